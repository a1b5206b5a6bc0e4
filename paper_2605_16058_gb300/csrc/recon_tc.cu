// Slice products on the tensor cores: Out_i = U_i diag(S_i) V_i^T (or Out_i -= ...; S may
// be null for S = 1, and V may be read transposed, which gives the rotation A_i V_i), the
// facewise product of the star-M product (Sec. 2.1, second step) for the factors of
// t-SVDM-I (uniform k) or t-SVDM-II (packed, slice i's columns offsets[i]..offsets[i+1]-1),
// FP32 data.  It is a dense contraction over the rank, so it runs on tcgen05:
//   D (128 rows a x 256 columns b, FP32 in TMEM) += A B^T,  A(a, c) = U(a, c) S(c),
//   B(b, c) = V(b, c), c over the slice's rank in K-blocks of 32.
// Every operand value enters as three BF16 terms x1 + x2 + x3 (residual <= 2^-27) and the
// six products of order >= 2^-24 are accumulated, so the result has FP32-level accuracy.
// One persistent CTA per SM (a kernel holding tensor memory runs one CTA per SM) takes
// output tiles (slice, a-tile, b-tile); 512 threads convert (four per row of A, two per
// row of B), one issues the MMAs, all drain TMEM.  Stages are double-buffered; every wait
// is bounded.  Loads run one K-block ahead: a block's values are requested before the
// previous block is converted, and a tile's first block while the previous tile's
// accumulator drains.  Nothing consumes a loaded value before the block's barrier (S(c)
// is loaded beside U and applied when the block is converted: a product formed at load
// time made every thread wait for its loads at each barrier, which doubled the time).
#include <cuda_bf16.h>

#include "common.cuh"
#include "tc.cuh"

namespace tsvdm {
namespace {

constexpr int RT = 512;                 // threads
constexpr int RM = 128, RN = 256, RK = 32;
constexpr uint32_t A_TERM = RM * 64;    // one BF16 term of the A tile (8 KB)
constexpr uint32_t B_TERM = RN * 64;    // one BF16 term of the B tile (16 KB)
constexpr uint32_t STAGE = 3 * A_TERM + 3 * B_TERM;   // 72 KB
constexpr unsigned RSPIN = 1u << 22;

struct ReconSmem {
  __align__(1024) unsigned char st[2][STAGE];
  uint64_t bar[2];                      // MMA completion per stage
  uint32_t tmem;
  int fail;
};

// SS: ||Out||^2 is accumulated (FP64); a separate instantiation, so that the product
// alone issues no FP64 instruction (predicated-off FP64 operations still occupy the FP64
// pipe, which runs at a small fraction of the FP32 rate on this GPU).
template <bool SS>
__global__ void __launch_bounds__(RT, 1)
    slice_products_tc_kernel(const float *__restrict__ U, const float *__restrict__ S,
                             const float *__restrict__ V, const int64_t *__restrict__ offsets,
                             int64_t k, int64_t n1, int64_t n2, int64_t n3,
                             float *__restrict__ Out, bool subtract, double *sumsq,
                             int *status, bool vtrans) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  ReconSmem &s = *reinterpret_cast<ReconSmem *>(((uintptr_t)smem_raw + 1023) & ~(uintptr_t)1023);
  constexpr int PA[6] = {0, 0, 1, 0, 2, 1}, PB[6] = {0, 1, 0, 2, 0, 1};
  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
  if (tid == 0) {
    tc::mbar_init(&s.bar[0], 1);
    tc::mbar_init(&s.bar[1], 1);
    tc::mbar_init_fence();
    s.fail = 0;
  }
  if (warp == 0) tc::tmem_alloc_n<RN>(&s.tmem);
  tc::fence_before_sync();
  __syncthreads();
  tc::fence_after_sync();
  const uint32_t tmem = s.tmem;
  const uint32_t idesc = tc::instr_desc(1, RM, RN);
  uint32_t phase = 0;
  auto wait = [&](int b) {
    const uint32_t par = (phase >> b) & 1u;
    if (!*(volatile int *)&s.fail && !tc::mbar_wait(&s.bar[b], par, RSPIN)) s.fail = 1;
    phase ^= 1u << b;
  };
  const int64_t ta = (n1 + RM - 1) / RM, tb = (n2 + RN - 1) / RN;
  const int64_t ntiles = n3 * ta * tb;
  double ss = 0.0;
  // operand values of K-block kb: A row a0 + (tid & 127), 8 columns of chunk tid >> 7;
  // B row b0 + (tid & 255), 16 columns of half tid >> 8
  const int ra = tid & 127, cha = tid >> 7;
  const int bh = tid >> 8;
  struct TileP {
    int64_t slice, a0, b0, c0, cnt;
    int nkb;
  };
  auto tparams = [&](int64_t tile) {
    TileP t;
    t.slice = tile / (ta * tb);
    t.a0 = ((tile / tb) % ta) * RM;
    t.b0 = (tile % tb) * RN;
    t.c0 = offsets ? offsets[t.slice] : t.slice * k;
    t.cnt = offsets ? offsets[t.slice + 1] - t.c0 : k;
    t.nkb = (int)((t.cnt + RK - 1) / RK);
    return t;
  };
  auto load_blk = [&](const TileP &t, int kb, float (&xa)[8], float &xs, float (&xb)[16]) {
    const int64_t arow = t.a0 + ra, bb = t.b0 + (tid & 255), c0 = t.c0, cnt = t.cnt;
#pragma unroll
    for (int e = 0; e < 8; ++e) {
      const int64_t c = (int64_t)kb * RK + cha * 8 + e;
      xa[e] = (arow < n1 && c < cnt) ? __ldg(U + (c0 + c) * n1 + arow) : 0.f;
    }
    {
      const int64_t c = (int64_t)kb * RK + cha * 8 + (lane & 7);
      xs = (S && c < cnt) ? __ldg(S + c0 + c) : 1.f;
    }
#pragma unroll
    for (int e = 0; e < 16; ++e) {
      const int64_t c = (int64_t)kb * RK + bh * 16 + e;
      // V(b, c) at (c0 + c) n2 + b, or (vtrans, uniform k) at c0 n2 + b k + c
      xb[e] = (bb < n2 && c < cnt)
                  ? __ldg(vtrans ? V + c0 * n2 + bb * k + c : V + (c0 + c) * n2 + bb)
                  : 0.f;
    }
  };
  float xa0[8], xs0, xb0[16], xa1[8], xs1, xb1[16];
  TileP cur = tparams(blockIdx.x);                 // the grid never exceeds the tile count
  if (cur.nkb > 0) load_blk(cur, 0, xa0, xs0, xb0);
  for (int64_t tile = blockIdx.x; tile < ntiles; tile += gridDim.x) {
    const int64_t slice = cur.slice, a0 = cur.a0, b0 = cur.b0;
    const int nkb = cur.nkb;
    // one K-block: the operands already in registers go to stage kb & 1 as three BF16
    // terms, the next block's values are loaded while this one's MMAs run
    auto run_blk = [&](int kb, float (&xa)[8], float &xs, float (&xb)[16],
                       float (&na)[8], float &ns, float (&nb)[16]) {
      const int b = kb & 1;
      if (kb + 1 < nkb) load_blk(cur, kb + 1, na, ns, nb);
      if (kb >= 2) wait(b);                        // the MMAs of K-block kb-2 read stage b
      unsigned char *st = s.st[b];
      {
        uint32_t w[3][4];
#pragma unroll
        for (int e = 0; e < 8; e += 2) {
          __nv_bfloat16 p0, p1, p2, q0, q1, q2;
          tc::split3(xa[e] * __shfl_sync(0xffffffffu, xs, e), p0, p1, p2);
          tc::split3(xa[e + 1] * __shfl_sync(0xffffffffu, xs, e + 1), q0, q1, q2);
          w[0][e / 2] = tc::pack2(p0, q0);
          w[1][e / 2] = tc::pack2(p1, q1);
          w[2][e / 2] = tc::pack2(p2, q2);
        }
        const uint32_t off = tc::sw64((uint32_t)ra, (uint32_t)cha);
#pragma unroll
        for (int u = 0; u < 3; ++u)
          *reinterpret_cast<uint4 *>(st + u * A_TERM + off) =
              make_uint4(w[u][0], w[u][1], w[u][2], w[u][3]);
      }
#pragma unroll
      for (int h = 0; h < 2; ++h) {
        const int ch = bh * 2 + h;
        uint32_t w[3][4];
#pragma unroll
        for (int e = 0; e < 8; e += 2) {
          __nv_bfloat16 p0, p1, p2, q0, q1, q2;
          tc::split3(xb[h * 8 + e], p0, p1, p2);
          tc::split3(xb[h * 8 + e + 1], q0, q1, q2);
          w[0][e / 2] = tc::pack2(p0, q0);
          w[1][e / 2] = tc::pack2(p1, q1);
          w[2][e / 2] = tc::pack2(p2, q2);
        }
        const uint32_t off = tc::sw64((uint32_t)(tid & 255), (uint32_t)ch);
#pragma unroll
        for (int u = 0; u < 3; ++u)
          *reinterpret_cast<uint4 *>(st + 3 * A_TERM + u * B_TERM + off) =
              make_uint4(w[u][0], w[u][1], w[u][2], w[u][3]);
      }
      tc::fence_proxy_async();
      tc::fence_before_sync();
      __syncthreads();
      if (tid == 0) {
        tc::fence_after_sync();
#pragma unroll
        for (int kk = 0; kk < 2; ++kk)
#pragma unroll
          for (int m = 0; m < 6; ++m) {
            const uint64_t da = tc::smem_desc(st + PA[m] * A_TERM + kk * 32, 512, 4);
            const uint64_t db = tc::smem_desc(st + 3 * A_TERM + PB[m] * B_TERM + kk * 32, 512, 4);
            tc::mma_f16(tmem, da, db, idesc, (kb > 0 || kk > 0 || m > 0) ? 1u : 0u);
          }
        tc::mma_commit(&s.bar[b]);
      }
    };
    for (int kb = 0; kb < nkb; kb += 2) {
      run_blk(kb, xa0, xs0, xb0, xa1, xs1, xb1);
      if (kb + 1 < nkb) run_blk(kb + 1, xa1, xs1, xb1, xa0, xs0, xb0);
    }
    // the next tile's first K-block is loaded while this tile's MMAs finish and its
    // accumulator drains (both register sets are free here)
    TileP nxt = cur;
    if (tile + gridDim.x < ntiles) {
      nxt = tparams(tile + gridDim.x);
      if (nxt.nkb > 0) load_blk(nxt, 0, xa0, xs0, xb0);
    }
    for (int kb = nkb >= 2 ? nkb - 2 : 0; kb < nkb; ++kb) wait(kb & 1);
    tc::fence_after_sync();
    // epilogue: warp w reads TMEM lanes 32 (w mod 4).. (rows) and columns (w / 4) * 64 ..
    {
      const int r = (warp & 3) * 32 + lane;
      const int64_t a = a0 + r;
      const uint32_t lane_base = (uint32_t)((warp & 3) * 32) << 16;
      float *O = Out + slice * n1 * n2;
      for (int j0 = (warp >> 2) * 64; j0 < (warp >> 2) * 64 + 64; j0 += 16) {
        float d[16];
        if (nkb > 0) {
          tc::tmem_ld16(tmem + lane_base + (uint32_t)j0, d);
        } else {
#pragma unroll
          for (int e = 0; e < 16; ++e) d[e] = 0.f;
        }
        if (a < n1) {
#pragma unroll
          for (int e = 0; e < 16; ++e) {
            const int64_t bcol = b0 + j0 + e;
            if (bcol < n2) {
              const float v = subtract ? O[a + n1 * bcol] - d[e] : d[e];
              O[a + n1 * bcol] = v;
              if constexpr (SS) ss += (double)v * (double)v;
            }
          }
        }
      }
    }
    tc::fence_before_sync();
    __syncthreads();                               // TMEM read before the next tile's MMAs
    cur = nxt;
  }
  if constexpr (SS) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) ss += __shfl_xor_sync(0xffffffffu, ss, o);
    if (lane == 0) atomicAdd(sumsq, ss);
  }
  tc::fence_before_sync();
  __syncthreads();
  if (warp == 0) {
    tc::fence_after_sync();
    tc::tmem_dealloc_n<RN>(tmem);
  }
  if (tid == 0 && s.fail && status) atomicOr(status, ST_TIMEOUT);
}

}  // namespace

cudaError_t slice_products_tc(const float *U, const float *S, const float *V,
                              const int64_t *offsets, int64_t k, int64_t n1, int64_t n2,
                              int64_t n3, float *Out, bool subtract_from_out, double *sumsq,
                              int *status, cudaStream_t st, bool vtrans) {
  const size_t smem = sizeof(ReconSmem) + 1024;
  auto kern = sumsq ? slice_products_tc_kernel<true> : slice_products_tc_kernel<false>;
  cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  if (e != cudaSuccess) return e;
  int dev = 0, sms = 0;
  if ((e = cudaGetDevice(&dev)) != cudaSuccess) return e;
  if ((e = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev)) != cudaSuccess)
    return e;
  const int64_t ntiles = n3 * ((n1 + RM - 1) / RM) * ((n2 + RN - 1) / RN);
  if (ntiles == 0) return cudaSuccess;
  const int grid = (int)(ntiles < sms ? ntiles : sms);
  kern<<<grid, RT, smem, st>>>(U, S, V, offsets, k, n1, n2, n3, Out, subtract_from_out, sumsq,
                               status, vtrans);
  return cudaGetLastError();
}

}  // namespace tsvdm
