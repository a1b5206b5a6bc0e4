// Second pass of the two-pass decompositions (Sec. 3.4): the other side of the kept triplets,
// Z_i = A_i^T K_i diag(1 / S_i), on the tensor cores for FP32 slices in the column layout
// (n1 >= n2; kd = n1 rows, od = n2 columns): A_i is the slice (column c of A_i is od-th
// column of the slice, kd contiguous values), K_i the emitted kept columns (column j at
// (base + j) kd, kd contiguous values), Z_i column j at (base + j) od.
//
// Both operands are K-major in memory (the contraction runs along the kd contiguous values),
// so a thread loads 16-byte vectors.  Every value enters as three BF16 terms x1 + x2 + x3
// (residual <= 2^-27) and the six products of order >= 2^-24 are accumulated in FP32
// (TMEM), FP32-level accuracy as the CUDA-core product it replaces.  Tile: 128 entries
// (od) x N <= 256 columns (the slice's kept count, in multiples of 16), contraction in
// K-blocks of 32; two stages, the next block's values loaded into registers while the
// current block's MMAs run.  One persistent CTA per SM (a kernel holding tensor memory runs
// one CTA per SM) walks (slice, entry tile, column tile) in order; every wait is bounded.
#include <cuda_bf16.h>

#include "common.cuh"
#include "tc.cuh"

namespace tsvdm {
namespace {

constexpr int QT = 512;                 // threads
constexpr int QM = 128, QN = 256, QK = 32;
constexpr uint32_t QA_TERM = QM * 64;   // one BF16 term of the A tile (8 KB)
constexpr uint32_t QB_TERM = QN * 64;   // one BF16 term of the B tile (16 KB)
constexpr uint32_t QSTAGE = 3 * QA_TERM + 3 * QB_TERM;   // 72 KB
constexpr unsigned QSPIN = 1u << 22;

struct CompleteSmem {
  __align__(1024) unsigned char st[2][QSTAGE];
  uint64_t bar[2];                      // MMA completion per stage
  uint32_t tmem;
  int fail;
};

__global__ void __launch_bounds__(QT, 1)
    complete_tc_kernel(const float *__restrict__ Ahat, int64_t kd, int64_t od, int64_t nslices,
                       int64_t k_uniform, const int *__restrict__ ranks,
                       const int64_t *__restrict__ offsets, const float *__restrict__ Kv,
                       const float *__restrict__ S, float *__restrict__ Ov, int *status) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  CompleteSmem &s =
      *reinterpret_cast<CompleteSmem *>(((uintptr_t)smem_raw + 1023) & ~(uintptr_t)1023);
  constexpr int PA[6] = {0, 0, 1, 0, 2, 1}, PB[6] = {0, 1, 0, 2, 0, 1};
  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
  if (tid == 0) {
    tc::mbar_init(&s.bar[0], 1);
    tc::mbar_init(&s.bar[1], 1);
    tc::mbar_init_fence();
    s.fail = 0;
  }
  if (warp == 0) tc::tmem_alloc_n<QN>(&s.tmem);
  tc::fence_before_sync();
  __syncthreads();
  tc::fence_after_sync();
  const uint32_t tmem = s.tmem;
  uint32_t phase = 0;
  auto wait = [&](int b) {
    const uint32_t par = (phase >> b) & 1u;
    if (!*(volatile int *)&s.fail && !tc::mbar_wait(&s.bar[b], par, QSPIN)) s.fail = 1;
    phase ^= 1u << b;
  };
  const int64_t nct = (od + QM - 1) / QM;
  const int64_t ntiles = nslices * nct * 2;
  const int nkb = (int)((kd + QK - 1) / QK);
  // operand rows of this thread: A row ra (an entry of the tile), B rows rb and rb + 128
  // (kept columns); 8 consecutive contraction values of each (quarter q of the K-block)
  const int ra = tid >> 2, q = tid & 3, rb = tid >> 2;
  for (int64_t tile = blockIdx.x; tile < ntiles; tile += gridDim.x) {
    const int64_t slice = tile / (nct * 2);
    const int64_t ct = (tile / 2) % nct, jt = tile % 2;
    const int64_t cnt = ranks ? (int64_t)ranks[slice] : k_uniform;
    const int64_t j0 = jt * QN;
    if (j0 >= cnt) continue;                      // the same decision in every thread
    const int64_t base = offsets ? offsets[slice] : slice * k_uniform;
    const int64_t ncols = cnt - j0 < QN ? cnt - j0 : QN;
    const uint32_t nn = (uint32_t)((ncols + 15) / 16 * 16);
    const int64_t c0 = ct * QM;
    const float *A = Ahat + slice * kd * od;
    const uint32_t idesc = tc::instr_desc(1, QM, nn);
    // 8 values of one operand row at contraction offset kb * 32 + q * 8 (zeros outside)
    auto load8v = [&](const float *row, bool valid, int kb, float (&x)[8]) {
      const int64_t r = (int64_t)kb * QK + q * 8;
      if (valid && r + 8 <= kd) {
        const float4 u = __ldg(reinterpret_cast<const float4 *>(row + r));
        const float4 w = __ldg(reinterpret_cast<const float4 *>(row + r + 4));
        x[0] = u.x; x[1] = u.y; x[2] = u.z; x[3] = u.w;
        x[4] = w.x; x[5] = w.y; x[6] = w.z; x[7] = w.w;
      } else {
#pragma unroll
        for (int e = 0; e < 8; ++e) x[e] = (valid && r + e < kd) ? __ldg(row + r + e) : 0.f;
      }
    };
    const bool va = c0 + ra < od;
    const float *arow = A + (c0 + ra) * kd;
    const bool vb0 = rb < ncols, vb1 = rb + 128 < ncols;
    const float *brow0 = Kv + (base + j0 + rb) * kd, *brow1 = Kv + (base + j0 + rb + 128) * kd;
    auto load_blk = [&](int kb, float (&xa)[8], float (&xb)[16]) {
      load8v(arow, va, kb, xa);
      float t0[8], t1[8];
      load8v(brow0, vb0, kb, t0);
      load8v(brow1, vb1, kb, t1);
#pragma unroll
      for (int e = 0; e < 8; ++e) {
        xb[e] = t0[e];
        xb[8 + e] = t1[e];
      }
    };
    // three BF16 terms of 8 values -> one 16-byte chunk per term of a swizzled row
    auto put8 = [&](unsigned char *tiles, uint32_t term_bytes, uint32_t row, const float *x) {
      uint32_t w[3][4];
#pragma unroll
      for (int e = 0; e < 8; e += 2) {
        __nv_bfloat16 p0, p1, p2, q0, q1, q2;
        tc::split3(x[e], p0, p1, p2);
        tc::split3(x[e + 1], q0, q1, q2);
        w[0][e / 2] = tc::pack2(p0, q0);
        w[1][e / 2] = tc::pack2(p1, q1);
        w[2][e / 2] = tc::pack2(p2, q2);
      }
      const uint32_t off = tc::sw64(row, (uint32_t)q);
#pragma unroll
      for (int u = 0; u < 3; ++u)
        *reinterpret_cast<uint4 *>(tiles + u * term_bytes + off) =
            make_uint4(w[u][0], w[u][1], w[u][2], w[u][3]);
    };
    auto run_blk = [&](int kb, float (&xa)[8], float (&xb)[16], float (&na)[8],
                       float (&nb)[16]) {
      const int b = kb & 1;
      if (kb >= 2) wait(b);                        // the MMAs of K-block kb-2 read stage b
      unsigned char *st = s.st[b];
      put8(st, QA_TERM, (uint32_t)ra, xa);
      put8(st + 3 * QA_TERM, QB_TERM, (uint32_t)rb, xb);
      if (nn > 128) put8(st + 3 * QA_TERM, QB_TERM, (uint32_t)(rb + 128), xb + 8);
      if (kb + 1 < nkb) load_blk(kb + 1, na, nb);
      tc::fence_proxy_async();
      tc::fence_before_sync();
      __syncthreads();
      if (tid == 0) {
        tc::fence_after_sync();
#pragma unroll
        for (int kk = 0; kk < 2; ++kk)
#pragma unroll
          for (int m = 0; m < 6; ++m) {
            const uint64_t da = tc::smem_desc(st + PA[m] * QA_TERM + kk * 32, 512, 4);
            const uint64_t db = tc::smem_desc(st + 3 * QA_TERM + PB[m] * QB_TERM + kk * 32, 512, 4);
            tc::mma_f16(tmem, da, db, idesc, (kb > 0 || kk > 0 || m > 0) ? 1u : 0u);
          }
        tc::mma_commit(&s.bar[b]);
      }
    };
    float xa0[8], xb0[16], xa1[8], xb1[16];
    load_blk(0, xa0, xb0);
    for (int kb = 0; kb < nkb; kb += 2) {
      run_blk(kb, xa0, xb0, xa1, xb1);
      if (kb + 1 < nkb) run_blk(kb + 1, xa1, xb1, xa0, xb0);
    }
    for (int kb = nkb >= 2 ? nkb - 2 : 0; kb < nkb; ++kb) wait(kb & 1);
    tc::fence_after_sync();
    // epilogue: warp w reads TMEM lanes 32 (w mod 4).. (entries) and columns (w / 4) * 64 ..
    {
      const int r = (warp & 3) * 32 + lane;
      const int64_t c = c0 + r;
      const uint32_t lane_base = (uint32_t)((warp & 3) * 32) << 16;
      for (int jj = (warp >> 2) * 64; jj < (warp >> 2) * 64 + 64; jj += 16) {
        if ((uint32_t)jj >= nn) break;
        float d[16];
        tc::tmem_ld16(tmem + lane_base + (uint32_t)jj, d);
        if (c < od) {
#pragma unroll
          for (int e = 0; e < 16; ++e) {
            const int64_t j = j0 + jj + e;
            if (j < cnt) {
              const float sj = S ? __ldg(S + base + j) : 1.f;
              const float inv = sj > 0.f ? 1.f / sj : 0.f;
              Ov[(base + j) * od + c] = d[e] * inv;
            }
          }
        }
      }
    }
    tc::fence_before_sync();
    __syncthreads();                               // TMEM read before the next tile's MMAs
  }
  tc::fence_before_sync();
  __syncthreads();
  if (warp == 0) {
    tc::fence_after_sync();
    tc::tmem_dealloc_n<QN>(tmem);
  }
  if (tid == 0 && s.fail && status) atomicOr(status, ST_TIMEOUT);
}


// K_i <- K_i R_i of the second pass (rotate_back): Ktmp(:, q) = K(:, 0..rho-1) R(:, perm[q])
// for every entry of the restricted Jacobi, on the tensor cores.  A = K (kd entries x rho,
// entries contiguous: per-element loads, one K-block value of eight per thread), B rows
// q = R's column perm[q] (rho contiguous values); tiles of 128 entries x N <= 256 output
// columns, the rank in K-blocks of 32; the same three-term split, stages and epilogue as
// complete_tc_kernel.
__global__ void __launch_bounds__(QT, 1)
    rotate_tc_kernel(const SliceDesc *__restrict__ desc, const int64_t *__restrict__ off,
                     int count, int64_t kd, const float *__restrict__ Kin,
                     float *__restrict__ Ktmp, int *status) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  CompleteSmem &s =
      *reinterpret_cast<CompleteSmem *>(((uintptr_t)smem_raw + 1023) & ~(uintptr_t)1023);
  constexpr int PA[6] = {0, 0, 1, 0, 2, 1}, PB[6] = {0, 1, 0, 2, 0, 1};
  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
  if (tid == 0) {
    tc::mbar_init(&s.bar[0], 1);
    tc::mbar_init(&s.bar[1], 1);
    tc::mbar_init_fence();
    s.fail = 0;
  }
  if (warp == 0) tc::tmem_alloc_n<QN>(&s.tmem);
  tc::fence_before_sync();
  __syncthreads();
  tc::fence_after_sync();
  const uint32_t tmem = s.tmem;
  uint32_t phase = 0;
  auto wait = [&](int b) {
    const uint32_t par = (phase >> b) & 1u;
    if (!*(volatile int *)&s.fail && !tc::mbar_wait(&s.bar[b], par, QSPIN)) s.fail = 1;
    phase ^= 1u << b;
  };
  const int64_t nct = (kd + QM - 1) / QM;
  const int64_t ntiles = (int64_t)count * nct * 2;
  const int ra = tid >> 2, q = tid & 3, rb = tid >> 2;
  for (int64_t tile = blockIdx.x; tile < ntiles; tile += gridDim.x) {
    const int64_t e = tile / (nct * 2);
    const int64_t ct = (tile / 2) % nct, jt = tile % 2;
    const SliceDesc d = desc[e];
    const int64_t rho = d.cols;
    const int64_t q0 = jt * QN;
    if (q0 >= rho) continue;                      // the same decision in every thread
    const int64_t base = off[e];
    const int64_t ncols = rho - q0 < QN ? rho - q0 : QN;
    const uint32_t nn = (uint32_t)((ncols + 15) / 16 * 16);
    const int64_t c0 = ct * QM;
    const int nkb = (int)((rho + QK - 1) / QK);
    const uint32_t idesc = tc::instr_desc(1, QM, nn);
    const float *R = reinterpret_cast<const float *>(d.V);
    const bool va = c0 + ra < kd;
    const float *acol = Kin + base * kd + c0 + ra;          // K(c0 + ra, l) at + l kd
    const bool vb0 = rb < ncols, vb1 = rb + 128 < ncols;
    const float *brow0 = vb0 ? R + (int64_t)d.perm[q0 + rb] * rho : R;
    const float *brow1 = vb1 ? R + (int64_t)d.perm[q0 + rb + 128] * rho : R;
    auto load_blk = [&](int kb, float (&xa)[8], float (&xb)[16]) {
      const int64_t l0 = (int64_t)kb * QK + q * 8;
#pragma unroll
      for (int u = 0; u < 8; ++u) {
        const int64_t l = l0 + u;
        xa[u] = (va && l < rho) ? __ldg(acol + l * kd) : 0.f;
        xb[u] = (vb0 && l < rho) ? __ldg(brow0 + l) : 0.f;
        xb[8 + u] = (vb1 && l < rho) ? __ldg(brow1 + l) : 0.f;
      }
    };
    auto put8 = [&](unsigned char *tiles, uint32_t term_bytes, uint32_t row, const float *x) {
      uint32_t w[3][4];
#pragma unroll
      for (int u = 0; u < 8; u += 2) {
        __nv_bfloat16 p0, p1, p2, q0_, q1, q2;
        tc::split3(x[u], p0, p1, p2);
        tc::split3(x[u + 1], q0_, q1, q2);
        w[0][u / 2] = tc::pack2(p0, q0_);
        w[1][u / 2] = tc::pack2(p1, q1);
        w[2][u / 2] = tc::pack2(p2, q2);
      }
      const uint32_t offs = tc::sw64(row, (uint32_t)q);
#pragma unroll
      for (int u = 0; u < 3; ++u)
        *reinterpret_cast<uint4 *>(tiles + u * term_bytes + offs) =
            make_uint4(w[u][0], w[u][1], w[u][2], w[u][3]);
    };
    auto run_blk = [&](int kb, float (&xa)[8], float (&xb)[16], float (&na)[8],
                       float (&nb)[16]) {
      const int b = kb & 1;
      if (kb >= 2) wait(b);                        // the MMAs of K-block kb-2 read stage b
      unsigned char *st = s.st[b];
      put8(st, QA_TERM, (uint32_t)ra, xa);
      put8(st + 3 * QA_TERM, QB_TERM, (uint32_t)rb, xb);
      if (nn > 128) put8(st + 3 * QA_TERM, QB_TERM, (uint32_t)(rb + 128), xb + 8);
      if (kb + 1 < nkb) load_blk(kb + 1, na, nb);
      tc::fence_proxy_async();
      tc::fence_before_sync();
      __syncthreads();
      if (tid == 0) {
        tc::fence_after_sync();
#pragma unroll
        for (int kk = 0; kk < 2; ++kk)
#pragma unroll
          for (int m = 0; m < 6; ++m) {
            const uint64_t da = tc::smem_desc(st + PA[m] * QA_TERM + kk * 32, 512, 4);
            const uint64_t db = tc::smem_desc(st + 3 * QA_TERM + PB[m] * QB_TERM + kk * 32, 512, 4);
            tc::mma_f16(tmem, da, db, idesc, (kb > 0 || kk > 0 || m > 0) ? 1u : 0u);
          }
        tc::mma_commit(&s.bar[b]);
      }
    };
    float xa0[8], xb0[16], xa1[8], xb1[16];
    load_blk(0, xa0, xb0);
    for (int kb = 0; kb < nkb; kb += 2) {
      run_blk(kb, xa0, xb0, xa1, xb1);
      if (kb + 1 < nkb) run_blk(kb + 1, xa1, xb1, xa0, xb0);
    }
    for (int kb = nkb >= 2 ? nkb - 2 : 0; kb < nkb; ++kb) wait(kb & 1);
    tc::fence_after_sync();
    {
      const int r = (warp & 3) * 32 + lane;
      const int64_t c = c0 + r;
      const uint32_t lane_base = (uint32_t)((warp & 3) * 32) << 16;
      for (int jj = (warp >> 2) * 64; jj < (warp >> 2) * 64 + 64; jj += 16) {
        if ((uint32_t)jj >= nn) break;
        float dv[16];
        tc::tmem_ld16(tmem + lane_base + (uint32_t)jj, dv);
        if (c < kd) {
#pragma unroll
          for (int u = 0; u < 16; ++u) {
            const int64_t qq = q0 + jj + u;
            if (qq < rho) Ktmp[(base + qq) * kd + c] = dv[u];
          }
        }
      }
    }
    tc::fence_before_sync();
    __syncthreads();                               // TMEM read before the next tile's MMAs
  }
  tc::fence_before_sync();
  __syncthreads();
  if (warp == 0) {
    tc::fence_after_sync();
    tc::tmem_dealloc_n<QN>(tmem);
  }
  if (tid == 0 && s.fail && status) atomicOr(status, ST_TIMEOUT);
}

}  // namespace

bool complete_tc_supported(const float *Ahat, const float *K, int64_t n1, int64_t n2,
                           bool transposed) {
  return !transposed && n1 >= 1 && n2 >= 1 && (n1 % 4) == 0 && ((uintptr_t)Ahat & 15) == 0 &&
         ((uintptr_t)K & 15) == 0;
}

cudaError_t complete_tc(const float *Ahat, int64_t n1, int64_t n2, int64_t nslices,
                        int64_t k_uniform, const int *ranks, const int64_t *offsets,
                        const float *K, const float *S, float *O, int *status, cudaStream_t st) {
  if (nslices <= 0) return cudaSuccess;
  const size_t smem = sizeof(CompleteSmem) + 1024;
  cudaError_t e = cudaFuncSetAttribute(complete_tc_kernel,
                                       cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  if (e != cudaSuccess) return e;
  int dev = 0, sms = 0;
  if ((e = cudaGetDevice(&dev)) != cudaSuccess) return e;
  if ((e = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev)) != cudaSuccess)
    return e;
  const int64_t ntiles = nslices * ((n2 + QM - 1) / QM) * 2;
  const int grid = (int)(ntiles < sms ? ntiles : sms);
  complete_tc_kernel<<<grid, QT, smem, st>>>(Ahat, n1, n2, nslices, k_uniform, ranks, offsets,
                                             K, S, O, status);
  return cudaGetLastError();
}

}  // namespace tsvdm

namespace tsvdm {

cudaError_t rotate_tc(const SliceDesc *desc, const int64_t *off, int count, int64_t kd,
                      const float *Kin, float *Ktmp, int *status, cudaStream_t st) {
  if (count <= 0) return cudaSuccess;
  const size_t smem = sizeof(CompleteSmem) + 1024;
  cudaError_t e = cudaFuncSetAttribute(rotate_tc_kernel,
                                       cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  if (e != cudaSuccess) return e;
  int dev = 0, sms = 0;
  if ((e = cudaGetDevice(&dev)) != cudaSuccess) return e;
  if ((e = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev)) != cudaSuccess)
    return e;
  const int64_t ntiles = (int64_t)count * ((kd + QM - 1) / QM) * 2;
  const int grid = (int)(ntiles < sms ? ntiles : sms);
  rotate_tc_kernel<<<grid, QT, smem, st>>>(desc, off, count, kd, Kin, Ktmp, status);
  return cudaGetLastError();
}

}  // namespace tsvdm
