// C (n x n) = alpha A^T B on the tensor cores, for FP32 column-major P x n operands A and B
// (P = n1 n2 rows).  This is the contraction of the backward pass, dL/dM = alpha R_(mat)^T
// X_(mat) (Sec. 3.3's adjoint of the mode-3 product), and of the data-driven transform, the
// mode-3 Gram A_(3) A_(3)^T (Sec. 2.2); both contract over the long mode, so the work is
// split over P and the partial n x n products are summed in FP64 in a fixed order.
//
// Precision (BF16x3, as the tensor-core TTM): x = x_hi + x_lo with x_hi = bf16(x),
// x_lo = bf16(x - x_hi); D += A_hi B_hi + A_hi B_lo + A_lo B_hi in FP32 (TMEM).
//
// Layout: one CTA owns a band of 128 rows of C (columns i0.. of A) and all npad <= 512
// columns of C (columns of B; n rounded up to 128) over a range of P; the accumulator is
// 128 TMEM lanes x npad columns.  Operand tiles are K-major (K = P, which is contiguous in a column of A or B),
// 64-byte rows of 32 BF16, 64-byte swizzle, so a column's 32 consecutive P-values are one
// tile row.  When A and B are the same matrix (the Gram) the A operand is rows i0.. of the
// B tile.  Warp roles (544 threads): warp 0 allocates TMEM and one of its threads issues the
// MMAs; warps 1..16 convert (eight threads per tile row, a 16-byte load each), with the next
// k-step's values in flight in registers, and finally drain TMEM into the FP64 partials.
// Stages rotate through full (written by every converter warp) and empty (read by the
// MMAs) barriers; every wait is bounded (ST_TIMEOUT); nothing traps.
#include <cuda_bf16.h>

#include "common.cuh"
#include "tc.cuh"

namespace tsvdm {
namespace {

constexpr int AT_THREADS = 544;        // warp 0 MMA + TMEM, warps 1..16 convert and drain
constexpr int AT_CONV = 512;           // converter threads
constexpr int AT_BM = 128;             // rows of C per CTA
constexpr int AT_BK = 32;              // P per k-step (one 64-byte BF16 row)
constexpr int AT_MAX_STAGES = 4;
constexpr int AT_MAX_ROWS = 8;         // tile rows per converter thread and k-step
constexpr unsigned AT_SPIN = 1u << 26;

struct AtbParams {
  const float *A, *B;
  int64_t P, n, chunk;                 // chunk: P per split (multiple of AT_BK)
  int npad, mbands, stages, same;
  uint32_t a_bytes, b_bytes, stage_bytes, tmem_cols;
  double *ws;                          // [split][n x n] FP64 partials
  int *status;
};

__global__ void __launch_bounds__(AT_THREADS, 1) atb_tc_kernel(AtbParams p) {
  extern __shared__ __align__(1024) unsigned char smem_raw[];
  unsigned char *smem = (unsigned char *)(((uintptr_t)smem_raw + 1023) & ~(uintptr_t)1023);
  const int S = p.stages;
  uint64_t *full = (uint64_t *)(smem + S * p.stage_bytes);
  uint64_t *empty = full + AT_MAX_STAGES;
  uint64_t *done = empty + AT_MAX_STAGES;
  uint32_t *tmem_slot = (uint32_t *)(done + 1);
  __shared__ int s_fail;
  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
  const int band = (int)(blockIdx.x % p.mbands);
  const int64_t split = blockIdx.x / p.mbands;
  const int64_t i0 = (int64_t)band * AT_BM;
  const int64_t pbeg = split * p.chunk;
  const int64_t pend = pbeg + p.chunk < p.P ? pbeg + p.chunk : p.P;
  const int nk = pend > pbeg ? (int)((pend - pbeg + AT_BK - 1) / AT_BK) : 0;
  if (tid == 0) {
    s_fail = 0;
    for (int s = 0; s < S; ++s) {
      tc::mbar_init(&full[s], AT_CONV / 32);
      tc::mbar_init(&empty[s], 1);
    }
    tc::mbar_init(done, 1);
    tc::mbar_init_fence();
  }
  if (warp == 0) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(
                     tc::smem_u32(tmem_slot)),
                 "r"(p.tmem_cols)
                 : "memory");
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
  }
  tc::fence_before_sync();
  __syncthreads();
  tc::fence_after_sync();
  const uint32_t tmem = *tmem_slot;
  auto wait = [&](uint64_t *bar, uint32_t par) -> bool {
    if (*(volatile int *)&s_fail) return false;
    if (!tc::mbar_wait(bar, par, AT_SPIN)) {
      s_fail = 1;
      return false;
    }
    return true;
  };
  const uint32_t a_off = 0u;                     // A tiles first (when separate), then B
  const uint32_t b_off = p.same ? 0u : p.a_bytes;

  if (warp == 0) {
    if (lane == 0) {
      // ---------------- MMA issuer
      for (int it = 0; it < nk; ++it) {
        const int s = it % S, u = it / S;
        if (!wait(&full[s], u & 1)) break;
        tc::fence_after_sync();
        unsigned char *st = smem + s * p.stage_bytes;
        // A: its own tiles, or rows i0.. of the B tiles (the Gram)
        unsigned char *ahi = p.same ? st + b_off + (uint32_t)i0 * 64 : st + a_off;
        unsigned char *alo = p.same ? st + b_off + (uint32_t)p.npad * 64 + (uint32_t)i0 * 64
                                    : st + a_off + AT_BM * 64;
        unsigned char *bhi = st + b_off, *blo = st + b_off + (uint32_t)p.npad * 64;
#pragma unroll
        for (int kk = 0; kk < AT_BK / 16; ++kk) {
          const uint32_t koff = kk * 32;
          for (int n0 = 0; n0 < p.npad; n0 += 256) {
            const uint32_t nn = p.npad - n0 < 256 ? (uint32_t)(p.npad - n0) : 256u;
            const uint32_t idesc = tc::instr_desc(1, AT_BM, nn);
            const uint32_t d = tmem + (uint32_t)n0;
            const uint64_t dah = tc::smem_desc(ahi + koff, 512, 4);
            const uint64_t dal = tc::smem_desc(alo + koff, 512, 4);
            const uint64_t dbh = tc::smem_desc(bhi + n0 * 64 + koff, 512, 4);
            const uint64_t dbl = tc::smem_desc(blo + n0 * 64 + koff, 512, 4);
            tc::mma_f16(d, dah, dbh, idesc, (it > 0 || kk > 0) ? 1u : 0u);
            tc::mma_f16(d, dah, dbl, idesc, 1u);
            tc::mma_f16(d, dal, dbh, idesc, 1u);
          }
        }
        tc::mma_commit(&empty[s]);
      }
      tc::mma_commit(done);
    }
  } else {
    // ---------------- converters: thread c owns tile rows g8, g8 + 64, ... (rows 0..127 of
    // the A tile when separate, then the npad rows of the B tile), 4 P-values each
    const int c = tid - 32, g8 = c >> 3, l8 = c & 7;
    const int rows = (p.same ? 0 : AT_BM) + p.npad;
    // operand column of tile row r (-1: zero padding)
    auto column = [&](int r, const float *&src) -> int64_t {
      if (!p.same && r < AT_BM) {
        src = p.A;
        return i0 + r < p.n ? i0 + r : -1;
      }
      const int j = p.same ? r : r - AT_BM;
      src = p.B;
      return j < p.n ? j : -1;
    };
    auto load = [&](int it, float4 (&v)[AT_MAX_ROWS]) {
      const int64_t p0 = pbeg + (int64_t)it * AT_BK + 4 * l8;
#pragma unroll
      for (int q = 0; q < AT_MAX_ROWS; ++q) {
        const int r = g8 + 64 * q;
        v[q] = make_float4(0.f, 0.f, 0.f, 0.f);
        if (r < rows && it < nk && p0 < pend) {
          const float *src;
          const int64_t col = column(r, src);
          if (col >= 0) v[q] = __ldcg(reinterpret_cast<const float4 *>(src + p.P * col + p0));
        }
      }
    };
    auto put = [&](unsigned char *st, const float4 (&v)[AT_MAX_ROWS]) {
#pragma unroll
      for (int q = 0; q < AT_MAX_ROWS; ++q) {
        const int r = g8 + 64 * q;
        if (r >= rows) break;
        const float x[4] = {v[q].x, v[q].y, v[q].z, v[q].w};
        uint32_t h[2], l[2];
#pragma unroll
        for (int e = 0; e < 2; ++e) {
          const __nv_bfloat16 h0 = __float2bfloat16_rn(x[2 * e]), h1 = __float2bfloat16_rn(x[2 * e + 1]);
          const __nv_bfloat16 l0 = __float2bfloat16_rn(x[2 * e] - __bfloat162float(h0));
          const __nv_bfloat16 l1 = __float2bfloat16_rn(x[2 * e + 1] - __bfloat162float(h1));
          h[e] = tc::pack2(h0, h1);
          l[e] = tc::pack2(l0, l1);
        }
        // tile and row within it; hi tile, then lo tile npad (or 128) rows further
        uint32_t base, tr, lo_step;
        if (!p.same && r < AT_BM) {
          base = a_off;
          tr = (uint32_t)r;
          lo_step = AT_BM * 64;
        } else {
          base = b_off;
          tr = (uint32_t)(p.same ? r : r - AT_BM);
          lo_step = (uint32_t)p.npad * 64;
        }
        const uint32_t off = base + tc::sw64(tr, (uint32_t)(l8 >> 1)) + (uint32_t)(l8 & 1) * 8;
        *reinterpret_cast<uint2 *>(st + off) = make_uint2(h[0], h[1]);
        *reinterpret_cast<uint2 *>(st + off + lo_step) = make_uint2(l[0], l[1]);
      }
    };
    // two register sets alternate (constant indices: no copy of a register in flight)
    float4 va[AT_MAX_ROWS], vb[AT_MAX_ROWS];
    load(0, va);
    auto step = [&](int it, float4 (&cur)[AT_MAX_ROWS], float4 (&nxt)[AT_MAX_ROWS]) -> bool {
      load(it + 1, nxt);
      const int s = it % S, u = it / S;
      if (u > 0 && !wait(&empty[s], (u - 1) & 1)) return false;
      put(smem + s * p.stage_bytes, cur);
      tc::fence_proxy_async();
      __syncwarp();
      if (lane == 0) tc::mbar_arrive(&full[s]);
      return true;
    };
    for (int it = 0; it < nk; it += 2) {
      if (!step(it, va, vb)) break;
      if (it + 1 < nk && !step(it + 1, vb, va)) break;
    }
    // ---------------- drain: warp w reads TMEM lanes 32 (w mod 4).. and a quarter of the
    // columns; rows i0 + lane.., FP64 partials of this split
    if (wait(done, 0) || nk == 0) {
      tc::fence_after_sync();
      const int qd = warp & 3, part = (warp - 1) >> 2;
      const int64_t i = i0 + qd * 32 + lane;
      const int cols = p.npad / 4;
      double *out = p.ws + split * p.n * p.n;
      for (int j0 = part * cols; j0 < (part + 1) * cols; j0 += 16) {
        float d[16];
        if (nk > 0) {
          tc::tmem_ld16(tmem + ((uint32_t)(qd * 32) << 16) + (uint32_t)j0, d);
        } else {
#pragma unroll
          for (int e = 0; e < 16; ++e) d[e] = 0.f;
        }
        if (i < p.n) {
#pragma unroll
          for (int e = 0; e < 16; ++e)
            if (j0 + e < p.n) out[i + p.n * (j0 + e)] = (double)d[e];
        }
      }
    }
  }
  tc::fence_before_sync();
  __syncthreads();
  if (warp == 0) {
    tc::fence_after_sync();
    asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem),
                 "r"(p.tmem_cols)
                 : "memory");
  }
  if (tid == 0 && s_fail && p.status) atomicOr(p.status, ST_TIMEOUT);
}

template <typename T>
__global__ void atb_tc_reduce_kernel(const double *__restrict__ ws, int64_t n, int64_t splits,
                                     const double *alpha, T *C) {
  const int64_t idx = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (idx >= n * n) return;
  double s = 0.0;
  for (int64_t z = 0; z < splits; ++z) s += ws[z * n * n + idx];   // fixed order
  C[idx] = (T)(s * (alpha ? *alpha : 1.0));
}

}  // namespace

bool atb_tc_supported(const float *A, const float *B, int64_t P, int64_t n) {
  return n >= 1 && n <= 512 && P >= 1 && (P % 4) == 0 && ((uintptr_t)A & 15) == 0 &&
         ((uintptr_t)B & 15) == 0;
}

cudaError_t atb_tc(const float *A, const float *B, int64_t P, int64_t n, float *C,
                   const double *alpha, double *ws, size_t ws_elems, int *status,
                   cudaStream_t st) {
  if (!atb_tc_supported(A, B, P, n)) return cudaErrorNotSupported;
  AtbParams p;
  p.A = A;
  p.B = B;
  p.P = P;
  p.n = n;
  p.same = A == B ? 1 : 0;
  // npad: a multiple of 128, so that the Gram's A bands (rows i0.. of the B tile) stay
  // inside the tile
  p.npad = (int)((n + 127) / 128 * 128);
  p.mbands = (int)((n + AT_BM - 1) / AT_BM);
  p.a_bytes = p.same ? 0u : 2u * AT_BM * 64;
  p.b_bytes = 2u * (uint32_t)p.npad * 64;
  p.stage_bytes = (p.a_bytes + p.b_bytes + 1023) & ~1023u;
  const int rows = (p.same ? 0 : AT_BM) + p.npad;
  if (rows > 64 * AT_MAX_ROWS) return cudaErrorNotSupported;
  p.stages = AT_MAX_STAGES;
  while (p.stages > 2 && (size_t)p.stages * p.stage_bytes + 2048 > 227 * 1024) --p.stages;
  if ((size_t)p.stages * p.stage_bytes + 2048 > 227 * 1024) return cudaErrorNotSupported;
  uint32_t cols = 32;
  while (cols < (uint32_t)p.npad) cols <<= 1;
  p.tmem_cols = cols;
  p.ws = ws;
  p.status = status;
  int dev = 0, sms = 0;
  cudaError_t e;
  if ((e = cudaGetDevice(&dev)) != cudaSuccess) return e;
  if ((e = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev)) != cudaSuccess)
    return e;
  // one wave of CTAs (one per SM): mbands x splits, splits bounded by the workspace
  int64_t splits = sms / p.mbands;
  if (splits < 1) splits = 1;
  const int64_t cap = (int64_t)(ws_elems / (size_t)(n * n));
  if (cap < 1) return cudaErrorInvalidValue;
  if (splits > cap) splits = cap;
  int64_t chunk = (P + splits - 1) / splits;
  chunk = (chunk + AT_BK - 1) / AT_BK * AT_BK;
  splits = (P + chunk - 1) / chunk;
  p.chunk = chunk;
  const size_t smem = (size_t)p.stages * p.stage_bytes + 2048;
  if ((e = cudaFuncSetAttribute(atb_tc_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                (int)smem)) != cudaSuccess)
    return e;
  atb_tc_kernel<<<(unsigned)(splits * p.mbands), AT_THREADS, smem, st>>>(p);
  if ((e = cudaGetLastError()) != cudaSuccess) return e;
  atb_tc_reduce_kernel<float><<<(unsigned)((n * n + 255) / 256), 256, 0, st>>>(ws, n, splits,
                                                                               alpha, C);
  return cudaGetLastError();
}

}  // namespace tsvdm
