// Mode-3 TTM on the 5th-generation tensor cores (tcgen05 + TMEM), fed by TMA.
//
// Y (P x J) = scale * X (P x n) B (n x J) [+ beta Z], the last-mode TTM as one GEMM
// (Sec. 3.1), B(t, i) = M(i, t) (forward) or M(t, i) (transposed).  One CTA owns a tile
// of 128 rows of X and ALL J <= 512 outputs (the accumulator lives in TMEM, 128 lanes x
// up to 512 FP32 columns), so X is read from HBM exactly once.
//
// Precision modes (FP32 accumulation in TMEM in both):
//   BF16x3  x = x_hi + x_lo with x_hi = bf16(x), x_lo = bf16(x - x_hi) (same split for B);
//           D += A_hi B_hi + A_hi B_lo + A_lo B_hi  (three kind::f16 MMAs per k-step)
//   TF32    D += A B with both operands rounded to TF32 (one kind::tf32 MMA per k-step)
//
// Persistent: one CTA per SM (a kernel that holds tensor memory runs one CTA per SM)
// loops over row tiles; the stage ring runs across tiles.  Warp roles (512 threads):
//   warp 0       TMA producer: the pre-converted K-major B tiles (swizzled) of each stage;
//   warp 1       TMEM allocation; one thread issues the MMAs and commits them (a tile's
//                first MMA waits until the epilogue has read the previous accumulator);
//   warps 4..11  converters (two threads per row, 16 t each): FP32 X, loaded from global
//                memory straight into registers two k-steps ahead (a warp's 32 rows are
//                128 contiguous bytes for each t), -> K-major swizzled operand tiles, so a
//                stage holds only the operands (three stages fit where the raw X tile left
//                room for two);
//   warps 12..15 epilogue (tcgen05.ld of its own TMEM lane -> scale -> a shared-memory
//                staging buffer of 32 columns -> one TMA bulk tensor store per 128 x 32
//                box, two buffers alternating; per-element stores when a beta Z term is
//                added), which overlaps the next tile's loads and conversions.  (Scalar
//                stores of 384 columns per row took longer than the tile's MMAs, and a
//                tile's MMAs wait for the epilogue to have read the single accumulator.)
// Every mbarrier wait is bounded; on expiry the kernel records ST_TIMEOUT in the status
// word, every role leaves its loop and TMEM is released.  Nothing traps.
#include <cuda.h>
#include <string.h>
#include <cuda_bf16.h>
#include <cudaTypedefs.h>

#include "common.cuh"
#include "tc.cuh"

namespace tsvdm {
namespace {

constexpr int TBM = 128;
constexpr int TBK = 32;
constexpr int MAX_STAGES = 6;
constexpr uint32_t EPI_COLS = 32;                 // columns per epilogue TMA store
constexpr uint32_t EPI_BUF = TBM * EPI_COLS * 4;  // one staging buffer (16 KB)
constexpr int TC_THREADS = 512;   // warps 0 TMA, 1 MMA + TMEM, 4-11 converters, 12-15 epilogue
constexpr unsigned SPIN_LIMIT = 1u << 26;

struct TcParams {
  int64_t P, n, J;
  int npad;          // J rounded up to 16 (J <= 256) or to 128 (J <= 512)
  int nsub;          // output columns of one CTA (npad); blockIdx.x picks the column group
  int box_rows;      // rows of one B tensor-map box (divides nsub, <= 256)
  int stages;        // pipeline depth (2..MAX_STAGES)
  int kt_count;      // ceil(n / TBK)
  int tma_store;     // 1: the epilogue writes Y through shared memory with TMA stores
  int prec;          // TSVDM_P_BF16X3 or TSVDM_P_TF32
  const float *X;
  float *Y;
  const float *Z;
  const double *scale_ptr, *beta_ptr;
  double *sumsq;
  int *status;
  uint32_t tmem_cols;
};

using tc::mbar_arrive;
using tc::mbar_expect_tx;
using tc::mbar_init;
using tc::mma_commit;
using tc::mma_f16;
using tc::mma_tf32;
using tc::smem_desc;
using tc::smem_u32;

__device__ __forceinline__ bool mbar_wait(uint64_t *bar, uint32_t par) {
  return tc::mbar_wait(bar, par, SPIN_LIMIT);
}
// M = 128 (one CTA's row tile), N = n
__device__ __forceinline__ uint32_t instr_desc(uint32_t fmt, uint32_t n) {
  return tc::instr_desc(fmt, TBM, n);
}

__device__ __forceinline__ void tma_load_2d(void *dst, const CUtensorMap *map, uint64_t *bar,
                                            int x, int y) {
  asm volatile(
      "cp.async.bulk.tensor.2d.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1, "
      "{%3, %4}], [%2];" ::"r"(smem_u32(dst)),
      "l"((uint64_t)map), "r"(smem_u32(bar)), "r"(x), "r"(y)
      : "memory");
}

// Shared memory of one CTA.  Offsets are multiples of 1024 bytes (swizzle atoms).
struct TcLayout {
  uint32_t raw, a, b, stage, total;
  uint32_t a_bytes, b_bytes;
};

__host__ __device__ inline TcLayout tc_layout(int npad, int prec, int stages) {
  TcLayout L;
  const uint32_t a = (prec == TSVDM_P_BF16X3) ? 2u * TBM * 64 : TBM * 128u;   // 16 KB
  const uint32_t b = (prec == TSVDM_P_BF16X3) ? 2u * npad * 64 : npad * 128u;
  L.a_bytes = a;
  L.b_bytes = b;
  L.raw = 0;
  L.a = 0;
  L.b = a;
  uint32_t st = a + b;
  st = (st + 1023) & ~1023u;
  L.stage = st;
  L.total = stages * st + 1024 + 2 * EPI_BUF;              // + barriers, epilogue buffers
  return L;
}

__global__ void __launch_bounds__(TC_THREADS, 1)
    ttm_tc_kernel(const __grid_constant__ CUtensorMap mapB, const __grid_constant__ CUtensorMap mapY,
                  TcParams p) {
  extern __shared__ __align__(1024) unsigned char smem_raw[];
  // align the dynamic shared memory base to 1024 bytes
  unsigned char *smem = (unsigned char *)(((uintptr_t)smem_raw + 1023) & ~(uintptr_t)1023);
  const int STAGES = p.stages;
  const TcLayout L = tc_layout(p.nsub, p.prec, STAGES);
  uint64_t *full = (uint64_t *)(smem + STAGES * L.stage);
  uint64_t *conv = full + MAX_STAGES;
  uint64_t *empty = conv + MAX_STAGES;
  uint64_t *tfull = empty + MAX_STAGES;        // a tile's accumulator is complete
  uint64_t *tempty = tfull + 1;                // the epilogue has read it (TMEM free)
  uint32_t *tmem_slot = (uint32_t *)(tempty + 1);
  float *ebuf = (float *)(smem + STAGES * L.stage + 1024);     // 2 x [32 cols][128 rows]
  __shared__ int s_fail;

  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
  const int n_base = blockIdx.y * p.nsub;      // first output column of this CTA
  const bool bf = p.prec == TSVDM_P_BF16X3;
  const int nk = p.kt_count;
  const int ntiles = (int)((p.P + TBM - 1) / TBM);

  if (tid == 0) {
    s_fail = 0;
    for (int s = 0; s < STAGES; ++s) {
      mbar_init(&full[s], 1);
      mbar_init(&conv[s], 256);
      mbar_init(&empty[s], 1);
    }
    mbar_init(tfull, 1);
    mbar_init(tempty, 128);
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  }
  if (warp == 1) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(
                     smem_u32(tmem_slot)),
                 "r"(p.tmem_cols)
                 : "memory");
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
  }
  asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
  __syncthreads();
  asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
  const uint32_t tmem = *tmem_slot;
  // bounded wait; after the first expiry every role stops waiting and leaves its loop
  auto wait = [&](uint64_t *bar, uint32_t par) -> bool {
    if (*(volatile int *)&s_fail) return false;
    if (!mbar_wait(bar, par)) {
      s_fail = 1;
      return false;
    }
    return true;
  };

  // Persistent: CTA b takes row tiles b, b + gridDim.x, ...; the stage ring runs across
  // tiles (iteration it = tiles before x nk + kt), so the TMA and the converters fill the
  // next tile's stages while the epilogue warps drain the accumulator of the last one.
  if (warp == 0 && lane == 0) {
    // ---------------- TMA producer: pre-split K-major B tiles
    const uint32_t bytes = L.b_bytes;
    const int ops = bf ? 2 : 1;
    const uint32_t row_bytes = bf ? 64 : 128;
    int it = 0;
    bool ok = true;
    for (int tile = blockIdx.x; tile < ntiles && ok; tile += gridDim.x) {
      for (int kt = 0; kt < nk; ++kt, ++it) {
        const int s = it % STAGES, u = it / STAGES;
        if (u > 0 && !wait(&empty[s], (u - 1) & 1)) { ok = false; break; }
        unsigned char *st = smem + s * L.stage;
        mbar_expect_tx(&full[s], bytes);
        for (int o = 0; o < ops; ++o)
          for (int r0 = 0; r0 < p.nsub; r0 += p.box_rows)
            tma_load_2d(st + L.b + (uint32_t)o * p.nsub * row_bytes + (uint32_t)r0 * row_bytes,
                        &mapB, &full[s], kt * TBK, o * p.npad + n_base + r0);
      }
    }
  } else if (warp == 1 && lane == 0) {
    // ---------------- MMA issuer
    const uint32_t fmt = bf ? 1u : 2u;
    const uint32_t sbo = bf ? 512u : 1024u;
    const uint32_t lay = bf ? 4u : 2u;
    const uint32_t row_bytes = bf ? 64u : 128u;
    const int ksub = bf ? TBK / 16 : TBK / 8;
    int it = 0, j = 0;
    bool ok = true;
    for (int tile = blockIdx.x; tile < ntiles && ok; tile += gridDim.x, ++j) {
      if (j > 0 && !wait(tempty, (j - 1) & 1)) break;      // accumulator drained
      asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
      for (int kt = 0; kt < nk; ++kt, ++it) {
        const int s = it % STAGES, u = it / STAGES;
        if (!wait(&conv[s], u & 1)) { ok = false; break; }
        asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
        unsigned char *st = smem + s * L.stage;
        for (int kk = 0; kk < ksub; ++kk) {
          const uint32_t koff = kk * 32;                    // 32 bytes per k-step
          for (int n0 = 0; n0 < p.nsub; n0 += 256) {
            const uint32_t nn = (p.nsub - n0) < 256 ? (uint32_t)(p.nsub - n0) : 256u;
            const uint32_t idesc = instr_desc(fmt, nn);
            const uint32_t d = tmem + (uint32_t)n0;
            const uint32_t acc = (kt > 0 || kk > 0) ? 1u : 0u;
            if (bf) {
              uint64_t ahi = smem_desc(st + L.a + koff, sbo, lay);
              uint64_t alo = smem_desc(st + L.a + TBM * 64 + koff, sbo, lay);
              uint64_t bhi = smem_desc(st + L.b + n0 * row_bytes + koff, sbo, lay);
              uint64_t blo = smem_desc(st + L.b + (uint32_t)p.nsub * row_bytes + n0 * row_bytes + koff,
                                       sbo, lay);
              mma_f16(d, ahi, bhi, idesc, acc);
              mma_f16(d, ahi, blo, idesc, 1u);
              mma_f16(d, alo, bhi, idesc, 1u);
            } else {
              uint64_t a = smem_desc(st + L.a + koff, sbo, lay);
              uint64_t b = smem_desc(st + L.b + n0 * row_bytes + koff, sbo, lay);
              mma_tf32(d, a, b, idesc, acc);
            }
          }
        }
        mma_commit(&empty[s]);
      }
      if (ok) mma_commit(tfull);
    }
  } else if (warp >= 4 && warp < 12) {
    // ---------------- converters (two threads per row, 16 t each): FP32 X -> K-major
    // swizzled operands
    const int row = (tid - 128) & 127, kh = (tid - 128) >> 7;
    double ss = 0.0;
    const bool do_ss = p.sumsq != nullptr;
    constexpr int KH = TBK / 2;
    // X(grow, t) for this thread's row and its 16 t of k-step kt (zero past P or n)
    auto load_x = [&](int tile, int kt, float (&x)[KH]) {
      const int64_t grow = (int64_t)tile * TBM + row;
      const bool rin = tile < ntiles && grow < p.P;
#pragma unroll
      for (int k = 0; k < KH; ++k) {
        const int64_t t = (int64_t)kt * TBK + kh * KH + k;
        x[k] = (rin && t < p.n) ? __ldg(p.X + grow + p.P * t) : 0.f;
      }
    };
    // the k-steps of this CTA in order: (tile, kt), tiles blockIdx.x, + gridDim.x, ...
    auto advance = [&](int &tile, int &kt) {
      if (++kt == nk) {
        kt = 0;
        tile += gridDim.x;
      }
    };
    float x[KH], xn1[KH], xn2[KH];
    int t1 = blockIdx.x, k1 = 0;
    load_x(t1, k1, x);
    advance(t1, k1);
    load_x(t1, k1, xn1);
    advance(t1, k1);
    int it = 0;
    bool ok = true;
    for (int tile = blockIdx.x; tile < ntiles && ok; tile += gridDim.x) {
      for (int kt = 0; kt < nk; ++kt, ++it) {
        const int s = it % STAGES, u = it / STAGES;
        load_x(t1, k1, xn2);                       // two k-steps ahead
        advance(t1, k1);
        if (!wait(&full[s], u & 1)) { ok = false; break; }
        unsigned char *st = smem + s * L.stage;
        if (do_ss) {
#pragma unroll
          for (int k = 0; k < KH; ++k) ss += (double)x[k] * (double)x[k];
        }
        if (bf) {
          unsigned char *ahi = st + L.a, *alo = st + L.a + TBM * 64;
#pragma unroll
          for (int cc = 0; cc < 2; ++cc) {
            const int c = kh * 2 + cc;
            uint32_t h[4], l[4];
#pragma unroll
            for (int q = 0; q < 4; ++q) {
              float x0 = x[cc * 8 + 2 * q], x1 = x[cc * 8 + 2 * q + 1];
              __nv_bfloat16 h0 = __float2bfloat16_rn(x0), h1 = __float2bfloat16_rn(x1);
              __nv_bfloat16 l0 = __float2bfloat16_rn(x0 - __bfloat162float(h0));
              __nv_bfloat16 l1 = __float2bfloat16_rn(x1 - __bfloat162float(h1));
              h[q] = (uint32_t)__bfloat16_as_ushort(h0) | ((uint32_t)__bfloat16_as_ushort(h1) << 16);
              l[q] = (uint32_t)__bfloat16_as_ushort(l0) | ((uint32_t)__bfloat16_as_ushort(l1) << 16);
            }
            const uint32_t off = (uint32_t)row * 64 + (((uint32_t)c ^ (((uint32_t)row >> 1) & 3)) << 4);
            *(uint4 *)(ahi + off) = make_uint4(h[0], h[1], h[2], h[3]);
            *(uint4 *)(alo + off) = make_uint4(l[0], l[1], l[2], l[3]);
          }
        } else {
          unsigned char *a = st + L.a;
#pragma unroll
          for (int cc = 0; cc < 4; ++cc) {
            const int c = kh * 4 + cc;
            uint32_t v[4];
#pragma unroll
            for (int q = 0; q < 4; ++q)
              asm("cvt.rna.tf32.f32 %0, %1;" : "=r"(v[q]) : "f"(x[cc * 4 + q]));
            const uint32_t off = (uint32_t)row * 128 + (((uint32_t)c ^ ((uint32_t)row & 7)) << 4);
            *(uint4 *)(a + off) = make_uint4(v[0], v[1], v[2], v[3]);
          }
        }
        asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
        mbar_arrive(&conv[s]);
#pragma unroll
        for (int k = 0; k < KH; ++k) {
          x[k] = xn1[k];
          xn1[k] = xn2[k];
        }
      }
    }
    if (do_ss) {
#pragma unroll
      for (int o = 16; o > 0; o >>= 1) ss += __shfl_xor_sync(0xffffffffu, ss, o);
      if (lane == 0) atomicAdd(p.sumsq, ss);
    }
  } else if (warp >= 12) {
    // ---------------- epilogue (thread = TMEM lane = row): scale, optional beta Z, store
    const int row = tid - 384;
    int echunk = 0;                      // staging chunks so far (over all tiles)
    const uint32_t lane_base = (uint32_t)(32 * (warp - 12)) << 16;
    const float scale = p.scale_ptr ? (float)(*p.scale_ptr) : 1.f;
    const float beta = p.beta_ptr ? (float)(*p.beta_ptr) : 0.f;
    int j = 0;
    for (int tile = blockIdx.x; tile < ntiles; tile += gridDim.x, ++j) {
      if (!wait(tfull, j & 1)) break;
      asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
      const int64_t grow = (int64_t)tile * TBM + row;
      if (p.tma_store) {
        // 32 columns at a time: TMEM -> staging buffer (column-major [32][128], conflict
        // free) -> one TMA store of the 128 x 32 box; two buffers alternate, and a buffer
        // is rewritten only after the store issued from it two chunks before has read it
        for (int c = 0; c * (int)EPI_COLS < p.nsub; ++c, ++echunk) {
          float *buf = ebuf + (echunk & 1) * (EPI_BUF / 4);
          if (row == 0 && echunk >= 2)
            asm volatile("cp.async.bulk.wait_group.read 1;" ::: "memory");
          asm volatile("bar.sync 1, 128;" ::: "memory");
          uint32_t v[32];
          asm volatile(
              "tcgen05.ld.sync.aligned.32x32b.x16.b32 {%0, %1, %2, %3, %4, %5, %6, %7, %8, %9, "
              "%10, %11, %12, %13, %14, %15}, [%16];"
              : "=r"(v[0]), "=r"(v[1]), "=r"(v[2]), "=r"(v[3]), "=r"(v[4]), "=r"(v[5]), "=r"(v[6]),
                "=r"(v[7]), "=r"(v[8]), "=r"(v[9]), "=r"(v[10]), "=r"(v[11]), "=r"(v[12]),
                "=r"(v[13]), "=r"(v[14]), "=r"(v[15])
              : "r"(tmem + lane_base + (uint32_t)(c * EPI_COLS)));
          asm volatile(
              "tcgen05.ld.sync.aligned.32x32b.x16.b32 {%0, %1, %2, %3, %4, %5, %6, %7, %8, %9, "
              "%10, %11, %12, %13, %14, %15}, [%16];"
              : "=r"(v[16]), "=r"(v[17]), "=r"(v[18]), "=r"(v[19]), "=r"(v[20]), "=r"(v[21]),
                "=r"(v[22]), "=r"(v[23]), "=r"(v[24]), "=r"(v[25]), "=r"(v[26]), "=r"(v[27]),
                "=r"(v[28]), "=r"(v[29]), "=r"(v[30]), "=r"(v[31])
              : "r"(tmem + lane_base + (uint32_t)(c * EPI_COLS + 16)));
          asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
#pragma unroll
          for (int e = 0; e < 32; ++e) buf[e * TBM + row] = scale * __uint_as_float(v[e]);
          asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
          asm volatile("bar.sync 1, 128;" ::: "memory");
          if (row == 0) {
            asm volatile(
                "cp.async.bulk.tensor.2d.global.shared::cta.bulk_group [%0, {%1, %2}], [%3];" ::"l"(
                    (uint64_t)&mapY),
                "r"((int)(tile * TBM)), "r"((int)(n_base + c * EPI_COLS)), "r"(smem_u32(buf))
                : "memory");
            asm volatile("cp.async.bulk.commit_group;" ::: "memory");
          }
        }
      } else {
      // 64 columns per TMEM round trip: four loads, one wait
      for (int j0 = 0; j0 < p.nsub; j0 += 64) {
        uint32_t v[64];
        const int nq = (p.nsub - j0) >= 64 ? 4 : (p.nsub - j0) / 16;
#pragma unroll
        for (int q = 0; q < 4; ++q) {
          if (q < nq)
            asm volatile(
                "tcgen05.ld.sync.aligned.32x32b.x16.b32 {%0, %1, %2, %3, %4, %5, %6, %7, %8, %9, "
                "%10, %11, %12, %13, %14, %15}, [%16];"
                : "=r"(v[16 * q + 0]), "=r"(v[16 * q + 1]), "=r"(v[16 * q + 2]), "=r"(v[16 * q + 3]),
                  "=r"(v[16 * q + 4]), "=r"(v[16 * q + 5]), "=r"(v[16 * q + 6]), "=r"(v[16 * q + 7]),
                  "=r"(v[16 * q + 8]), "=r"(v[16 * q + 9]), "=r"(v[16 * q + 10]), "=r"(v[16 * q + 11]),
                  "=r"(v[16 * q + 12]), "=r"(v[16 * q + 13]), "=r"(v[16 * q + 14]), "=r"(v[16 * q + 15])
                : "r"(tmem + lane_base + (uint32_t)(j0 + 16 * q)));
        }
        asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
        if (grow < p.P) {
#pragma unroll
          for (int e = 0; e < 64; ++e) {
            const int64_t col = n_base + j0 + e;
            if (e < 16 * nq && col < p.J) {
              float y = scale * __uint_as_float(v[e]);
              if (p.Z) y = fmaf(beta, p.Z[grow + p.P * col], y);
              p.Y[grow + p.P * col] = y;
            }
          }
        }
      }
      }
      asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
      mbar_arrive(tempty);
    }
  }
  // the thread that issued the epilogue's TMA stores waits for them before the CTA ends
  if (warp >= 12 && tid == 384 && p.tma_store)
    asm volatile("cp.async.bulk.wait_group 0;" ::: "memory");
  asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
  __syncthreads();
  if (warp == 1) {
    asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
    asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem),
                 "r"(p.tmem_cols)
                 : "memory");
  }
  if (tid == 0 && s_fail) atomicOr(p.status, ST_TIMEOUT);
}

// Bk: operand B of the TTM in K-major layout, [ops][npad][kpad] (K contiguous), zero
// padded.  BF16x3: ops = 2 (hi, lo) bf16; TF32: ops = 1, FP32 rounded to TF32.
__global__ void prep_b_kernel(const float *__restrict__ M, int64_t n, int64_t J, bool transB,
                              int npad, int kpad, int prec, void *Bk) {
  const int64_t idx = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (idx >= (int64_t)npad * kpad) return;
  const int64_t i = idx / kpad, t = idx % kpad;     // output column i, contraction index t
  float b = 0.f;
  if (i < J && t < n) b = transB ? M[t + n * i] : M[i + J * t];
  if (prec == TSVDM_P_BF16X3) {
    __nv_bfloat16 h = __float2bfloat16_rn(b);
    __nv_bfloat16 l = __float2bfloat16_rn(b - __bfloat162float(h));
    __nv_bfloat16 *o = (__nv_bfloat16 *)Bk;
    o[i * kpad + t] = h;
    o[(int64_t)npad * kpad + i * kpad + t] = l;
  } else {
    uint32_t v;
    asm("cvt.rna.tf32.f32 %0, %1;" : "=r"(v) : "f"(b));
    ((uint32_t *)Bk)[i * kpad + t] = v;
  }
}

PFN_cuTensorMapEncodeTiled_v12000 get_encode() {
  static PFN_cuTensorMapEncodeTiled_v12000 fn = nullptr;
  if (!fn) {
    cudaDriverEntryPointQueryResult q;
    void *f = nullptr;
    if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &f, 12000, cudaEnableDefault,
                                         &q) == cudaSuccess &&
        q == cudaDriverEntryPointSuccess)
      fn = (PFN_cuTensorMapEncodeTiled_v12000)f;
  }
  return fn;
}

}  // namespace

static int tc_npad(int64_t J) { return J <= 256 ? (int)((J + 15) / 16 * 16) : (int)((J + 127) / 128 * 128); }

size_t ttm_tc_workspace(int64_t n, int64_t J) {
  int64_t npad = tc_npad(J), kpad = (n + TBK - 1) / TBK * TBK;
  return (size_t)2 * npad * kpad * 2 + 4096;           // bf16 hi+lo (tf32 needs the same)
}

bool ttm_tc_supported(int64_t P, int64_t n, int64_t J, const void *X, const void *Y) {
  if (J < 1 || J > 512 || n < 1 || P < 1) return false;
  if ((P % 4) != 0) return false;                      // 16-byte row stride of the X view
  if (((uintptr_t)X & 15) != 0 || ((uintptr_t)Y & 3) != 0) return false;
  if (P > (int64_t)0x7fffffff) return false;
  return get_encode() != nullptr;
}

cudaError_t ttm_tc(const float *X, int64_t P, int64_t n, const float *M, int64_t J, bool transB,
                   int prec, float *Y, void *ws, size_t ws_bytes, double *sumsq,
                   const double *scale_ptr, const double *beta_ptr, const float *Z, int *status,
                   cudaStream_t st) {
  if (!ttm_tc_supported(P, n, J, X, Y)) return cudaErrorNotSupported;
  if (prec != TSVDM_P_BF16X3 && prec != TSVDM_P_TF32) return cudaErrorInvalidValue;
  const int npad = tc_npad(J);
  const int kpad = (int)((n + TBK - 1) / TBK * TBK);
  // One CTA owns all J outputs of its row tile (measured faster than splitting J over two
  // CTAs, which re-converts X and halves the MMA work per stage).
  const int nsplit = 1;
  const int nsub = npad;
  const int box_rows = npad <= 256 ? npad : 128;
  if (ws_bytes < ttm_tc_workspace(n, J)) return cudaErrorInvalidValue;
  void *Bk = (void *)(((uintptr_t)ws + 255) & ~(uintptr_t)255);
  {
    int64_t cnt = (int64_t)npad * kpad;
    prep_b_kernel<<<(unsigned)((cnt + 255) / 256), 256, 0, st>>>(M, n, J, transB, npad, kpad, prec,
                                                                  Bk);
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return e;
  }
  auto enc = get_encode();
  CUtensorMap mapB, mapY;
  // the epilogue stores Y (P x J, column-major) with TMA when Y is 16-byte aligned and no
  // beta Z term is added (the backward's dX keeps the per-element stores)
  const bool tma_store = Z == nullptr && ((uintptr_t)Y & 15) == 0;
  memset(&mapY, 0, sizeof(mapY));
  if (tma_store) {
    cuuint64_t dims[2] = {(cuuint64_t)P, (cuuint64_t)J};
    cuuint64_t strides[1] = {(cuuint64_t)P * 4};
    cuuint32_t box[2] = {TBM, EPI_COLS};
    cuuint32_t es[2] = {1, 1};
    if (enc(&mapY, CU_TENSOR_MAP_DATA_TYPE_FLOAT32, 2, (void *)Y, dims, strides, box, es,
            CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_NONE,
            CU_TENSOR_MAP_L2_PROMOTION_NONE, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE) != CUDA_SUCCESS)
      return cudaErrorInvalidValue;
  }
  {
    const bool bf = prec == TSVDM_P_BF16X3;
    const int ops = bf ? 2 : 1;
    cuuint64_t dims[2] = {(cuuint64_t)kpad, (cuuint64_t)npad * ops};
    cuuint64_t strides[1] = {(cuuint64_t)kpad * (bf ? 2 : 4)};
    cuuint32_t box[2] = {TBK, (cuuint32_t)box_rows};
    cuuint32_t es[2] = {1, 1};
    if (enc(&mapB, bf ? CU_TENSOR_MAP_DATA_TYPE_BFLOAT16 : CU_TENSOR_MAP_DATA_TYPE_FLOAT32, 2, Bk,
            dims, strides, box, es, CU_TENSOR_MAP_INTERLEAVE_NONE,
            bf ? CU_TENSOR_MAP_SWIZZLE_64B : CU_TENSOR_MAP_SWIZZLE_128B,
            CU_TENSOR_MAP_L2_PROMOTION_L2_256B, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE) != CUDA_SUCCESS)
      return cudaErrorInvalidValue;
  }
  TcParams p;
  p.P = P;
  p.n = n;
  p.J = J;
  p.npad = npad;
  p.nsub = nsub;
  p.box_rows = box_rows;
  p.kt_count = kpad / TBK;
  p.prec = prec;
  p.tma_store = tma_store ? 1 : 0;
  p.X = X;
  p.Y = Y;
  p.Z = Z;
  p.scale_ptr = scale_ptr;
  p.beta_ptr = beta_ptr;
  p.sumsq = sumsq;
  p.status = status;
  uint32_t cols = 32;
  while (cols < (uint32_t)nsub) cols <<= 1;
  p.tmem_cols = cols;
  // the deepest pipeline that fits (one CTA per SM)
  int stages = MAX_STAGES;
  while (stages > 2 && tc_layout(nsub, prec, stages).total + 1024 > 227 * 1024) --stages;
  p.stages = stages;
  const TcLayout L = tc_layout(nsub, prec, stages);
  const size_t smem = L.total + 1024;
  cudaError_t e = cudaFuncSetAttribute(ttm_tc_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                       (int)smem);
  if (e != cudaSuccess) return e;
  // persistent: one CTA per SM (a kernel holding tensor memory runs one CTA per SM)
  int dev = 0, sms = 0;
  if ((e = cudaGetDevice(&dev)) != cudaSuccess) return e;
  if ((e = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev)) != cudaSuccess)
    return e;
  const int64_t ntiles = (P + TBM - 1) / TBM;
  const dim3 grid((unsigned)(ntiles < sms ? ntiles : sms), (unsigned)nsplit);
  ttm_tc_kernel<<<grid, TC_THREADS, smem, st>>>(mapB, mapY, p);
  return cudaGetLastError();
}

}  // namespace tsvdm

