// Batched one-sided Jacobi SVD of the frontal slices (the per-slice svd of Algorithm 1,
// Sec. 3.2), laid out for GB300.
//
// Method: block one-sided (Hestenes) Jacobi.  A slice W (rows x cols, rows >= cols,
// column-major, in place) is cut into column blocks of width B = W2/2.  One sweep runs
// the round-robin tournament over the blocks (nb-1 rounds of nb/2 disjoint block
// pairs).  For a block pair (I, J):
//   1. G = [W_I W_J]^T [W_I W_J]   (W2 x W2 Gram, FP32 (or FP64) FMA, rows streamed
//      through shared memory in chunks);
//   2. if some |g_ij| > tol sqrt(g_ii g_jj): one cyclic sweep of two-sided Jacobi on G
//      (round-robin over all W2 (W2-1)/2 pairs; rotation angle, convergence test, G and
//      the accumulated rotation Q in the storage precision);
//   3. [W_I W_J] <- [W_I W_J] Q and [V_I V_J] <- [V_I V_J] Q.
// A column pair is rotated exactly as in the scalar method: zeta = (b - a) / (2 g),
// t = sign(zeta) / (|zeta| + sqrt(1 + zeta^2)), c = 1/sqrt(1+t^2), s = c t,
// w_i' = c w_i - s w_j, w_j' = s w_i + c w_j.  A slice has converged after a sweep in
// which no block pair needed a rotation (the scalar stopping rule, applied to Grams
// formed fresh from the current columns).
//
// GB300 mapping: a thread-block cluster of CL CTAs owns one slice at a time (CTAs of a
// cluster are co-scheduled, so the per-round barrier.cluster is safe); CTA r takes block
// pairs r, r+CL, ... of each round.  The slice and its V stay in global memory, which is
// L2-resident because only (clusters in flight) slices are live at once; global loads
// bypass L1 (ld.global.cg) because other CTAs of the cluster rewrite the columns
// between rounds.  Clusters are persistent and pull slice indices from an atomic
// counter.  Every loop is bounded (sweep cap), and no device code traps.
#include <cooperative_groups.h>
#include <cuda_bf16.h>

#include "common.cuh"
#include "tc.cuh"

namespace cg = cooperative_groups;

namespace tsvdm {
namespace {

constexpr int NT = 256;

template <typename T> struct Vec16;
template <> struct Vec16<float> { using type = float4; static constexpr int N = 4; };
template <> struct Vec16<double> { using type = double2; static constexpr int N = 2; };

template <typename T, int W2, int NS_ = 3>
struct Cfg {
  static constexpr int B = W2 / 2;                    // block width
  static constexpr int RC = 4096 / W2;                // rows per pipelined chunk
  static constexpr int NS = NS_;                      // pipeline stages
  static constexpr int VN = Vec16<T>::N;
  static constexpr int LDR = RC + VN;                 // chunk column stride (elements)
  static constexpr int TD = W2 / 4;                   // Gram tiles per dimension
  static constexpr int TILES = TD * TD;
  static constexpr int KG = NT / TILES;               // Gram K-groups
  static constexpr int CPW = W2 / 8;                  // apply: columns per warp
  static constexpr int RPT = RC / 32;                 // apply: rows per thread
  static constexpr int CHUNK = W2 * LDR;
  static constexpr int GPART = KG * W2 * W2;
  static constexpr int BUF = NS * CHUNK > GPART ? NS * CHUNK : GPART;
  static_assert(NT % TILES == 0, "tiles must divide the block");
  static_assert(RC % (KG * VN) == 0, "K-groups must tile the chunk");
  static_assert(RC % 32 == 0, "apply rows");
};

__device__ __forceinline__ void rr_pair(int n, int round, int q, int &a, int &b) {
  // circle method: players 0..n-1 (n even), rounds 0..n-2, pairs q = 0..n/2-1
  if (q == 0) {
    a = n - 1;
    b = round;
  } else {
    a = (round + q) % (n - 1);
    b = (round - q + (n - 1)) % (n - 1);
  }
  if (a > b) {
    int t = a;
    a = b;
    b = t;
  }
}

template <typename T>
__device__ __forceinline__ T ldcg(const T *p) { return __ldcg(p); }

// Packed upper triangle of a symmetric W2 x W2 matrix: entry (i, j), i <= j.
template <int W2>
__device__ __forceinline__ int tri(int i, int j) {
  const int lo = min(i, j), hi = max(i, j);
  // row lo starts at lo W2 - lo (lo - 1) / 2; lo (2 W2 - 1 - lo) is even
  return hi + (int)(((unsigned)lo * (unsigned)(2 * W2 - 1 - lo)) >> 1);
}

// The 2 x 2 block of G on rows (pair p) x columns (pair q) after J_p^T B J_q, written
// with explicit FMAs so that every caller computes bit-identical values.
template <typename T>
__device__ __forceinline__ void rot_block(T b00, T b01, T b10, T b11, T c1, T s1, T c2, T s2,
                                          T &o00, T &o01, T &o10, T &o11) {
  const T r00 = fma(c1, b00, -(s1 * b10)), r01 = fma(c1, b01, -(s1 * b11));
  const T r10 = fma(s1, b00, c1 * b10), r11 = fma(s1, b01, c1 * b11);
  o00 = fma(c2, r00, -(s2 * r01));
  o01 = fma(s2, r00, c2 * r01);
  o10 = fma(c2, r10, -(s2 * r11));
  o11 = fma(s2, r10, c2 * r11);
}

constexpr int MAXSORT = 1024;        // slices with more columns keep the natural order
constexpr int XLD = 33;              // row stride of the cross-sweep Gram quadrants

template <typename T, int W2, int NS>
struct Smem {
  static constexpr bool QCOL = false;    // Q row-major
  T buf[Cfg<T, W2, NS>::BUF];            // streamed chunk / Gram partials
  T G[2][W2 * (W2 + 1) / 2];         // Gram, packed upper triangle, double-buffered
  __align__(16) T Q[W2 * W2];        // accumulated rotation, Q(r, j) at Q[r*W2 + j]
  T cs[2][W2];                       // c, s per pair, slot = step parity
  T dd[2][W2];                       // updated diagonal per pair
  int pi[2][W2 / 2], pj[2][W2 / 2];
  int rot[2][W2 / 2];
  int pos[2][W2];                    // 2 * pair + role of every column in the step
  int gcur;                          // buffer of G holding the current Gram
  int col[W2];                       // global column of local column c (-1 = padding)
  int any_rot;                       // this block pair rotated
  int step_rot;                      // the last inner sweep rotated
  int sweep_any;                     // this CTA rotated in this sweep
  int nonfinite;
  long long nrot;
  int slice[2];
  int vote[2];
  int ord[MAXSORT];                  // column order of the current sweep
};

// Barrier of the threads that work on one block pair: the whole CTA (FMA kernel), or one
// 256-thread group of the tensor-core kernel (named barrier 1 + group).
struct CtaBar {
  __device__ __forceinline__ void sync() const { __syncthreads(); }
  __device__ __forceinline__ int sync_or(int v) const { return __syncthreads_or(v); }
};
struct GroupBar {
  int id;
  __device__ __forceinline__ void sync() const {
    asm volatile("bar.sync %0, %1;" ::"r"(id), "n"(NT) : "memory");
  }
  __device__ __forceinline__ int sync_or(int v) const {
    int r;
    asm volatile(
        "{\n .reg .pred p, q;\n setp.ne.s32 p, %1, 0;\n bar.red.or.pred q, %2, %3, p;\n"
        " selp.s32 %0, 1, 0, q;\n}\n"
        : "=r"(r)
        : "r"(v), "r"(id), "n"(NT)
        : "memory");
    return r;
  }
};

// Shared memory of the tensor-core variant (FP32 slices, block pairs of 64 columns).  The
// member names match Smem, so the inner Gram sweep is shared.  3 CTAs fit on an SM.
struct SmemTc {
  static constexpr int W2 = 64;
  static constexpr bool QCOL = true;       // Q column-major
  // operand tiles (Gram: two 16 KB [128 x 32] TF32 tiles; apply: the hi and lo
  // [128 x 32] tiles of one K-block), then the Gram epilogue scratch and the sort keys
  __align__(1024) unsigned char op[32768];
  union {
    struct {
      union {
        // full inner sweeps (the first round of a sweep): Gram, packed upper triangle,
        // double-buffered
        float G[2][W2 * (W2 + 1) / 2];
        // cross inner sweeps: the Gram's quadrants I x I, I x J and J x J (I = local
        // columns 0..31, J = 32..63), row stride XLD, updated in place
        float X3[3][32 * XLD];
      };
      __align__(16) float Q[W2 * W2];      // accumulated rotation, column-major: Q(r, j) at Q[j*W2 + r]
    };
    // the apply's B operand, (Q - I) split into TF32 hi (first 16 KB) and lo, each two
    // K-blocks of [64 output columns x 32 K] (G and Q are dead while it lives)
    __align__(1024) unsigned char bq[32768];
  };
  float cs[2][W2];
  float dd[2][W2];
  int pi[2][W2 / 2], pj[2][W2 / 2];
  int rot[2][W2 / 2];
  int pos[2][W2];
  int gcur;
  int col[W2];
  int any_rot;
  int step_rot;
  int sweep_any;
  int nonfinite;
  long long nrot;
  int slice[2];
  int vote[2];
  int ord[MAXSORT];
  uint64_t bar[3];                         // MMA completion: Gram tiles 0 and 1, apply
  uint32_t tmem;                           // TMEM base (64 FP32 columns x 128 lanes)
  int fail;                                // a bounded wait ran out
  int wk[4];                               // work item broadcast to the group
  int reopen;                              // this worker closed a sweep that continues
};

template <typename SM>
__device__ __forceinline__ float *sort_keys(SM &s) { return reinterpret_cast<float *>(s.buf); }
__device__ __forceinline__ float *sort_keys(SmemTc &s) { return reinterpret_cast<float *>(s.op); }

__device__ __forceinline__ void cp_async16(void *smem, const void *gmem, int src_bytes) {
  unsigned sa = (unsigned)__cvta_generic_to_shared(smem);
  asm volatile("cp.async.cg.shared.global [%0], [%1], 16, %2;\n" ::"r"(sa), "l"(gmem),
               "r"(src_bytes));
}
__device__ __forceinline__ void cp_async_commit() { asm volatile("cp.async.commit_group;\n" ::); }
template <int N>
__device__ __forceinline__ void cp_async_wait() { asm volatile("cp.async.wait_group %0;\n" ::"n"(N)); }

// Stage chunk `ck` (rows ck*RC .. +RC of the W2 columns col[]) into buffer `dst`.
// Aligned case (lda a multiple of the 16-byte vector): asynchronous 16-byte copies with
// zero fill past the last row and for padding columns.  Otherwise plain loads.
template <typename T, int W2, int NS>
__device__ __forceinline__ void stage_chunk(const int *col, const T *__restrict__ Wsl, int rows,
                                            int lda, bool aligned, int ck, T *dst) {
  using C = Cfg<T, W2, NS>;
  const int r0 = ck * C::RC;
  if (aligned) {
    constexpr int VPC = C::RC / C::VN;                // vectors per column
    for (int idx = threadIdx.x; idx < W2 * VPC; idx += NT) {
      int c = idx / VPC, v = idx % VPC;
      int gc = col[c];
      int r = r0 + v * C::VN;
      int valid = rows - r;
      valid = valid < 0 ? 0 : (valid > C::VN ? C::VN : valid);
      if (gc < 0) valid = 0;
      const T *src = Wsl + (valid > 0 ? (int64_t)gc * lda + r : 0);
      cp_async16(dst + c * C::LDR + v * C::VN, src, valid * (int)sizeof(T));
    }
  } else {
    for (int idx = threadIdx.x; idx < W2 * C::RC; idx += NT) {
      int c = idx / C::RC, r = idx % C::RC;
      int gc = col[c];
      T v = T(0);
      if (gc >= 0 && r0 + r < rows) v = ldcg(Wsl + (int64_t)gc * lda + r0 + r);
      dst[c * C::LDR + r] = v;
    }
  }
}

// Gram G = Wc^T Wc for the W2 columns of the block pair (columns col[]), rows streamed
// through an NS-stage cp.async pipeline (one barrier per chunk).
template <typename T, int W2, int NS>
__device__ void gram(Smem<T, W2, NS> &s, const T *__restrict__ Wsl, int rows, int lda) {
  using C = Cfg<T, W2, NS>;
  using V = typename Vec16<T>::type;
  const int tid = threadIdx.x;
  const int kg = tid / C::TILES;
  const int tile = tid % C::TILES;
  const int ti = tile / C::TD, tj = tile % C::TD;
  const bool aligned = (lda % C::VN) == 0 && ((uintptr_t)Wsl & 15) == 0;
  const int nck = (rows + C::RC - 1) / C::RC;
  T acc[4][4];
#pragma unroll
  for (int e = 0; e < 4; ++e)
#pragma unroll
    for (int f = 0; f < 4; ++f) acc[e][f] = T(0);
#pragma unroll
  for (int c = 0; c < C::NS - 1; ++c) {
    if (c < nck) stage_chunk<T, W2, NS>(s.col, Wsl, rows, lda, aligned, c, s.buf + (c % C::NS) * C::CHUNK);
    cp_async_commit();
  }
  for (int ck = 0; ck < nck; ++ck) {
    cp_async_wait<C::NS - 2>();
    __syncthreads();
    {
      int nx = ck + C::NS - 1;
      if (nx < nck) stage_chunk<T, W2, NS>(s.col, Wsl, rows, lda, aligned, nx, s.buf + (nx % C::NS) * C::CHUNK);
      cp_async_commit();
    }
    const T *ch = s.buf + (ck % C::NS) * C::CHUNK;
#pragma unroll 2
    for (int r = kg * C::VN; r < C::RC; r += C::KG * C::VN) {
      T a[4][C::VN], b[4][C::VN];
#pragma unroll
      for (int e = 0; e < 4; ++e) {
        V va = *reinterpret_cast<const V *>(ch + (ti + C::TD * e) * C::LDR + r);
        V vb = *reinterpret_cast<const V *>(ch + (tj + C::TD * e) * C::LDR + r);
        const T *pa = reinterpret_cast<const T *>(&va);
        const T *pb = reinterpret_cast<const T *>(&vb);
#pragma unroll
        for (int u = 0; u < C::VN; ++u) {
          a[e][u] = pa[u];
          b[e][u] = pb[u];
        }
      }
#pragma unroll
      for (int u = 0; u < C::VN; ++u)
#pragma unroll
        for (int e = 0; e < 4; ++e)
#pragma unroll
          for (int f = 0; f < 4; ++f) acc[e][f] = fma(a[e][u], b[f][u], acc[e][f]);
    }
  }
  cp_async_wait<0>();
  __syncthreads();
  // reduce the K-groups in a fixed order
  T *gp = s.buf;
#pragma unroll
  for (int e = 0; e < 4; ++e)
#pragma unroll
    for (int f = 0; f < 4; ++f)
      gp[(kg * W2 + (ti + C::TD * e)) * W2 + (tj + C::TD * f)] = acc[e][f];
  __syncthreads();
  for (int idx = tid; idx < W2 * W2; idx += NT) {
    int i = idx / W2, j = idx % W2;
    if (i > j) continue;
    T sum = T(0);
    for (int g = 0; g < C::KG; ++g) sum += gp[(g * W2 + i) * W2 + j];
    s.G[0][tri<W2>(i, j)] = sum;
  }
  if (tid == 0) s.gcur = 0;
  __syncthreads();
}

// Pair k of step `step` of one inner sweep.  full: the round-robin over all W2 columns
// (W2-1 steps); cross: only pairs (i in block I, j in block J), B steps of B pairs.
template <int W2>
__device__ __forceinline__ void inner_pair(bool full, int step, int k, int &i, int &j) {
  if (full) {
    rr_pair(W2, step, k, i, j);
  } else {
    i = k;
    j = W2 / 2 + (k + step) % (W2 / 2);
  }
}

// Convergence test |g| > tol sqrt(a b)  <=>  g^2 > tol^2 a b (a, b >= 0), decided in FP64.
// decide64 puts single-precision products in front of the FP64 comparison: they carry
// relative errors below 1e-6, so outside a 2% band around the threshold they give the FP64
// answer, and the FP64 products run only inside the band (or when a single-precision
// product over- or underflows).  The decision is always the FP64 one.  The FP64 test is a
// call, so that it stays a branch taken by the few lanes in the band: predicated FP64
// instructions still occupy the FP64 pipe, whose rate is a small fraction of the FP32 rate
// on this GPU.
__device__ __noinline__ bool exceeds(double a, double b, double g, double tol2) {
  return isfinite(a) && isfinite(b) && g * g > tol2 * (a * b);
}
template <typename T>
__device__ __forceinline__ bool decide64(T a, T b, T g, double tol2) {
  const float af = (float)a, bf = (float)b, gf = (float)g;
  const float lhs = gf * gf, rhs = (float)tol2 * (af * bf);
  if (lhs < 1e30f && rhs < 1e30f && rhs > 1e-30f) {
    if (lhs < 0.98f * rhs) return false;
    if (lhs > 1.02f * rhs) return true;
  }
  return exceeds((double)a, (double)b, (double)g, tol2);
}

// Single-precision form of the test (the opt-in FP32 angle mode of FP32 slices; the
// threshold tol ~ 4 sqrt(m) 2^-24 is itself a rounding-level quantity, so deciding it in
// FP32 moves it by ~1e-7 relative): g^2 > tol^2 a b while the products stay in the normal
// range, else the overflow-free |g| > tol sqrt(a) sqrt(b).
__device__ __forceinline__ bool rot_test_f32(float a, float b, float g, float tol, float tol2) {
  const float lhs = g * g, rhs = tol2 * (a * b);
  if (lhs < 1e30f && rhs < 1e30f && rhs > 1e-30f) return lhs > rhs;
  return fabsf(g) > tol * (sqrtf(fmaxf(a, 0.f)) * sqrtf(fmaxf(b, 0.f)));
}

// a32: FP32 slices decide in FP32 (opt-in); otherwise, and always for FP64 slices, in FP64.
template <typename T>
__device__ __forceinline__ bool rot_test(T a, T b, T g, double tol, double tol2, bool a32) {
  if constexpr (sizeof(T) == 4) {
    if (a32) return rot_test_f32(a, b, g, (float)tol, (float)tol2);
  }
  return decide64(a, b, g, tol2);
}

// Rotation of a pair in FP64 from its Gram entries a = g_ii, b = g_jj, g = g_ij:
//   zeta = (b - a) / (2 g);  t = sign(zeta) / (|zeta| + sqrt(1 + zeta^2))
//     = sign(zeta) |2g| / (|b - a| + sqrt((b - a)^2 + 4 g^2))   (|t| <= 1),
// c = 1 / sqrt(1 + t^2), s = c t, and the rotated diagonal a - t g, b + t g.
__device__ __forceinline__ void angle64(double a, double b, double g, double &c, double &sn,
                                        double &da, double &db) {
  const double h = b - a, g2 = 2.0 * g;
  double t = fabs(g2) / (fabs(h) + sqrt(fma(h, h, g2 * g2)));
  if ((h >= 0.0) != (g2 >= 0.0)) t = -t;
  c = rsqrt(fma(t, t, 1.0));
  sn = c * t;
  da = fma(-t, g, a);
  db = fma(t, g, b);
}

// The FP64 rotation angle of an FP32 slice's pair, with few FP64 operations (the FP64 rate
// of the GPU is a small fraction of its FP32 rate).  The angle t = tan(theta) solves
// f(t) = g (t^2 - 1) + h t = 0 (t^2 + 2 zeta t - 1 = 0 times g; h = b - a), whose derivative
// f'(t) = 2 g t + h has magnitude sqrt(h^2 + 4 g^2) at the root: from the FP32 estimate t0
// (absolute error d, |t| <= 1) one Newton step leaves about d^2 / 2 plus the rounding of
// f(t0).  f(t0) is the cancelling part and is evaluated in FP64 from the FP32 inputs (nine
// FP64-pipe instructions, conversions included); the step f(t0) / f'(t0) is small against
// t0 (|d| ~ 1e-7 |t|), so it is formed in FP32 from f(t0) rounded to FP32 and t = t0 - step
// is the one FP32 rounding of the refined angle.  The rotation then takes that angle in the
// slice's precision: c = 1 / sqrt(1 + t^2), s = c t and the rotated diagonal a - t g, b + t g
// (the values the FP32 rotation is applied with).
__device__ __forceinline__ void angle64_f32(float a, float b, float g, float &c, float &sn,
                                            float &da, float &db) {
  const float hf = b - a, g2f = 2.f * g;
  float t0 = fabsf(g2f) / (fabsf(hf) + hypotf(hf, g2f));
  if ((hf >= 0.f) != (g2f >= 0.f)) t0 = -t0;
  const double G = g, T = t0, H = (double)b - (double)a;
  const float f = (float)fma(G, fma(T, T, -1.0), H * T);       // f(t0) in FP64, then rounded
  const float rf = __frcp_rn(fmaf(g2f, t0, hf));   // 1 / f'(t0); |f'| >= 2 |g| > 0 (infinite
                                                    // only for denormal pairs)
  const float t = isfinite(rf) ? t0 - f * rf : t0;
  // correctly rounded 1/sqrt: an approximate reciprocal square root biased c (and the
  // column norms, over thousands of rotations) by ~1e-5
  c = __frsqrt_rn(fmaf(t, t, 1.f));
  sn = c * t;
  da = fmaf(-t, g, a);
  db = fmaf(t, g, b);
}

// The same rotation in FP32 (the opt-in FP32 angle mode).  c is the correctly rounded
// 1/sqrt: an approximate reciprocal square root biased c (and the column norms, over
// thousands of rotations) by ~1e-5.
__device__ __forceinline__ void angle32(float a, float b, float g, float &c, float &sn,
                                        float &da, float &db) {
  const float h = b - a, g2 = 2.f * g;
  float t = fabsf(g2) / (fabsf(h) + hypotf(h, g2));
  if ((h >= 0.f) != (g2 >= 0.f)) t = -t;
  c = __frsqrt_rn(fmaf(t, t, 1.f));
  sn = c * t;
  da = fmaf(-t, g, a);
  db = fmaf(t, g, b);
}

// Rotation of one pair from its current Gram entries (a = g_ii, b = g_jj, g = g_ij),
// stored in slot `sl` as pair k.  The test and the angle run in FP64 (from the FP32 Gram
// entries of an FP32 slice, whose rotation then takes the angle rounded to FP32), or in
// FP32 when a32 is set for an FP32 slice.
template <typename T, int W2, int NS, typename SM>
__device__ __forceinline__ void pair_angle(SM &s, int sl, int k, int i, int j, T a, T b, T g,
                                           double tol, double tol2, bool a32) {
  s.pi[sl][k] = i;
  s.pj[sl][k] = j;
  s.pos[sl][i] = 2 * k;
  s.pos[sl][j] = 2 * k + 1;
  int rot = 0;
  if (!(isfinite(a) && isfinite(b))) {
    s.nonfinite = 1;
  } else if (rot_test(a, b, g, tol, tol2, a32)) {
    bool done = false;
    if constexpr (sizeof(T) == 4) {
      if (a32) {
        float c, sn, da, db;
        angle32(a, b, g, c, sn, da, db);
        s.cs[sl][2 * k] = c;
        s.cs[sl][2 * k + 1] = sn;
        s.dd[sl][2 * k] = da;
        s.dd[sl][2 * k + 1] = db;
        done = true;
      }
    }
    if (!done) {
      if constexpr (sizeof(T) == 4) {
        float c, sn, da, db;
        angle64_f32(a, b, g, c, sn, da, db);
        s.cs[sl][2 * k] = c;
        s.cs[sl][2 * k + 1] = sn;
        s.dd[sl][2 * k] = da;
        s.dd[sl][2 * k + 1] = db;
      } else {
        double c, sn, da, db;
        angle64(a, b, g, c, sn, da, db);
        s.cs[sl][2 * k] = (T)c;
        s.cs[sl][2 * k + 1] = (T)sn;
        s.dd[sl][2 * k] = (T)da;
        s.dd[sl][2 * k + 1] = (T)db;
      }
    }
    rot = 1;
    s.any_rot = 1;
    s.step_rot = 1;
    atomicAdd((unsigned long long *)&s.nrot, 1ull);
  }
  if (!rot) {
    s.cs[sl][2 * k] = T(1);
    s.cs[sl][2 * k + 1] = T(0);
  }
  s.rot[sl][k] = rot;
}

// One cyclic two-sided Jacobi sweep on G (all pairs when `full`, else only pairs across
// the two blocks), accumulating the rotations in Q.  Sets s.any_rot and s.step_rot.
//
// One barrier per step: while warps 0..6 apply step s to the Gram (read from one buffer,
// written to the other) and to Q, the last warp already computes the angles of step s+1
// from the Gram before step s and the rotations of step s, with the same 2 x 2
// arithmetic the update warps use, so both see bit-identical entries.
template <typename T, int W2, int NS, typename SM, typename Bar>
__device__ void inner_sweep(SM &s, double tol, bool full, bool first, int tid, const Bar &bar,
                            bool a32) {
  constexpr int NP = W2 / 2;
  constexpr int AW = NT / 32 - 1;          // the angle warp
  constexpr int NU = NT - 32;              // update threads
  const double tol2 = tol * tol;
  const int g0 = s.gcur;
  // fresh-Gram convergence test |g| > tol sqrt(a b) (the same test pair_angle applies)
  int need = 0;
  for (int idx = tid; idx < W2 * W2; idx += NT) {
    int i = idx / W2, j = idx % W2;
    if (i < j && (full || (i < NP && j >= NP))) {
      const T a = s.G[g0][tri<W2>(i, i)], b = s.G[g0][tri<W2>(j, j)], g = s.G[g0][tri<W2>(i, j)];
      if (rot_test(a, b, g, tol, tol2, a32)) need = 1;
    }
  }
  bar.sync();                        // every thread has read step_rot of the previous call
  if (tid == 0) {
    s.step_rot = 0;
    if (first) s.any_rot = 0;
  }
  if (!bar.sync_or(need)) return;
  if (first) {
    for (int idx = tid; idx < W2 * W2; idx += NT) s.Q[idx] = (idx / W2 == idx % W2) ? T(1) : T(0);
  }
  const int nsteps = full ? W2 - 1 : NP;
  const int warp = tid >> 5, lane = tid & 31;
  // the 2 x 2 blocks (pp <= qq) of pair slots this update thread owns in every step:
  // block blk = tid + t NU, rows of the packed upper triangle of an NP x NP grid
  constexpr int NB = NP * (NP + 1) / 2;
  constexpr int BPT = (NB + NU - 1) / NU;
  int bpp[BPT], bqq[BPT];
#pragma unroll
  for (int t = 0; t < BPT; ++t) {
    const int blk = tid + t * NU;
    bpp[t] = -1;
    bqq[t] = 0;
    if (warp != AW && blk < NB) {
      int pp = 0, start = 0;
      while (start + (NP - pp) <= blk) {
        start += NP - pp;
        ++pp;
      }
      bpp[t] = pp;
      bqq[t] = pp + (blk - start);
    }
  }
  if (warp == AW && lane < NP) {     // angles of step 0 from the fresh Gram
    int i, j;
    inner_pair<W2>(full, 0, lane, i, j);
    pair_angle<T, W2, NS>(s, 0, lane, i, j, s.G[g0][tri<W2>(i, i)], s.G[g0][tri<W2>(j, j)],
                          s.G[g0][tri<W2>(i, j)], tol, tol2, a32);
  }
  bar.sync();
  for (int step = 0; step < nsteps; ++step) {
    const int sl = step & 1;
    const T *Gs = s.G[g0 ^ (step & 1)];
    T *Gd = s.G[g0 ^ ((step + 1) & 1)];
    if (warp == AW) {
      if (lane < NP && step + 1 < nsteps) {
        int i, j;
        inner_pair<W2>(full, step + 1, lane, i, j);
        const int pi_ = s.pos[sl][i], pj_ = s.pos[sl][j];
        const int p = pi_ >> 1, q = pj_ >> 1, ri = pi_ & 1, rj = pj_ & 1;
        T a = s.rot[sl][p] ? s.dd[sl][pi_] : Gs[tri<W2>(i, i)];
        T b = s.rot[sl][q] ? s.dd[sl][pj_] : Gs[tri<W2>(j, j)];
        T g;
        if (p == q) {
          g = s.rot[sl][p] ? T(0) : Gs[tri<W2>(i, j)];
        } else {
          // the block the update warps form: rows of the lower pair index, columns of the
          // higher one, so the entry is bit-identical to the one they store
          const int pl = p < q ? p : q, ph = p < q ? q : p;
          const int rl = p < q ? ri : rj, rh = p < q ? rj : ri;
          const int i1 = s.pi[sl][pl], j1 = s.pj[sl][pl], i2 = s.pi[sl][ph], j2 = s.pj[sl][ph];
          T o[4];
          rot_block(Gs[tri<W2>(i1, i2)], Gs[tri<W2>(i1, j2)], Gs[tri<W2>(j1, i2)],
                    Gs[tri<W2>(j1, j2)], s.cs[sl][2 * pl], s.cs[sl][2 * pl + 1], s.cs[sl][2 * ph],
                    s.cs[sl][2 * ph + 1], o[0], o[1], o[2], o[3]);
          g = o[2 * rl + rh];
        }
        pair_angle<T, W2, NS>(s, sl ^ 1, lane, i, j, a, b, g, tol, tol2, a32);
      }
    } else {
      // G_{s+1} = J^T G_s J on the blocks pp <= qq (the rest is their transpose)
#pragma unroll
      for (int t = 0; t < BPT; ++t) {
        const int pp = bpp[t], qq = bqq[t];
        if (pp < 0) continue;
        const int i1 = s.pi[sl][pp], j1 = s.pj[sl][pp];
        if (pp == qq) {
          if (s.rot[sl][pp]) {
            Gd[tri<W2>(i1, i1)] = s.dd[sl][2 * pp];
            Gd[tri<W2>(j1, j1)] = s.dd[sl][2 * pp + 1];
            Gd[tri<W2>(i1, j1)] = T(0);
          } else {
            Gd[tri<W2>(i1, i1)] = Gs[tri<W2>(i1, i1)];
            Gd[tri<W2>(j1, j1)] = Gs[tri<W2>(j1, j1)];
            Gd[tri<W2>(i1, j1)] = Gs[tri<W2>(i1, j1)];
          }
          continue;
        }
        const int i2 = s.pi[sl][qq], j2 = s.pj[sl][qq];
        T o00, o01, o10, o11;
        rot_block(Gs[tri<W2>(i1, i2)], Gs[tri<W2>(i1, j2)], Gs[tri<W2>(j1, i2)],
                  Gs[tri<W2>(j1, j2)], s.cs[sl][2 * pp], s.cs[sl][2 * pp + 1],
                  s.cs[sl][2 * qq], s.cs[sl][2 * qq + 1], o00, o01, o10, o11);
        Gd[tri<W2>(i1, i2)] = o00;
        Gd[tri<W2>(i1, j2)] = o01;
        Gd[tri<W2>(j1, i2)] = o10;
        Gd[tri<W2>(j1, j2)] = o11;
      }
      if constexpr (SM::QCOL) {
        // Q <- Q J on a column-major Q: item (pair k, rows 4 r4 .. 4 r4 + 3), one 16-byte
        // load and store per column; a warp's items cover two pairs' full columns
        constexpr int R4 = W2 / 4;
        for (int it = tid; it < NP * R4; it += NU) {
          const int k = it / R4, r4 = it % R4;
          if (!s.rot[sl][k]) continue;
          const T c = s.cs[sl][2 * k], sn = s.cs[sl][2 * k + 1];
          float4 *qi = reinterpret_cast<float4 *>(&s.Q[s.pi[sl][k] * W2]) + r4;
          float4 *qj = reinterpret_cast<float4 *>(&s.Q[s.pj[sl][k] * W2]) + r4;
          const float4 x = *qi, y = *qj;
          *qi = make_float4(c * x.x - sn * y.x, c * x.y - sn * y.y, c * x.z - sn * y.z,
                            c * x.w - sn * y.w);
          *qj = make_float4(sn * x.x + c * y.x, sn * x.y + c * y.y, sn * x.z + c * y.z,
                            sn * x.w + c * y.w);
        }
      } else {
        // Q <- Q J: lane -> pair k = lane mod NP and a row offset; a warp covers 32 / NP
        // rows at a time (distinct columns of a row across the pairs)
        constexpr int RPW = 32 / NP;
        const int k = lane % NP;
        if (s.rot[sl][k]) {
          const int i = s.pi[sl][k], j = s.pj[sl][k];
          const T c = s.cs[sl][2 * k], sn = s.cs[sl][2 * k + 1];
          for (int r = warp * RPW + lane / NP; r < W2; r += (NU / 32) * RPW) {
            const T x = s.Q[r * W2 + i], y = s.Q[r * W2 + j];
            s.Q[r * W2 + i] = c * x - sn * y;
            s.Q[r * W2 + j] = sn * x + c * y;
          }
        }
      }
    }
    bar.sync();
  }
  if (tid == 0) s.gcur = g0 ^ (nsteps & 1);
  bar.sync();
}

// [Wsl(:, col)] <- [Wsl(:, col)] Q, rows streamed through the cp.async pipeline; results
// go straight from registers to global memory (each chunk's rows are read before they
// are overwritten, and no other CTA touches these columns during the round).
template <typename T, int W2, int NS>
__device__ void apply_q(Smem<T, W2, NS> &s, T *__restrict__ Wsl, int rows, int lda) {
  using C = Cfg<T, W2, NS>;
  const int tid = threadIdx.x;
  const int lane = tid & 31, warp = tid >> 5;
  const bool aligned = (lda % C::VN) == 0 && ((uintptr_t)Wsl & 15) == 0;
  const int nck = (rows + C::RC - 1) / C::RC;
  const int j0 = warp * C::CPW;
#pragma unroll
  for (int c = 0; c < C::NS - 1; ++c) {
    if (c < nck) stage_chunk<T, W2, NS>(s.col, Wsl, rows, lda, aligned, c, s.buf + (c % C::NS) * C::CHUNK);
    cp_async_commit();
  }
  for (int ck = 0; ck < nck; ++ck) {
    cp_async_wait<C::NS - 2>();
    __syncthreads();
    {
      int nx = ck + C::NS - 1;
      if (nx < nck) stage_chunk<T, W2, NS>(s.col, Wsl, rows, lda, aligned, nx, s.buf + (nx % C::NS) * C::CHUNK);
      cp_async_commit();
    }
    const T *ch = s.buf + (ck % C::NS) * C::CHUNK;
    T acc[C::RPT][C::CPW];
#pragma unroll
    for (int q = 0; q < C::RPT; ++q)
#pragma unroll
      for (int e = 0; e < C::CPW; ++e) acc[q][e] = T(0);
#pragma unroll 4
    for (int c = 0; c < W2; ++c) {
      T qv[C::CPW];                   // Q(c, j0 .. j0+CPW-1): contiguous, 16-byte loads
      if constexpr ((C::CPW * sizeof(T)) % 16 == 0) {
        using V = typename Vec16<T>::type;
#pragma unroll
        for (int e = 0; e < C::CPW; e += C::VN) {
          V v = *reinterpret_cast<const V *>(&s.Q[c * W2 + j0 + e]);
          const T *pv = reinterpret_cast<const T *>(&v);
#pragma unroll
          for (int u = 0; u < C::VN; ++u) qv[e + u] = pv[u];
        }
      } else {
#pragma unroll
        for (int e = 0; e < C::CPW; ++e) qv[e] = s.Q[c * W2 + j0 + e];
      }
#pragma unroll
      for (int q = 0; q < C::RPT; ++q) {
        T a = ch[c * C::LDR + lane + 32 * q];
#pragma unroll
        for (int e = 0; e < C::CPW; ++e) acc[q][e] = fma(a, qv[e], acc[q][e]);
      }
    }
    const int r0 = ck * C::RC;
#pragma unroll
    for (int e = 0; e < C::CPW; ++e) {
      int gc = s.col[j0 + e];
      if (gc < 0) continue;
#pragma unroll
      for (int q = 0; q < C::RPT; ++q) {
        int r = r0 + lane + 32 * q;
        if (r < rows) __stcg(Wsl + (int64_t)gc * lda + r, acc[q][e]);
      }
    }
  }
  cp_async_wait<0>();
  __syncthreads();
}

// ---------------------------------------------------------------- tensor-core products
// The Gram enters the tensor cores as x = h + l, h = tf32(x), l = tf32(x - h) (x - h is
// exact; |x - h - l| <= 2^-22 |x|): its rounding only steers the rotation angles and the
// stopping test (whose threshold is ~4 sqrt(m) 2^-24), never the columns themselves.

constexpr unsigned TC_SPIN = 1u << 22;

// Bounded wait for the next completion of barrier b (phase bits in `phase`, identical in
// every thread because every thread waits on every completion).  After one expiry the
// CTA stops waiting; the host sees ST_TIMEOUT.
__device__ __forceinline__ void tc_wait(SmemTc &s, int b, uint32_t &phase) {
  const uint32_t par = (phase >> b) & 1u;
  if (!*(volatile int *)&s.fail && !tc::mbar_wait(&s.bar[b], par, TC_SPIN)) s.fail = 1;
  phase ^= 1u << b;
}

// Eight consecutive rows r .. r+7 of one column (zeros past `rows` or for padding).
__device__ __forceinline__ void load8(const float *src, int r, int rows, bool vec, float (&v)[8]) {
  if (src != nullptr && vec && r + 8 <= rows) {
    const float4 a = __ldcg(reinterpret_cast<const float4 *>(src + r));
    const float4 b = __ldcg(reinterpret_cast<const float4 *>(src + r + 4));
    v[0] = a.x; v[1] = a.y; v[2] = a.z; v[3] = a.w;
    v[4] = b.x; v[5] = b.y; v[6] = b.z; v[7] = b.w;
  } else {
#pragma unroll
    for (int e = 0; e < 8; ++e) v[e] = (src != nullptr && r + e < rows) ? __ldcg(src + r + e) : 0.f;
  }
}

// 16-byte chunk `ch` (4 TF32 values) of row `row` of a K-major 128-byte-swizzled tile.
__device__ __forceinline__ void put_chunk(unsigned char *tile, uint32_t row, uint32_t ch,
                                          uint32_t a, uint32_t b, uint32_t c, uint32_t d) {
  *reinterpret_cast<uint4 *>(tile + row * 128 + ((ch ^ (row & 7)) << 4)) = make_uint4(a, b, c, d);
}

// G = W_c^T W_c of the 64 columns col[] on the tensor cores.  Rows stream in chunks of 32
// (K); a chunk's tile holds H (rows 0..63, one per column) over L (rows 64..127), so one
// MMA with A = the whole tile (M = 128) and B = its first 64 rows (N = 64) accumulates
// [H^T H ; L^T H] in TMEM.  Then G = H^T H + L^T H + (L^T H)^T, summed in that order.
// Two tiles alternate.  Each thread copies its own 8 rows of a column GRING - 1 chunks
// ahead (cp.async into a private slot of a ring in the G / Q area, dead until the
// epilogue), so it needs no barrier to read them back; unaligned columns load directly.
constexpr int GRING = 4;
__device__ void gram_tc(SmemTc &s, const float *__restrict__ Wsl, int rows, int lda,
                        uint32_t &phase, int tid, const GroupBar &bar, bool cross) {
  constexpr int W2 = SmemTc::W2;
  constexpr int GK = 32;
  static_assert(GRING * W2 * GK * sizeof(float) <= sizeof(SmemTc::bq), "Gram ring");
  const int c = tid >> 2, q = tid & 3;             // column, 8-row quarter of the chunk
  const bool vec = (lda & 3) == 0 && ((uintptr_t)Wsl & 15) == 0;
  const int gc = s.col[c];
  const float *src = gc >= 0 ? Wsl + (int64_t)gc * lda : nullptr;
  const int nck = (rows + GK - 1) / GK;
  const uint32_t idesc = tc::instr_desc(2, 128, W2);
  float *ring = reinterpret_cast<float *>(s.bq) + c * GK + q * 8;   // + slot * W2 * GK
  // one commit group per chunk (empty past the end), so wait_group counts chunks
  auto stage = [&](int ck) {
    if (vec && ck < nck) {
      const int r = ck * GK + q * 8;
      int valid = rows - r;
      valid = valid < 0 ? 0 : (valid > 8 ? 8 : valid);
      const float *g0 = src != nullptr && valid > 0 ? src + r : Wsl;
      const int b0 = src != nullptr ? (valid > 4 ? 4 : valid) * 4 : 0;
      const int b1 = src != nullptr ? (valid > 4 ? valid - 4 : 0) * 4 : 0;
      float *dst = ring + (ck % GRING) * (W2 * GK);
      cp_async16(dst, g0, b0);
      cp_async16(dst + 4, b1 > 0 ? g0 + 4 : g0, b1);
    }
    cp_async_commit();
  };
#pragma unroll
  for (int k = 0; k < GRING - 1; ++k) stage(k);
  float v[8];
  for (int ck = 0; ck < nck; ++ck) {
    const int b = ck & 1;
    stage(ck + GRING - 1);
    if (vec) {
      cp_async_wait<GRING - 1>();
      const float4 a0 = *reinterpret_cast<const float4 *>(ring + (ck % GRING) * (W2 * GK));
      const float4 a1 = *reinterpret_cast<const float4 *>(ring + (ck % GRING) * (W2 * GK) + 4);
      v[0] = a0.x; v[1] = a0.y; v[2] = a0.z; v[3] = a0.w;
      v[4] = a1.x; v[5] = a1.y; v[6] = a1.z; v[7] = a1.w;
    } else {
      load8(src, ck * GK + q * 8, rows, false, v);
    }
    if (ck >= 2) tc_wait(s, b, phase);             // the MMAs of chunk ck-2 read tile b
    unsigned char *tile = s.op + b * 16384;
    uint32_t h[8], l[8];
#pragma unroll
    for (int e = 0; e < 8; ++e) {
      h[e] = tc::tf32_rna(v[e]);
      l[e] = tc::tf32_rna(v[e] - __uint_as_float(h[e]));
    }
    put_chunk(tile, c, 2 * q, h[0], h[1], h[2], h[3]);
    put_chunk(tile, c, 2 * q + 1, h[4], h[5], h[6], h[7]);
    put_chunk(tile, 64 + c, 2 * q, l[0], l[1], l[2], l[3]);
    put_chunk(tile, 64 + c, 2 * q + 1, l[4], l[5], l[6], l[7]);
    tc::fence_proxy_async();
    bar.sync();
    if (tid == 0) {
      tc::fence_after_sync();
#pragma unroll
      for (int kk = 0; kk < GK / 8; ++kk) {
        const uint64_t d = tc::smem_desc(tile + kk * 32, 1024, 2);
        tc::mma_tf32(s.tmem, d, d, idesc, (ck > 0 || kk > 0) ? 1u : 0u);
      }
      tc::mma_commit(&s.bar[b]);
    }
  }
  cp_async_wait<0>();                              // the ring area becomes G below
  for (int ck = nck >= 2 ? nck - 2 : 0; ck < nck; ++ck) tc_wait(s, ck & 1, phase);
  tc::fence_after_sync();
  // epilogue: warps 2, 3 park L^T H (TMEM lanes 64..127) in the tile area, XOR-swizzled
  // S[i][j] at i*64 + (j ^ i) (conflict-free by rows and by columns); warps 0, 1 add it to
  // their H^T H rows
  float *S = reinterpret_cast<float *>(s.op);
  const int warp = tid >> 5, lane = tid & 31;
  if (warp == 2 || warp == 3) {
    const int i = (warp - 2) * 32 + lane;
#pragma unroll
    for (int j0 = 0; j0 < W2; j0 += 16) {
      float d[16];
      tc::tmem_ld16(s.tmem + ((uint32_t)(warp * 32) << 16) + j0, d);
#pragma unroll
      for (int e = 0; e < 16; ++e) S[i * 64 + ((j0 + e) ^ i)] = d[e];
    }
  }
  tc::fence_before_sync();
  bar.sync();
  if (cross) {
    // quadrants for the cross sweeps: warp 0 writes rows 0..31 of I x I and I x J, warp 1
    // rows 32..63 of J x J (both triangles of the diagonal quadrants)
    if (warp == 0) {
      float *A = s.X3[0], *B = s.X3[1];
#pragma unroll
      for (int j0 = 0; j0 < W2; j0 += 16) {
        float d[16];
        tc::tmem_ld16(s.tmem + j0, d);
#pragma unroll
        for (int e = 0; e < 16; ++e) {
          const int j = j0 + e;
          const float g = (d[e] + S[lane * 64 + (j ^ lane)]) + S[j * 64 + (lane ^ j)];
          if (j < 32)
            A[lane * XLD + j] = g;
          else
            B[lane * XLD + (j - 32)] = g;
        }
      }
    } else if (warp == 1) {
      float *C = s.X3[2];
      const int i = 32 + lane;
#pragma unroll
      for (int j0 = 32; j0 < W2; j0 += 16) {
        float d[16];
        tc::tmem_ld16(s.tmem + ((uint32_t)32 << 16) + j0, d);
#pragma unroll
        for (int e = 0; e < 16; ++e) {
          const int j = j0 + e;
          C[lane * XLD + (j - 32)] = (d[e] + S[i * 64 + (j ^ i)]) + S[j * 64 + (i ^ j)];
        }
      }
    }
  } else if (warp < 2) {
    const int i = warp * 32 + lane;
#pragma unroll
    for (int j0 = 0; j0 < W2; j0 += 16) {
      float d[16];
      tc::tmem_ld16(s.tmem + ((uint32_t)(warp * 32) << 16) + j0, d);
#pragma unroll
      for (int e = 0; e < 16; ++e) {
        const int j = j0 + e;
        if (j >= i) s.G[0][tri<W2>(i, j)] = (d[e] + S[i * 64 + (j ^ i)]) + S[j * 64 + (i ^ j)];
      }
    }
  }
  if (tid == 0) s.gcur = 0;
  tc::fence_before_sync();
  bar.sync();
}

// The rotation apply needs FP32 accuracy (its rounding accumulates in the columns over the
// sweeps), so it splits every value into three BF16 terms x = x1 + x2 + x3 (each the
// rounding of what the previous ones leave; |x - x1 - x2 - x3| <= 2^-27 |x|) and forms the
// six products whose order is at least 2^-24: x1 y1, x1 y2, x2 y1, x1 y3, x3 y1, x2 y2.
using tc::pack2;
using tc::split3;
using tc::sw64;

constexpr uint32_t AP_TERM = 8192;    // one term of the apply's A tile: [128 rows x 32 K] BF16
constexpr uint32_t BQ_TERM = 8192;    // one term of (Q - I): 2 K-blocks x [64 x 32] BF16
constexpr uint32_t BQ_KB = 4096;

// B operand of the apply from the accumulated rotation: (Q - I)(c, c') split into three
// BF16 terms, K-major (row c', K = c), two K-blocks of 32.  Overwrites G and Q.
__device__ void build_bq(SmemTc &s, int tid, const GroupBar &bar) {
  constexpr int W2 = SmemTc::W2;
  float qv[W2 * W2 / NT];
#pragma unroll
  for (int m = 0; m < W2 * W2 / NT; ++m) {
    const int idx = tid + NT * m, cp = idx >> 6, c = idx & 63;
    qv[m] = s.Q[cp * W2 + c] - (c == cp ? 1.f : 0.f);
  }
  bar.sync();
#pragma unroll
  for (int m = 0; m < W2 * W2 / NT; ++m) {
    const int idx = tid + NT * m, cp = idx >> 6, c = idx & 63;
    __nv_bfloat16 t[3];
    split3(qv[m], t[0], t[1], t[2]);
    const uint32_t kb = (uint32_t)c >> 5, k = (uint32_t)c & 31;
    const uint32_t off = kb * BQ_KB + sw64((uint32_t)cp, k >> 3) + (k & 7) * 2;
#pragma unroll
    for (int u = 0; u < 3; ++u)
      *reinterpret_cast<__nv_bfloat16 *>(s.bq + u * BQ_TERM + off) = t[u];
  }
  tc::fence_proxy_async();
  bar.sync();
}

// W(:, col) <- W(:, col) + W(:, col) (Q - I) on the tensor cores, 128 rows at a time.
// Thread t owns row r = t mod 128 of the chunk and, in each K-block kb, the 16 columns
// kb*32 + (t/128)*16 ..: it loads them, writes their three BF16 terms into the A tiles and,
// after the MMAs, reads the same 16 columns of its TMEM lane and stores x + D.  Adding the
// correction W (Q - I) in FP32 keeps the accumulator's rounding away from the columns'
// norms (Q -> I as the sweeps converge).
__device__ void apply_tc(SmemTc &s, float *__restrict__ W, int rows, int lda, uint32_t &phase,
                         int tid, const GroupBar &bar) {
  constexpr int W2 = SmemTc::W2;
  // (A term, B term) of the six products
  constexpr int PA[6] = {0, 0, 1, 0, 2, 1}, PB[6] = {0, 1, 0, 2, 0, 1};
  const int warp = tid >> 5;
  const int r = tid & 127, hh = tid >> 7;
  const uint32_t idesc = tc::instr_desc(1, 128, W2);
  const uint32_t lane_base = (uint32_t)((warp & 3) * 32) << 16;
  const int nck = (rows + 127) / 128;
  for (int ck = 0; ck < nck; ++ck) {
    const int row = ck * 128 + r;
    const bool rin = row < rows;
    float x[32];
#pragma unroll
    for (int kb = 0; kb < 2; ++kb)
#pragma unroll
      for (int e = 0; e < 16; ++e) {
        const int gc = s.col[kb * 32 + hh * 16 + e];
        x[kb * 16 + e] = (rin && gc >= 0) ? __ldcg(W + (int64_t)gc * lda + row) : 0.f;
      }
#pragma unroll
    for (int kb = 0; kb < 2; ++kb) {
      if (kb == 1) tc_wait(s, 2, phase);           // the K-block 0 MMAs read the tiles
#pragma unroll
      for (int h8 = 0; h8 < 2; ++h8) {              // 8 columns = one 16-byte chunk per term
        uint32_t w[3][4];
#pragma unroll
        for (int e = 0; e < 8; e += 2) {
          __nv_bfloat16 a0, a1, a2, b0, b1, b2;
          split3(x[kb * 16 + h8 * 8 + e], a0, a1, a2);
          split3(x[kb * 16 + h8 * 8 + e + 1], b0, b1, b2);
          w[0][e / 2] = pack2(a0, b0);
          w[1][e / 2] = pack2(a1, b1);
          w[2][e / 2] = pack2(a2, b2);
        }
        const uint32_t off = sw64((uint32_t)r, (uint32_t)(hh * 2 + h8));
#pragma unroll
        for (int u = 0; u < 3; ++u)
          *reinterpret_cast<uint4 *>(s.op + u * AP_TERM + off) =
              make_uint4(w[u][0], w[u][1], w[u][2], w[u][3]);
      }
      tc::fence_proxy_async();
      tc::fence_before_sync();
      bar.sync();
      if (tid == 0) {
        tc::fence_after_sync();
#pragma unroll
        for (int kk = 0; kk < 2; ++kk) {
#pragma unroll
          for (int m = 0; m < 6; ++m) {
            const uint64_t a = tc::smem_desc(s.op + PA[m] * AP_TERM + kk * 32, 512, 4);
            const uint64_t b =
                tc::smem_desc(s.bq + PB[m] * BQ_TERM + kb * BQ_KB + kk * 32, 512, 4);
            tc::mma_f16(s.tmem, a, b, idesc, (kb > 0 || kk > 0 || m > 0) ? 1u : 0u);
          }
        }
        tc::mma_commit(&s.bar[2]);
      }
    }
    tc_wait(s, 2, phase);                          // D complete, tiles free
    tc::fence_after_sync();
#pragma unroll
    for (int kb = 0; kb < 2; ++kb) {
      float d[16];
      tc::tmem_ld16(s.tmem + lane_base + (uint32_t)(kb * 32 + hh * 16), d);
#pragma unroll
      for (int e = 0; e < 16; ++e) {
        const int gc = s.col[kb * 32 + hh * 16 + e];
        if (rin && gc >= 0) __stcg(W + (int64_t)gc * lda + row, x[kb * 16 + e] + d[e]);
      }
    }
    tc::fence_before_sync();
    bar.sync();                                    // TMEM read before the next chunk's MMAs
  }
}

// Rotation of pair k from its Gram entries a = g_ii, b = g_jj, g = g_ij (FP32 slices): the
// test and angle of pair_angle (FP64, or FP32 when a32), stored in slot `sl` (c, s;
// rotated diagonal; flag).
__device__ __forceinline__ void cross_angle(SmemTc &s, int sl, int k, float a, float b, float g,
                                            float tol, float tol2, double tol2d, bool a32) {
  int rot = 0;
  float c = 1.f, sn = 0.f;
  if (!(isfinite(a) && isfinite(b))) {
    s.nonfinite = 1;
  } else if (a32 ? rot_test_f32(a, b, g, tol, tol2) : decide64(a, b, g, tol2d)) {
    float da, db;
    if (a32)
      angle32(a, b, g, c, sn, da, db);
    else
      angle64_f32(a, b, g, c, sn, da, db);
    s.dd[sl][2 * k] = da;
    s.dd[sl][2 * k + 1] = db;
    rot = 1;
    s.any_rot = 1;
    s.step_rot = 1;
    atomicAdd((unsigned long long *)&s.nrot, 1ull);
  }
  s.cs[sl][2 * k] = c;
  s.cs[sl][2 * k + 1] = sn;
  s.rot[sl][k] = rot;
}

// Block (p, q), p <= q, of the c-th non-hand-over block of the 32 x 32 pair grid in row
// order (the hand-over blocks (k, k + 1) and (0, 31) removed): row 0 holds 30 of them,
// row p in 1..30 holds 31 - p, row 31 one.
__device__ __forceinline__ void cross_block(int c, int &p, int &q) {
  p = 0;
  int cnt = 30;
  while (c >= cnt) {
    c -= cnt;
    ++p;
    cnt = p <= 30 ? 31 - p : 1;
  }
  if (p == 0)
    q = c == 0 ? 0 : c + 1;
  else if (p <= 30)
    q = c == 0 ? p : p + 1 + c;
  else
    q = 31;
}

// Q <- Q J of a cross step on the column-major Q, item `it` = (pair k, rows 4 r4 .. 4 r4 +
// 3): columns k and 32 + (k + step) mod 32, one 16-byte load and store per column.
__device__ __forceinline__ void cross_q_item(SmemTc &s, const float2 *cs2, int it, int step) {
  constexpr int W2 = SmemTc::W2, R4 = W2 / 4;
  const int k = it / R4, r4 = it % R4;
  const float2 ck = cs2[k];
  if (ck.y == 0.f) return;
  const float c = ck.x, sn = ck.y;
  float4 *qi = reinterpret_cast<float4 *>(&s.Q[k * W2]) + r4;
  float4 *qj = reinterpret_cast<float4 *>(&s.Q[(W2 / 2 + ((k + step) & 31)) * W2]) + r4;
  const float4 x = *qi, y = *qj;
  *qi = make_float4(c * x.x - sn * y.x, c * x.y - sn * y.y, c * x.z - sn * y.z,
                    c * x.w - sn * y.w);
  *qj = make_float4(sn * x.x + c * y.x, sn * x.y + c * y.y, sn * x.z + c * y.z,
                    sn * x.w + c * y.w);
}

// One cross inner sweep of the tensor-core worker: every pair of a local column i < 32 with
// a local column 32 + j, in 32 steps (step t pairs column k with column 32 + (k + t) mod 32),
// on the quadrant storage X3 (A = I x I, B = I x J, C = J x J), accumulating the rotations
// in Q.  Sets s.any_rot and s.step_rot.
//
// Thread-owned 2 x 2 blocks, updated in place.  In step t, block (p, q) (p <= q) holds
//   A(p, q), B(p, (q + t) mod 32), B(q, (p + t) mod 32), C((p + t) mod 32, (q + t) mod 32),
// the rows and columns of pairs p and q; no two blocks share an entry, so a block is read
// and rewritten by its owner alone, and blocks of two non-rotating pairs are skipped.  The
// next step's pair k joins column k with the J column of pair k + 1, so its cross entry is
// in block (k, k + 1) (block (0, 31) for k = 31).  Lane k of the last warp owns that block:
// it rotates it and forms pair k's next rotation from the entry it has just computed, while
// the other warps rotate the remaining blocks and most of Q (the split below balances the
// warps).  One barrier per step.  With row stride 33 the loads and stores of a warp's
// blocks fall on distinct banks.
__device__ void inner_sweep_cross(SmemTc &s, double tol, bool first, int tid,
                                  const GroupBar &bar, bool a32) {
  constexpr int W2 = SmemTc::W2;
  constexpr int NP = W2 / 2;
  constexpr int NB = NP * (NP + 1) / 2;
  constexpr int AW = NT / 32 - 1;          // the angle warp
  constexpr int NU = NT - 32;              // update threads
  constexpr int BPT = 3;
  constexpr int NOWN = NB - NP;            // blocks of the update threads
  // work split per step (the cost of a block is about three Q items): warps 0..4 take two
  // blocks and three Q items, warps 5 and 6 two or three blocks and no Q item, the angle
  // warp its hand-over block, the rotations and one Q item (with FP64 angles, whose
  // arithmetic lengthens the angle warp's step, warp 5 takes that Q item)
  constexpr int QW = 5 * 32;               // update threads that rotate Q
  constexpr int XT = 5 * 32;               // first update thread with a third block
  static_assert(2 * NU + (NOWN - 2 * NU) == NOWN && NOWN - 2 * NU <= NU - XT, "block split");
  static_assert(3 * QW + 32 == NP * (W2 / 4), "Q item split");
  float *A = s.X3[0], *B = s.X3[1], *C = s.X3[2];
  const float tolf = (float)tol, tol2f = (float)(tol * tol);
  const double tol2d = tol * tol;
  const int warp = tid >> 5, lane = tid & 31;
  // fresh-Gram convergence test |g| > tol sqrt(a b) over the cross pairs
  int need = 0;
  for (int idx = tid; idx < NP * NP; idx += NT) {
    const int i = idx >> 5, j = idx & 31;
    const float a = A[i * XLD + i], b = C[j * XLD + j], g = B[i * XLD + j];
    if (a32 ? rot_test_f32(a, b, g, tolf, tol2f) : decide64(a, b, g, tol2d)) need = 1;
  }
  bar.sync();                        // every thread has read step_rot of the previous call
  if (tid == 0) {
    s.step_rot = 0;
    if (first) s.any_rot = 0;
  }
  if (!bar.sync_or(need)) return;
  if (first) {
    for (int idx = tid; idx < W2 * W2; idx += NT) s.Q[idx] = (idx / W2 == idx % W2) ? 1.f : 0.f;
  }
  // update threads: blocks tid, tid + NU and (threads XT ..) 2 NU + tid - XT of the
  // non-hand-over blocks
  int bp[BPT], bq[BPT];
#pragma unroll
  for (int t = 0; t < BPT; ++t) {
    const int c = t < 2 ? tid + t * NU : 2 * NU + (tid - XT);
    bp[t] = -1;
    bq[t] = 0;
    if (warp != AW && (t < 2 || (tid >= XT && c < NOWN))) cross_block(c, bp[t], bq[t]);
  }
  // angle warp: lane k owns block (hp, hq) and forms pair k's rotations; the entry it
  // needs is o01 of (k, k + 1) or o10 of (0, NP - 1)
  const int hp = lane < NP - 1 ? lane : 0, hq = lane < NP - 1 ? lane + 1 : NP - 1;
  const int kq = (lane + 1) & 31;
  if (warp == AW)                    // rotations of step 0: pair k = columns k, 32 + k
    cross_angle(s, 0, lane, A[lane * XLD + lane], C[lane * XLD + lane], B[lane * XLD + lane],
                tolf, tol2f, tol2d, a32);
  bar.sync();
  for (int step = 0; step < NP; ++step) {
    const int sl = step & 1;
    if (warp == AW) {
      const int rp = s.rot[sl][hp], rq = s.rot[sl][hq];
      const int sp = (hp + step) & 31, sq = (hq + step) & 31;
      const bool more = step + 1 < NP;
      if (rp || rq || more) {
        float o00, o01, o10, o11;
        rot_block(A[hp * XLD + hq], B[hp * XLD + sq], B[hq * XLD + sp], C[sp * XLD + sq],
                  s.cs[sl][2 * hp], s.cs[sl][2 * hp + 1], s.cs[sl][2 * hq],
                  s.cs[sl][2 * hq + 1], o00, o01, o10, o11);
        if (rp || rq) {
          A[hp * XLD + hq] = o00;
          B[hp * XLD + sq] = o01;
          B[hq * XLD + sp] = o10;
          C[sp * XLD + sq] = o11;
          C[sq * XLD + sp] = o11;
        }
        if (more) {
          // the diagonal entries are the rotated ones if those pairs rotated, else
          // unchanged in place
          const int skq = (kq + step) & 31;
          const float a = s.rot[sl][lane] ? s.dd[sl][2 * lane] : A[lane * XLD + lane];
          const float b = s.rot[sl][kq] ? s.dd[sl][2 * kq + 1] : C[skq * XLD + skq];
          cross_angle(s, sl ^ 1, lane, a, b, lane < NP - 1 ? o01 : o10, tolf, tol2f, tol2d,
                      a32);
        }
      }
    } else {
      // (c, s) of the step's pairs; a pair with s == 0 is the identity (a non-rotating pair
      // carries (1, 0); a rotation whose tangent underflowed has c = 1, s = 0 and leaves its
      // diagonal unchanged), so s != 0 decides whether a pair moves
      const float2 *cs2 = reinterpret_cast<const float2 *>(s.cs[sl]);
#pragma unroll
      for (int t = 0; t < BPT; ++t) {
        const int p = bp[t], q = bq[t];
        if (p < 0) continue;
        const float2 cp = cs2[p], cq = cs2[q];
        const bool rp = cp.y != 0.f, rq = cq.y != 0.f;
        const int sp = (p + step) & 31, sq = (q + step) & 31;
        if (p == q) {
          if (rp) {
            A[p * XLD + p] = s.dd[sl][2 * p];
            C[sp * XLD + sp] = s.dd[sl][2 * p + 1];
            B[p * XLD + sp] = 0.f;
          }
          continue;
        }
        if (!(rp || rq)) continue;
        float o00, o01, o10, o11;
        rot_block(A[p * XLD + q], B[p * XLD + sq], B[q * XLD + sp], C[sp * XLD + sq], cp.x,
                  cp.y, cq.x, cq.y, o00, o01, o10, o11);
        A[p * XLD + q] = o00;
        B[p * XLD + sq] = o01;
        B[q * XLD + sp] = o10;
        C[sp * XLD + sq] = o11;
        C[sq * XLD + sp] = o11;
      }
      if (tid < QW)
        for (int u = 0; u < 3; ++u) cross_q_item(s, cs2, tid + u * QW, step);
      else if (!a32 && tid < QW + 32)   // FP64 angles: warp 5 takes the angle warp's Q item
        cross_q_item(s, cs2, 3 * QW + (tid - QW), step);
    }
    if (warp == AW && a32)
      cross_q_item(s, reinterpret_cast<const float2 *>(s.cs[sl]), 3 * QW + lane, step);
    bar.sync();
  }
}

// This slice's matrices: the uniform batch of one tensor, or a per-slice descriptor.
template <typename T>
struct SliceView {
  T *W, *V;
  float *nrm2;
  int rows, cols;
};
template <typename T>
__device__ __forceinline__ SliceView<T> slice_view(const JacobiParams &p, int slice) {
  SliceView<T> v;
  if (p.desc) {
    const SliceDesc d = p.desc[slice];
    v.W = reinterpret_cast<T *>(d.A);
    v.V = reinterpret_cast<T *>(d.V);
    v.nrm2 = d.norm2;
    v.rows = d.rows;
    v.cols = d.cols;
  } else {
    v.W = reinterpret_cast<T *>(p.A) + (int64_t)slice * p.sA;
    v.V = reinterpret_cast<T *>(p.V) + (int64_t)slice * p.sV;
    v.nrm2 = p.norm2 ? p.norm2 + (int64_t)slice * p.cols : nullptr;
    v.rows = p.rows;
    v.cols = p.cols;
  }
  return v;
}

// de Rijk ordering: s.ord = the columns by decreasing norm (ties: lower index first), from
// the squared norms the previous sweep left in nrm (bitonic sort of a power-of-two key
// array); the first sweep keeps 0..cols-1.
template <typename SM, typename Bar>
__device__ void sort_columns(SM &s, const float *nrm, int cols, bool first, int tid,
                             const Bar &bar) {
  int p2 = 1;
  while (p2 < cols) p2 <<= 1;
  float *key = sort_keys(s);
  for (int c = tid; c < p2; c += NT) {
    key[c] = c < cols ? (first ? -(float)c : __ldcg(nrm + c)) : -INFINITY;
    s.ord[c] = c;
  }
  bar.sync();
  for (int k = 2; k <= p2; k <<= 1) {
    for (int j = k >> 1; j > 0; j >>= 1) {
      for (int t = tid; t < p2; t += NT) {
        int u = t ^ j;
        if (u > t) {
          float kt = key[t], ku = key[u];
          int it = s.ord[t], iu = s.ord[u];
          bool t_first = (kt > ku) || (kt == ku && it < iu);
          if (((t & k) == 0) ? !t_first : t_first) {
            key[t] = ku; key[u] = kt;
            s.ord[t] = iu; s.ord[u] = it;
          }
        }
      }
      bar.sync();
    }
  }
}

// Local columns of block pair (bi, bj) of the sweep's order (-1 = padding).
template <int W2, typename SM>
__device__ __forceinline__ void pair_columns(SM &s, int bi, int bj, int cols, bool sorted,
                                             int tid) {
  constexpr int B = W2 / 2;
  if (tid < W2) {
    int lc = (tid < B) ? bi * B + tid : bj * B + (tid - B);
    s.col[tid] = lc < cols ? (sorted ? s.ord[lc] : lc) : -1;
  }
}

template <typename T, int W2, int NS>
__global__ void __launch_bounds__(NT, NS == 2 ? 3 : 2) jacobi_kernel(JacobiParams p) {
  using C = Cfg<T, W2, NS>;
  extern __shared__ __align__(16) unsigned char smem_raw[];
  Smem<T, W2, NS> &s = *reinterpret_cast<Smem<T, W2, NS> *>(smem_raw);
  cg::cluster_group cluster = cg::this_cluster();
  const int crank = (int)cluster.block_rank();
  const int csize = (int)cluster.num_blocks();
  const int tid = threadIdx.x;
  const double tol = p.tol;
  const CtaBar bar;

  for (int iter = 0;; ++iter) {
    const int par = iter & 1;
    if (crank == 0 && tid == 0) s.slice[par] = atomicAdd(p.queue, 1);
    cluster.sync();
    const int slice = *cluster.map_shared_rank(&s.slice[par], 0);
    if (slice >= p.nslices) break;
    const SliceView<T> v = slice_view<T>(p, slice);
    int nb = (v.cols + C::B - 1) / C::B;
    if (nb & 1) ++nb;
    if (nb < 2) nb = 2;

    // V = I (this CTA initialises columns crank, crank + csize, ...); a warm start keeps the
    // caller's V (the slice then holds W V)
    if (!p.warm && !p.novec)
      for (int c = crank; c < v.cols; c += csize)
        for (int r = tid; r < v.cols; r += NT)
          __stcg(v.V + (int64_t)c * v.cols + r, r == c ? T(1) : T(0));
    if (tid == 0) {
      s.nrot = 0;
      s.nonfinite = 0;
    }
    cluster.sync();

    const bool sorted = v.nrm2 != nullptr && v.cols <= MAXSORT;
    int converged = 0, sweep = 0;
    for (sweep = 1; sweep <= p.max_sweeps; ++sweep) {
      if (tid == 0) s.sweep_any = 0;
      if (sorted) sort_columns(s, v.nrm2, v.cols, sweep == 1, tid, bar);
      for (int round = 0; round < nb - 1; ++round) {
        for (int q = crank; q < nb / 2; q += csize) {
          int bi, bj;
          rr_pair(nb, round, q, bi, bj);
          pair_columns<W2>(s, bi, bj, v.cols, sorted, tid);
          __syncthreads();
          gram<T, W2, NS>(s, v.W, v.rows, v.rows);
          for (int is = 0; is < p.inner_sweeps; ++is) {
            inner_sweep<T, W2, NS>(s, tol, round == 0, is == 0, tid, bar, p.angle32 != 0);
            if (!s.step_rot) break;
          }
          __syncthreads();
          if (sorted && tid < W2 && s.col[tid] >= 0)     // squared norms after this step
            __stcg(v.nrm2 + s.col[tid], (float)s.G[s.gcur][tri<W2>(tid, tid)]);
          if (s.any_rot) {
            if (tid == 0) s.sweep_any = 1;
            apply_q<T, W2, NS>(s, v.W, v.rows, v.rows);
            if (!p.novec) apply_q<T, W2, NS>(s, v.V, v.cols, v.cols);
          }
          __syncthreads();
        }
        __threadfence();
        cluster.sync();
      }
      // cluster-wide vote: did anybody rotate during this sweep?
      if (tid == 0) s.vote[sweep & 1] = s.sweep_any;
      cluster.sync();
      int any = 0;
      for (int r = 0; r < csize; ++r) any |= *cluster.map_shared_rank(&s.vote[sweep & 1], r);
      if (!any) {
        converged = 1;
        break;
      }
    }
    if (tid == 0) {
      atomicAdd((unsigned long long *)&p.rots[slice], (unsigned long long)s.nrot);
      if (s.nonfinite) atomicOr(p.status, ST_NONFINITE);
      if (crank == 0) {
        p.sweeps[slice] = converged ? sweep : -1;
        if (!converged) atomicOr(p.status, ST_NOCONV);
      }
    }
  }
  cluster.sync();  // keep shared memory alive until every CTA has read the slice index
}

// ---------------------------------------------------------------- tensor-core kernel
// A kernel that holds tensor memory runs one CTA per SM, so the tensor-core variant is one
// persistent CTA per SM made of TC_GROUPS 256-thread groups ("workers").  Each worker has
// its own shared memory (SmemTc), named barrier, MMA barriers and 64 TMEM columns.
//
// Work is scheduled GPU-wide at the granularity of one block pair, so that slices whose
// iteration runs longer than others do not leave SMs idle at the end.  Per slice (SliceCtx
// in global memory): sn = (sweep << 32) | next ticket, a ticket t of sweep w being the
// block pair q = t mod np of round t / np (np = nb / 2 pairs, nb - 1 rounds); done = pairs
// of the sweep completed; rot = whether a pair rotated.  Per block: a version counter = the
// pairs that have finished with it.  Block b enters exactly one pair per round, so the pair
// of round r of sweep w may start when both its blocks have version (w - 1)(nb - 1) + r;
// tickets are handed out in increasing order and a pair only waits for pairs with smaller
// tickets, so the earliest unfinished ticket can always run (no deadlock).  The worker that
// completes the last pair of a sweep closes it: the slice has converged if no pair rotated
// (the stopping rule of the scalar method), else it sorts the columns by the squared norms
// the sweep left (all of its pairs are done, so they are final), stores that order for the
// slice in global memory and opens the next sweep's tickets; every worker takes its block
// pair's columns from the stored order (the first sweep uses the natural order).  A worker
// takes the next ticket of its current slice, else starts a new slice, else helps any open
// slice (warp 0 of the worker examines 32 slices at a time), and only takes a ticket whose
// two blocks are already free, so the pair runs without waiting (the earliest unfinished
// ticket always becomes free; versions only grow).  Every wait is bounded; on expiry the
// kernel raises a global abort flag and ST_TIMEOUT.
constexpr int TC_GROUPS = 3;
constexpr uint32_t TC_COLS = 256;     // TMEM columns of the CTA (64 per group, power of two)
constexpr unsigned SCHED_SPIN = 1u << 24;   // polls of a dependency or idle wait (~1 us each)

struct SliceCtx {
  unsigned long long sn;   // (sweep << 32) | next ticket; sweep 0 = not started
  int done;                // pairs of the current sweep completed
  int rot[2];              // a pair rotated, by sweep parity
  int finished;            // converged or capped
  int pad[2];
};
struct SchedHdr {
  int fin;                 // slices finished
  int abort;               // a wait ran out: everybody leaves
  int pad[14];
};

__host__ __device__ inline int tc_blocks(int cols) {
  int nb = (cols + 31) / 32;
  if (nb & 1) ++nb;
  return nb < 2 ? 2 : nb;
}

enum { WK_EXIT = 0, WK_START = 1, WK_PAIR = 2 };

__device__ __forceinline__ int vload(const int *p) { return *(const volatile int *)p; }
__device__ __forceinline__ unsigned long long vload64(const unsigned long long *p) {
  return *(const volatile unsigned long long *)p;
}

// Takes ticket (sweep, t) of slice sl if one is open and its two blocks are already free
// (so that the worker does not wait; the earliest unfinished ticket always becomes free).
__device__ bool take_ticket(SliceCtx *ctx, const int *ver, int nbmax, const JacobiParams &p,
                            int sl, int &sweep, int &t) {
  SliceCtx &c = ctx[sl];
  // (a finished slice has handed out all tickets of its last sweep: tk >= total below)
  const int cols = p.desc ? p.desc[sl].cols : p.cols;
  const int nb = tc_blocks(cols), np = nb / 2;
  const unsigned total = (unsigned)(np * (nb - 1));
  for (int attempt = 0; attempt < 4; ++attempt) {
    const unsigned long long sn = vload64(&c.sn);
    const int w = (int)(sn >> 32);
    const unsigned tk = (unsigned)sn;
    if (w == 0 || tk >= total) return false;
    {
      const int round = (int)(tk / np), q = (int)(tk % np);
      int bi, bj;
      rr_pair(nb, round, q, bi, bj);
      const int need = (w - 1) * (nb - 1) + round;
      const int *v = ver + (int64_t)sl * nbmax;
      if (vload(v + bi) < need || vload(v + bj) < need) return false;
    }
    if (atomicCAS(&c.sn, sn, sn + 1) == sn) {
      sweep = w;
      t = (int)tk;
      return true;
    }
  }
  return false;
}

// Warp-wide search over the started slices (every lane of the calling warp): lane l looks
// at slice (first + base + l) mod started for base = 0, 32, ..; the lowest lane that sees a
// free ticket tries to take it.  Returns the slice (ticket in sweep, t; same in all lanes),
// or -1.
__device__ int scan_tickets(SliceCtx *ctx, const int *ver, int nbmax, const JacobiParams &p,
                            int first, int started, int &sweep, int &t) {
  const int lane = threadIdx.x & 31;
  for (int base = 0; base < started; base += 32) {
    const int k = base + lane;
    const int cand = k < started ? (first + k) % started : -1;
    bool free = false;
    if (cand >= 0) {
      const unsigned long long sn = vload64(&ctx[cand].sn);
      const int w = (int)(sn >> 32);
      const unsigned tk = (unsigned)sn;
      const int cols = p.desc ? p.desc[cand].cols : p.cols;
      const int nb = tc_blocks(cols), np = nb / 2;
      if (w != 0 && tk < (unsigned)(np * (nb - 1))) {
        const int round = (int)(tk / np), q = (int)(tk % np);
        int bi, bj;
        rr_pair(nb, round, q, bi, bj);
        const int need = (w - 1) * (nb - 1) + round;
        const int *v = ver + (int64_t)cand * nbmax;
        free = vload(v + bi) >= need && vload(v + bj) >= need;
      }
    }
    unsigned m = __ballot_sync(0xffffffffu, free);
    while (m) {
      const int src = __ffs(m) - 1;
      int got = 0, w = 0, tt = 0;
      if (lane == src) got = take_ticket(ctx, ver, nbmax, p, cand, w, tt) ? 1 : 0;
      got = __shfl_sync(0xffffffffu, got, src);
      if (got) {
        sweep = __shfl_sync(0xffffffffu, w, src);
        t = __shfl_sync(0xffffffffu, tt, src);
        return __shfl_sync(0xffffffffu, cand, src);
      }
      m &= m - 1;
    }
  }
  return -1;
}

__global__ void __launch_bounds__(NT * TC_GROUPS, 1) jacobi_tc_kernel(JacobiParams p) {
  constexpr int W2 = SmemTc::W2;
  extern __shared__ __align__(16) unsigned char smem_raw[];
  __shared__ uint32_t tmem_base;
  // the swizzled operand tiles need 1024-byte alignment (the launch adds the slack)
  SmemTc *groups =
      reinterpret_cast<SmemTc *>(((uintptr_t)smem_raw + 1023) & ~(uintptr_t)1023);
  const int g = threadIdx.x / NT, tid = threadIdx.x % NT;
  // the inner sweeps see the group's warps rotated by g, so that their angle warp (the
  // last one) is physical warp 7 - g: the three groups' angle warps, which carry the FP64
  // angle arithmetic, sit on different SM sub-partitions
  const int vtid = (tid + 32 * g) % NT;
  SmemTc &s = groups[g];
  const unsigned spin = p.wait_polls > 0 ? (unsigned)p.wait_polls : SCHED_SPIN;
  const GroupBar gbar{1 + g};
  const double tol = p.tol;
  SchedHdr *hdr = reinterpret_cast<SchedHdr *>(p.sched);
  SliceCtx *ctx = reinterpret_cast<SliceCtx *>(hdr + 1);
  const int nbmax = tc_blocks(p.max_cols);
  int *ver = reinterpret_cast<int *>(ctx + p.nslices);
  int *ordg = reinterpret_cast<int *>(ver + (int64_t)p.nslices * nbmax);   // column orders
  if (tid == 0) {
    for (int b = 0; b < 3; ++b) tc::mbar_init(&s.bar[b], 1);
    tc::mbar_init_fence();
    s.fail = 0;
  }
  if (threadIdx.x < 32) tc::tmem_alloc_n<TC_COLS>(&tmem_base);
  tc::fence_before_sync();
  __syncthreads();
  tc::fence_after_sync();
  if (tid == 0) s.tmem = tmem_base + 64u * (uint32_t)g;
  gbar.sync();

  uint32_t phase = 0;
  int cur = -1;                        // slice this worker prefers (warp 0's view)
  bool queue_open = true;
  const int worker = blockIdx.x * TC_GROUPS + g;
  for (;;) {
    // ---- warp 0 finds the next work item (lane 0 decides) and broadcasts it
    if (tid < 32) {
      int kind = WK_EXIT, sl = -1, w = 0, t = 0;
      for (unsigned idle = 0;; ++idle) {
        int stop = 0;
        if (tid == 0) {
          stop = vload(&hdr->abort);
          if (!stop && cur >= 0 && take_ticket(ctx, ver, nbmax, p, cur, w, t)) {
            kind = WK_PAIR;
            sl = cur;
          } else if (!stop && queue_open) {
            const int n = atomicAdd(p.queue, 1);
            if (n < p.nslices) {
              kind = WK_START;
              sl = n;
            } else {
              queue_open = false;
            }
          }
        }
        stop = __shfl_sync(0xffffffffu, stop, 0);
        kind = __shfl_sync(0xffffffffu, kind, 0);
        if (stop || kind != WK_EXIT) break;
        const int started = min(vload(p.queue), p.nslices);
        const int got = scan_tickets(ctx, ver, nbmax, p, worker % (started > 0 ? started : 1),
                                     started, w, t);
        if (got >= 0) {
          kind = WK_PAIR;
          sl = got;
          cur = got;
          break;
        }
        int fin = 0;
        if (tid == 0) fin = vload(&hdr->fin) >= p.nslices;
        if (__shfl_sync(0xffffffffu, fin, 0)) break;
        if (idle >= spin) {
          if (tid == 0) {
            atomicExch(&hdr->abort, 1);
            s.fail = 1;
          }
          break;
        }
        __nanosleep(1000);
      }
      if (tid == 0) {
        __threadfence();               // what the ticket's publisher wrote is visible
        s.wk[0] = kind;
        s.wk[1] = sl;
        s.wk[2] = w;
        s.wk[3] = t;
      }
    }
    gbar.sync();
    const int kind = s.wk[0], slice = s.wk[1], sweep = s.wk[2], ticket = s.wk[3];
    if (kind == WK_EXIT) break;
    const SliceView<float> v = slice_view<float>(p, slice);
    if (kind == WK_START) {
      // V = I (a warm start keeps the caller's V), then open sweep 1
      if (!p.warm && !p.novec)
        for (int c = 0; c < v.cols; ++c)
          for (int r = tid; r < v.cols; r += NT)
            __stcg(v.V + (int64_t)c * v.cols + r, r == c ? 1.f : 0.f);
      __threadfence();
      gbar.sync();
      if (tid == 0) {
        cur = slice;
        atomicExch(&ctx[slice].sn, 1ull << 32);
      }
      continue;
    }
    // ---- one block pair of slice `slice`, sweep `sweep`
    SliceCtx &c = ctx[slice];
    const int nb = tc_blocks(v.cols), np = nb / 2;
    const int round = ticket / np, q = ticket % np;
    int bi, bj;
    rr_pair(nb, round, q, bi, bj);
    const bool sorted = v.nrm2 != nullptr && v.cols <= MAXSORT;
    // both blocks have finished the previous round (checked when the ticket was taken)
    if (tid == 0) {
      s.nrot = 0;
      s.nonfinite = 0;
    }
    if (tid < W2) {
      // this pair's columns in the sweep's order (natural in the first sweep)
      constexpr int B = W2 / 2;
      const int lc = (tid < B) ? bi * B + tid : bj * B + (tid - B);
      s.col[tid] = lc < v.cols ? (sorted && sweep > 1 ? __ldcg(ordg + (int64_t)slice * p.max_cols + lc)
                                                      : lc)
                               : -1;
    }
    gbar.sync();
    // the first round of a sweep also rotates within each block (full inner sweeps), the
    // others only across the two blocks
    const bool cross = round != 0;
    gram_tc(s, v.W, v.rows, v.rows, phase, tid, gbar, cross);
    for (int is = 0; is < p.inner_sweeps; ++is) {
      if (cross)
        inner_sweep_cross(s, tol, is == 0, vtid, gbar, p.angle32 != 0);
      else
        inner_sweep<float, W2, 2>(s, tol, true, is == 0, vtid, gbar, p.angle32 != 0);
      if (!s.step_rot) break;
    }
    gbar.sync();
    if (sorted && tid < W2 && s.col[tid] >= 0) {   // squared norms after this step
      const int c = tid & 31;
      __stcg(v.nrm2 + s.col[tid], !cross ? s.G[s.gcur][tri<W2>(tid, tid)]
                                         : s.X3[tid < 32 ? 0 : 2][c * XLD + c]);
    }
    if (s.any_rot) {
      build_bq(s, tid, gbar);
      apply_tc(s, v.W, v.rows, v.rows, phase, tid, gbar);
      if (!p.novec) apply_tc(s, v.V, v.cols, v.cols, phase, tid, gbar);
    }
    __threadfence();
    gbar.sync();
    if (tid == 0) {
      const int rotated = s.any_rot;
      if (s.nrot) atomicAdd((unsigned long long *)&p.rots[slice], (unsigned long long)s.nrot);
      if (s.nonfinite) atomicOr(p.status, ST_NONFINITE);
      if (rotated) atomicOr(&c.rot[sweep & 1], 1);
      __threadfence();
      atomicAdd(ver + (int64_t)slice * nbmax + bi, 1);
      atomicAdd(ver + (int64_t)slice * nbmax + bj, 1);
      const int d = atomicAdd(&c.done, 1) + 1;
      int reopen = 0;
      if (d == np * (nb - 1)) {
        // last pair of the sweep: close it
        __threadfence();
        const int any = vload(&c.rot[sweep & 1]);
        if (!any || sweep >= p.max_sweeps) {
          p.sweeps[slice] = any ? -1 : sweep;
          if (any) atomicOr(p.status, ST_NOCONV);
          c.finished = 1;
          __threadfence();
          atomicAdd(&hdr->fin, 1);
        } else {
          reopen = 1;
        }
      }
      s.reopen = reopen;
    }
    gbar.sync();
    if (s.reopen) {
      // the next sweep: the column order by the norms this sweep left, then its tickets
      if (sorted) {
        sort_columns(s, v.nrm2, v.cols, false, tid, gbar);
        int *og = ordg + (int64_t)slice * p.max_cols;
        for (int k = tid; k < v.cols; k += NT) __stcg(og + k, s.ord[k]);
      }
      __threadfence();
      gbar.sync();
      if (tid == 0) {
        c.rot[(sweep + 1) & 1] = 0;
        c.done = 0;
        __threadfence();
        atomicExch(&c.sn, (unsigned long long)(sweep + 1) << 32);
      }
    }
  }
  tc::fence_before_sync();
  __syncthreads();                                 // every group has finished
  tc::fence_after_sync();
  if (threadIdx.x < 32) tc::tmem_dealloc_n<TC_COLS>(tmem_base);
  if (tid == 0 && s.fail) atomicOr(p.status, ST_TIMEOUT);
}

template <typename T, int W2, int NS>
cudaError_t launch_jacobi(const JacobiParams &p, cudaStream_t st, int cluster_hint,
                          int grid_hint) {
  auto kern = jacobi_kernel<T, W2, NS>;
  size_t smem = sizeof(Smem<T, W2, NS>);
  cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  if (e != cudaSuccess) return e;
  cudaFuncSetAttribute(kern, cudaFuncAttributeNonPortableClusterSizeAllowed, 1);
  int nb = (p.cols + W2 / 2 - 1) / (W2 / 2);
  if (nb & 1) ++nb;
  if (nb < 2) nb = 2;
  int cl = 1;
  int want = cluster_hint > 0 ? cluster_hint : (W2 >= 64 ? 4 : 16);
  while (cl * 2 <= want && cl * 2 <= nb / 2) cl *= 2;
  cudaLaunchConfig_t cfg = {};
  cudaLaunchAttribute attr[1];
  attr[0].id = cudaLaunchAttributeClusterDimension;
  cfg.blockDim = dim3(NT);
  cfg.dynamicSmemBytes = smem;
  cfg.stream = st;
  cfg.attrs = attr;
  cfg.numAttrs = 1;
  int max_clusters = 0;
  for (;;) {
    attr[0].val.clusterDim.x = cl;
    attr[0].val.clusterDim.y = 1;
    attr[0].val.clusterDim.z = 1;
    cfg.gridDim = dim3(cl);
    e = cudaOccupancyMaxActiveClusters(&max_clusters, kern, &cfg);
    if (e == cudaSuccess && max_clusters > 0) break;
    cudaGetLastError();
    if (cl == 1) return e == cudaSuccess ? cudaErrorInvalidConfiguration : e;
    cl /= 2;
  }
  // All co-resident clusters (measured faster than keeping the slices in flight within L2).
  int nclusters = max_clusters;
  if (grid_hint > 0) nclusters = grid_hint;
  if (nclusters > p.nslices) nclusters = p.nslices;
  if (nclusters < 1) nclusters = 1;
  cfg.gridDim = dim3(nclusters * cl);
  return cudaLaunchKernelEx(&cfg, kern, p);
}

size_t sched_bytes_for(int64_t nslices, int64_t max_cols) {
  return sizeof(SchedHdr) + (size_t)nslices * sizeof(SliceCtx) +
         (size_t)nslices * (size_t)tc_blocks((int)max_cols) * sizeof(int) +
         (size_t)nslices * (size_t)max_cols * sizeof(int);     // column orders
}

// grid_hint: CTAs (0 = one per SM).  The scheduler state is zeroed here, in stream order.
cudaError_t launch_jacobi_tc(const JacobiParams &p, cudaStream_t st, int grid_hint) {
  static_assert(TC_GROUPS * sizeof(SmemTc) + 1024 <= 227 * 1024, "shared memory of a CTA");
  if (p.sched == nullptr || p.nslices < 1) return cudaErrorInvalidValue;
  const size_t smem = (size_t)TC_GROUPS * sizeof(SmemTc) + 1024;
  cudaError_t e = cudaFuncSetAttribute(jacobi_tc_kernel,
                                       cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  if (e != cudaSuccess) return e;
  int dev = 0, sms = 0, per_sm = 0;
  if ((e = cudaGetDevice(&dev)) != cudaSuccess) return e;
  if ((e = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev)) != cudaSuccess)
    return e;
  e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, jacobi_tc_kernel, NT * TC_GROUPS,
                                                     smem);
  if (e != cudaSuccess) return e;
  if (per_sm < 1) return cudaErrorInvalidConfiguration;
  // every CTA resident at once (workers wait on one another through global memory)
  int grid = sms * per_sm;
  if (grid_hint > 0 && grid_hint < grid) grid = grid_hint;
  if ((e = cudaMemsetAsync(p.sched, 0, p.sched_bytes, st)) != cudaSuccess) return e;
  jacobi_tc_kernel<<<grid, NT * TC_GROUPS, smem, st>>>(p);
  return cudaGetLastError();
}

// ---------------------------------------------------------------- finalize
// sigma_j = ||w_j|| and a stable descending order (ties: lower column first).
template <typename T>
__global__ void __launch_bounds__(256) finalize_kernel(const T *__restrict__ A, int64_t sA,
                                                       int rows, int cols, T *sig, int *perm,
                                                       int p2, const SliceDesc *desc) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  T *key = reinterpret_cast<T *>(smem_raw);
  int *idx = reinterpret_cast<int *>(key + p2);
  int slice = blockIdx.x;
  const T *W = A + (int64_t)slice * sA;
  if (desc) {                       // batched: each slice carries its own matrices
    const SliceDesc d = desc[blockIdx.x];
    W = reinterpret_cast<const T *>(d.A);
    rows = d.rows;
    cols = d.cols;
    sig = reinterpret_cast<T *>(d.sig);
    perm = d.perm;
    slice = 0;
    p2 = 1;
    while (p2 < cols) p2 <<= 1;
  }
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  for (int j = warp; j < p2; j += 8) {
    T acc = T(0);
    if (j < cols)
      for (int r = lane; r < rows; r += 32) {
        T v = W[(int64_t)j * rows + r];
        acc = fma(v, v, acc);
      }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) acc += __shfl_xor_sync(0xffffffffu, acc, o);
    if (lane == 0) {
      key[j] = j < cols ? sqrt(acc) : T(-1);
      idx[j] = j;
    }
  }
  __syncthreads();
  // bitonic sort: descending key, ascending index on ties
  for (int k = 2; k <= p2; k <<= 1) {
    for (int j = k >> 1; j > 0; j >>= 1) {
      for (int t = threadIdx.x; t < p2; t += blockDim.x) {
        int u = t ^ j;
        if (u > t) {
          bool up = ((t & k) == 0);
          T kt = key[t], ku = key[u];
          int it = idx[t], iu = idx[u];
          bool t_first = (kt > ku) || (kt == ku && it < iu);   // t precedes u in output
          if (up ? !t_first : t_first) {
            key[t] = ku; key[u] = kt;
            idx[t] = iu; idx[u] = it;
          }
        }
      }
      __syncthreads();
    }
  }
  for (int j = threadIdx.x; j < cols; j += blockDim.x) {
    sig[(int64_t)slice * cols + j] = key[j];
    perm[(int64_t)slice * cols + j] = idx[j];
  }
}

// ---------------------------------------------------------------- emit
// (bv, bi) <- the larger magnitude, first index on ties; bv starts at -1 (empty).
template <typename T>
__device__ __forceinline__ void merge_max(T a, int i, T &bv, int &bi) {
  if (a > bv || (a == bv && i < bi)) {
    bv = a;
    bi = i;
  }
}
template <typename T>
__device__ __forceinline__ void argmax_abs(T v, int i, T &bv, int &bi) { merge_max(fabs(v), i, bv, bi); }

template <typename T>
__global__ void __launch_bounds__(256) emit_kernel(const T *__restrict__ A, int64_t sA,
                                                   const T *__restrict__ Vw, int64_t sV,
                                                   int rows, int cols, bool transposed,
                                                   const T *__restrict__ sig,
                                                   const int *__restrict__ perm,
                                                   int64_t k_uniform, const int *ranks,
                                                   const int64_t *offsets, T *U, T *S, T *V) {
  const int q = blockIdx.x;
  const int slice = blockIdx.y;
  int64_t count = ranks ? (int64_t)ranks[slice] : k_uniform;
  if (q >= count) return;
  int64_t colbase = offsets ? offsets[slice] : (int64_t)slice * k_uniform;
  const int j = perm[(int64_t)slice * cols + q];
  const T sg = sig[(int64_t)slice * cols + q];
  const T *wcol = A + (int64_t)slice * sA + (int64_t)j * rows;     // rows entries, scaled 1/sg
  const T *zcol = Vw ? Vw + (int64_t)slice * sV + (int64_t)j * cols : nullptr;   // cols entries
  if (!Vw) {
    // no right vectors: the work matrix's side only (U of a non-transposed slice, sign-fixed
    // on itself; V of a transposed one, sign decided after the other side is formed)
    __shared__ T k_bv[8];
    __shared__ int k_bi[8];
    __shared__ T k_sign;
    const T inv0 = sg > T(0) ? T(1) / sg : T(0);
    T bv0 = T(-1);
    int bi0 = 0x7fffffff;
    if (!transposed)
      for (int a = threadIdx.x; a < rows; a += blockDim.x) argmax_abs(wcol[a] * inv0, a, bv0, bi0);
    for (int o = 16; o > 0; o >>= 1) {
      T ov = __shfl_xor_sync(0xffffffffu, bv0, o);
      int oi = __shfl_xor_sync(0xffffffffu, bi0, o);
      merge_max(ov, oi, bv0, bi0);
    }
    if ((threadIdx.x & 31) == 0) {
      k_bv[threadIdx.x >> 5] = bv0;
      k_bi[threadIdx.x >> 5] = bi0;
    }
    __syncthreads();
    if (threadIdx.x == 0) {
      T b = T(-1);
      int i = 0x7fffffff;
      for (int w = 0; w < (int)(blockDim.x >> 5); ++w) merge_max(k_bv[w], k_bi[w], b, i);
      k_sign = (b > T(0) && wcol[i] * inv0 < T(0)) ? T(-1) : T(1);
      S[colbase + q] = sg;
    }
    __syncthreads();
    T *out = transposed ? V + (colbase + q) * rows : U + (colbase + q) * rows;
    for (int a = threadIdx.x; a < rows; a += blockDim.x) out[a] = k_sign * (wcol[a] * inv0);
    return;
  }
  const T inv = sg > T(0) ? T(1) / sg : T(0);
  // left vector: W-part (non-transposed) or Z-part (transposed)
  const int nl = transposed ? cols : rows;
  const int nr = transposed ? rows : cols;
  __shared__ T sbv[8];
  __shared__ int sbi[8];
  __shared__ T s_sign;
  T bv = T(-1);
  int bi = 0x7fffffff;
  for (int a = threadIdx.x; a < nl; a += blockDim.x) {
    T v = transposed ? zcol[a] : wcol[a] * inv;
    argmax_abs(v, a, bv, bi);
  }
  for (int o = 16; o > 0; o >>= 1) {
    T ov = __shfl_xor_sync(0xffffffffu, bv, o);
    int oi = __shfl_xor_sync(0xffffffffu, bi, o);
    merge_max(ov, oi, bv, bi);
  }
  if ((threadIdx.x & 31) == 0) {
    sbv[threadIdx.x >> 5] = bv;
    sbi[threadIdx.x >> 5] = bi;
  }
  __syncthreads();
  if (threadIdx.x == 0) {
    T b = T(-1);
    int i = 0x7fffffff;
    for (int w = 0; w < (int)(blockDim.x >> 5); ++w) merge_max(sbv[w], sbi[w], b, i);
    T ref;
    if (b > T(0)) {
      ref = transposed ? zcol[i] : wcol[i] * inv;
    } else {
      // zero left vector: take the sign from the right vector
      T b2 = T(-1);
      int i2 = 0x7fffffff;
      for (int a = 0; a < nr; ++a) argmax_abs(transposed ? wcol[a] * inv : zcol[a], a, b2, i2);
      ref = b2 > T(0) ? (transposed ? wcol[i2] * inv : zcol[i2]) : T(1);
    }
    s_sign = ref < T(0) ? T(-1) : T(1);
    S[colbase + q] = sg;
  }
  __syncthreads();
  const T sgn = s_sign;
  const int64_t n1 = nl, n2 = nr;
  T *Ucol = U + (colbase + q) * n1;
  T *Vcol = V + (colbase + q) * n2;
  for (int a = threadIdx.x; a < nl; a += blockDim.x)
    Ucol[a] = sgn * (transposed ? zcol[a] : wcol[a] * inv);
  for (int b = threadIdx.x; b < nr; b += blockDim.x)
    Vcol[b] = sgn * (transposed ? wcol[b] * inv : zcol[b]);
}

template <typename T>
__global__ void transpose_kernel(const T *__restrict__ A, int64_t m, int64_t p, T *__restrict__ B) {
  __shared__ T tile[32][33];
  const int64_t slice = blockIdx.z;
  const T *a = A + slice * m * p;
  T *b = B + slice * m * p;
  int64_t i0 = (int64_t)blockIdx.x * 32, j0 = (int64_t)blockIdx.y * 32;
  for (int y = threadIdx.y; y < 32; y += 8) {
    int64_t i = i0 + threadIdx.x, j = j0 + y;
    if (i < m && j < p) tile[y][threadIdx.x] = a[i + m * j];
  }
  __syncthreads();
  for (int y = threadIdx.y; y < 32; y += 8) {
    int64_t j = j0 + threadIdx.x, i = i0 + y;
    if (i < m && j < p) b[j + p * i] = tile[threadIdx.x][y];
  }
}

}  // namespace

size_t jacobi_sched_bytes(int64_t nslices, int64_t max_cols) {
  return sched_bytes_for(nslices, max_cols);
}

template <typename T>
cudaError_t jacobi_run(const JacobiParams &p, cudaStream_t st, int width_hint, int cluster_hint,
                       int grid_hint, int stages) {
  if constexpr (sizeof(T) == 4) {
    // tensor-core Gram / apply: block pairs of 64 columns (slices of >= 64 columns under
    // the automatic choice; any width when asked for explicitly)
    if (p.engine == JACOBI_TC || (p.engine == JACOBI_AUTO && p.cols >= 64 &&
                                  (width_hint == 0 || width_hint == 64)))
      return launch_jacobi_tc(p, st, grid_hint);
  }
  int w = width_hint;
  if (w != 16 && w != 32 && w != 64) w = p.cols <= 8 ? 16 : (p.cols <= 16 || p.cols < 256 ? 32 : 64);
  const bool two = stages == 2 || (stages == 0 && w == 64);
  if (w == 16) return two ? launch_jacobi<T, 16, 2>(p, st, cluster_hint, grid_hint)
                          : launch_jacobi<T, 16, 3>(p, st, cluster_hint, grid_hint);
  if (w == 32) return two ? launch_jacobi<T, 32, 2>(p, st, cluster_hint, grid_hint)
                          : launch_jacobi<T, 32, 3>(p, st, cluster_hint, grid_hint);
  return two ? launch_jacobi<T, 64, 2>(p, st, cluster_hint, grid_hint)
             : launch_jacobi<T, 64, 3>(p, st, cluster_hint, grid_hint);
}

template <typename T>
cudaError_t jacobi_finalize(const T *A, int64_t sA, int rows, int cols, int nslices, T *sig,
                            int *perm, cudaStream_t st) {
  int p2 = 1;
  while (p2 < cols) p2 <<= 1;
  size_t smem = (size_t)p2 * (sizeof(T) + sizeof(int));
  auto kern = finalize_kernel<T>;
  if (smem > 48 * 1024) {
    cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
  }
  kern<<<nslices, 256, smem, st>>>(A, sA, rows, cols, sig, perm, p2, nullptr);
  return cudaGetLastError();
}

template <typename T>
cudaError_t jacobi_finalize_desc(const SliceDesc *desc, int nslices, int max_cols,
                                 cudaStream_t st) {
  int p2 = 1;
  while (p2 < max_cols) p2 <<= 1;
  size_t smem = (size_t)p2 * (sizeof(T) + sizeof(int));
  auto kern = finalize_kernel<T>;
  if (smem > 48 * 1024) {
    cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
  }
  kern<<<nslices, 256, smem, st>>>(nullptr, 0, 0, 0, nullptr, nullptr, p2, desc);
  return cudaGetLastError();
}

template <typename T>
cudaError_t emit_factors(const T *A, int64_t sA, const T *Vw, int64_t sV, int rows, int cols,
                         int nslices, bool transposed, const T *sig, const int *perm,
                         int64_t k_uniform, const int *ranks, const int64_t *offsets, T *U,
                         T *S, T *V, cudaStream_t st) {
  int gx = ranks ? cols : (int)k_uniform;
  if (gx <= 0 || nslices <= 0) return cudaSuccess;
  emit_kernel<T><<<dim3(gx, nslices), 256, 0, st>>>(A, sA, Vw, sV, rows, cols, transposed, sig,
                                                    perm, k_uniform, ranks, offsets, U, S, V);
  return cudaGetLastError();
}

template <typename T>
cudaError_t transpose_slices(const T *A, int64_t m, int64_t p, int64_t nslices, T *B,
                             cudaStream_t st) {
  dim3 grid((unsigned)((m + 31) / 32), (unsigned)((p + 31) / 32), (unsigned)nslices);
  transpose_kernel<T><<<grid, dim3(32, 8), 0, st>>>(A, m, p, B);
  return cudaGetLastError();
}

#define INST(T)                                                                               \
  template cudaError_t jacobi_run<T>(const JacobiParams &, cudaStream_t, int, int, int, int); \
  template cudaError_t jacobi_finalize<T>(const T *, int64_t, int, int, int, T *, int *,      \
                                          cudaStream_t);                                      \
  template cudaError_t jacobi_finalize_desc<T>(const SliceDesc *, int, int, cudaStream_t);    \
  template cudaError_t emit_factors<T>(const T *, int64_t, const T *, int64_t, int, int, int, \
                                       bool, const T *, const int *, int64_t, const int *,    \
                                       const int64_t *, T *, T *, T *, cudaStream_t);         \
  template cudaError_t transpose_slices<T>(const T *, int64_t, int64_t, int64_t, T *,         \
                                           cudaStream_t);
INST(float)
INST(double)
#undef INST

}  // namespace tsvdm
