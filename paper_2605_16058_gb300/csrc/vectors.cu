// Second pass of the two-pass decompositions (Sec. 3.4's strategies that compute the
// singular values first and the vectors of the kept triplets afterwards).
//
// The first pass is the one-sided Jacobi without right vectors: the slice's work matrix
// ends as W = A V with orthogonal columns of norms sigma_j, so the work matrix's side of
// every triplet is W's normalised column (U_k for the kept ones), and it is emitted from
// there.  The other side of the kept triplets follows from the slice itself: Z = A^T U_k
// (A V_k for the transposed layout), a batched product of the slice (transposed) with the
// emitted vectors.  In exact arithmetic Z = V_k S_k Q with Q orthogonal (U_k differs from
// the singular vectors by a rotation within the kept subspace), so the columns of Z are not
// orthogonal once the product amplifies that rotation by sigma_l / sigma_j.  A restricted
// one-sided Jacobi of Z (rho_i columns, the same Jacobi kernels) gives Z R = V_k S_k exactly
// up to its own rounding; then V_k = the normalised columns of Z R, U_k <- U_k R, and the
// singular values are the column norms of Z R.
#include "common.cuh"

namespace tsvdm {
namespace {

constexpr int CT = 64;          // output tile: CT entries x CT columns
constexpr int CK = 32;          // contraction step
constexpr int NT = 256;

// O(:, j) = A(:, :)^T K(:, j) / S_j over slice blockIdx.z: A(r, c) is Ahat_i(r, c) (rows
// r < n1, non-transposed) or Ahat_i(c, r) (transposed); K has kd entries per column, O has
// od.  Thread (tx, ty) owns entries c0 + tx + 16 e and columns j0 + ty + 16 f.
template <typename T>
__global__ void __launch_bounds__(NT) complete_kernel(const T *__restrict__ Ahat, int64_t n1,
                                                      int64_t n2, bool transposed,
                                                      int64_t k_uniform,
                                                      const int *__restrict__ ranks,
                                                      const int64_t *__restrict__ offsets,
                                                      const T *__restrict__ Kv,
                                                      const T *__restrict__ S,
                                                      T *__restrict__ Ov) {
  __shared__ T As[CK][CT + 1];
  __shared__ T Ks[CK][CT + 1];
  const int64_t slice = blockIdx.z;
  const int64_t cnt = ranks ? (int64_t)ranks[slice] : k_uniform;
  const int64_t j0 = (int64_t)blockIdx.y * CT;
  if (j0 >= cnt) return;
  const int64_t base = offsets ? offsets[slice] : slice * k_uniform;
  const int64_t kd = transposed ? n2 : n1, od = transposed ? n1 : n2;
  const int64_t c0 = (int64_t)blockIdx.x * CT;
  const T *A = Ahat + slice * n1 * n2;
  const int tid = threadIdx.x, tx = tid % 16, ty = tid / 16;
  T acc[4][4];
#pragma unroll
  for (int e = 0; e < 4; ++e)
#pragma unroll
    for (int f = 0; f < 4; ++f) acc[e][f] = T(0);
  for (int64_t r0 = 0; r0 < kd; r0 += CK) {
#pragma unroll
    for (int u = 0; u < CK * CT / NT; ++u) {
      const int idx = tid + u * NT;
      int r, c;
      if (transposed) {                    // A(r, c) = Ahat_i[c + n1 r]: c contiguous
        r = idx / CT;
        c = idx % CT;
      } else {                             // A(r, c) = Ahat_i[r + n1 c]: r contiguous
        c = idx / CK;
        r = idx % CK;
      }
      const int64_t gr = r0 + r, gc = c0 + c;
      T v = T(0);
      if (gr < kd && gc < od) v = transposed ? A[gc + n1 * gr] : A[gr + n1 * gc];
      As[r][c] = v;
      const int jj = idx / CK, rr = idx % CK;
      const int64_t gj = j0 + jj, grr = r0 + rr;
      Ks[rr][jj] = (gj < cnt && grr < kd) ? Kv[(base + gj) * kd + grr] : T(0);
    }
    __syncthreads();
#pragma unroll 8
    for (int rr = 0; rr < CK; ++rr) {
      T a[4], k[4];
#pragma unroll
      for (int e = 0; e < 4; ++e) a[e] = As[rr][tx + 16 * e];
#pragma unroll
      for (int f = 0; f < 4; ++f) k[f] = Ks[rr][ty + 16 * f];
#pragma unroll
      for (int e = 0; e < 4; ++e)
#pragma unroll
        for (int f = 0; f < 4; ++f) acc[e][f] = fma(a[e], k[f], acc[e][f]);
    }
    __syncthreads();
  }
#pragma unroll
  for (int f = 0; f < 4; ++f) {
    const int64_t j = j0 + ty + 16 * f;
    if (j >= cnt) continue;
    const T s = S ? S[base + j] : T(1);
    const T inv = s > T(0) ? T(1) / s : T(0);
#pragma unroll
    for (int e = 0; e < 4; ++e) {
      const int64_t c = c0 + tx + 16 * e;
      if (c < od) Ov[(base + j) * od + c] = acc[e][f] * inv;
    }
  }
}

// Assembly after the restricted Jacobi of entry d (slice columns at offset off[d], rho =
// desc[d].cols): the Jacobi left Zr = Z R in place (desc[d].A, od x rho), R in desc[d].V
// (rho x rho) and the descending order of Zr's column norms in desc[d].sig / perm.  Output
// column q takes original column j = perm[q]:
//   Otmp(:, q) = Zr(:, j) / sig_q          (blockIdx.x == 0 tiles: od entries)
//   Ktmp(:, q) = K(:, 0..rho-1) R(:, j)   (kd entries, a tiled product over rho)
//   S(q) = sig_q
// Thread (tx, ty) owns entries c0 + tx + 16 e of columns q0 + ty + 16 f.
template <typename T>
__global__ void __launch_bounds__(NT) rotate_back_kernel(const SliceDesc *__restrict__ desc,
                                                         const int64_t *__restrict__ off,
                                                         int64_t kd, int64_t od,
                                                         const T *__restrict__ Kin,
                                                         T *__restrict__ Ktmp,
                                                         T *__restrict__ Otmp, T *__restrict__ S) {
  __shared__ T Ks[CK][CT + 1];
  __shared__ T Rs[CK][CT + 1];
  const SliceDesc d = desc[blockIdx.z];
  const int rho = d.cols;
  const int64_t q0 = (int64_t)blockIdx.y * CT;
  if (q0 >= rho) return;
  const int64_t base = off[blockIdx.z];
  const T *R = reinterpret_cast<const T *>(d.V);
  const T *sig = reinterpret_cast<const T *>(d.sig);
  const int *perm = d.perm;
  const int tid = threadIdx.x, tx = tid % 16, ty = tid / 16;
  if (blockIdx.x == 0) {
    // the other side: gather and scale whole columns
    const T *Zr = reinterpret_cast<const T *>(d.A);
    for (int f = 0; f < 4; ++f) {
      const int64_t q = q0 + ty + 16 * f;
      if (q >= rho) break;
      const int j = perm[q];
      const T sg = sig[q];
      const T inv = sg > T(0) ? T(1) / sg : T(0);
      for (int64_t c = tx; c < od; c += 16) Otmp[(base + q) * od + c] = Zr[(int64_t)j * od + c] * inv;
      if (tx == 0) S[base + q] = sg;
    }
  }
  if (blockIdx.x == 0) return;
  const int64_t c0 = (int64_t)(blockIdx.x - 1) * CT;
  T acc[4][4];
#pragma unroll
  for (int e = 0; e < 4; ++e)
#pragma unroll
    for (int f = 0; f < 4; ++f) acc[e][f] = T(0);
  for (int l0 = 0; l0 < rho; l0 += CK) {
#pragma unroll
    for (int u = 0; u < CK * CT / NT; ++u) {
      const int idx = tid + u * NT;
      // K(c, l): entries c contiguous
      const int l = idx / CT, c = idx % CT;
      const int64_t gl = l0 + l, gc = c0 + c;
      Ks[l][c] = (gl < rho && gc < kd) ? Kin[(base + gl) * kd + gc] : T(0);
      // R(l, perm q): l contiguous
      const int qq = idx / CK, ll = idx % CK;
      const int64_t gq = q0 + qq, gll = l0 + ll;
      Rs[ll][qq] = (gq < rho && gll < rho) ? R[(int64_t)perm[gq] * rho + gll] : T(0);
    }
    __syncthreads();
#pragma unroll 8
    for (int ll = 0; ll < CK; ++ll) {
      T a[4], r[4];
#pragma unroll
      for (int e = 0; e < 4; ++e) a[e] = Ks[ll][tx + 16 * e];
#pragma unroll
      for (int f = 0; f < 4; ++f) r[f] = Rs[ll][ty + 16 * f];
#pragma unroll
      for (int e = 0; e < 4; ++e)
#pragma unroll
        for (int f = 0; f < 4; ++f) acc[e][f] = fma(a[e], r[f], acc[e][f]);
    }
    __syncthreads();
  }
#pragma unroll
  for (int f = 0; f < 4; ++f) {
    const int64_t q = q0 + ty + 16 * f;
    if (q >= rho) continue;
#pragma unroll
    for (int e = 0; e < 4; ++e) {
      const int64_t c = c0 + tx + 16 * e;
      if (c < kd) Ktmp[(base + q) * kd + c] = acc[e][f];
    }
  }
}

template <typename T>
__device__ __forceinline__ void take_max(T a, int i, T &bv, int &bi) {
  if (a > bv || (a == bv && i < bi)) {
    bv = a;
    bi = i;
  }
}

// Index of the largest |x[0 .. n-1]| (first on ties) over the block, -1 if all are zero.
template <typename T>
__device__ int block_argmax_abs(const T *x, int64_t n) {
  __shared__ T sv[NT / 32];
  __shared__ int si[NT / 32];
  __shared__ int res;
  T bv = T(-1);
  int bi = 0x7fffffff;
  for (int64_t a = threadIdx.x; a < n; a += NT) take_max(fabs(x[a]), (int)a, bv, bi);
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) {
    const T ov = __shfl_xor_sync(0xffffffffu, bv, o);
    const int oi = __shfl_xor_sync(0xffffffffu, bi, o);
    take_max(ov, oi, bv, bi);
  }
  if ((threadIdx.x & 31) == 0) {
    sv[threadIdx.x >> 5] = bv;
    si[threadIdx.x >> 5] = bi;
  }
  __syncthreads();
  if (threadIdx.x == 0) {
    T b = T(-1);
    int i = 0x7fffffff;
    for (int w = 0; w < NT / 32; ++w) take_max(sv[w], si[w], b, i);
    res = b > T(0) ? i : -1;
  }
  __syncthreads();
  const int r = res;
  __syncthreads();
  return r;
}

template <typename T>
__global__ void __launch_bounds__(NT) signfix_kernel(int64_t n1, int64_t n2, int64_t k_uniform,
                                                     const int *__restrict__ ranks,
                                                     const int64_t *__restrict__ offsets,
                                                     T *U, T *V) {
  const int64_t slice = blockIdx.y, j = blockIdx.x;
  const int64_t cnt = ranks ? (int64_t)ranks[slice] : k_uniform;
  if (j >= cnt) return;
  const int64_t col = (offsets ? offsets[slice] : slice * k_uniform) + j;
  T *u = U + col * n1, *v = V + col * n2;
  int i = block_argmax_abs(u, n1);
  T ref = T(1);
  if (i >= 0) {
    ref = u[i];
  } else {
    i = block_argmax_abs(v, n2);
    if (i >= 0) ref = v[i];
  }
  if (ref < T(0)) {
    for (int64_t a = threadIdx.x; a < n1; a += NT) u[a] = -u[a];
    for (int64_t b = threadIdx.x; b < n2; b += NT) v[b] = -v[b];
  }
}

}  // namespace

template <typename T>
cudaError_t complete_vectors(const T *Ahat, int64_t n1, int64_t n2, int64_t nslices,
                             bool transposed, int64_t k_uniform, const int *ranks,
                             const int64_t *offsets, int64_t max_rank, T *U, const T *S, T *V,
                             cudaStream_t st) {
  if (nslices <= 0 || max_rank <= 0) return cudaSuccess;
  const int64_t od = transposed ? n1 : n2;
  dim3 grid((unsigned)((od + CT - 1) / CT), (unsigned)((max_rank + CT - 1) / CT),
            (unsigned)nslices);
  complete_kernel<T><<<grid, NT, 0, st>>>(Ahat, n1, n2, transposed, k_uniform, ranks, offsets,
                                          transposed ? V : U, S, transposed ? U : V);
  return cudaGetLastError();
}

template <typename T>
cudaError_t rotate_back(const SliceDesc *desc, const int64_t *off, int count, int max_rho,
                        int64_t kd, int64_t od, const T *Kin, T *Ktmp, T *Otmp, T *S,
                        cudaStream_t st, bool gather_only) {
  if (count <= 0 || max_rho <= 0) return cudaSuccess;
  // gather_only: Otmp and S alone (Ktmp = K R is formed elsewhere)
  dim3 grid((unsigned)(gather_only ? 1 : 1 + (kd + CT - 1) / CT),
            (unsigned)((max_rho + CT - 1) / CT), (unsigned)count);
  rotate_back_kernel<T><<<grid, NT, 0, st>>>(desc, off, kd, od, Kin, Ktmp, Otmp, S);
  return cudaGetLastError();
}

template <typename T>
cudaError_t emit_signfix(int64_t n1, int64_t n2, int64_t nslices, int64_t k_uniform,
                         const int *ranks, const int64_t *offsets, int64_t max_rank, T *U, T *V,
                         cudaStream_t st) {
  if (nslices <= 0 || max_rank <= 0) return cudaSuccess;
  signfix_kernel<T><<<dim3((unsigned)max_rank, (unsigned)nslices), NT, 0, st>>>(
      n1, n2, k_uniform, ranks, offsets, U, V);
  return cudaGetLastError();
}

#define INST(T)                                                                                \
  template cudaError_t complete_vectors<T>(const T *, int64_t, int64_t, int64_t, bool, int64_t, \
                                           const int *, const int64_t *, int64_t, T *,          \
                                           const T *, T *, cudaStream_t);                       \
  template cudaError_t emit_signfix<T>(int64_t, int64_t, int64_t, int64_t, const int *,         \
                                       const int64_t *, int64_t, T *, T *, cudaStream_t);      \
  template cudaError_t rotate_back<T>(const SliceDesc *, const int64_t *, int, int, int64_t,    \
                                      int64_t, const T *, T *, T *, T *, cudaStream_t, bool);
INST(float)
INST(double)
#undef INST

}  // namespace tsvdm
