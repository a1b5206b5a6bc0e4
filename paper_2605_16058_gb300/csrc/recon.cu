// Slice-wise products for reconstruction and the backward pass.
//
//  slice_products: Out_i = U_i diag(S_i) V_i^T  (or Out_i -= ...), the facewise product of
//    the star-M product (Sec. 2.1, second step) for the factors of t-SVDM-I (uniform k) or
//    t-SVDM-II (packed, slice i's columns at offsets[i]..offsets[i+1]-1).  64 x 64 output
//    tiles per CTA, K (rank) steps of 16.  Optionally accumulates ||Out||_F^2 in FP64.
//  gemm_atb: C = alpha A^T B for column-major P x n operands (the n x n gradient
//    R_(mat)^T X_(mat)), split over P into partial tiles that are summed in a fixed order
//    in FP64.
#include "common.cuh"

namespace tsvdm {
namespace {

constexpr int TM = 64, TN = 64, TK = 16, NT = 256;

template <typename T>
__global__ void __launch_bounds__(NT) slice_products_kernel(
    const T *__restrict__ U, const T *__restrict__ S, const T *__restrict__ V,
    const int64_t *__restrict__ offsets, int64_t k, int64_t n1, int64_t n2, T *__restrict__ Out,
    bool subtract, double *sumsq, bool vtrans) {
  __shared__ __align__(16) T Us[TK][TM];
  __shared__ __align__(16) T Vs[TK][TN];
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  const int64_t slice = blockIdx.z;
  const int64_t a0 = (int64_t)blockIdx.x * TM, b0 = (int64_t)blockIdx.y * TN;
  const int64_t c0 = offsets ? offsets[slice] : slice * k;
  const int64_t cnt = offsets ? offsets[slice + 1] - c0 : k;
  T acc[2][8];
#pragma unroll
  for (int q = 0; q < 2; ++q)
#pragma unroll
    for (int e = 0; e < 8; ++e) acc[q][e] = T(0);
  for (int64_t q0 = 0; q0 < cnt; q0 += TK) {
#pragma unroll
    for (int u = 0; u < TK * TM / NT; ++u) {
      int idx = tid + u * NT;
      int t = idx / TM, r = idx % TM;
      int64_t a = a0 + r, c = q0 + t;
      T v = T(0);
      if (a < n1 && c < cnt) v = U[(c0 + c) * n1 + a] * (S ? S[c0 + c] : T(1));
      Us[t][r] = v;
    }
#pragma unroll
    for (int u = 0; u < TK * TN / NT; ++u) {
      int idx = tid + u * NT;
      int t = idx / TN, r = idx % TN;
      int64_t b = b0 + r, c = q0 + t;
      T v = T(0);
      if (b < n2 && c < cnt) v = vtrans ? V[c0 * n2 + b * k + c] : V[(c0 + c) * n2 + b];
      Vs[t][r] = v;
    }
    __syncthreads();
#pragma unroll
    for (int kk = 0; kk < TK; ++kk) {
      T x[2], y[8];
#pragma unroll
      for (int q = 0; q < 2; ++q) x[q] = Us[kk][lane + 32 * q];
#pragma unroll
      for (int e = 0; e < 8; ++e) y[e] = Vs[kk][warp * 8 + e];
#pragma unroll
      for (int q = 0; q < 2; ++q)
#pragma unroll
        for (int e = 0; e < 8; ++e) acc[q][e] = fma(x[q], y[e], acc[q][e]);
    }
    __syncthreads();
  }
  double ss = 0.0;
  T *O = Out + slice * n1 * n2;
#pragma unroll
  for (int e = 0; e < 8; ++e) {
    int64_t b = b0 + warp * 8 + e;
    if (b >= n2) continue;
#pragma unroll
    for (int q = 0; q < 2; ++q) {
      int64_t a = a0 + lane + 32 * q;
      if (a >= n1) continue;
      T v = subtract ? O[a + n1 * b] - acc[q][e] : acc[q][e];
      O[a + n1 * b] = v;
      ss += (double)v * (double)v;
    }
  }
  if (sumsq) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) ss += __shfl_xor_sync(0xffffffffu, ss, o);
    if (lane == 0) atomicAdd(sumsq, ss);
  }
}

template <typename T>
__global__ void __launch_bounds__(NT) atb_partial_kernel(const T *__restrict__ A,
                                                         const T *__restrict__ B, int64_t P,
                                                         int64_t n, int64_t chunk,
                                                         double *__restrict__ ws) {
  __shared__ __align__(16) T As[TK][TM];
  __shared__ __align__(16) T Bs[TK][TN];
  const int tid = threadIdx.x;
  const int ti = tid % 16, tj = tid / 16;      // 4 x 4 outputs: rows ti + 16 e, cols tj + 16 f
  const int64_t i0 = (int64_t)blockIdx.x * TM, j0 = (int64_t)blockIdx.y * TN;
  const int64_t rbeg = (int64_t)blockIdx.z * chunk;
  const int64_t rend = rbeg + chunk < P ? rbeg + chunk : P;
  T acc[4][4];
#pragma unroll
  for (int e = 0; e < 4; ++e)
#pragma unroll
    for (int f = 0; f < 4; ++f) acc[e][f] = T(0);
  for (int64_t r0 = rbeg; r0 < rend; r0 += TK) {
#pragma unroll
    for (int u = 0; u < TK * TM / NT; ++u) {
      int idx = tid + u * NT;
      int c = idx / TK, r = idx % TK;     // consecutive threads walk rows of one column
      int64_t row = r0 + r;
      T va = T(0), vb = T(0);
      if (row < rend) {
        if (i0 + c < n) va = A[row + P * (i0 + c)];
        if (j0 + c < n) vb = B[row + P * (j0 + c)];
      }
      As[r][c] = va;
      Bs[r][c] = vb;
    }
    __syncthreads();
#pragma unroll
    for (int kk = 0; kk < TK; ++kk) {
      T x[4], y[4];
#pragma unroll
      for (int e = 0; e < 4; ++e) x[e] = As[kk][ti + 16 * e];
#pragma unroll
      for (int f = 0; f < 4; ++f) y[f] = Bs[kk][tj + 16 * f];
#pragma unroll
      for (int e = 0; e < 4; ++e)
#pragma unroll
        for (int f = 0; f < 4; ++f) acc[e][f] = fma(x[e], y[f], acc[e][f]);
    }
    __syncthreads();
  }
  double *out = ws + (int64_t)blockIdx.z * n * n;
#pragma unroll
  for (int e = 0; e < 4; ++e)
#pragma unroll
    for (int f = 0; f < 4; ++f) {
      int64_t i = i0 + ti + 16 * e, j = j0 + tj + 16 * f;
      if (i < n && j < n) out[i + n * j] = (double)acc[e][f];
    }
}

template <typename T>
__global__ void atb_reduce_kernel(const double *__restrict__ ws, int64_t n, int64_t splits,
                                  const double *alpha, T *C) {
  int64_t idx = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (idx >= n * n) return;
  double s = 0.0;
  for (int64_t z = 0; z < splits; ++z) s += ws[z * n * n + idx];
  C[idx] = (T)(s * (alpha ? *alpha : 1.0));
}

// scal[SC_E] = ||R||^2, scal[SC_XNORM2] = ||X||^2  ->  L, alpha, beta
__global__ void backward_scalars_kernel(double *scal, double dL) {
  double E = scal[SC_E], x2 = scal[SC_XNORM2];
  if (E > 0.0 && x2 > 0.0) {
    double xn = sqrt(x2), rE = sqrt(E);
    double L = rE / xn;
    scal[SC_LOSS] = L;
    scal[SC_ALPHA] = dL / (rE * xn);
    scal[SC_BETA] = -dL * L / x2;
  } else {
    scal[SC_LOSS] = 0.0;
    scal[SC_ALPHA] = 0.0;
    scal[SC_BETA] = 0.0;
  }
}

}  // namespace

template <typename T>
cudaError_t slice_products(const T *U, const T *S, const T *V, const int64_t *offsets,
                           int64_t k, int64_t n1, int64_t n2, int64_t n3, T *Out,
                           bool subtract_from_out, double *sumsq, cudaStream_t st) {
  dim3 grid((unsigned)((n1 + TM - 1) / TM), (unsigned)((n2 + TN - 1) / TN), (unsigned)n3);
  slice_products_kernel<T><<<grid, NT, 0, st>>>(U, S, V, offsets, k, n1, n2, Out,
                                                subtract_from_out, sumsq, false);
  return cudaGetLastError();
}

template <typename T>
cudaError_t slice_rotate(const T *A, const T *V, int64_t rows, int64_t cols, int64_t n3, T *Out,
                         bool tensor_cores, int *status, cudaStream_t st) {
  if constexpr (sizeof(T) == 4) {
    if (tensor_cores)
      return slice_products_tc(A, nullptr, V, nullptr, cols, rows, cols, n3, Out, false,
                               nullptr, status, st, true);
  }
  dim3 grid((unsigned)((rows + TM - 1) / TM), (unsigned)((cols + TN - 1) / TN), (unsigned)n3);
  slice_products_kernel<T><<<grid, NT, 0, st>>>(A, nullptr, V, nullptr, cols, rows, cols, Out,
                                                false, nullptr, true);
  return cudaGetLastError();
}

template <typename T>
cudaError_t gemm_atb(const T *A, const T *B, int64_t P, int64_t n, T *C, const double *alpha,
                     double *ws, size_t ws_elems, cudaStream_t st) {
  int64_t splits = (int64_t)(ws_elems / (size_t)(n * n));
  if (splits > 1024) splits = 1024;
  if (splits < 1) return cudaErrorInvalidValue;
  int64_t chunk = (P + splits - 1) / splits;
  chunk = (chunk + TK - 1) / TK * TK;
  splits = (P + chunk - 1) / chunk;
  dim3 grid((unsigned)((n + TM - 1) / TM), (unsigned)((n + TN - 1) / TN), (unsigned)splits);
  atb_partial_kernel<T><<<grid, NT, 0, st>>>(A, B, P, n, chunk, ws);
  cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) return e;
  atb_reduce_kernel<T><<<(unsigned)((n * n + 255) / 256), 256, 0, st>>>(ws, n, splits, alpha, C);
  return cudaGetLastError();
}

cudaError_t backward_scalars(double *scal, double dL, cudaStream_t st) {
  backward_scalars_kernel<<<1, 1, 0, st>>>(scal, dL);
  return cudaGetLastError();
}

#define INST(T)                                                                             \
  template cudaError_t slice_products<T>(const T *, const T *, const T *, const int64_t *,  \
                                         int64_t, int64_t, int64_t, int64_t, T *, bool,     \
                                         double *, cudaStream_t);                           \
  template cudaError_t slice_rotate<T>(const T *, const T *, int64_t, int64_t, int64_t, T *, \
                                       bool, int *, cudaStream_t);                          \
  template cudaError_t gemm_atb<T>(const T *, const T *, int64_t, int64_t, T *,             \
                                   const double *, double *, size_t, cudaStream_t);
INST(float)
INST(double)
#undef INST

}  // namespace tsvdm
