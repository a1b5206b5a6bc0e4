// Mode-3 tensor-times-matrix on CUDA cores (Sec. 2.1 definition, Sec. 3.1 "last-mode TTM
// is one GEMM"): the column-major n1 x n2 x n3 tensor is the (P = n1 n2) x n3 matrix X,
// and Y = X B with B(t, i) = M(i, t) (forward, Y = X x_3 M) or B(t, i) = M(t, i)
// (transB, Y = X x_3 M^T).  FP32 or FP64 FMA; 128 x 64 output tiles, k-steps of 16.
// Epilogue: Y = scale * (X B) + beta * Z with scale and beta read from device memory
// (so the backward pass needs no host round trip).  Optionally accumulates ||X||_F^2 in
// FP64 from the tiles it loads.
#include "common.cuh"

namespace tsvdm {
namespace {

constexpr int BM = 128, BN = 64, BK = 16, NT = 256;

template <typename T>
__global__ void __launch_bounds__(NT) ttm_kernel(const T *__restrict__ X, int64_t P, int64_t n,
                                                 const T *__restrict__ M, int64_t ldm, int64_t J,
                                                 bool transB, T *__restrict__ Y,
                                                 const double *scale_ptr, const double *beta_ptr,
                                                 const T *__restrict__ Z, double *sumsq) {
  __shared__ __align__(16) T Xs[BK][BM];
  __shared__ __align__(16) T Bs[BK][BN];
  const int tid = threadIdx.x;
  const int lane = tid & 31, warp = tid >> 5;
  const int64_t row0 = (int64_t)blockIdx.x * BM;
  const int64_t col0 = (int64_t)blockIdx.y * BN;
  const bool do_sumsq = sumsq != nullptr && blockIdx.y == 0;
  double ss = 0.0;
  T acc[4][8];
#pragma unroll
  for (int q = 0; q < 4; ++q)
#pragma unroll
    for (int e = 0; e < 8; ++e) acc[q][e] = T(0);
  for (int64_t k0 = 0; k0 < n; k0 += BK) {
#pragma unroll
    for (int u = 0; u < BK * BM / NT; ++u) {
      int idx = tid + u * NT;
      int t = idx / BM, r = idx % BM;
      int64_t row = row0 + r, kt = k0 + t;
      T v = T(0);
      if (row < P && kt < n) v = X[row + P * kt];
      if (do_sumsq) ss += (double)v * (double)v;
      Xs[t][r] = v;
    }
#pragma unroll
    for (int u = 0; u < BK * BN / NT; ++u) {
      int idx = tid + u * NT;
      int t = idx / BN, c = idx % BN;
      int64_t kt = k0 + t, col = col0 + c;
      T v = T(0);
      if (kt < n && col < J) v = transB ? M[kt + ldm * col] : M[col + ldm * kt];
      Bs[t][c] = v;
    }
    __syncthreads();
#pragma unroll
    for (int kk = 0; kk < BK; ++kk) {
      T a[4], b[8];
#pragma unroll
      for (int q = 0; q < 4; ++q) a[q] = Xs[kk][lane + 32 * q];
#pragma unroll
      for (int e = 0; e < 8; ++e) b[e] = Bs[kk][warp * 8 + e];
#pragma unroll
      for (int q = 0; q < 4; ++q)
#pragma unroll
        for (int e = 0; e < 8; ++e) acc[q][e] = fma(a[q], b[e], acc[q][e]);
    }
    __syncthreads();
  }
  const T scale = scale_ptr ? (T)(*scale_ptr) : T(1);
  const T beta = beta_ptr ? (T)(*beta_ptr) : T(0);
#pragma unroll
  for (int e = 0; e < 8; ++e) {
    int64_t col = col0 + warp * 8 + e;
    if (col >= J) continue;
#pragma unroll
    for (int q = 0; q < 4; ++q) {
      int64_t row = row0 + lane + 32 * q;
      if (row >= P) continue;
      T v = scale * acc[q][e];
      if (Z) v = fma(beta, Z[row + P * col], v);
      Y[row + P * col] = v;
    }
  }
  if (do_sumsq) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) ss += __shfl_xor_sync(0xffffffffu, ss, o);
    if (lane == 0) atomicAdd(sumsq, ss);
  }
}

template <typename T>
__global__ void sumsq_kernel(const T *__restrict__ X, int64_t count, double *out) {
  double ss = 0.0;
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < count;
       i += (int64_t)gridDim.x * blockDim.x) {
    double v = (double)X[i];
    ss += v * v;
  }
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) ss += __shfl_xor_sync(0xffffffffu, ss, o);
  __shared__ double part[32];
  if ((threadIdx.x & 31) == 0) part[threadIdx.x >> 5] = ss;
  __syncthreads();
  if (threadIdx.x == 0) {
    double t = 0.0;
    for (int w = 0; w < (int)(blockDim.x >> 5); ++w) t += part[w];
    atomicAdd(out, t);
  }
}

// out[0] = 1 / ||M(:,0)||^2 (so that M^T * out[0] inverts a multiple of an orthogonal M)
template <typename T>
__global__ void inv_scale_kernel(const T *__restrict__ M, int64_t n, double *out) {
  double ss = 0.0;
  for (int64_t t = threadIdx.x; t < n; t += blockDim.x) {
    double v = (double)M[t];
    ss += v * v;
  }
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) ss += __shfl_xor_sync(0xffffffffu, ss, o);
  __shared__ double part[32];
  if ((threadIdx.x & 31) == 0) part[threadIdx.x >> 5] = ss;
  __syncthreads();
  if (threadIdx.x == 0) {
    double t = 0.0;
    for (int w = 0; w < (int)(blockDim.x >> 5); ++w) t += part[w];
    out[0] = t > 0.0 ? 1.0 / t : 0.0;
  }
}

}  // namespace

template <typename T>
cudaError_t ttm_simt(const T *X, int64_t P, int64_t n, const T *M, int64_t ldm, int64_t J,
                     bool transB, T *Y, const double *scale_ptr, const double *beta_ptr,
                     const T *Z, double *sumsq, cudaStream_t st) {
  if (P <= 0 || J <= 0) return cudaSuccess;
  dim3 grid((unsigned)((P + BM - 1) / BM), (unsigned)((J + BN - 1) / BN));
  ttm_kernel<T><<<grid, NT, 0, st>>>(X, P, n, M, ldm, J, transB, Y, scale_ptr, beta_ptr, Z,
                                     sumsq);
  return cudaGetLastError();
}

template <typename T>
cudaError_t sumsq(const T *X, int64_t count, double *out, cudaStream_t st) {
  if (count <= 0) return cudaSuccess;
  int64_t blocks = (count + 255) / 256;
  if (blocks > 152 * 8) blocks = 152 * 8;
  sumsq_kernel<T><<<(unsigned)blocks, 256, 0, st>>>(X, count, out);
  return cudaGetLastError();
}

template <typename T>
cudaError_t inv_scale(const T *M, int64_t n, double *out, cudaStream_t st) {
  inv_scale_kernel<T><<<1, 256, 0, st>>>(M, n, out);
  return cudaGetLastError();
}

#define INST(T)                                                                              \
  template cudaError_t ttm_simt<T>(const T *, int64_t, int64_t, const T *, int64_t, int64_t, \
                                   bool, T *, const double *, const double *, const T *,     \
                                   double *, cudaStream_t);                                  \
  template cudaError_t sumsq<T>(const T *, int64_t, double *, cudaStream_t);                 \
  template cudaError_t inv_scale<T>(const T *, int64_t, double *, cudaStream_t);
INST(float)
INST(double)
#undef INST

}  // namespace tsvdm
