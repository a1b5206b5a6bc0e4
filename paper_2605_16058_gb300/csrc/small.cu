// Small dense n x n kernels for the learned orthogonal transform (an extension of the
// paper, whose M is user-supplied, Sec. 2.2 "Choice of M"):
//   Cayley map   W = A^T - A,  Z = (I + W)^{-1} (Gauss-Jordan, no pivoting: the symmetric
//                part of I + W is I, so every leading minor is positive),
//                Q = Z (I - W),  M = Q M0;
//   its adjoint  dQ = dM M0^T,  dW = -Z^T dQ (Q + I)^T,  dA = dW^T - dW;
//   Adam         (Kingma & Ba) elementwise update.
#include "common.cuh"

namespace tsvdm {
namespace {

// C = op(A) op(B) (+ diag shift handled by callers), one thread per output.
// opA(i,l) = transA ? A[l + n i] : A[i + n l]
template <typename T>
__global__ void small_gemm_kernel(int64_t n, const T *A, bool transA, const T *B, bool transB,
                                  T *C, T alpha) {
  int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  int64_t j = blockIdx.y;
  if (i >= n) return;
  T acc = T(0);
  for (int64_t l = 0; l < n; ++l) {
    T a = transA ? A[l + n * i] : A[i + n * l];
    T b = transB ? B[j + n * l] : B[l + n * j];
    acc = fma(a, b, acc);
  }
  C[i + n * j] = alpha * acc;
}

// work (n x 2n, column-major: [I + W | I]) -> Gauss-Jordan -> Z = right half
template <typename T>
__global__ void __launch_bounds__(1024) cayley_gj_kernel(int64_t n, const T *Ain, T *aug, T *Z,
                                                         T *ImW) {
  const int64_t ld = n;
  for (int64_t idx = threadIdx.x; idx < n * n; idx += blockDim.x) {
    int64_t i = idx % n, j = idx / n;
    T w = Ain[j + n * i] - Ain[i + n * j];      // W = A^T - A  (W[i,j] = A[j,i] - A[i,j])
    aug[i + ld * j] = (i == j ? T(1) : T(0)) + w;
    aug[i + ld * (n + j)] = (i == j) ? T(1) : T(0);
    ImW[i + n * j] = (i == j ? T(1) : T(0)) - w;
  }
  __syncthreads();
  __shared__ T s_piv;
  for (int64_t k = 0; k < n; ++k) {
    if (threadIdx.x == 0) s_piv = T(1) / aug[k + ld * k];
    __syncthreads();
    const T pinv = s_piv;
    for (int64_t j = threadIdx.x; j < 2 * n; j += blockDim.x) aug[k + ld * j] *= pinv;
    __syncthreads();
    for (int64_t idx = threadIdx.x; idx < n * 2 * n; idx += blockDim.x) {
      int64_t i = idx % n, j = idx / n;
      if (i == k) continue;
      T f = aug[i + ld * k];
      if (j == k) continue;
      aug[i + ld * j] -= f * aug[k + ld * j];
    }
    __syncthreads();
    for (int64_t i = threadIdx.x; i < n; i += blockDim.x)
      if (i != k) aug[i + ld * k] = T(0);
    __syncthreads();
  }
  for (int64_t idx = threadIdx.x; idx < n * n; idx += blockDim.x) {
    int64_t i = idx % n, j = idx / n;
    Z[i + n * j] = aug[i + ld * (n + j)];
  }
}

template <typename T>
__global__ void add_identity_kernel(int64_t n, const T *Q, T *out) {
  int64_t idx = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (idx >= n * n) return;
  out[idx] = Q[idx] + ((idx % n) == (idx / n) ? T(1) : T(0));
}

template <typename T>
__global__ void skew_grad_kernel(int64_t n, const T *dW, T *dA) {
  int64_t idx = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (idx >= n * n) return;
  int64_t i = idx % n, j = idx / n;
  dA[idx] = dW[j + n * i] - dW[idx];
}

template <typename T>
__global__ void adam_kernel(int64_t count, T *p, const T *g, T *m1, T *m2, double lr, double b1,
                            double b2, double eps, double c1, double c2) {
  int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= count) return;
  double gi = (double)g[i];
  double a = b1 * (double)m1[i] + (1.0 - b1) * gi;
  double b = b2 * (double)m2[i] + (1.0 - b2) * gi * gi;
  m1[i] = (T)a;
  m2[i] = (T)b;
  double mh = a / c1, vh = b / c2;
  p[i] = (T)((double)p[i] - lr * mh / (sqrt(vh) + eps));
}

template <typename T>
cudaError_t gemm_small(int64_t n, const T *A, bool tA, const T *B, bool tB, T *C, T alpha,
                       cudaStream_t st) {
  dim3 grid((unsigned)((n + 127) / 128), (unsigned)n);
  small_gemm_kernel<T><<<grid, 128, 0, st>>>(n, A, tA, B, tB, C, alpha);
  return cudaGetLastError();
}

}  // namespace

template <typename T>
cudaError_t small_cayley(int64_t n, const T *A, const T *M0, T *M, T *Z, T *Q, T *work,
                         cudaStream_t st) {
  // work: the n x 2n augmented matrix [I + W | I]; M temporarily holds I - W.
  cayley_gj_kernel<T><<<1, 1024, 0, st>>>(n, A, work, Z, M);
  cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) return e;
  if ((e = gemm_small<T>(n, Z, false, M, false, Q, T(1), st)) != cudaSuccess) return e;
  return gemm_small<T>(n, Q, false, M0, false, M, T(1), st);
}

template <typename T>
cudaError_t small_cayley_backward(int64_t n, const T *M0, const T *Z, const T *Q, const T *dM,
                                  T *dA, T *work, cudaStream_t st) {
  // work: 3 n^2
  T *dQ = work, *T1 = work + n * n, *QpI = work + 2 * n * n;
  cudaError_t e;
  if ((e = gemm_small<T>(n, dM, false, M0, true, dQ, T(1), st)) != cudaSuccess) return e;
  if ((e = gemm_small<T>(n, Z, true, dQ, false, T1, T(1), st)) != cudaSuccess) return e;
  add_identity_kernel<T><<<(unsigned)((n * n + 255) / 256), 256, 0, st>>>(n, Q, QpI);
  if ((e = cudaGetLastError()) != cudaSuccess) return e;
  // dW = -T1 (Q+I)^T  -> store in dQ
  if ((e = gemm_small<T>(n, T1, false, QpI, true, dQ, T(-1), st)) != cudaSuccess) return e;
  skew_grad_kernel<T><<<(unsigned)((n * n + 255) / 256), 256, 0, st>>>(n, dQ, dA);
  return cudaGetLastError();
}

template <typename T>
cudaError_t small_adam(int64_t count, T *param, const T *grad, T *m1, T *m2, int64_t step,
                       double lr, double b1, double b2, double eps, cudaStream_t st) {
  double c1 = 1.0 - pow(b1, (double)step), c2 = 1.0 - pow(b2, (double)step);
  adam_kernel<T><<<(unsigned)((count + 255) / 256), 256, 0, st>>>(count, param, grad, m1, m2, lr,
                                                                  b1, b2, eps, c1, c2);
  return cudaGetLastError();
}

#define INST(T)                                                                             \
  template cudaError_t small_cayley<T>(int64_t, const T *, const T *, T *, T *, T *, T *,   \
                                       cudaStream_t);                                       \
  template cudaError_t small_cayley_backward<T>(int64_t, const T *, const T *, const T *,   \
                                                const T *, T *, T *, cudaStream_t);         \
  template cudaError_t small_adam<T>(int64_t, T *, const T *, T *, T *, int64_t, double,    \
                                     double, double, double, cudaStream_t);
INST(float)
INST(double)
#undef INST

}  // namespace tsvdm
