// Internal declarations shared by the CUDA translation units of libtsvdm.
#pragma once
#include <cuda_runtime.h>
#include <stdint.h>

#include "tsvdm.h"

namespace tsvdm {

// Device status word bits (OR-ed by kernels, read back by the host).
enum : int {
  ST_NOCONV = 1,
  ST_NONFINITE = 2,
  ST_TIMEOUT = 4,
};

// Device scalars kept in the plan (FP64).
enum : int {
  SC_XNORM2 = 0,    // ||X||_F^2
  SC_TOTAL = 1,     // sum of all sigma^2
  SC_DISCARD = 2,   // sum of discarded sigma^2
  SC_TAU = 3,       // t-SVDM-II threshold (a sigma^2 value)
  SC_E = 4,         // backward: ||R||_F^2
  SC_ALPHA = 5,     // backward: scale of the adjoint TTM
  SC_BETA = 6,      // backward: scale of X in dX
  SC_LOSS = 7,      // backward: L
  SC_TOTRANK = 8,   // t-SVDM-II: total rank (as double, exact below 2^53)
  SC_COUNT = 16
};

// ---- launch helpers implemented in the .cu files (all asynchronous on `st`) ----

// Mode-3 TTM as a (P x n) x (n x J) product.  B(t,i) = M[i + ldm*t] (forward, M is J x n)
// or M[t + ldm*i] (transB, M^T applied).  `scale_ptr` (device double, nullable) multiplies
// the product; `beta_ptr` (device double, nullable) adds beta * Z[row + P*i] (Z same shape
// as Y).  `sumsq` (device double, nullable) accumulates sum over X of x^2.
template <typename T>
cudaError_t ttm_simt(const T *X, int64_t P, int64_t n, const T *M, int64_t ldm, int64_t J,
                     bool transB, T *Y, const double *scale_ptr, const double *beta_ptr,
                     const T *Z, double *sumsq, cudaStream_t st);

// Tensor-core (tcgen05) TTM in BF16x3 or TF32, FP32 accumulation; same semantics as
// ttm_simt with ldm = n for the forward case (M is J x n, J <= 512).  Returns
// cudaErrorNotSupported when the shape or alignment cannot use it.
size_t ttm_tc_workspace(int64_t n, int64_t J);
bool ttm_tc_supported(int64_t P, int64_t n, int64_t J, const void *X, const void *Y);
cudaError_t ttm_tc(const float *X, int64_t P, int64_t n, const float *M, int64_t J, bool transB,
                   int prec, float *Y, void *ws, size_t ws_bytes, double *sumsq,
                   const double *scale_ptr, const double *beta_ptr, const float *Z, int *status,
                   cudaStream_t st);

// Orthonormal DCT-II (inverse: its transpose, DCT-III) along mode 3 of `batch` consecutive
// P x n column-major views (view q at X + q P n), n a power of two <= 4096, from the
// twiddle tables of dct_tables (device); Y must not overlap X.
template <typename T>
cudaError_t dct_mode3(const T *X, int64_t P, int64_t n, int64_t batch, bool inverse,
                      const void *tables, T *Y, cudaStream_t st);
// Elements (complex pairs) of the tables of one mode length n: n/2 forward and n/2 inverse
// FFT twiddles, n post-twiddles (forward) and n pre-twiddles (inverse).
inline int64_t dct_table_pairs(int64_t n) { return 2 * (n > 1 ? n / 2 : 1) + 2 * n; }

// Transposed copy of each m x p slice (rows x cols) into p x m.
template <typename T>
cudaError_t transpose_slices(const T *A, int64_t m, int64_t p, int64_t nslices, T *B,
                             cudaStream_t st);

// One slice of a batched decomposition (tensors of different shapes in one launch).
struct SliceDesc {
  void *A;             // rows x cols work matrix (column-major, lda = rows)
  void *V;             // cols x cols rotations
  float *norm2;        // cols squared norms (de Rijk ordering)
  void *sig;           // cols sorted singular values (finalize output)
  int *perm;           // cols column permutation (finalize output)
  int rows, cols;
};

struct JacobiParams {
  void *A;             // slice s work matrix at A + s*sA: rows x cols, column-major
  void *V;             // slice s rotations at V + s*sV: cols x cols
  int64_t sA, sV;
  int rows, cols;      // rows >= cols
  int nslices;
  double tol;
  int max_sweeps;
  int *queue;          // slice counter, zeroed before the launch
  int *status;         // status word
  int *sweeps;         // [nslices] sweeps executed (-1 = cap reached)
  long long *rots;     // [nslices] rotations applied
  float *norm2;        // [nslices * cols] squared column norms (nullptr: natural order)
  int inner_sweeps;    // Gram sweeps per block pair (>= 1)
  const SliceDesc *desc; // per-slice matrices (batched), or nullptr (uniform, A/V/sA/sV)
  int engine;          // JACOBI_AUTO / JACOBI_FMA / JACOBI_TC (Gram and apply products)
  void *sched;         // tensor-core kernel's scheduler state (jacobi_sched_bytes), zeroed
  size_t sched_bytes;  //   by jacobi_run before the launch
  int max_cols;        // largest cols of any slice (sizes the scheduler state)
  int warm;            // 1: V already holds the starting rotation (warm start), keep it
  int angle32;         // FP32 slices: 1 = rotation test and angle in FP32, 0 = in FP64
  long long wait_polls;  // polls of the tensor-core kernel's dependency and idle waits
                         //   (0 = the default bound)
  int novec;           // 1: no right vectors (V is neither initialised nor rotated)
};
enum { JACOBI_AUTO = 0, JACOBI_FMA = 1, JACOBI_TC = 2 };

template <typename T>
cudaError_t jacobi_run(const JacobiParams &p, cudaStream_t st, int width_hint, int cluster_hint,
                       int grid_hint, int stages);
// Scheduler state of the tensor-core Jacobi for nslices slices of at most max_cols columns.
size_t jacobi_sched_bytes(int64_t nslices, int64_t max_cols);

// sigma (sorted descending) and the column permutation of each slice.
template <typename T>
cudaError_t jacobi_finalize(const T *A, int64_t sA, int rows, int cols, int nslices, T *sig,
                            int *perm, cudaStream_t st);

template <typename T>
cudaError_t jacobi_finalize_desc(const SliceDesc *desc, int nslices, int max_cols,
                                 cudaStream_t st);

// Writes normalised, sign-fixed factors of slices (see emit in jacobi.cu).  Vw == nullptr
// (a decomposition without right vectors): only the work matrix's side is written (U for
// non-transposed slices, sign-fixed; V for transposed ones, sign left to emit_signfix) and
// S; complete_vectors then forms the other side.
template <typename T>
cudaError_t emit_factors(const T *A, int64_t sA, const T *Vw, int64_t sV, int rows, int cols,
                         int nslices, bool transposed, const T *sig, const int *perm,
                         int64_t k_uniform, const int *ranks, const int64_t *offsets, T *U,
                         T *S, T *V, cudaStream_t st);
// Second pass of a decomposition without right vectors: for every emitted column j of slice
// i (uniform k, or packed ranks/offsets), the vector of the other side from the slice
// Ahat_i (n1 x n2, column-major, slices n1 n2 apart) and the emitted one:
//   non-transposed (n1 >= n2): V(:, j) = Ahat_i^T U(:, j) / S_j
//   transposed     (n1 <  n2): U(:, j) = Ahat_i   V(:, j) / S_j    (0 where S_j = 0)
template <typename T>
cudaError_t complete_vectors(const T *Ahat, int64_t n1, int64_t n2, int64_t nslices,
                             bool transposed, int64_t k_uniform, const int *ranks,
                             const int64_t *offsets, int64_t max_rank, T *U, const T *S, T *V,
                             cudaStream_t st);
// After the restricted Jacobi of the second pass (entries desc[0..count-1], Zr in place of
// the other side, R, sig and perm in the entry): the other side's columns Zr(:, perm q) /
// sig_q into Otmp, the emitted side rotated, K R(:, perm q), into Ktmp, sig_q into S
// (gather_only: Otmp and S alone).
template <typename T>
cudaError_t rotate_back(const SliceDesc *desc, const int64_t *off, int count, int max_rho,
                        int64_t kd, int64_t od, const T *Kin, T *Ktmp, T *Otmp, T *S,
                        cudaStream_t st, bool gather_only = false);
// Ktmp = K R(:, perm) of rotate_back for FP32 entries on the tensor cores (three-term BF16
// split, FP32-level accuracy).
cudaError_t rotate_tc(const SliceDesc *desc, const int64_t *off, int count, int64_t kd,
                      const float *Kin, float *Ktmp, int *status, cudaStream_t st);
// Sign rule after complete_vectors on transposed slices: the largest-magnitude entry of
// each U column positive (ties: the first), V flipped with it; a zero U column takes the
// sign of its V column.
template <typename T>
cudaError_t emit_signfix(int64_t n1, int64_t n2, int64_t nslices, int64_t k_uniform,
                         const int *ranks, const int64_t *offsets, int64_t max_rank, T *U, T *V,
                         cudaStream_t st);

// t-SVDM-II selection (Algorithm 2) on the sorted singular values sig (cols x nslices),
// over the whole GPU (select_launches kernels and one memset).  ws holds
// select_workspace_bytes(cols, nslices) bytes; status (nullable) receives ST_NONFINITE for
// NaN, infinite or negative values.
size_t select_workspace_bytes(int64_t cols, int64_t nslices);
int select_launches(bool fp64);
template <typename T>
cudaError_t select_ranks(const T *sig, int cols, int nslices, double eps, void *ws,
                         double *scal, int *ranks, int64_t *offsets, int *status,
                         cudaStream_t st);

// The selection of one t-SVDM-II tensor of a batch (one CTA each).
struct SelectSeg {
  const void *sig;     // cols x nslices, descending per slice
  int cols, nslices;
  double eps;
  void *keys;          // 2 * cols * nslices 64-bit keys
  double *scal;        // SC_COUNT scalars
  int *ranks;
  int64_t *offsets;
};
template <typename T>
cudaError_t select_segments(const SelectSeg *segs, int count, cudaStream_t st);
template <typename T>
cudaError_t trunc_sums(const T *sig, int cols, int nslices, int64_t k, double *scal,
                       cudaStream_t st);

// Per-slice product Out_i = [Base_i -] U_i diag(S_i) V_i^T.
template <typename T>
cudaError_t slice_products(const T *U, const T *S, const T *V, const int64_t *offsets,
                           int64_t k, int64_t n1, int64_t n2, int64_t n3, T *Out,
                           bool subtract_from_out, double *sumsq, cudaStream_t st);
// The same product for FP32 factors on the tensor cores (three-term BF16 split, FP32-level
// accuracy); a bounded wait that runs out sets ST_TIMEOUT in *status.
cudaError_t slice_products_tc(const float *U, const float *S, const float *V,
                              const int64_t *offsets, int64_t k, int64_t n1, int64_t n2,
                              int64_t n3, float *Out, bool subtract_from_out, double *sumsq,
                              int *status, cudaStream_t st, bool vtrans = false);
// Out_i = A_i V_i for column-major A_i (rows x cols) and V_i (cols x cols), slice strides
// rows*cols and cols*cols (the warm start of the slice SVDs): the slice product with S = 1
// and V read transposed.
template <typename T>
cudaError_t slice_rotate(const T *A, const T *V, int64_t rows, int64_t cols, int64_t n3, T *Out,
                         bool tensor_cores, int *status, cudaStream_t st);

// C (n x n) = alpha * A^T B with A, B column-major P x n; split over P; alpha from device.
template <typename T>
cudaError_t gemm_atb(const T *A, const T *B, int64_t P, int64_t n, T *C, const double *alpha,
                     double *ws, size_t ws_elems, cudaStream_t st);

// Z_i = A_i^T K_i diag(1 / S_i) of complete_vectors for FP32 slices in the column layout on
// the tensor cores (three-term BF16 split, FP32-level accuracy); complete_tc_supported says
// whether the layout and alignment allow it.
bool complete_tc_supported(const float *Ahat, const float *K, int64_t n1, int64_t n2,
                           bool transposed);
cudaError_t complete_tc(const float *Ahat, int64_t n1, int64_t n2, int64_t nslices,
                        int64_t k_uniform, const int *ranks, const int64_t *offsets,
                        const float *K, const float *S, float *O, int *status, cudaStream_t st);

// The same product for FP32 operands on the tensor cores (BF16x3, FP32 accumulation, FP64
// split sums); n <= 512, P a multiple of 4, 16-byte aligned operands (atb_tc_supported).
bool atb_tc_supported(const float *A, const float *B, int64_t P, int64_t n);
cudaError_t atb_tc(const float *A, const float *B, int64_t P, int64_t n, float *C,
                   const double *alpha, double *ws, size_t ws_elems, int *status,
                   cudaStream_t st);

template <typename T>
cudaError_t sumsq(const T *X, int64_t count, double *out, cudaStream_t st);

cudaError_t backward_scalars(double *scal, double dL, cudaStream_t st);

// Orthogonality defect and squared norm of M's first column (scale of M^{-1} = M^T/c^2).
template <typename T>
cudaError_t inv_scale(const T *M, int64_t n, double *out, cudaStream_t st);

template <typename T>
cudaError_t small_cayley(int64_t n, const T *A, const T *M0, T *M, T *Z, T *Q, T *work,
                         cudaStream_t st);
template <typename T>
cudaError_t small_cayley_backward(int64_t n, const T *M0, const T *Z, const T *Q, const T *dM,
                                  T *dA, T *work, cudaStream_t st);
template <typename T>
cudaError_t small_adam(int64_t count, T *param, const T *grad, T *m1, T *m2, int64_t step,
                       double lr, double b1, double b2, double eps, cudaStream_t st);

}  // namespace tsvdm
