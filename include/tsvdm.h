/*
 * tsvdm.h - C ABI of the GB300 (sm_103a) star-M truncated tensor SVD library.
 *
 * The operations follow arXiv 2605.16058 ("High-Performance star-M SVD for Big Data
 * Compression"):
 *   - mode-3 TTM  Ahat = A x_3 M                         (Sec. 2.1, Sec. 3.1)
 *   - t-SVDM-I: per-slice truncated SVD at uniform rank k (Sec. 3.3, Fig. 1)
 *   - t-SVDM-II: global sigma^2 threshold from a relative error tolerance, per-slice
 *     ranks rho_i and a variable-rank packed format       (Algorithm 2, Sec. 3.4)
 *   - reconstruction  X_k = (U S V^T per slice) x_3 M^{-1} (Sec. 2.1, Sec. 2.2)
 *   - the gradient of the truncation error with respect to X and M (an extension: the
 *     paper has no differentiation; see tsvdm_backward).
 *
 * Conventions shared by every entry point
 *   Layout   column-major throughout.  An n1 x n2 x n3 tensor X has X(a,b,t) at
 *            X[a + n1*b + n1*n2*t]; frontal slice t is contiguous (Sec. 3).  An n x n
 *            matrix M has M(i,t) at M[i + n*t]; row i of M forms output slice i.
 *   Types    dtype TSVDM_F32 means every tensor/matrix argument is float, TSVDM_F64
 *            means double.  Sizes are int64_t.
 *   Memory   tensor arguments are caller-owned.  Unless an entry point says otherwise
 *            they must be DEVICE pointers.  tsvdm_fixed_rank and tsvdm_tolerance also
 *            accept HOST pointers (pageable or pinned; detected per pointer): inputs
 *            are copied in and outputs copied out on the plan's stream, through
 *            staging buffers the plan allocates on the first such call and keeps.
 *            Calls that allocate device memory after plan creation (each once per
 *            plan, kept until tsvdm_plan_destroy): the first host-pointer call (staging),
 *            tsvdm_data_transform (its one-slice plan), tsvdm_plan_set_warm_start (enable),
 *            tsvdm_plan_set_vectors (SECOND_PASS) and tsvdm_plan_set_transform (DCT2
 *            tables); tsvdm_probe_peak allocates and frees
 *            a status word.  Every other call allocates nothing.
 *   Streams  work is enqueued on the plan's stream.  Calls return once the work is
 *            enqueued, except where a host output (rel_err, total_rank, loss) is
 *            requested: those calls synchronise the stream before returning.
 *   Errors   argument errors are detected on the host and returned at once, with
 *            nothing enqueued.  Errors found on the device (no convergence, non-finite
 *            values, a bounded wait that ran out) are recorded in the plan's status
 *            word; synchronous calls return them, and tsvdm_last_status() reads them
 *            after the caller has synchronised the stream.  No device code traps.
 *   Threads  a plan may be used by one host thread at a time.
 */
#ifndef TSVDM_H
#define TSVDM_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef enum {
  TSVDM_OK = 0,
  TSVDM_EINVAL = 1,      /* bad argument: sizes, null pointer, k outside [1, min(n1,n2)],
                            eps outside (0,1), dtype/precision mismatch               */
  TSVDM_ENOTORTHO = 2,   /* the operation needs an orthogonal M (t-SVDM-II, original-
                            domain factors) and the plan was not created with one     */
  TSVDM_ENOCONV = 3,     /* a slice's Jacobi iteration reached the sweep cap; outputs
                            are written from the last iterate                        */
  TSVDM_ENONFINITE = 4,  /* NaN or Inf met in the transformed slices                  */
  TSVDM_ETIMEOUT = 5,    /* a bounded device-side wait ran out                        */
  TSVDM_ENOMEM = 6,      /* device or pinned-host allocation failed                   */
  TSVDM_ECAPACITY = 7,   /* t-SVDM-II: the output capacity is below the total rank    */
  TSVDM_ECUDA = 8,       /* a CUDA runtime call failed                                */
  TSVDM_ENOTSUP = 9,     /* combination not supported (e.g. TF32 precision with F64)  */
  TSVDM_ESCRATCH = 10    /* the problem exceeds the fixed scratch of an allocation-free
                            entry point                                               */
} tsvdm_status;

typedef enum { TSVDM_F32 = 0, TSVDM_F64 = 1 } tsvdm_dtype;

/* Arithmetic of the mode-3 TTMs.  The slice SVDs run in the storage precision (FP32
 * data and rotations for F32, with the rotation angle and the convergence test in FP64;
 * FP64 for F64); see tsvdm_plan_set_engine for the engine of their dense products and
 * tsvdm_plan_set_angle_precision for the angle arithmetic.
 *   TSVDM_P_FP64    FP64 CUDA-core products (dtype F64 only)
 *   TSVDM_P_FP32    FP32 CUDA-core products (dtype F32)
 *   TSVDM_P_TF32    one TF32 tensor-core product, FP32 accumulation (dtype F32)
 *   TSVDM_P_BF16X3  split x = hi + lo in BF16, hi*hi + hi*lo + lo*hi on tensor cores,
 *                   FP32 accumulation (dtype F32)                                   */
typedef enum {
  TSVDM_P_FP64 = 0,
  TSVDM_P_FP32 = 1,
  TSVDM_P_TF32 = 2,
  TSVDM_P_BF16X3 = 3
} tsvdm_prec;

typedef struct tsvdm_plan_s *tsvdm_plan;

/* Create a plan for n1 x n2 x n3 tensors (Sec. 2.2 problem statement: A in
 * R^{m x p x n}, invertible M in R^{n x n}).  The plan owns all device workspace
 * (allocated here, about (n1 n2 + min(n1,n2)^2) n3 elements plus O(n1 n2 + n3^2)), the
 * device status word and the tile choices.  m_is_orthogonal declares M to be a
 * nonzero multiple of an orthogonal matrix (Sec. 2.1): then M^{-1} = M^T / c^2 with
 * c^2 = ||M(:,0)||^2, and t-SVDM-II is allowed.  stream is a cudaStream_t (NULL = the
 * default stream).  Returns EINVAL for non-positive sizes, ENOTSUP for a precision the
 * dtype cannot use, ENOMEM if the workspace cannot be allocated. */
tsvdm_status tsvdm_plan_create(int64_t n1, int64_t n2, int64_t n3, tsvdm_dtype dtype,
                               tsvdm_prec prec, int m_is_orthogonal, void *stream,
                               tsvdm_plan *out);
tsvdm_status tsvdm_plan_destroy(tsvdm_plan plan);

/* Plans for d-way tensors, 3 <= d <= TSVDM_MAX_ORDER (the order-d star-M product of
 * Sec. 2.1 applied to every mode k >= 3; the paper's higher-order layouts such as a 6-way
 * reanalysis tensor).  X is n_1 x n_2 x ... x n_d, column-major (n_1 fastest); the transform
 * is Ahat = X x_3 M_3 x_4 M_4 ... x_d M_d, and the slice SVDs run over all N = n_3 ... n_d
 * trailing index combinations (slice index i_3 + n_3 i_4 + n_3 n_4 i_5 + ...).  On such a
 * plan every entry point's M argument is the concatenation of M_3, M_4, ..., M_d (each
 * n_k x n_k column-major, stored one after the other; for inverse transforms and
 * reconstruction the same matrices on an orthogonal plan, else their inverses), and the
 * factors are laid out as for a 3-way tensor with n3 = N (U n_1 x k x N, S k x N,
 * V n_2 x k x N; packed t-SVDM-II factors likewise).  m_is_orthogonal declares every M_k a
 * nonzero multiple of an orthogonal matrix.  tsvdm_backward returns ENOTSUP on a d-way
 * plan with d > 3; the batch API is 3-way.  d = 3 gives an ordinary plan.  EINVAL for d
 * outside [3, TSVDM_MAX_ORDER] or non-positive dims. */
#define TSVDM_MAX_ORDER 8
tsvdm_status tsvdm_plan_create_dway(int d, const int64_t *dims, tsvdm_dtype dtype,
                                    tsvdm_prec prec, int m_is_orthogonal, void *stream,
                                    tsvdm_plan *out);

/* Jacobi controls.  tol is the relative off-diagonal threshold
 * |a_i^T a_j| <= tol ||a_i|| ||a_j|| under which a column pair counts as orthogonal
 * (<= 0 restores the default: 4 sqrt(m) u with u the unit roundoff of the dtype);
 * max_sweeps caps the sweeps per slice (<= 0 restores the default 40).  A slice that
 * is still rotating after max_sweeps sets TSVDM_ENOCONV. */
tsvdm_status tsvdm_plan_set_jacobi(tsvdm_plan plan, double tol, int max_sweeps);

/* Launch shape of the batched Jacobi kernel (for tuning; 0 = automatic).  block_width:
 * columns of a block pair (16, 32 or 64); cluster_size: CTAs that share one slice
 * (1..16, powers of two, capped by the block pairs of a round and by the device);
 * clusters: clusters launched (slices in flight); stages: row-chunk pipeline depth
 * (2 or 3); ordering: 1 = columns re-ordered by decreasing norm at every sweep
 * (de Rijk), 2 = natural column order; inner_sweeps: Gram sweeps per block pair
 * (1..8; default 2: the first over all pairs in a sweep's first round, the others over the
 * pairs across the two blocks).  EINVAL for other values. */
tsvdm_status tsvdm_plan_set_tuning(tsvdm_plan plan, int block_width, int cluster_size,
                                   int clusters, int stages, int ordering, int inner_sweeps);

/* Engine of the dense products inside the slice SVDs (the block Gram G = W^T W and the
 * rotation apply W <- W Q of every block pair of the one-sided Jacobi, Sec. 3.2's
 * per-slice svd):
 *   TSVDM_JACOBI_AUTO  tensor cores for F32 plans, FMA for F64 (default; see below)
 *   TSVDM_JACOBI_FMA   FP32 / FP64 FMA on the CUDA cores
 *   TSVDM_JACOBI_TC    tcgen05 tensor cores (F32 only).  Gram: every element split as
 *                      x = h + l, h = tf32(x), l = tf32(x - h), G = H^T H + L^T H + H^T L.
 *                      Apply: W + W (Q - I) with W and Q - I split into three BF16 terms
 *                      (x1 + x2 + x3, residual <= 2^-27 |x|) and the six products of order
 *                      >= 2^-24.  FP32 accumulation.  Block pairs are 64 columns.
 *                      One persistent CTA per SM of three 256-thread workers that take
 *                      block pairs of any slice in progress (dataflow order within a
 *                      slice); under tsvdm_plan_set_tuning, clusters caps the CTAs
 *                      launched, cluster_size and stages are ignored.
 * AUTO uses TC for F32 slices of at least 64 columns unless block_width asks for 16 or 32.
 * The engine also selects, for F32 plans, how the other dense products are formed: the
 * slice products U_i diag(S_i) V_i^T of tsvdm_reconstruct and tsvdm_backward and, for
 * two-pass vectors, Z_i = A_i^T U_k and U_k R_i (tensor cores under AUTO and TC: three-term
 * BF16 split, FP32-level accuracy; FMA otherwise), and dL/dM of tsvdm_backward and the
 * mode-3 Gram of tsvdm_data_transform (tensor cores under AUTO and TC: two-term BF16
 * split, three products, FP32 accumulation, FP64 sums over the split of the long mode;
 * FMA with FP64 sums otherwise).
 * ENOTSUP for TC on an F64 plan, EINVAL for other values. */
/* Data-driven transform (Sec. 2.2: M as the transposed matrix of left singular vectors of
 * the mode-3 unfolding A_(3), an n3 x (n1 n2) matrix; an upfront SVD of the unfolding).
 * Writes the orthogonal n3 x n3 M (column-major; device or host pointer) for the tensor X
 * (n1 x n2 x n3, device or host) of a 3-way plan.  The left singular vectors of A_(3) are
 * the eigenvectors of G = A_(3) A_(3)^T = X_mat^T X_mat (formed with FP64 partial sums in
 * a fixed order); they come from the library's own Jacobi SVD of G (a one-slice plan kept
 * inside this plan, allocated on the first call), by decreasing singular value, each with
 * its largest-magnitude entry positive (rows of M with equal singular values are defined
 * only up to a rotation).  Synchronises the plan's stream.  ENOTSUP on a d-way plan. */
tsvdm_status tsvdm_data_transform(tsvdm_plan plan, const void *X, void *M);

/* Warm start of the slice SVDs, for sequences of closely related tensors (learned-M
 * training, where M changes by one optimiser step at a time; streaming data).  Once
 * enabled, every decomposition after the first starts each slice's one-sided Jacobi from
 * the previous decomposition's right vectors V_i: the slice becomes Ahat_i V_i (a slice
 * product on the engine of tsvdm_plan_set_engine) and the rotations accumulate onto V_i,
 * so a slice that changed little converges in a few sweeps.  The stopping rule and the
 * outputs are those of a cold start (to the Jacobi tolerance; in FP32 the orthogonality of
 * V can drift by ~1e-6 per call over long sequences).  Every call of this function makes
 * the next decomposition start cold (call it again after a device-reported error);
 * enable = 0 turns warm starts off.  The first enable allocates rows x cols x n3 elements
 * of scratch (ENOMEM if that fails). */
tsvdm_status tsvdm_plan_set_warm_start(tsvdm_plan plan, int enable);

typedef enum {
  TSVDM_JACOBI_AUTO = 0,
  TSVDM_JACOBI_FMA = 1,
  TSVDM_JACOBI_TC = 2
} tsvdm_jacobi_engine;
tsvdm_status tsvdm_plan_set_engine(tsvdm_plan plan, int engine);

/* Arithmetic of the rotation test and angle of the slice SVDs for F32 plans (the scalar
 * method's zeta = (b - a) / (2 g), t = sign(zeta) / (|zeta| + sqrt(1 + zeta^2)),
 * c = 1 / sqrt(1 + t^2), s = c t, and the test |g| > tol sqrt(a b), on the FP32 Gram
 * entries a = ||w_i||^2, b = ||w_j||^2, g = w_i^T w_j; Sec. 3.2's per-slice svd):
 *   TSVDM_ANGLE_FP64  (default) the test is decided and t, c, s and the rotated diagonal
 *                     are computed in FP64, then rounded to FP32 for the rotation;
 *   TSVDM_ANGLE_FP32  both in FP32 (opt-in: cheaper on GPUs whose FP64 rate is low; the
 *                     rotation is applied to freshly formed Grams, so the angle's rounding
 *                     moves the convergence rate, not the accuracy of the columns).
 * F64 plans always use FP64.  EINVAL for other values. */
typedef enum { TSVDM_ANGLE_FP64 = 0, TSVDM_ANGLE_FP32 = 1 } tsvdm_angle_prec;
tsvdm_status tsvdm_plan_set_angle_precision(tsvdm_plan plan, int angles);

/* How the singular vectors are formed (Sec. 3.4's strategies for t-SVDM-II; the same two
 * forms serve t-SVDM-I):
 *   TSVDM_VECTORS_ACCUMULATE   (default; the "truncate" strategy) one pass: every slice's
 *                              Jacobi accumulates its rotations into V, the kept triplets
 *                              are taken from the full decomposition;
 *   TSVDM_VECTORS_SECOND_PASS  two passes (the compute-efficient strategy): the Jacobi runs
 *                              without right vectors (the slices' singular values, and the
 *                              work matrix W = A V whose normalised columns are one side of
 *                              each triplet); the ranks are chosen; then only the kept
 *                              triplets' other side is formed from the slice itself,
 *                              v_j = A^T u_j / sigma_j (u_j = A v_j / sigma_j for n1 < n2;
 *                              0 where sigma_j = 0), in the plan's precision.  Its rounding
 *                              error is about u ||A|| / sigma_j per vector, the order of the
 *                              rank-k subspace error of the one-pass form (u ||A|| / gap).
 * A warm-started decomposition (tsvdm_plan_set_warm_start) always uses the one-pass form.
 * The first SECOND_PASS on a plan with n1 >= n2 allocates n1 n2 n3 elements (a copy of the
 * transformed slices that the Jacobi works on, so that the second pass reads the slices
 * themselves); ENOMEM if that fails.  EINVAL for other values. */
typedef enum { TSVDM_VECTORS_ACCUMULATE = 0, TSVDM_VECTORS_SECOND_PASS = 1 } tsvdm_vectors;
tsvdm_status tsvdm_plan_set_vectors(tsvdm_plan plan, int mode);

/* Transform of the plan (Sec. 2.2; the paper's transform is the orthonormal DCT, which can
 * be applied in O(n log n) instead of as a dense product):
 *   TSVDM_TRANSFORM_DENSE  (default) the caller's M, as a dense mode-3 product (TTM);
 *   TSVDM_TRANSFORM_DCT2   the orthonormal DCT-II, M(i, t) = s_i cos(pi i (2t + 1) / (2n))
 *                          with s_0 = sqrt(1/n), s_i = sqrt(2/n), and its transpose for
 *                          inverse transforms, by a fast kernel (an n-point FFT of each
 *                          mode-3 fiber in shared memory; one read and one write of the
 *                          tensor); on d-way plans one DCT-II per trailing mode.  The M
 *                          arguments of the decompositions, transforms and reconstruction
 *                          must still be non-NULL but are not read; tsvdm_backward, whose
 *                          gradient is with respect to a dense M, reads and uses M.
 * DCT2 needs an orthogonal plan (EINVAL otherwise) and every transformed mode length a
 * power of two <= 4096 (ENOTSUP otherwise); it allocates the twiddle tables (about 3 n
 * complex values per mode) once.  EINVAL for other values. */
typedef enum { TSVDM_TRANSFORM_DENSE = 0, TSVDM_TRANSFORM_DCT2 = 1 } tsvdm_transform_kind;
tsvdm_status tsvdm_plan_set_transform(tsvdm_plan plan, int kind);

/* Bound of the waits of the tensor-core slice-SVD kernel's scheduler (a worker waiting for
 * the two column blocks of its block pair, or for work to appear): after `polls` polls
 * (about a microsecond each) the kernel stops every worker and the call reports
 * TSVDM_ETIMEOUT (tsvdm_last_status; the outputs are then undefined).  0 restores the
 * default (2^24 polls, several seconds).  The plan stays usable after a timeout.  EINVAL for
 * polls < 0 or above 2^32 - 1. */
tsvdm_status tsvdm_plan_set_wait_limit(tsvdm_plan plan, int64_t polls);

/* Y = X x_3 M (inverse = 0) or Y = X x_3 M^{-1} (inverse = 1), Sec. 2.1.  For
 * inverse = 1 on an orthogonal plan, M is the forward matrix and M^T / c^2 is applied;
 * on a non-orthogonal plan, M must already hold M^{-1}.  X, Y: n1 x n2 x n3 device,
 * X and Y must not overlap.  M: n3 x n3 device. */
tsvdm_status tsvdm_transform(tsvdm_plan plan, const void *X, const void *M, int inverse,
                             void *Y);

/* t-SVDM-I (Sec. 3.3; Fig. 1): Ahat = X x_3 M, then the leading k singular triplets of
 * every frontal slice of Ahat.  Outputs, all caller-owned (device or host):
 *   U  n1 x k x n3   U(:,j,i) = j-th left singular vector of Ahat(:,:,i)
 *   S  k x n3        S(j,i) = j-th singular value of slice i, descending in j
 *   V  n2 x k x n3   right singular vectors
 * Signs: the largest-magnitude entry of each left vector is positive.
 * original_domain = 0 returns the transform-domain factors Uhat, Shat, Vhat (the
 * compressed form, Fig. 1); 1 returns them mapped back by M^{-1} along mode 3 (Sec.
 * 2.2), which needs an orthogonal plan (else ENOTORTHO); S is then f-diagonal data
 * S(j,:) = Shat(j,:) x M^{-T}, not sorted and possibly negative.
 * rel_err (host, nullable): sqrt(sum of discarded sigma^2 / sum of all sigma^2), which
 * equals ||X - X_k||_F / ||X||_F when M is a multiple of an orthogonal matrix
 * (Eckart-Young, Sec. 2.3); NaN on a non-orthogonal plan.  Requesting it synchronises. */
tsvdm_status tsvdm_fixed_rank(tsvdm_plan plan, const void *X, const void *M, int64_t k,
                              void *U, void *S, void *V, int original_domain,
                              double *rel_err);

/* t-SVDM-II (Algorithm 2, "truncate" strategy of Sec. 3.4), orthogonal plans only
 * (else ENOTORTHO).  eps in (0,1).  Steps: the full t-SVDM of X; v = all sigma^2
 * sorted ascending; w = cumulative sums (FP64); J = the largest index with
 * w_J / sum(v) < eps^2 (J = 0: nothing is discarded); tau = v_J;
 * rho_i = #{sigma_{j,i}^2 > tau} (values equal to tau are discarded).
 * Outputs (caller-owned; device or host):
 *   ranks    int32 [n3]       rho_i
 *   offsets  int64 [n3 + 1]   exclusive prefix sum of rho; offsets[n3] = total rank
 *   U  n1 x capacity, S  capacity, V  n2 x capacity: slice i's triplets occupy columns
 *            offsets[i] .. offsets[i+1]-1 (variable-rank format, no padding)
 *   total_rank (host, required)   sum of rho_i
 *   rel_err  (host, nullable)     sqrt(sum of discarded sigma^2 / sum of all sigma^2)
 * U, S, V may all be NULL: only ranks, offsets and total_rank are produced and the
 * factors stay in the plan for tsvdm_tolerance_pack.  If capacity < total rank the call
 * returns ECAPACITY after writing ranks/offsets/total_rank; the factors also stay in
 * the plan.  Always synchronises (the total rank is read back). */
tsvdm_status tsvdm_tolerance(tsvdm_plan plan, const void *X, const void *M, double eps,
                             int32_t *ranks, int64_t *offsets, void *U, void *S, void *V,
                             int64_t capacity, int64_t *total_rank, double *rel_err);

/* Packs the factors kept by the most recent tsvdm_tolerance call on this plan into
 * device buffers U (n1 x capacity), S (capacity), V (n2 x capacity).  ECAPACITY if
 * capacity is below that call's total rank; EINVAL if no tolerance call preceded.  With
 * TSVDM_VECTORS_SECOND_PASS the second pass runs here, and only one pack follows each
 * tsvdm_tolerance call (a second one returns EINVAL). */
tsvdm_status tsvdm_tolerance_pack(tsvdm_plan plan, void *U, void *S, void *V,
                                  int64_t capacity);

/* X_k = (U_i diag(S_i) V_i^T for every slice i) x_3 M^{-1}  (Sec. 2.1 third step).
 * Factors are transform-domain, on the device.  offsets == NULL: uniform rank k,
 * U n1 x k x n3, S k x n3, V n2 x k x n3.  offsets != NULL (device int64 [n3+1]):
 * packed variable-rank factors as produced by tsvdm_tolerance (k is ignored).
 * M: forward matrix on an orthogonal plan, else M^{-1}.  Xk: n1 x n2 x n3 device. */
tsvdm_status tsvdm_reconstruct(tsvdm_plan plan, const void *U, const void *S, const void *V,
                               const int64_t *offsets, int64_t k, const void *M, void *Xk);

/* Gradient of the t-SVDM-I truncation loss (an extension; the paper has no
 * differentiation):  L(X, M) = sqrt(E) / ||X||_F,  E = sum_i sum_{j>k} sigma_j(Ahat_i)^2,
 * Ahat = X x_3 M.  With R_i = Ahat_i - U_i S_i V_i^T (the residual of the rank-k
 * truncation, from the forward factors U, S, V of tsvdm_fixed_rank in the transform
 * domain), dE/dAhat_i = 2 R_i where sigma_k > sigma_{k+1}, so
 *   dX = dL * [ (R x_3 M^T) / (sqrt(E) ||X||) - L X / ||X||^2 ]     (n1 x n2 x n3)
 *   dM = dL * R_(3)-view^T X_(3)-view / (sqrt(E) ||X||)             (n3 x n3)
 * where the views are the (n1 n2) x n3 column-major matrices.  dL is the upstream
 * scalar.  dX and dM are device, nullable.  E = 0 gives L = 0 and zero gradients.
 * loss (nullable) receives L: a device pointer is written on the stream without
 * synchronising, a host pointer after synchronising. */
tsvdm_status tsvdm_backward(tsvdm_plan plan, const void *X, const void *M, int64_t k,
                            const void *U, const void *S, const void *V, double dL,
                            void *dX, void *dM, double *loss);

/* Device-detected status of the plan's work so far (ENOCONV, ENONFINITE, ETIMEOUT or
 * OK).  Synchronises the plan's stream, then clears the word. */
tsvdm_status tsvdm_last_status(tsvdm_plan plan);

/* Number of Jacobi sweeps and rotations executed by the most recent decomposition on
 * this plan (summed over slices); synchronises.  Either pointer may be NULL. */
tsvdm_status tsvdm_plan_stats(tsvdm_plan plan, int64_t *sweeps, int64_t *rotations);

const char *tsvdm_strerror(tsvdm_status s);

/* Per-stage instrumentation (not in the paper, which reports stage timings only in
 * prose, Sec. 3.4 and Sec. 4).  With enable != 0, later calls on the plan record CUDA
 * events on the plan's stream around each stage.  tsvdm_plan_profile_read synchronises
 * and returns, for the most recent call, the stage times in milliseconds
 * (ms[TSVDM_STAGE_COUNT], 0 for stages that did not run) and the number of kernels the
 * call launched (launches, nullable). */
typedef enum {
  TSVDM_STAGE_TTM = 0,        /* mode-3 TTMs (forward and back-transform)            */
  TSVDM_STAGE_TRANSPOSE = 1,  /* slice transposition for n1 < n2                     */
  TSVDM_STAGE_JACOBI = 2,     /* batched one-sided Jacobi sweeps                     */
  TSVDM_STAGE_FINALIZE = 3,   /* column norms and per-slice descending order         */
  TSVDM_STAGE_SELECT = 4,     /* t-SVDM-II threshold (tail sums), ranks, offsets     */
  TSVDM_STAGE_EMIT = 5,       /* normalised, sign-fixed factor output / packing      */
  TSVDM_STAGE_OTHER = 6,      /* reductions, products and small kernels              */
  TSVDM_STAGE_COUNT = 7
} tsvdm_stage;
tsvdm_status tsvdm_plan_profile(tsvdm_plan plan, int enable);
tsvdm_status tsvdm_plan_profile_read(tsvdm_plan plan, float *ms, int64_t *launches);

/* Measured peak rates for roofline fractions (instrumentation; the paper has no
 * counterpart).  Runs one warm-up and one timed launch of a kernel that does nothing but the
 * unit's instruction on every SM, and returns the rate in TFLOP/s (synchronises; allocates
 * and frees a 4-byte status word):
 *   TSVDM_PROBE_FP32_FMA  FP32 FMA on the CUDA cores (256-thread CTAs, full occupancy,
 *                         8 independent chains per thread), iters FMAs per chain
 *   TSVDM_PROBE_TF32_MMA  tcgen05.mma kind::tf32, M = 128, N = 256, K = 8, one CTA per SM,
 *                         iters MMAs per SM, operands in shared memory
 *   TSVDM_PROBE_BF16_MMA  the same with kind::f16 (BF16, K = 16)
 *   TSVDM_PROBE_FP64_FMA  FP64 FMA on the CUDA cores, as the FP32 probe
 * EINVAL for another unit or iters < 1; ETIMEOUT if the MMA completion wait ran out. */
typedef enum {
  TSVDM_PROBE_FP32_FMA = 0,
  TSVDM_PROBE_TF32_MMA = 1,
  TSVDM_PROBE_BF16_MMA = 2,
  TSVDM_PROBE_FP64_FMA = 3
} tsvdm_probe_unit;
tsvdm_status tsvdm_probe_peak(int unit, int64_t iters, void *stream, double *tflops);

/* ---- learned orthogonal transform (extension) -------------------------------------
 * Cayley form M(A) = (I + W)^{-1} (I - W) M0 with W = A^T - A skew-symmetric.
 * All pointers are n x n device matrices of the given dtype unless stated otherwise;
 * stream is a cudaStream_t.  tsvdm_cayley writes M and keeps Z = (I + W)^{-1} and
 * Q = Z (I - W) in the caller's buffers for the backward; work holds 2 n^2 elements.
 * (I + W) is always invertible for skew W and is solved by Gauss-Jordan elimination
 * without pivoting (its symmetric part is I, so no pivot vanishes). */
tsvdm_status tsvdm_cayley(int64_t n, tsvdm_dtype dtype, const void *A, const void *M0,
                          void *M, void *Z, void *Q, void *work, void *stream);
/* dA = (dW)^T - dW with dW = -Z^T (dM M0^T) (Q + I)^T; work holds 3 n^2 elements. */
tsvdm_status tsvdm_cayley_backward(int64_t n, tsvdm_dtype dtype, const void *M0,
                                   const void *Z, const void *Q, const void *dM, void *dA,
                                   void *work, void *stream);
/* One Adam step (Kingma & Ba) over count elements, in place: step is 1-based. */
tsvdm_status tsvdm_adam(int64_t count, tsvdm_dtype dtype, void *param, const void *grad,
                        void *m1, void *m2, int64_t step, double lr, double beta1,
                        double beta2, double eps, void *stream);

/* ---- batches of tensors with uneven shapes (one persistent Jacobi launch, graph) ----
 * The spec batching extension of t-SVDM-I / t-SVDM-II (Sec. 3.3, Algorithm 2):
 * count tensors, each with its own n1 x n2 x n3, orthogonal M and mode, decomposed by one
 * stream of work whose dominant step is a single persistent Jacobi launch over every
 * slice of every tensor (longest slices first).  Nothing is read back to the host, so the
 * whole run can be captured once into a CUDA graph (tsvdm_batch_capture) and replayed
 * (tsvdm_batch_launch).  M must be a multiple of an orthogonal matrix; min(n1,n2) <= 1024. */
typedef struct {
  int64_t n1, n2, n3;
  int mode;        /* 0: t-SVDM-I with rank k; 1: t-SVDM-II with tolerance eps */
  int64_t k;
  double eps;
} tsvdm_batch_desc;

typedef struct {
  const void *X, *M;   /* device inputs (column-major n1 x n2 x n3, n3 x n3) */
  void *U, *S, *V;     /* device outputs.  mode 0: U n1 x k x n3, S k x n3, V n2 x k x n3.
                          mode 1: packed, capacity n3 min(n1,n2) columns (U n1 x cap,
                          S cap, V n2 x cap), slice i at offsets[i]..offsets[i+1]-1 */
  int32_t *ranks;      /* mode 1: device [n3] (nullable) */
  int64_t *offsets;    /* mode 1: device [n3 + 1] (nullable) */
  double *rel_err;     /* device double (nullable): sqrt(discarded / total sigma^2) */
} tsvdm_batch_io;

typedef struct tsvdm_batch_s *tsvdm_batch;

/* Allocates the workspace of all tensors (EINVAL for a bad descriptor). */
tsvdm_status tsvdm_batch_create(const tsvdm_batch_desc *descs, int count, tsvdm_dtype dtype,
                                tsvdm_prec prec, void *stream, tsvdm_batch *out);
tsvdm_status tsvdm_batch_destroy(tsvdm_batch b);
/* Enqueues one decomposition of every tensor (io[count]) on the batch's stream. */
tsvdm_status tsvdm_batch_run(tsvdm_batch b, const tsvdm_batch_io *io);
/* Runs once, then captures one run into a CUDA graph (io pointers are baked in).  The
 * batch must have been created on a non-default stream (EINVAL otherwise). */
tsvdm_status tsvdm_batch_capture(tsvdm_batch b, const tsvdm_batch_io *io);
/* Replays the captured graph on the batch's stream. */
tsvdm_status tsvdm_batch_launch(tsvdm_batch b);
/* Autotuner: times the Jacobi launch for each candidate (F32 batches whose slices all
 * have >= 64 columns: the tensor-core engine; and the FMA engine with block width 32/64,
 * cluster size 1/2/4, pipeline stages 2/3) on these inputs and keeps the fastest; choice
 * (nullable, int[4]) receives width, cluster size, stages (0 = the tensor-core engine,
 * reported with cluster size 1) and the best time in microseconds.  Until tuned, a batch
 * uses TSVDM_JACOBI_AUTO (tsvdm_plan_set_engine). */
tsvdm_status tsvdm_batch_tune(tsvdm_batch b, const tsvdm_batch_io *io, int *choice);
/* Synchronises; sweeps and rotations summed over all slices of the last run, and the
 * device-detected status (ENOCONV, ENONFINITE, ETIMEOUT or OK, then cleared). */
tsvdm_status tsvdm_batch_status(tsvdm_batch b, int64_t *sweeps, int64_t *rotations);
/* Kernel launches in one replay of the captured graph (its kernel nodes), in *kernels.
 * EINVAL before tsvdm_batch_capture. */
tsvdm_status tsvdm_batch_graph_kernels(tsvdm_batch b, int64_t *kernels);

/* Allocation-free t-SVDM-II rank choice.  The paper has no counterpart: it exists for
 * callers that must not call cudaMalloc (a process whose device memory is all handed to
 * another allocator up front, or a service that forbids allocation on its request path
 * because a driver allocation can synchronise the device and take milliseconds).
 * It is the same computation as the selection inside tsvdm_tolerance, on given singular
 * values, with its scratch in a fixed array of about 2.1 MiB built into the library (held
 * on every GPU that loads it until the process exits) instead of a plan.
 *   sigma    device float [cols x nslices], column i = slice i's singular values sorted
 *            in descending order (e.g. S of tsvdm_fixed_rank with k = min(n1, n2)); they
 *            must be finite and non-negative (-0 counts as 0)
 *   eps      relative tolerance in (0, 1)
 *   ranks    device int32 [nslices]; offsets device int64 [nslices + 1] (as tsvdm_tolerance)
 *   summary  device double [4] or NULL: sum of all sigma^2, sum of discarded sigma^2,
 *            tau (a sigma^2 value, -1 when nothing is discarded), total rank
 *   stream   cudaStream_t
 * At most 262,144 singular values per call (cols * nslices); larger problems return
 * TSVDM_ESCRATCH without launching anything.  Nothing is allocated.  The call is
 * asynchronous: a NaN, infinite or negative value is reported on the device, as NaN in all
 * four summary entries with every rank and offset 0.  Each call looks up the scratch's
 * device address on the current device (a host-side lookup; the first one on a device may
 * load the library's device code, so make the first call before any stream capture).
 * Every call shares the scratch and clears what must start at zero itself, so calls whose
 * work overlaps on the GPU race: issue them on one stream. */
tsvdm_status tsvdm_select_ranks_noalloc(const float *sigma, int64_t cols, int64_t nslices,
                                        double eps, int32_t *ranks, int64_t *offsets,
                                        double *summary, void *stream);

#ifdef __cplusplus
}
#endif
#endif /* TSVDM_H */
