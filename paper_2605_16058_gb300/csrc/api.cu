// C ABI of libtsvdm (declared in include/tsvdm.h): plans, argument checks, host-buffer
// staging and the order of the device kernels for each operation.
#include <math.h>
#include <stdlib.h>
#include <string.h>

#include <new>
#include <vector>

#include "common.cuh"

using namespace tsvdm;

enum { SC_INVSCALE = 9 };
enum { STG_X = 0, STG_M, STG_U, STG_S, STG_V, STG_RANKS, STG_OFF, STG_COUNT };

struct tsvdm_plan_s {
  int64_t n1 = 0, n2 = 0, n3 = 0;
  tsvdm_dtype dtype = TSVDM_F32;
  tsvdm_prec prec = TSVDM_P_FP32;
  int ortho = 0;
  cudaStream_t st = nullptr;
  int transposed = 0;
  int64_t rows = 0, cols = 0;
  size_t esz = 4;
  void *Ahat = nullptr, *Wt = nullptr, *Vw = nullptr, *sig = nullptr, *keys = nullptr;
  int *perm = nullptr, *sweeps = nullptr, *status = nullptr, *queue = nullptr;
  int *ranks_ws = nullptr;
  int64_t *off_ws = nullptr;
  long long *rots = nullptr;
  float *norm2 = nullptr;
  void *sched = nullptr;
  size_t sched_bytes = 0;
  int sort_cols = 1;
  double *scal = nullptr;
  double *splitk = nullptr;
  size_t splitk_elems = 0;
  void *tc_ws = nullptr;
  size_t tc_ws_bytes = 0;
  double tol = 0.0;
  int max_sweeps = 40;
  int width_hint = 0, cluster_hint = 0, grid_hint = 0, stages_hint = 0, inner_sweeps = 2;
  int engine = JACOBI_AUTO;
  int angle32 = 0;           // FP32 slices: rotation test and angle in FP32 (opt-in)
  long long wait_polls = 0;  // bound of the tensor-core Jacobi's scheduler waits (0: default)
  int vec_mode = 0;          // TSVDM_VECTORS_ACCUMULATE / TSVDM_VECTORS_SECOND_PASS
  // TSVDM_TRANSFORM_DCT2: transforms by the orthonormal DCT-II through the fast kernels,
  // with twiddle tables per transformed mode (element offsets dct_off[m] into dct_tab)
  int xform = 0;
  void *dct_tab = nullptr;
  int64_t dct_off[TSVDM_MAX_ORDER] = {};
  int twopass = 0;           // the last decomposition ran without right vectors
  // second pass: one restricted-Jacobi entry per slice with kept columns (device arrays of
  // n3 entries, their host images, and the restricted Jacobi's sweep counts)
  SliceDesc *tp_desc = nullptr;
  int64_t *tp_off = nullptr;
  int *tp_sweeps = nullptr;
  void *tp_sig = nullptr;    // the restricted Jacobi's singular values and order (cols n3)
  int *tp_perm = nullptr;
  std::vector<SliceDesc> tp_hdesc;
  std::vector<int64_t> tp_hoff;
  std::vector<int> tp_hranks;
  // d-way tensors: the trailing modes (dims td[0..dw-1], n3 = their product), one matrix
  // per mode, concatenated in the M buffer at element offsets mo[]; dw = 0: 3-way plan
  int dw = 0;
  int64_t td[TSVDM_MAX_ORDER] = {}, mo[TSVDM_MAX_ORDER] = {}, msum = 0;
  void *dtmp = nullptr;      // ping-pong buffer of the per-mode TTMs (n1 n2 n3 elements)
  // warm start of the slice SVDs: the next decomposition starts from the V in Vw
  int warm = 0, warm_valid = 0;
  void *warm_buf = nullptr;  // A_i V_i (rows cols n3 elements)
  // data-driven transform: a one-slice n3 x n3 plan for the SVD of the mode-3 Gram, and its
  // buffers (Gram, 1 x 1 identity, U, S, V)
  tsvdm_plan_s *dsub = nullptr;
  void *dbuf = nullptr;
  int tol_valid = 0;
  int64_t tol_total = 0;
  void *stage[STG_COUNT] = {};
  size_t stage_bytes[STG_COUNT] = {};
  // instrumentation
  int profile = 0;
  cudaEvent_t ev[2 * TSVDM_STAGE_COUNT] = {};
  int ran[TSVDM_STAGE_COUNT] = {};
  int64_t launches = 0;
};

namespace {

tsvdm_status from_cuda(cudaError_t e) {
  if (e == cudaSuccess) return TSVDM_OK;
  if (e == cudaErrorMemoryAllocation) return TSVDM_ENOMEM;
  return TSVDM_ECUDA;
}

#define CK(expr)                                    \
  do {                                              \
    cudaError_t _e = (expr);                        \
    if (_e != cudaSuccess) return from_cuda(_e);    \
  } while (0)

bool is_device_ptr(const void *p) {
  if (!p) return true;
  cudaPointerAttributes a;
  cudaError_t e = cudaPointerGetAttributes(&a, p);
  if (e != cudaSuccess) {
    cudaGetLastError();
    return false;
  }
  return a.type == cudaMemoryTypeDevice || a.type == cudaMemoryTypeManaged;
}

double default_tol(const tsvdm_plan_s *p) {
  double u = p->dtype == TSVDM_F32 ? ldexp(1.0, -24) : ldexp(1.0, -53);
  return 4.0 * sqrt((double)p->rows) * u;
}

// The Jacobi's matrix: the transposed copy, or (a decomposition without right vectors on a
// non-transposed plan) a copy of Ahat, which the second pass then reads; else Ahat itself.
void *work_matrix(tsvdm_plan_s *p) {
  return (p->transposed || p->twopass) ? p->Wt : p->Ahat;
}

// Start of a call: forget the previous call's stage record.
void begin_call(tsvdm_plan_s *p) {
  p->launches = 0;
  for (int i = 0; i < TSVDM_STAGE_COUNT; ++i) p->ran[i] = 0;
}
// Brackets a stage with events when profiling (a stage may run more than once per call;
// the bracket then spans from its first start to its last end).
void stage_begin(tsvdm_plan_s *p, int s) {
  if (p->profile && !p->ran[s]) cudaEventRecord(p->ev[2 * s], p->st);
}
void stage_end(tsvdm_plan_s *p, int s, int nlaunch) {
  p->launches += nlaunch;
  if (p->profile) cudaEventRecord(p->ev[2 * s + 1], p->st);
  p->ran[s] = 1;
}

// Device buffer for a caller pointer: the pointer itself when it is device memory, else
// a staging buffer of `bytes` (grown on demand) filled from host when `copy_in`.
tsvdm_status stage_in(tsvdm_plan_s *p, int slot, const void *ptr, size_t bytes, bool copy_in,
                      void **dev, bool *staged) {
  *staged = false;
  *dev = const_cast<void *>(ptr);
  if (ptr == nullptr || is_device_ptr(ptr)) return TSVDM_OK;
  if (p->stage_bytes[slot] < bytes) {
    if (p->stage[slot]) cudaFree(p->stage[slot]);
    p->stage[slot] = nullptr;
    p->stage_bytes[slot] = 0;
    CK(cudaMalloc(&p->stage[slot], bytes));
    p->stage_bytes[slot] = bytes;
  }
  *dev = p->stage[slot];
  *staged = true;
  if (copy_in && bytes) CK(cudaMemcpyAsync(*dev, ptr, bytes, cudaMemcpyHostToDevice, p->st));
  return TSVDM_OK;
}

tsvdm_status read_status(tsvdm_plan_s *p) {
  int s = 0;
  CK(cudaMemcpyAsync(&s, p->status, sizeof(int), cudaMemcpyDeviceToHost, p->st));
  CK(cudaStreamSynchronize(p->st));
  if (s) CK(cudaMemsetAsync(p->status, 0, sizeof(int), p->st));
  if (s & ST_NONFINITE) return TSVDM_ENONFINITE;
  if (s & ST_TIMEOUT) return TSVDM_ETIMEOUT;
  if (s & ST_NOCONV) return TSVDM_ENOCONV;
  return TSVDM_OK;
}

// One mode-3 TTM in the plan's precision: tensor cores (tcgen05) for TF32 / BF16x3 when
// the shape allows it, CUDA cores otherwise.
template <typename T>
cudaError_t ttm_any(tsvdm_plan_s *p, const T *X, int64_t P, const T *M, bool transB, T *Y,
                    const double *scale, const double *beta, const T *Z, double *sumsq) {
  const int64_t n = p->n3;
  if constexpr (sizeof(T) == 4) {
    if ((p->prec == TSVDM_P_TF32 || p->prec == TSVDM_P_BF16X3) && p->tc_ws &&
        ttm_tc_supported(P, n, n, X, Y))
      return ttm_tc((const float *)X, P, n, (const float *)M, n, transB, (int)p->prec, (float *)Y,
                    p->tc_ws, p->tc_ws_bytes, sumsq, scale, beta, (const float *)Z, p->status,
                    p->st);
  }
  return ttm_simt<T>(X, P, n, M, n, n, transB, Y, scale, beta, Z, sumsq, p->st);
}

// Elements of the transform argument: n3^2, or the concatenated per-mode matrices.
int64_t m_elems(const tsvdm_plan_s *p) { return p->dw ? p->msum : p->n3 * p->n3; }

// Y = X x_3 M (or M^{-1}) on a (P x n) column-major view, n explicit.
template <typename T>
cudaError_t ttm_n(tsvdm_plan_s *p, const T *X, int64_t P, int64_t n, const T *M, bool transB,
                  T *Y, const double *scale) {
  if constexpr (sizeof(T) == 4) {
    if ((p->prec == TSVDM_P_TF32 || p->prec == TSVDM_P_BF16X3) && p->tc_ws &&
        ttm_tc_supported(P, n, n, X, Y))
      return ttm_tc((const float *)X, P, n, (const float *)M, n, transB, (int)p->prec, (float *)Y,
                    p->tc_ws, p->tc_ws_bytes, nullptr, scale, nullptr, nullptr, p->status, p->st);
  }
  return ttm_simt<T>(X, P, n, M, n, n, transB, Y, scale, nullptr, nullptr, nullptr, p->st);
}

// d-way: Y = X x_3 M_3 x_4 M_4 ... (or the inverses) for a tensor of P0 x td[0] x td[1] x ...
// (P0 = n1 n2 for the data, n1 k / n2 k / k for factors).  The mode-(3+m) product is a
// batch over the trailing index q of (P_m x td[m]) mode-3 products, P_m = P0 prod_{i<m}
// td[i]; the modes commute.  Results ping-pong between Y and the plan's buffer so that the
// last mode lands in Y (X is never written).
template <typename T>
tsvdm_status transform_dway(tsvdm_plan_s *p, const T *X, int64_t P0, const T *M, bool inverse,
                            T *Y) {
  const int d = p->dw;
  int nl = 0;
  stage_begin(p, TSVDM_STAGE_TTM);
  int64_t Pm = P0;
  const T *src = X;
  for (int m = 0; m < d; ++m) {
    const int64_t nm = p->td[m];
    int64_t Qm = 1;
    for (int i = m + 1; i < d; ++i) Qm *= p->td[i];
    T *dst = ((d - 1 - m) % 2 == 0) ? Y : (T *)p->dtmp;
    const T *Mm = M + p->mo[m];
    const double *scale = nullptr;
    bool transB = false;
    if (inverse && p->ortho && p->xform != TSVDM_TRANSFORM_DCT2) {
      CK(inv_scale<T>(Mm, nm, p->scal + SC_INVSCALE, p->st));
      scale = p->scal + SC_INVSCALE;
      transB = true;
      ++nl;
    }
    if (p->xform == TSVDM_TRANSFORM_DCT2) {                      // M is not read
      CK(dct_mode3<T>(src, Pm, nm, Qm, inverse, (const char *)p->dct_tab + p->dct_off[m], dst,
                      p->st));
      ++nl;
    } else {
      for (int64_t q = 0; q < Qm; ++q) {
        CK(ttm_n<T>(p, src + q * Pm * nm, Pm, nm, Mm, transB, dst + q * Pm * nm, scale));
        nl += (p->prec == TSVDM_P_TF32 || p->prec == TSVDM_P_BF16X3) ? 2 : 1;
      }
    }
    src = dst;
    Pm *= nm;
  }
  stage_end(p, TSVDM_STAGE_TTM, nl);
  return TSVDM_OK;
}

template <typename T>
tsvdm_status run_ttm(tsvdm_plan_s *p, const T *X, int64_t P, const T *M, bool inverse, T *Y,
                     double *sumsq) {
  if (p->dw) return transform_dway<T>(p, X, P, M, inverse, Y);
  const int64_t n = p->n3;
  stage_begin(p, TSVDM_STAGE_TTM);
  if (p->xform == TSVDM_TRANSFORM_DCT2 && !sumsq) {
    CK(dct_mode3<T>(X, P, n, 1, inverse, p->dct_tab, Y, p->st));
    stage_end(p, TSVDM_STAGE_TTM, 1);
    return TSVDM_OK;
  }
  int nl = 1;
  const bool tc = (p->prec == TSVDM_P_TF32 || p->prec == TSVDM_P_BF16X3);
  if (!inverse) {
    CK(ttm_any<T>(p, X, P, M, false, Y, nullptr, nullptr, nullptr, sumsq));
  } else if (p->ortho) {
    CK(inv_scale<T>(M, n, p->scal + SC_INVSCALE, p->st));
    CK(ttm_any<T>(p, X, P, M, true, Y, p->scal + SC_INVSCALE, nullptr, nullptr, sumsq));
    nl = 2;
  } else {
    CK(ttm_any<T>(p, X, P, M, false, Y, nullptr, nullptr, nullptr, sumsq));
  }
  if (tc) nl += 1;   // the B-operand preparation kernel
  stage_end(p, TSVDM_STAGE_TTM, nl);
  return TSVDM_OK;
}

// Algorithm 1: Ahat = X x_3 M, then the slice SVDs (sorted sigma and permutation kept).
template <typename T>
tsvdm_status decompose(tsvdm_plan_s *p, const T *X, const T *M) {
  p->tol_valid = 0;
  const int64_t P = p->n1 * p->n2;
  tsvdm_status s = run_ttm<T>(p, X, P, M, false, (T *)p->Ahat, nullptr);
  if (s != TSVDM_OK) return s;
  // two passes (Sec. 3.4): singular values first, the kept vectors afterwards; a warm start
  // needs the right vectors, so it keeps the one-pass form
  p->twopass = (p->vec_mode == TSVDM_VECTORS_SECOND_PASS && !p->warm) ? 1 : 0;
  if (p->transposed) {
    stage_begin(p, TSVDM_STAGE_TRANSPOSE);
    CK(transpose_slices<T>((const T *)p->Ahat, p->n1, p->n2, p->n3, (T *)p->Wt, p->st));
    stage_end(p, TSVDM_STAGE_TRANSPOSE, 1);
  } else if (p->twopass) {
    stage_begin(p, TSVDM_STAGE_TRANSPOSE);
    CK(cudaMemcpyAsync(p->Wt, p->Ahat, p->esz * p->n1 * p->n2 * p->n3, cudaMemcpyDeviceToDevice,
                       p->st));
    stage_end(p, TSVDM_STAGE_TRANSPOSE, 0);
  }
  CK(cudaMemsetAsync(p->queue, 0, sizeof(int), p->st));
  CK(cudaMemsetAsync(p->rots, 0, sizeof(long long) * p->n3, p->st));
  const bool warm = p->warm && p->warm_valid;
  if (warm) {
    // start from the previous right vectors: the slice becomes A_i V_i, V starts at V_i
    stage_begin(p, TSVDM_STAGE_OTHER);
    CK(slice_rotate<T>((const T *)work_matrix(p), (const T *)p->Vw, p->rows, p->cols, p->n3,
                       (T *)p->warm_buf, sizeof(T) == 4 && p->engine != JACOBI_FMA, p->status,
                       p->st));
    CK(cudaMemcpyAsync(work_matrix(p), p->warm_buf, p->esz * p->rows * p->cols * p->n3,
                       cudaMemcpyDeviceToDevice, p->st));
    stage_end(p, TSVDM_STAGE_OTHER, 1);
  }
  JacobiParams jp{};
  jp.A = work_matrix(p);
  jp.V = p->Vw;
  jp.sA = p->rows * p->cols;
  jp.sV = p->cols * p->cols;
  jp.rows = (int)p->rows;
  jp.cols = (int)p->cols;
  jp.nslices = (int)p->n3;
  jp.tol = p->tol > 0 ? p->tol : default_tol(p);
  jp.max_sweeps = p->max_sweeps;
  jp.queue = p->queue;
  jp.status = p->status;
  jp.sweeps = p->sweeps;
  jp.rots = p->rots;
  jp.norm2 = p->sort_cols ? p->norm2 : nullptr;
  jp.inner_sweeps = p->inner_sweeps;
  jp.desc = nullptr;
  jp.engine = p->engine;
  jp.warm = warm ? 1 : 0;
  jp.angle32 = p->angle32;
  jp.wait_polls = p->wait_polls;
  jp.novec = p->twopass;
  jp.sched = p->sched;
  jp.sched_bytes = p->sched_bytes;
  jp.max_cols = (int)p->cols;
  stage_begin(p, TSVDM_STAGE_JACOBI);
  CK(jacobi_run<T>(jp, p->st, p->width_hint, p->cluster_hint, p->grid_hint, p->stages_hint));
  stage_end(p, TSVDM_STAGE_JACOBI, 1);
  stage_begin(p, TSVDM_STAGE_FINALIZE);
  CK(jacobi_finalize<T>((const T *)work_matrix(p), jp.sA, jp.rows, jp.cols, jp.nslices,
                        (T *)p->sig, p->perm, p->st));
  stage_end(p, TSVDM_STAGE_FINALIZE, 1);
  p->warm_valid = p->warm;           // Vw now holds every slice's right vectors
  return TSVDM_OK;
}

// Second pass of a decomposition without right vectors (Sec. 3.4), after the emitted side
// K (U, or V for transposed slices) and S: Z = A^T K (A K) into the other side's buffer O,
// a restricted one-sided Jacobi of every slice's Z (its kept columns only), then O = the
// normalised columns of Z R, K <- K R, S = their norms (descending), and the sign rule.
// Ahat and the work matrix are free by then and hold the rotated copies.
template <typename T>
tsvdm_status second_pass(tsvdm_plan_s *p, int64_t k, const int *ranks, const int64_t *offsets,
                         T *U, T *S, T *V, int *nl) {
  const bool tr = p->transposed != 0;
  const int64_t kd = p->rows, od = p->cols, n3 = p->n3;
  T *Kout = tr ? V : U, *Oout = tr ? U : V;
  const int64_t maxr = ranks ? p->cols : k;
  bool done_tc = false;
  if constexpr (sizeof(T) == 4) {
    // tensor cores (three-term BF16 split) unless the FMA engine was chosen
    if (p->engine != JACOBI_FMA &&
        complete_tc_supported((const float *)p->Ahat, (const float *)Kout, p->n1, p->n2, tr)) {
      CK(complete_tc((const float *)p->Ahat, p->n1, p->n2, n3, k, ranks, offsets,
                     (const float *)Kout, nullptr, (float *)Oout, p->status, p->st));
      done_tc = true;
    }
  }
  if (!done_tc)
    CK(complete_vectors<T>((const T *)p->Ahat, p->n1, p->n2, n3, tr, k, ranks, offsets, maxr, U,
                           nullptr, V, p->st));
  // the kept columns of every slice (ranks are read back: the descriptors are built here)
  p->tp_hranks.assign(n3, (int)k);
  if (ranks) {
    CK(cudaMemcpyAsync(p->tp_hranks.data(), ranks, sizeof(int) * n3, cudaMemcpyDeviceToHost,
                       p->st));
    CK(cudaStreamSynchronize(p->st));
  }
  p->tp_hdesc.clear();
  p->tp_hoff.clear();
  int64_t col = 0, roff = 0;
  int max_rho = 0, min_rho = 1 << 30;
  for (int64_t i = 0; i < n3; ++i) {
    const int rho = p->tp_hranks[i];
    if (rho >= 1) {
      SliceDesc d;
      d.A = Oout + col * od;
      d.V = (T *)p->Vw + roff;
      d.norm2 = p->norm2 + col;
      d.sig = (T *)p->tp_sig + col;
      d.perm = p->tp_perm + col;
      d.rows = (int)od;
      d.cols = rho;
      p->tp_hdesc.push_back(d);
      p->tp_hoff.push_back(col);
      max_rho = rho > max_rho ? rho : max_rho;
      min_rho = rho < min_rho ? rho : min_rho;
    }
    col += rho;
    roff += (int64_t)rho * rho;
  }
  const int count = (int)p->tp_hdesc.size();
  if (count == 0) return TSVDM_OK;
  const int64_t total = col;
  CK(cudaMemcpyAsync(p->tp_desc, p->tp_hdesc.data(), sizeof(SliceDesc) * count,
                     cudaMemcpyHostToDevice, p->st));
  CK(cudaMemcpyAsync(p->tp_off, p->tp_hoff.data(), sizeof(int64_t) * count,
                     cudaMemcpyHostToDevice, p->st));
  CK(cudaMemsetAsync(p->queue, 0, sizeof(int), p->st));
  JacobiParams jp{};
  jp.rows = 0;
  jp.cols = min_rho;
  jp.nslices = count;
  jp.tol = p->tol > 0 ? p->tol
                      : 4.0 * sqrt((double)od) * (sizeof(T) == 4 ? ldexp(1.0, -24) : ldexp(1.0, -53));
  jp.max_sweeps = p->max_sweeps;
  jp.queue = p->queue;
  jp.status = p->status;
  jp.sweeps = p->tp_sweeps;
  jp.rots = p->rots;
  jp.norm2 = nullptr;
  jp.inner_sweeps = 1;      // Z's columns are nearly orthogonal: one Gram sweep per block pair
  jp.desc = p->tp_desc;
  jp.engine = (sizeof(T) == 4 && p->engine != JACOBI_FMA) ? JACOBI_TC : JACOBI_FMA;
  jp.sched = p->sched;
  jp.sched_bytes = p->sched_bytes;
  jp.max_cols = max_rho;
  jp.angle32 = p->angle32;
  jp.wait_polls = p->wait_polls;
  CK(jacobi_run<T>(jp, p->st, 0, 0, 0, 0));
  CK(jacobi_finalize_desc<T>(p->tp_desc, count, max_rho, p->st));
  T *Ktmp = (T *)p->Ahat, *Otmp = (T *)p->Wt;
  bool rotated = false;
  if constexpr (sizeof(T) == 4) {
    if (p->engine != JACOBI_FMA) {
      // the gather of the other side on the CUDA cores, K R on the tensor cores
      CK(rotate_back<T>(p->tp_desc, p->tp_off, count, max_rho, kd, od, Kout, Ktmp, Otmp, S,
                        p->st, true));
      CK(rotate_tc(p->tp_desc, p->tp_off, count, kd, (const float *)Kout, (float *)Ktmp,
                   p->status, p->st));
      *nl += 1;
      rotated = true;
    }
  }
  if (!rotated)
    CK(rotate_back<T>(p->tp_desc, p->tp_off, count, max_rho, kd, od, Kout, Ktmp, Otmp, S, p->st));
  CK(cudaMemcpyAsync(Kout, Ktmp, sizeof(T) * kd * total, cudaMemcpyDeviceToDevice, p->st));
  CK(cudaMemcpyAsync(Oout, Otmp, sizeof(T) * od * total, cudaMemcpyDeviceToDevice, p->st));
  CK(emit_signfix<T>(p->n1, p->n2, n3, k, ranks, offsets, maxr, U, V, p->st));
  *nl += 5;
  return TSVDM_OK;
}

template <typename T>
tsvdm_status emit(tsvdm_plan_s *p, int64_t k, const int *ranks, const int64_t *offsets, T *U,
                  T *S, T *V) {
  stage_begin(p, TSVDM_STAGE_EMIT);
  CK(emit_factors<T>((const T *)work_matrix(p), p->rows * p->cols,
                     p->twopass ? nullptr : (const T *)p->Vw, p->cols * p->cols, (int)p->rows,
                     (int)p->cols, (int)p->n3, p->transposed != 0, (const T *)p->sig, p->perm, k,
                     ranks, offsets, U, S, V, p->st));
  int nl = 1;
  if (p->twopass) {
    tsvdm_status s = second_pass<T>(p, k, ranks, offsets, U, S, V, &nl);
    if (s != TSVDM_OK) return s;
  }
  stage_end(p, TSVDM_STAGE_EMIT, nl);
  return TSVDM_OK;
}

template <typename T>
tsvdm_status fixed_rank_impl(tsvdm_plan_s *p, const void *X, const void *M, int64_t k, void *U,
                             void *S, void *V, int original_domain, double *rel_err) {
  const size_t e = p->esz;
  const int64_t n1 = p->n1, n2 = p->n2, n3 = p->n3;
  void *dX, *dM, *dU, *dS, *dV;
  bool sX, sM, sU, sS, sV;
  tsvdm_status s;
  if ((s = stage_in(p, STG_X, X, e * n1 * n2 * n3, true, &dX, &sX)) != TSVDM_OK) return s;
  if ((s = stage_in(p, STG_M, M, e * m_elems(p), true, &dM, &sM)) != TSVDM_OK) return s;
  if ((s = stage_in(p, STG_U, U, e * n1 * k * n3, false, &dU, &sU)) != TSVDM_OK) return s;
  if ((s = stage_in(p, STG_S, S, e * k * n3, false, &dS, &sS)) != TSVDM_OK) return s;
  if ((s = stage_in(p, STG_V, V, e * n2 * k * n3, false, &dV, &sV)) != TSVDM_OK) return s;
  if ((s = decompose<T>(p, (const T *)dX, (const T *)dM)) != TSVDM_OK) return s;
  if ((s = emit<T>(p, k, nullptr, nullptr, (T *)dU, (T *)dS, (T *)dV)) != TSVDM_OK) return s;
  if (rel_err) {
    stage_begin(p, TSVDM_STAGE_OTHER);
    CK(trunc_sums<T>((const T *)p->sig, (int)p->cols, (int)n3, k, p->scal, p->st));
    stage_end(p, TSVDM_STAGE_OTHER, 1);
  }
  if (original_domain) {
    T *tmp = (T *)p->Ahat;   // free once the factors are emitted
    struct { void *buf; int64_t P; } f[3] = {{dU, n1 * k}, {dS, k}, {dV, n2 * k}};
    for (auto &x : f) {
      if ((s = run_ttm<T>(p, (const T *)x.buf, x.P, (const T *)dM, true, tmp, nullptr)) != TSVDM_OK)
        return s;
      CK(cudaMemcpyAsync(x.buf, tmp, e * x.P * n3, cudaMemcpyDeviceToDevice, p->st));
    }
  }
  if (sU) CK(cudaMemcpyAsync(U, dU, e * n1 * k * n3, cudaMemcpyDeviceToHost, p->st));
  if (sS) CK(cudaMemcpyAsync(S, dS, e * k * n3, cudaMemcpyDeviceToHost, p->st));
  if (sV) CK(cudaMemcpyAsync(V, dV, e * n2 * k * n3, cudaMemcpyDeviceToHost, p->st));
  if (rel_err || sU || sS || sV) {
    double sc[SC_COUNT];
    CK(cudaMemcpyAsync(sc, p->scal, sizeof(sc), cudaMemcpyDeviceToHost, p->st));
    CK(cudaStreamSynchronize(p->st));
    if (rel_err) {
      if (!p->ortho) *rel_err = NAN;
      else *rel_err = sc[SC_TOTAL] > 0 ? sqrt(sc[SC_DISCARD] / sc[SC_TOTAL]) : 0.0;
    }
    return read_status(p);
  }
  return TSVDM_OK;
}

template <typename T>
tsvdm_status tolerance_impl(tsvdm_plan_s *p, const void *X, const void *M, double eps,
                            int32_t *ranks, int64_t *offsets, void *U, void *S, void *V,
                            int64_t capacity, int64_t *total_rank, double *rel_err) {
  const size_t e = p->esz;
  const int64_t n1 = p->n1, n2 = p->n2, n3 = p->n3;
  void *dX, *dM;
  bool sX, sM;
  tsvdm_status s;
  if ((s = stage_in(p, STG_X, X, e * n1 * n2 * n3, true, &dX, &sX)) != TSVDM_OK) return s;
  if ((s = stage_in(p, STG_M, M, e * m_elems(p), true, &dM, &sM)) != TSVDM_OK) return s;
  if ((s = decompose<T>(p, (const T *)dX, (const T *)dM)) != TSVDM_OK) return s;
  stage_begin(p, TSVDM_STAGE_SELECT);
  CK(select_ranks<T>((const T *)p->sig, (int)p->cols, (int)n3, eps, p->keys, p->scal,
                     p->ranks_ws, p->off_ws, p->status, p->st));
  stage_end(p, TSVDM_STAGE_SELECT, select_launches(sizeof(T) == 8));
  double sc[SC_COUNT];
  CK(cudaMemcpyAsync(sc, p->scal, sizeof(sc), cudaMemcpyDeviceToHost, p->st));
  if (ranks)
    CK(cudaMemcpyAsync(ranks, p->ranks_ws, sizeof(int32_t) * n3, cudaMemcpyDefault, p->st));
  if (offsets)
    CK(cudaMemcpyAsync(offsets, p->off_ws, sizeof(int64_t) * (n3 + 1), cudaMemcpyDefault, p->st));
  CK(cudaStreamSynchronize(p->st));
  const int64_t tot = (int64_t)sc[SC_TOTRANK];
  *total_rank = tot;
  if (rel_err) *rel_err = sc[SC_TOTAL] > 0 ? sqrt(sc[SC_DISCARD] / sc[SC_TOTAL]) : 0.0;
  p->tol_valid = 1;
  p->tol_total = tot;
  tsvdm_status dev = read_status(p);
  if (!U && !S && !V) return dev;
  if (capacity < tot) return TSVDM_ECAPACITY;
  if ((s = tsvdm_tolerance_pack(p, U, S, V, capacity)) != TSVDM_OK) return s;
  return dev;
}

template <typename T>
tsvdm_status pack_impl(tsvdm_plan_s *p, void *U, void *S, void *V) {
  const size_t e = p->esz;
  const int64_t tot = p->tol_total;
  void *dU, *dS, *dV;
  bool sU, sS, sV;
  tsvdm_status s;
  if ((s = stage_in(p, STG_U, U, e * p->n1 * (tot > 0 ? tot : 1), false, &dU, &sU)) != TSVDM_OK) return s;
  if ((s = stage_in(p, STG_S, S, e * (tot > 0 ? tot : 1), false, &dS, &sS)) != TSVDM_OK) return s;
  if ((s = stage_in(p, STG_V, V, e * p->n2 * (tot > 0 ? tot : 1), false, &dV, &sV)) != TSVDM_OK) return s;
  if (tot > 0) {
    if ((s = emit<T>(p, 0, p->ranks_ws, p->off_ws, (T *)dU, (T *)dS, (T *)dV)) != TSVDM_OK) return s;
    if (p->twopass) p->tol_valid = 0;   // the second pass used the kept slices as scratch
    if (sU) CK(cudaMemcpyAsync(U, dU, e * p->n1 * tot, cudaMemcpyDeviceToHost, p->st));
    if (sS) CK(cudaMemcpyAsync(S, dS, e * tot, cudaMemcpyDeviceToHost, p->st));
    if (sV) CK(cudaMemcpyAsync(V, dV, e * p->n2 * tot, cudaMemcpyDeviceToHost, p->st));
  }
  if (sU || sS || sV) CK(cudaStreamSynchronize(p->st));
  return TSVDM_OK;
}

// C = alpha A^T B over the long mode: tensor cores for FP32 plans unless the FMA engine was
// chosen (tsvdm_plan_set_engine) or the shape does not fit, CUDA cores otherwise.
template <typename T>
cudaError_t atb_any(tsvdm_plan_s *p, const T *A, const T *B, int64_t P, int64_t n, T *C,
                    const double *alpha) {
  if constexpr (sizeof(T) == 4) {
    if (p->engine != JACOBI_FMA && atb_tc_supported((const float *)A, (const float *)B, P, n))
      return atb_tc((const float *)A, (const float *)B, P, n, (float *)C, alpha, p->splitk,
                    p->splitk_elems, p->status, p->st);
  }
  return gemm_atb<T>(A, B, P, n, C, alpha, p->splitk, p->splitk_elems, p->st);
}

// Out_i (+)= U_i diag(S_i) V_i^T: tensor cores for FP32 plans unless the FMA engine was
// chosen (tsvdm_plan_set_engine), CUDA cores otherwise.
template <typename T>
cudaError_t products(tsvdm_plan_s *p, const T *U, const T *S, const T *V,
                     const int64_t *offsets, int64_t k, int64_t n3, T *Out, bool subtract,
                     double *sumsq) {
  if constexpr (sizeof(T) == 4) {
    if (p->engine != JACOBI_FMA)
      return slice_products_tc(U, S, V, offsets, k, p->n1, p->n2, n3, Out, subtract, sumsq,
                               p->status, p->st);
  }
  return slice_products<T>(U, S, V, offsets, k, p->n1, p->n2, n3, Out, subtract, sumsq, p->st);
}

template <typename T>
tsvdm_status reconstruct_impl(tsvdm_plan_s *p, const void *U, const void *S, const void *V,
                              const int64_t *offsets, int64_t k, const void *M, void *Xk) {
  p->tol_valid = 0;
  stage_begin(p, TSVDM_STAGE_OTHER);
  CK(products<T>(p, (const T *)U, (const T *)S, (const T *)V, offsets, k, p->n3,
                 (T *)p->Ahat, false, nullptr));
  stage_end(p, TSVDM_STAGE_OTHER, 1);
  return run_ttm<T>(p, (const T *)p->Ahat, p->n1 * p->n2, (const T *)M, true, (T *)Xk, nullptr);
}

template <typename T>
tsvdm_status backward_impl(tsvdm_plan_s *p, const void *X, const void *M, int64_t k,
                           const void *U, const void *S, const void *V, double dL, void *dX,
                           void *dM, double *loss) {
  p->tol_valid = 0;
  const int64_t P = p->n1 * p->n2, n = p->n3;
  CK(cudaMemsetAsync(p->scal, 0, sizeof(double) * SC_COUNT, p->st));
  tsvdm_status s = run_ttm<T>(p, (const T *)X, P, (const T *)M, false, (T *)p->Ahat,
                              p->scal + SC_XNORM2);
  if (s != TSVDM_OK) return s;
  stage_begin(p, TSVDM_STAGE_OTHER);
  CK(products<T>(p, (const T *)U, (const T *)S, (const T *)V, nullptr, k, n, (T *)p->Ahat,
                 true, p->scal + SC_E));
  CK(backward_scalars(p->scal, dL, p->st));
  stage_end(p, TSVDM_STAGE_OTHER, 2);
  if (dX) {
    stage_begin(p, TSVDM_STAGE_TTM);
    CK(ttm_any<T>(p, (const T *)p->Ahat, P, (const T *)M, true, (T *)dX, p->scal + SC_ALPHA,
                  p->scal + SC_BETA, (const T *)X, nullptr));
    stage_end(p, TSVDM_STAGE_TTM, 1);
  }
  if (dM) {
    stage_begin(p, TSVDM_STAGE_OTHER);
    CK(atb_any<T>(p, (const T *)p->Ahat, (const T *)X, P, n, (T *)dM, p->scal + SC_ALPHA));
    stage_end(p, TSVDM_STAGE_OTHER, 2);
  }
  if (loss && is_device_ptr(loss)) {
    CK(cudaMemcpyAsync(loss, p->scal + SC_LOSS, sizeof(double), cudaMemcpyDeviceToDevice, p->st));
  } else if (loss) {
    double sc[SC_COUNT];
    CK(cudaMemcpyAsync(sc, p->scal, sizeof(sc), cudaMemcpyDeviceToHost, p->st));
    CK(cudaStreamSynchronize(p->st));
    *loss = sc[SC_LOSS];
  }
  return TSVDM_OK;
}

bool valid_plan(tsvdm_plan p) { return p != nullptr && p->Ahat != nullptr; }

void free_plan(tsvdm_plan_s *p) {
  void *bufs[] = {p->dct_tab, p->tp_desc, p->tp_off, p->tp_sweeps, p->tp_sig, p->tp_perm, p->Ahat, p->Wt, p->Vw, p->sig, p->keys,
                  p->perm, p->sweeps, p->status,
                  p->queue, p->ranks_ws, p->off_ws, p->rots, p->scal, p->splitk, p->tc_ws,
                  p->norm2, p->sched, p->dtmp, p->warm_buf};
  for (void *b : bufs)
    if (b) cudaFree(b);
  if (p->dsub) free_plan(p->dsub);
  if (p->dbuf) cudaFree(p->dbuf);
  for (int i = 0; i < STG_COUNT; ++i)
    if (p->stage[i]) cudaFree(p->stage[i]);
  for (int i = 0; i < 2 * TSVDM_STAGE_COUNT; ++i)
    if (p->ev[i]) cudaEventDestroy(p->ev[i]);
  delete p;
}

}  // namespace

// Data-driven M (Sec. 2.2): the transposed left singular vectors of the mode-3 unfolding,
// i.e. the eigenvectors of G = X_mat^T X_mat, from the library's own Jacobi SVD of G.
template <typename T>
tsvdm_status data_transform_impl(tsvdm_plan_s *p, const void *X, void *M) {
  const int64_t P = p->n1 * p->n2, n = p->n3;
  const size_t e = p->esz;
  void *dX, *dM;
  bool sX, sM;
  tsvdm_status s;
  if ((s = stage_in(p, STG_X, X, e * P * n, true, &dX, &sX)) != TSVDM_OK) return s;
  if ((s = stage_in(p, STG_M, M, e * n * n, false, &dM, &sM)) != TSVDM_OK) return s;
  if (!p->dsub) {
    tsvdm_plan sub = nullptr;
    s = tsvdm_plan_create(n, n, 1, p->dtype, p->dtype == TSVDM_F32 ? TSVDM_P_FP32 : TSVDM_P_FP64,
                          1, p->st, &sub);
    if (s != TSVDM_OK) return s;
    sub->engine = p->engine;
    sub->angle32 = p->angle32;
    if (cudaMalloc(&p->dbuf, e * (3 * n * n + n + 16)) != cudaSuccess) {
      cudaGetLastError();
      free_plan(sub);
      return TSVDM_ENOMEM;
    }
    p->dsub = sub;
  }
  T *G = (T *)p->dbuf, *one = G + n * n, *U = one + 16, *S = U + n * n, *V = S + n;
  const T unit = T(1);
  CK(cudaMemcpyAsync(one, &unit, sizeof(T), cudaMemcpyHostToDevice, p->st));
  stage_begin(p, TSVDM_STAGE_OTHER);
  CK(atb_any<T>(p, (const T *)dX, (const T *)dX, P, n, G, nullptr));
  stage_end(p, TSVDM_STAGE_OTHER, 2);
  // G = W diag(sigma) W^T (symmetric PSD): the one-slice t-SVD with M = [1] gives W in U
  if ((s = fixed_rank_impl<T>(p->dsub, G, one, n, U, S, V, 0, nullptr)) != TSVDM_OK) return s;
  stage_begin(p, TSVDM_STAGE_OTHER);
  CK(transpose_slices<T>(U, n, n, 1, (T *)dM, p->st));         // M = W^T
  stage_end(p, TSVDM_STAGE_OTHER, 1);
  if (sM) CK(cudaMemcpyAsync(M, dM, e * n * n, cudaMemcpyDeviceToHost, p->st));
  CK(cudaStreamSynchronize(p->st));
  return TSVDM_OK;
}

extern "C" {

const char *tsvdm_strerror(tsvdm_status s) {
  switch (s) {
    case TSVDM_OK: return "success";
    case TSVDM_EINVAL: return "invalid argument";
    case TSVDM_ENOTORTHO: return "operation needs an orthogonal transform M";
    case TSVDM_ENOCONV: return "Jacobi iteration reached the sweep cap";
    case TSVDM_ENONFINITE: return "non-finite value in the transformed slices";
    case TSVDM_ETIMEOUT: return "a bounded device wait ran out";
    case TSVDM_ENOMEM: return "out of memory";
    case TSVDM_ECAPACITY: return "output capacity below the total rank";
    case TSVDM_ECUDA: return "CUDA runtime error";
    case TSVDM_ENOTSUP: return "not supported";
    case TSVDM_ESCRATCH: return "problem exceeds the fixed scratch of the allocation-free entry point";
  }
  return "unknown status";
}

tsvdm_status tsvdm_plan_create(int64_t n1, int64_t n2, int64_t n3, tsvdm_dtype dtype,
                               tsvdm_prec prec, int m_is_orthogonal, void *stream,
                               tsvdm_plan *out) {
  if (!out) return TSVDM_EINVAL;
  *out = nullptr;
  if (n1 <= 0 || n2 <= 0 || n3 <= 0) return TSVDM_EINVAL;
  if (n1 > (1 << 30) || n2 > (1 << 30) || n3 > (1 << 30)) return TSVDM_EINVAL;
  if (dtype != TSVDM_F32 && dtype != TSVDM_F64) return TSVDM_EINVAL;
  if (dtype == TSVDM_F64 && prec != TSVDM_P_FP64) return TSVDM_ENOTSUP;
  if (dtype == TSVDM_F32 && prec != TSVDM_P_FP32 && prec != TSVDM_P_TF32 &&
      prec != TSVDM_P_BF16X3)
    return TSVDM_ENOTSUP;
  tsvdm_plan_s *p = new (std::nothrow) tsvdm_plan_s();
  if (!p) return TSVDM_ENOMEM;
  p->n1 = n1;
  p->n2 = n2;
  p->n3 = n3;
  p->dtype = dtype;
  p->prec = prec;
  p->ortho = m_is_orthogonal ? 1 : 0;
  p->st = (cudaStream_t)stream;
  p->esz = dtype == TSVDM_F32 ? 4 : 8;
  p->transposed = n1 < n2;
  p->rows = n1 < n2 ? n2 : n1;
  p->cols = n1 < n2 ? n1 : n2;
  const size_t e = p->esz;
  const size_t nx = (size_t)n1 * n2 * n3;
  const size_t nv = (size_t)p->cols * p->cols * n3;
  const size_t ns = (size_t)p->cols * n3;
  p->splitk_elems = (size_t)n3 * n3;
  {
    size_t splits = (size_t)8 * 1024 * 1024 / ((size_t)n3 * n3);
    if (splits < 1) splits = 1;
    if (splits > 256) splits = 256;
    p->splitk_elems *= splits;
  }
  cudaError_t err = cudaSuccess;
#define AL(ptr, bytes) \
  if (err == cudaSuccess) err = cudaMalloc((void **)&(ptr), (bytes) > 0 ? (bytes) : 16)
  AL(p->Ahat, e * nx);
  if (p->transposed) AL(p->Wt, e * nx);
  AL(p->Vw, e * nv);
  AL(p->sig, e * ns);
  AL(p->perm, sizeof(int) * ns);
  AL(p->keys, select_workspace_bytes(p->cols, n3));
  AL(p->sweeps, sizeof(int) * n3);
  AL(p->rots, sizeof(long long) * n3);
  AL(p->norm2, sizeof(float) * ns);
  AL(p->status, sizeof(int));
  AL(p->queue, sizeof(int));
  p->sched_bytes = jacobi_sched_bytes(n3, p->cols);
  AL(p->sched, p->sched_bytes);
  AL(p->ranks_ws, sizeof(int) * n3);
  AL(p->tp_desc, sizeof(SliceDesc) * n3);
  AL(p->tp_off, sizeof(int64_t) * n3);
  AL(p->tp_sweeps, sizeof(int) * n3);
  AL(p->off_ws, sizeof(int64_t) * (n3 + 1));
  AL(p->scal, sizeof(double) * SC_COUNT);
  AL(p->splitk, sizeof(double) * p->splitk_elems);
  if (prec == TSVDM_P_TF32 || prec == TSVDM_P_BF16X3) {
    p->tc_ws_bytes = ttm_tc_workspace(n3, n3);
    AL(p->tc_ws, p->tc_ws_bytes);
  }
#undef AL
  if (err == cudaSuccess) err = cudaMemset(p->status, 0, sizeof(int));
  if (err == cudaSuccess) err = cudaMemset(p->scal, 0, sizeof(double) * SC_COUNT);
  if (err != cudaSuccess) {
    cudaGetLastError();
    free_plan(p);
    return err == cudaErrorMemoryAllocation ? TSVDM_ENOMEM : TSVDM_ECUDA;
  }
  *out = p;
  return TSVDM_OK;
}

tsvdm_status tsvdm_plan_create_dway(int d, const int64_t *dims, tsvdm_dtype dtype,
                                    tsvdm_prec prec, int m_is_orthogonal, void *stream,
                                    tsvdm_plan *out) {
  if (!out || !dims) return TSVDM_EINVAL;
  *out = nullptr;
  if (d < 3 || d > TSVDM_MAX_ORDER) return TSVDM_EINVAL;
  int64_t n3 = 1;
  for (int i = 2; i < d; ++i) {
    if (dims[i] <= 0 || dims[i] > (1 << 30)) return TSVDM_EINVAL;
    if (n3 > ((int64_t)1 << 30) / dims[i]) return TSVDM_EINVAL;
    n3 *= dims[i];
  }
  tsvdm_plan p = nullptr;
  tsvdm_status s = tsvdm_plan_create(dims[0], dims[1], n3, dtype, prec, m_is_orthogonal, stream,
                                     &p);
  if (s != TSVDM_OK) return s;
  if (d > 3) {
    p->dw = d - 2;
    int64_t off = 0;
    for (int m = 0; m < p->dw; ++m) {
      p->td[m] = dims[2 + m];
      p->mo[m] = off;
      off += dims[2 + m] * dims[2 + m];
    }
    p->msum = off;
    if (cudaMalloc(&p->dtmp, p->esz * (size_t)p->n1 * p->n2 * n3) != cudaSuccess) {
      cudaGetLastError();
      free_plan(p);
      return TSVDM_ENOMEM;
    }
  }
  *out = p;
  return TSVDM_OK;
}

tsvdm_status tsvdm_plan_destroy(tsvdm_plan plan) {
  if (!plan) return TSVDM_EINVAL;
  cudaStreamSynchronize(plan->st);
  free_plan(plan);
  return TSVDM_OK;
}

tsvdm_status tsvdm_plan_set_jacobi(tsvdm_plan plan, double tol, int max_sweeps) {
  if (!valid_plan(plan)) return TSVDM_EINVAL;
  plan->tol = tol > 0 ? tol : 0.0;
  plan->max_sweeps = max_sweeps > 0 ? max_sweeps : 40;
  return TSVDM_OK;
}

tsvdm_status tsvdm_plan_set_tuning(tsvdm_plan plan, int block_width, int cluster_size,
                                   int clusters, int stages, int ordering, int inner_sweeps) {
  if (!valid_plan(plan)) return TSVDM_EINVAL;
  if (block_width != 0 && block_width != 16 && block_width != 32 && block_width != 64)
    return TSVDM_EINVAL;
  if (cluster_size < 0 || cluster_size > 16 || clusters < 0) return TSVDM_EINVAL;
  if (stages != 0 && stages != 2 && stages != 3) return TSVDM_EINVAL;
  if (ordering < 0 || ordering > 2) return TSVDM_EINVAL;
  if (inner_sweeps < 0 || inner_sweeps > 8) return TSVDM_EINVAL;
  plan->inner_sweeps = inner_sweeps > 0 ? inner_sweeps : 2;
  plan->width_hint = block_width;
  plan->stages_hint = stages;
  plan->sort_cols = ordering == 2 ? 0 : 1;
  plan->cluster_hint = cluster_size;
  plan->grid_hint = clusters;
  return TSVDM_OK;
}

tsvdm_status tsvdm_plan_set_engine(tsvdm_plan plan, int engine) {
  if (!valid_plan(plan)) return TSVDM_EINVAL;
  if (engine != TSVDM_JACOBI_AUTO && engine != TSVDM_JACOBI_FMA && engine != TSVDM_JACOBI_TC)
    return TSVDM_EINVAL;
  if (engine == TSVDM_JACOBI_TC && plan->dtype != TSVDM_F32) return TSVDM_ENOTSUP;
  plan->engine = engine == TSVDM_JACOBI_TC ? JACOBI_TC
                                           : (engine == TSVDM_JACOBI_FMA ? JACOBI_FMA : JACOBI_AUTO);
  return TSVDM_OK;
}

tsvdm_status tsvdm_plan_set_angle_precision(tsvdm_plan plan, int angles) {
  if (!valid_plan(plan)) return TSVDM_EINVAL;
  if (angles != TSVDM_ANGLE_FP64 && angles != TSVDM_ANGLE_FP32) return TSVDM_EINVAL;
  plan->angle32 = angles == TSVDM_ANGLE_FP32 ? 1 : 0;
  return TSVDM_OK;
}

tsvdm_status tsvdm_plan_set_vectors(tsvdm_plan plan, int mode) {
  if (!valid_plan(plan)) return TSVDM_EINVAL;
  if (mode != TSVDM_VECTORS_ACCUMULATE && mode != TSVDM_VECTORS_SECOND_PASS) return TSVDM_EINVAL;
  if (mode == TSVDM_VECTORS_SECOND_PASS) {
    const size_t ns = (size_t)plan->cols * plan->n3;
    cudaError_t e = cudaSuccess;
    if (!plan->Wt) e = cudaMalloc(&plan->Wt, plan->esz * (size_t)plan->n1 * plan->n2 * plan->n3);
    if (e == cudaSuccess && !plan->tp_sig) e = cudaMalloc(&plan->tp_sig, plan->esz * ns);
    if (e == cudaSuccess && !plan->tp_perm) e = cudaMalloc((void **)&plan->tp_perm, sizeof(int) * ns);
    if (e != cudaSuccess) {
      cudaGetLastError();
      return TSVDM_ENOMEM;
    }
  }
  plan->vec_mode = mode;
  plan->tol_valid = 0;
  return TSVDM_OK;
}

tsvdm_status tsvdm_plan_set_transform(tsvdm_plan plan, int kind) {
  if (!valid_plan(plan)) return TSVDM_EINVAL;
  if (kind == TSVDM_TRANSFORM_DENSE) {
    plan->xform = kind;
    plan->tol_valid = 0;
    return TSVDM_OK;
  }
  if (kind != TSVDM_TRANSFORM_DCT2 || !plan->ortho) return TSVDM_EINVAL;
  const int modes = plan->dw ? plan->dw : 1;
  int64_t len[TSVDM_MAX_ORDER];
  int64_t pairs = 0;
  for (int m = 0; m < modes; ++m) {
    len[m] = plan->dw ? plan->td[m] : plan->n3;
    if (len[m] < 1 || len[m] > 4096 || (len[m] & (len[m] - 1)) != 0) return TSVDM_ENOTSUP;
    pairs += dct_table_pairs(len[m]);
  }
  // twiddle tables, computed in double precision and stored in the plan's precision
  std::vector<double> h((size_t)pairs * 2);
  int64_t off[TSVDM_MAX_ORDER];
  int64_t at = 0;
  const double pi = 3.14159265358979323846;
  for (int m = 0; m < modes; ++m) {
    off[m] = at;
    const int64_t n = len[m], nh = n > 1 ? n / 2 : 1;
    double *fw = h.data() + 2 * at, *iw = fw + 2 * nh, *post = iw + 2 * nh, *pre = post + 2 * n;
    for (int64_t j = 0; j < nh; ++j) {
      const double a = 2.0 * pi * (double)j / (double)n;
      fw[2 * j] = cos(a);
      fw[2 * j + 1] = -sin(a);
      iw[2 * j] = cos(a);
      iw[2 * j + 1] = sin(a);
    }
    for (int64_t k = 0; k < n; ++k) {
      const double sk = sqrt((k == 0 ? 1.0 : 2.0) / (double)n);
      const double a = pi * (double)k / (2.0 * (double)n);
      post[2 * k] = sk * cos(a);
      post[2 * k + 1] = -sk * sin(a);
      pre[2 * k] = cos(a) / (sk * (double)n);
      pre[2 * k + 1] = sin(a) / (sk * (double)n);
    }
    at += dct_table_pairs(n);
  }
  const size_t bytes = (size_t)pairs * 2 * plan->esz;
  if (plan->dct_tab) cudaFree(plan->dct_tab);
  plan->dct_tab = nullptr;
  if (cudaMalloc(&plan->dct_tab, bytes) != cudaSuccess) {
    cudaGetLastError();
    return TSVDM_ENOMEM;
  }
  cudaError_t e;
  if (plan->dtype == TSVDM_F64) {
    e = cudaMemcpy(plan->dct_tab, h.data(), bytes, cudaMemcpyHostToDevice);
  } else {
    std::vector<float> f(h.size());
    for (size_t i = 0; i < h.size(); ++i) f[i] = (float)h[i];
    e = cudaMemcpy(plan->dct_tab, f.data(), bytes, cudaMemcpyHostToDevice);
  }
  if (e != cudaSuccess) return from_cuda(e);
  for (int m = 0; m < modes; ++m) plan->dct_off[m] = off[m] * 2 * (int64_t)plan->esz;
  plan->xform = kind;
  plan->tol_valid = 0;
  return TSVDM_OK;
}

tsvdm_status tsvdm_plan_set_wait_limit(tsvdm_plan plan, int64_t polls) {
  if (!valid_plan(plan) || polls < 0 || polls > 0xffffffffLL) return TSVDM_EINVAL;
  plan->wait_polls = polls;
  return TSVDM_OK;
}

tsvdm_status tsvdm_data_transform(tsvdm_plan plan, const void *X, void *M) {
  if (!valid_plan(plan) || !X || !M) return TSVDM_EINVAL;
  if (plan->dw) return TSVDM_ENOTSUP;
  begin_call(plan);
  if (plan->dtype == TSVDM_F32) return data_transform_impl<float>(plan, X, M);
  return data_transform_impl<double>(plan, X, M);
}

tsvdm_status tsvdm_plan_set_warm_start(tsvdm_plan plan, int enable) {
  if (!valid_plan(plan)) return TSVDM_EINVAL;
  plan->warm_valid = 0;              // the next decomposition starts cold
  plan->warm = 0;
  if (!enable) return TSVDM_OK;
  if (!plan->warm_buf &&
      cudaMalloc(&plan->warm_buf, plan->esz * (size_t)plan->rows * plan->cols * plan->n3) !=
          cudaSuccess) {
    cudaGetLastError();
    plan->warm_buf = nullptr;
    return TSVDM_ENOMEM;
  }
  plan->warm = 1;
  return TSVDM_OK;
}

tsvdm_status tsvdm_transform(tsvdm_plan plan, const void *X, const void *M, int inverse,
                             void *Y) {
  if (!valid_plan(plan) || !X || !M || !Y || X == Y) return TSVDM_EINVAL;
  begin_call(plan);
  plan->tol_valid = 0;
  const int64_t P = plan->n1 * plan->n2;
  if (plan->dtype == TSVDM_F32)
    return run_ttm<float>(plan, (const float *)X, P, (const float *)M, inverse != 0, (float *)Y,
                          nullptr);
  return run_ttm<double>(plan, (const double *)X, P, (const double *)M, inverse != 0, (double *)Y,
                         nullptr);
}

tsvdm_status tsvdm_fixed_rank(tsvdm_plan plan, const void *X, const void *M, int64_t k, void *U,
                              void *S, void *V, int original_domain, double *rel_err) {
  if (!valid_plan(plan) || !X || !M || !U || !S || !V) return TSVDM_EINVAL;
  begin_call(plan);
  if (k < 1 || k > plan->cols) return TSVDM_EINVAL;
  if (original_domain && !plan->ortho) return TSVDM_ENOTORTHO;
  if (plan->dtype == TSVDM_F32)
    return fixed_rank_impl<float>(plan, X, M, k, U, S, V, original_domain, rel_err);
  return fixed_rank_impl<double>(plan, X, M, k, U, S, V, original_domain, rel_err);
}

tsvdm_status tsvdm_tolerance(tsvdm_plan plan, const void *X, const void *M, double eps,
                             int32_t *ranks, int64_t *offsets, void *U, void *S, void *V,
                             int64_t capacity, int64_t *total_rank, double *rel_err) {
  if (!valid_plan(plan) || !X || !M || !total_rank) return TSVDM_EINVAL;
  begin_call(plan);
  if (!(eps > 0.0 && eps < 1.0)) return TSVDM_EINVAL;
  if ((U || S || V) && !(U && S && V)) return TSVDM_EINVAL;
  if (capacity < 0) return TSVDM_EINVAL;
  if (!plan->ortho) return TSVDM_ENOTORTHO;
  if (plan->dtype == TSVDM_F32)
    return tolerance_impl<float>(plan, X, M, eps, ranks, offsets, U, S, V, capacity, total_rank,
                                 rel_err);
  return tolerance_impl<double>(plan, X, M, eps, ranks, offsets, U, S, V, capacity, total_rank,
                                rel_err);
}

tsvdm_status tsvdm_tolerance_pack(tsvdm_plan plan, void *U, void *S, void *V, int64_t capacity) {
  if (!valid_plan(plan) || !U || !S || !V) return TSVDM_EINVAL;
  if (!plan->tol_valid) return TSVDM_EINVAL;
  if (capacity < plan->tol_total) return TSVDM_ECAPACITY;
  if (plan->dtype == TSVDM_F32) return pack_impl<float>(plan, U, S, V);
  return pack_impl<double>(plan, U, S, V);
}

tsvdm_status tsvdm_reconstruct(tsvdm_plan plan, const void *U, const void *S, const void *V,
                               const int64_t *offsets, int64_t k, const void *M, void *Xk) {
  if (!valid_plan(plan) || !U || !S || !V || !M || !Xk) return TSVDM_EINVAL;
  begin_call(plan);
  if (!offsets && (k < 1 || k > plan->cols)) return TSVDM_EINVAL;
  if (plan->dtype == TSVDM_F32)
    return reconstruct_impl<float>(plan, U, S, V, offsets, k, M, Xk);
  return reconstruct_impl<double>(plan, U, S, V, offsets, k, M, Xk);
}

tsvdm_status tsvdm_backward(tsvdm_plan plan, const void *X, const void *M, int64_t k,
                            const void *U, const void *S, const void *V, double dL, void *dX,
                            void *dM, double *loss) {
  if (!valid_plan(plan) || !X || !M || !U || !S || !V) return TSVDM_EINVAL;
  if (plan->dw) return TSVDM_ENOTSUP;
  begin_call(plan);
  if (k < 1 || k > plan->cols) return TSVDM_EINVAL;
  if (plan->dtype == TSVDM_F32)
    return backward_impl<float>(plan, X, M, k, U, S, V, dL, dX, dM, loss);
  return backward_impl<double>(plan, X, M, k, U, S, V, dL, dX, dM, loss);
}

tsvdm_status tsvdm_plan_profile(tsvdm_plan plan, int enable) {
  if (!valid_plan(plan)) return TSVDM_EINVAL;
  if (enable && !plan->ev[0]) {
    for (int i = 0; i < 2 * TSVDM_STAGE_COUNT; ++i) CK(cudaEventCreate(&plan->ev[i]));
  }
  plan->profile = enable ? 1 : 0;
  return TSVDM_OK;
}

tsvdm_status tsvdm_plan_profile_read(tsvdm_plan plan, float *ms, int64_t *launches) {
  if (!valid_plan(plan)) return TSVDM_EINVAL;
  if (launches) *launches = plan->launches;
  if (!ms) return TSVDM_OK;
  CK(cudaStreamSynchronize(plan->st));
  for (int s = 0; s < TSVDM_STAGE_COUNT; ++s) {
    ms[s] = 0.f;
    if (plan->profile && plan->ran[s]) CK(cudaEventElapsedTime(&ms[s], plan->ev[2 * s], plan->ev[2 * s + 1]));
  }
  return TSVDM_OK;
}

tsvdm_status tsvdm_last_status(tsvdm_plan plan) {
  if (!valid_plan(plan)) return TSVDM_EINVAL;
  return read_status(plan);
}

tsvdm_status tsvdm_plan_stats(tsvdm_plan plan, int64_t *sweeps, int64_t *rotations) {
  if (!valid_plan(plan)) return TSVDM_EINVAL;
  const int64_t n = plan->n3;
  int *sw = (int *)malloc(sizeof(int) * n);
  long long *ro = (long long *)malloc(sizeof(long long) * n);
  if (!sw || !ro) {
    free(sw);
    free(ro);
    return TSVDM_ENOMEM;
  }
  cudaError_t e = cudaMemcpyAsync(sw, plan->sweeps, sizeof(int) * n, cudaMemcpyDeviceToHost, plan->st);
  if (e == cudaSuccess)
    e = cudaMemcpyAsync(ro, plan->rots, sizeof(long long) * n, cudaMemcpyDeviceToHost, plan->st);
  if (e == cudaSuccess) e = cudaStreamSynchronize(plan->st);
  if (e == cudaSuccess) {
    int64_t a = 0, b = 0;
    for (int64_t i = 0; i < n; ++i) {
      a += sw[i] > 0 ? sw[i] : 0;
      b += ro[i];
    }
    if (sweeps) *sweeps = a;
    if (rotations) *rotations = b;
  }
  free(sw);
  free(ro);
  return from_cuda(e);
}

tsvdm_status tsvdm_cayley(int64_t n, tsvdm_dtype dtype, const void *A, const void *M0, void *M,
                          void *Z, void *Q, void *work, void *stream) {
  if (n <= 0 || !A || !M0 || !M || !Z || !Q || !work) return TSVDM_EINVAL;
  cudaStream_t st = (cudaStream_t)stream;
  if (dtype == TSVDM_F32)
    return from_cuda(small_cayley<float>(n, (const float *)A, (const float *)M0, (float *)M,
                                         (float *)Z, (float *)Q, (float *)work, st));
  if (dtype == TSVDM_F64)
    return from_cuda(small_cayley<double>(n, (const double *)A, (const double *)M0, (double *)M,
                                          (double *)Z, (double *)Q, (double *)work, st));
  return TSVDM_EINVAL;
}

tsvdm_status tsvdm_cayley_backward(int64_t n, tsvdm_dtype dtype, const void *M0, const void *Z,
                                   const void *Q, const void *dM, void *dA, void *work,
                                   void *stream) {
  if (n <= 0 || !M0 || !Z || !Q || !dM || !dA || !work) return TSVDM_EINVAL;
  cudaStream_t st = (cudaStream_t)stream;
  if (dtype == TSVDM_F32)
    return from_cuda(small_cayley_backward<float>(n, (const float *)M0, (const float *)Z,
                                                  (const float *)Q, (const float *)dM, (float *)dA,
                                                  (float *)work, st));
  if (dtype == TSVDM_F64)
    return from_cuda(small_cayley_backward<double>(n, (const double *)M0, (const double *)Z,
                                                   (const double *)Q, (const double *)dM,
                                                   (double *)dA, (double *)work, st));
  return TSVDM_EINVAL;
}

tsvdm_status tsvdm_adam(int64_t count, tsvdm_dtype dtype, void *param, const void *grad,
                        void *m1, void *m2, int64_t step, double lr, double beta1, double beta2,
                        double eps, void *stream) {
  if (count <= 0 || !param || !grad || !m1 || !m2 || step < 1) return TSVDM_EINVAL;
  cudaStream_t st = (cudaStream_t)stream;
  if (dtype == TSVDM_F32)
    return from_cuda(small_adam<float>(count, (float *)param, (const float *)grad, (float *)m1,
                                       (float *)m2, step, lr, beta1, beta2, eps, st));
  if (dtype == TSVDM_F64)
    return from_cuda(small_adam<double>(count, (double *)param, (const double *)grad,
                                        (double *)m1, (double *)m2, step, lr, beta1, beta2, eps,
                                        st));
  return TSVDM_EINVAL;
}

}  // extern "C"
