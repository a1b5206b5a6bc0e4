// Batched t-SVDM of many tensors with uneven shapes, mixing t-SVDM-I (rank k) and
// t-SVDM-II (tolerance eps), in one stream of work that can be captured once into a CUDA
// graph and replayed.  The dominant step is ONE persistent Jacobi launch over every slice
// of every tensor (slice descriptors, longest slices first so the tail is short).
//
//   per tensor   mode-3 TTM (tensor cores for TF32/BF16x3 when the shape allows);
//                transposition of slices when n1 < n2
//   one launch   batched one-sided Jacobi over all slices (persistent clusters)
//   one launch   finalize (norms, per-slice order) over all slices
//   one launch   t-SVDM-II selection, one CTA per tolerance tensor
//   per tensor   factor emission (uniform k or packed variable rank)
//   one launch   relative errors of all tensors
// t-SVDM-II outputs use the full capacity n3 min(n1,n2) columns, so nothing is read back
// and the whole batch runs without a host synchronisation.
#include <math.h>
#include <stdlib.h>
#include <string.h>

#include <algorithm>
#include <new>
#include <vector>

#include "common.cuh"

using namespace tsvdm;

namespace {

struct Item {
  tsvdm_batch_desc d;
  int64_t rows, cols;
  bool transposed;
  size_t off_ahat, off_wt, off_vw, off_sig;   // element offsets in the T arena
  size_t off_perm, off_norm2, off_ranks;      // int / float arena offsets
  size_t off_offs, off_keys, off_scal;        // int64 / key / double arena offsets
  int64_t first_slice;
};

struct RelErrArg {
  const double *scal;
  double *out;
};

__global__ void rel_err_kernel(const RelErrArg *args, int count) {
  int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= count || !args[i].out) return;
  double tot = args[i].scal[SC_TOTAL], dis = args[i].scal[SC_DISCARD];
  *args[i].out = tot > 0.0 ? sqrt(dis / tot) : 0.0;
}

tsvdm_status from_cuda(cudaError_t e) {
  if (e == cudaSuccess) return TSVDM_OK;
  if (e == cudaErrorMemoryAllocation) return TSVDM_ENOMEM;
  return TSVDM_ECUDA;
}
#define CKB(expr)                                   \
  do {                                              \
    cudaError_t _e = (expr);                        \
    if (_e != cudaSuccess) return from_cuda(_e);    \
  } while (0)

}  // namespace

struct tsvdm_batch_s {
  std::vector<Item> items;
  tsvdm_dtype dtype = TSVDM_F32;
  tsvdm_prec prec = TSVDM_P_FP32;
  cudaStream_t st = nullptr;
  size_t esz = 4;
  int64_t total_slices = 0;
  int max_cols = 0, min_cols = 1 << 30, max_rows = 0;
  void *arena = nullptr;        // T elements
  int *iarena = nullptr;        // perm, ranks
  float *farena = nullptr;      // norm2
  int64_t *larena = nullptr;    // offsets
  unsigned long long *karena = nullptr;   // selection scratch (FP64 tail sums)
  double *darena = nullptr;     // scalars
  SliceDesc *desc = nullptr;    // device
  SelectSeg *segs = nullptr;    // device
  int nsegs = 0;
  RelErrArg *relargs = nullptr; // device
  void *tc_ws = nullptr;
  size_t tc_ws_bytes = 0;
  int *status = nullptr, *queue = nullptr, *sweeps = nullptr;
  void *sched = nullptr;
  size_t sched_bytes = 0;
  long long *rots = nullptr;
  std::vector<RelErrArg> h_rel;
  // Jacobi launch shape (autotuned)
  int width = 0, cluster = 2, clusters = 0, stages = 0, engine = JACOBI_AUTO;
  double tol = 0.0;
  int max_sweeps = 40;
  // graph
  cudaGraph_t graph = nullptr;
  cudaGraphExec_t exec = nullptr;
  float last_jacobi_ms = 0.f;
  cudaEvent_t ev[2] = {nullptr, nullptr};
};

namespace {

template <typename T>
tsvdm_status run_batch(tsvdm_batch_s *b, const tsvdm_batch_io *io, bool timed) {
  cudaStream_t st = b->st;
  T *arena = (T *)b->arena;
  for (size_t i = 0; i < b->items.size(); ++i) {
    const Item &it = b->items[i];
    const int64_t P = it.d.n1 * it.d.n2, n = it.d.n3;
    T *Ahat = arena + it.off_ahat;
    cudaError_t e = cudaErrorNotSupported;
    if constexpr (sizeof(T) == 4) {
      if ((b->prec == TSVDM_P_TF32 || b->prec == TSVDM_P_BF16X3) &&
          ttm_tc_supported(P, n, n, io[i].X, Ahat))
        e = ttm_tc((const float *)io[i].X, P, n, (const float *)io[i].M, n, false, (int)b->prec,
                   (float *)Ahat, b->tc_ws, b->tc_ws_bytes, nullptr, nullptr, nullptr, nullptr,
                   b->status, st);
    }
    if (e == cudaErrorNotSupported)
      e = ttm_simt<T>((const T *)io[i].X, P, n, (const T *)io[i].M, n, n, false, Ahat, nullptr,
                      nullptr, nullptr, nullptr, st);
    CKB(e);
    if (it.transposed)
      CKB(transpose_slices<T>(Ahat, it.d.n1, it.d.n2, n, arena + it.off_wt, st));
  }
  CKB(cudaMemsetAsync(b->queue, 0, sizeof(int), st));
  CKB(cudaMemsetAsync(b->rots, 0, sizeof(long long) * b->total_slices, st));
  JacobiParams jp{};
  memset(&jp, 0, sizeof(jp));
  jp.rows = 0;
  jp.cols = b->min_cols;     // caps the cluster at the smallest slice's block pairs
  jp.nslices = (int)b->total_slices;
  jp.tol = b->tol > 0 ? b->tol
                      : 4.0 * sqrt((double)b->max_rows) *
                            (sizeof(T) == 4 ? ldexp(1.0, -24) : ldexp(1.0, -53));
  jp.max_sweeps = b->max_sweeps;
  jp.queue = b->queue;
  jp.status = b->status;
  jp.sweeps = b->sweeps;
  jp.rots = b->rots;
  jp.norm2 = nullptr;
  jp.inner_sweeps = 2;
  jp.desc = b->desc;
  jp.engine = b->engine;
  jp.sched = b->sched;
  jp.sched_bytes = b->sched_bytes;
  jp.max_cols = b->max_cols;
  if (timed) CKB(cudaEventRecord(b->ev[0], st));
  CKB(jacobi_run<T>(jp, st, b->width, b->cluster, b->clusters, b->stages));
  if (timed) CKB(cudaEventRecord(b->ev[1], st));
  CKB(jacobi_finalize_desc<T>(b->desc, (int)b->total_slices, b->max_cols, st));
  if (b->nsegs) CKB(select_segments<T>(b->segs, b->nsegs, st));
  for (size_t i = 0; i < b->items.size(); ++i) {
    const Item &it = b->items[i];
    const T *W = it.transposed ? arena + it.off_wt : arena + it.off_ahat;
    const T *sig = arena + it.off_sig;
    const int *perm = b->iarena + it.off_perm;
    double *scal = b->darena + it.off_scal;
    if (it.d.mode == 0) {
      CKB(emit_factors<T>(W, it.rows * it.cols, arena + it.off_vw, it.cols * it.cols, (int)it.rows,
                          (int)it.cols, (int)it.d.n3, it.transposed, sig, perm, it.d.k, nullptr,
                          nullptr, (T *)io[i].U, (T *)io[i].S, (T *)io[i].V, st));
      CKB(trunc_sums<T>(sig, (int)it.cols, (int)it.d.n3, it.d.k, scal, st));
    } else {
      const int *ranks = b->iarena + it.off_ranks;
      const int64_t *offs = b->larena + it.off_offs;
      CKB(emit_factors<T>(W, it.rows * it.cols, arena + it.off_vw, it.cols * it.cols, (int)it.rows,
                          (int)it.cols, (int)it.d.n3, it.transposed, sig, perm, 0, ranks, offs,
                          (T *)io[i].U, (T *)io[i].S, (T *)io[i].V, st));
      if (io[i].ranks)
        CKB(cudaMemcpyAsync(io[i].ranks, ranks, sizeof(int32_t) * it.d.n3,
                            cudaMemcpyDeviceToDevice, st));
      if (io[i].offsets)
        CKB(cudaMemcpyAsync(io[i].offsets, offs, sizeof(int64_t) * (it.d.n3 + 1),
                            cudaMemcpyDeviceToDevice, st));
    }
  }
  rel_err_kernel<<<(unsigned)((b->items.size() + 127) / 128), 128, 0, st>>>(b->relargs,
                                                                           (int)b->items.size());
  CKB(cudaGetLastError());
  return TSVDM_OK;
}

// The relative-error targets are caller pointers: refresh the device argument table.
tsvdm_status upload_rel_targets(tsvdm_batch_s *b, const tsvdm_batch_io *io, bool blocking) {
  for (size_t i = 0; i < b->items.size(); ++i) b->h_rel[i].out = io[i].rel_err;
  const size_t bytes = sizeof(RelErrArg) * b->items.size();
  if (blocking) {
    CKB(cudaStreamSynchronize(b->st));
    CKB(cudaMemcpy(b->relargs, b->h_rel.data(), bytes, cudaMemcpyHostToDevice));
  } else {
    CKB(cudaMemcpyAsync(b->relargs, b->h_rel.data(), bytes, cudaMemcpyHostToDevice, b->st));
    CKB(cudaStreamSynchronize(b->st));   // the host table may be rewritten by the next call
  }
  return TSVDM_OK;
}

tsvdm_status run_any(tsvdm_batch_s *b, const tsvdm_batch_io *io, bool timed) {
  return b->dtype == TSVDM_F32 ? run_batch<float>(b, io, timed) : run_batch<double>(b, io, timed);
}

void free_batch(tsvdm_batch_s *b) {
  if (b->exec) cudaGraphExecDestroy(b->exec);
  if (b->graph) cudaGraphDestroy(b->graph);
  void *bufs[] = {b->arena, b->iarena, b->farena, b->larena, b->karena, b->darena, b->desc,
                  b->segs, b->relargs, b->tc_ws, b->status, b->queue, b->sweeps, b->rots,
                  b->sched};
  for (void *p : bufs)
    if (p) cudaFree(p);
  for (auto &e : b->ev)
    if (e) cudaEventDestroy(e);
  delete b;
}

}  // namespace

extern "C" {

tsvdm_status tsvdm_batch_create(const tsvdm_batch_desc *descs, int count, tsvdm_dtype dtype,
                                tsvdm_prec prec, void *stream, tsvdm_batch *out) {
  if (!descs || count < 1 || !out) return TSVDM_EINVAL;
  *out = nullptr;
  if (dtype != TSVDM_F32 && dtype != TSVDM_F64) return TSVDM_EINVAL;
  if (dtype == TSVDM_F64 && prec != TSVDM_P_FP64) return TSVDM_ENOTSUP;
  if (dtype == TSVDM_F32 && prec == TSVDM_P_FP64) return TSVDM_ENOTSUP;
  tsvdm_batch_s *b = new (std::nothrow) tsvdm_batch_s();
  if (!b) return TSVDM_ENOMEM;
  b->dtype = dtype;
  b->prec = prec;
  b->st = (cudaStream_t)stream;
  b->esz = dtype == TSVDM_F32 ? 4 : 8;
  size_t nT = 0, nI = 0, nF = 0, nL = 0, nK = 0, nD = 0;
  int64_t max_n3 = 1;
  for (int i = 0; i < count; ++i) {
    const tsvdm_batch_desc &d = descs[i];
    if (d.n1 < 1 || d.n2 < 1 || d.n3 < 1 || d.n1 > (1 << 20) || d.n2 > (1 << 20) ||
        d.n3 > 65535) {
      delete b;
      return TSVDM_EINVAL;
    }
    const int64_t r = d.n1 < d.n2 ? d.n1 : d.n2;
    if ((d.mode == 0 && (d.k < 1 || d.k > r)) || (d.mode == 1 && !(d.eps > 0 && d.eps < 1)) ||
        (d.mode != 0 && d.mode != 1) || r > 1024) {
      delete b;
      return TSVDM_EINVAL;
    }
    Item it;
    it.d = d;
    it.transposed = d.n1 < d.n2;
    it.rows = it.transposed ? d.n2 : d.n1;
    it.cols = r;
    // every region starts on a 256-byte boundary (vector loads and asynchronous copies of
    // the slices need at least 16-byte aligned bases)
    auto up = [](size_t v) { return (v + 63) & ~(size_t)63; };
    const size_t nx = (size_t)d.n1 * d.n2 * d.n3;
    it.off_ahat = nT; nT = up(nT + nx);
    it.off_wt = nT; if (it.transposed) nT = up(nT + nx);
    it.off_vw = nT; nT = up(nT + (size_t)r * r * d.n3);
    it.off_sig = nT; nT = up(nT + (size_t)r * d.n3);
    it.off_perm = nI; nI = up(nI + (size_t)r * d.n3);
    it.off_ranks = nI; nI = up(nI + (size_t)d.n3);
    it.off_norm2 = nF; nF = up(nF + (size_t)r * d.n3);
    it.off_offs = nL; nL = up(nL + (size_t)d.n3 + 1);
    it.off_keys = nK; if (d.mode == 1) nK = up(nK + 2 * (size_t)r * d.n3);
    it.off_scal = nD; nD = up(nD + SC_COUNT);
    it.first_slice = b->total_slices;
    b->total_slices += d.n3;
    b->max_cols = std::max<int>(b->max_cols, (int)r);
    b->max_rows = std::max<int>(b->max_rows, (int)it.rows);
    b->min_cols = std::min<int>(b->min_cols, (int)r);
    max_n3 = std::max<int64_t>(max_n3, d.n3);
    b->items.push_back(it);
  }
  cudaError_t e = cudaSuccess;
#define ALB(p, bytes) \
  if (e == cudaSuccess) e = cudaMalloc((void **)&(p), (bytes) > 0 ? (bytes) : 16)
  ALB(b->arena, b->esz * nT);
  ALB(b->iarena, sizeof(int) * nI);
  ALB(b->farena, sizeof(float) * nF);
  ALB(b->larena, sizeof(int64_t) * nL);
  ALB(b->karena, sizeof(unsigned long long) * nK);
  ALB(b->darena, sizeof(double) * nD);
  ALB(b->desc, sizeof(SliceDesc) * b->total_slices);
  ALB(b->segs, sizeof(SelectSeg) * count);
  ALB(b->relargs, sizeof(RelErrArg) * count);
  ALB(b->status, sizeof(int));
  ALB(b->queue, sizeof(int));
  ALB(b->sweeps, sizeof(int) * b->total_slices);
  ALB(b->rots, sizeof(long long) * b->total_slices);
  b->sched_bytes = jacobi_sched_bytes(b->total_slices, b->max_cols);
  ALB(b->sched, b->sched_bytes);
  if (prec == TSVDM_P_TF32 || prec == TSVDM_P_BF16X3) {
    b->tc_ws_bytes = ttm_tc_workspace(max_n3, max_n3);
    ALB(b->tc_ws, b->tc_ws_bytes);
  }
#undef ALB
  if (e == cudaSuccess) e = cudaEventCreate(&b->ev[0]);
  if (e == cudaSuccess) e = cudaEventCreate(&b->ev[1]);
  if (e != cudaSuccess) {
    cudaGetLastError();
    free_batch(b);
    return e == cudaErrorMemoryAllocation ? TSVDM_ENOMEM : TSVDM_ECUDA;
  }
  // slice descriptors, longest slices (rows * cols^2) first
  std::vector<SliceDesc> hd;
  hd.reserve(b->total_slices);
  std::vector<std::pair<double, size_t>> order;
  for (const Item &it : b->items) {
    unsigned char *base = (unsigned char *)b->arena;
    for (int64_t s = 0; s < it.d.n3; ++s) {
      SliceDesc sd;
      const size_t work = it.transposed ? it.off_wt : it.off_ahat;
      sd.A = base + b->esz * (work + (size_t)s * it.rows * it.cols);
      sd.V = base + b->esz * (it.off_vw + (size_t)s * it.cols * it.cols);
      sd.norm2 = b->farena + it.off_norm2 + (size_t)s * it.cols;
      sd.sig = base + b->esz * (it.off_sig + (size_t)s * it.cols);
      sd.perm = b->iarena + it.off_perm + (size_t)s * it.cols;
      sd.rows = (int)it.rows;
      sd.cols = (int)it.cols;
      order.push_back({(double)it.rows * it.cols * it.cols, hd.size()});
      hd.push_back(sd);
    }
  }
  std::stable_sort(order.begin(), order.end(),
                   [](const std::pair<double, size_t> &a, const std::pair<double, size_t> &c) {
                     return a.first > c.first;
                   });
  std::vector<SliceDesc> sorted;
  sorted.reserve(hd.size());
  for (auto &o : order) sorted.push_back(hd[o.second]);
  std::vector<SelectSeg> hs;
  for (const Item &it : b->items) {
    RelErrArg ra;
    ra.scal = b->darena + it.off_scal;
    ra.out = nullptr;
    b->h_rel.push_back(ra);
    if (it.d.mode != 1) continue;
    SelectSeg g;
    g.sig = (unsigned char *)b->arena + b->esz * it.off_sig;
    g.cols = (int)it.cols;
    g.nslices = (int)it.d.n3;
    g.eps = it.d.eps;
    g.keys = b->karena + it.off_keys;
    g.scal = b->darena + it.off_scal;
    g.ranks = b->iarena + it.off_ranks;
    g.offsets = b->larena + it.off_offs;
    hs.push_back(g);
  }
  b->nsegs = (int)hs.size();
  e = cudaMemcpy(b->desc, sorted.data(), sizeof(SliceDesc) * sorted.size(), cudaMemcpyHostToDevice);
  if (e == cudaSuccess && !hs.empty())
    e = cudaMemcpy(b->segs, hs.data(), sizeof(SelectSeg) * hs.size(), cudaMemcpyHostToDevice);
  if (e == cudaSuccess) e = cudaMemset(b->status, 0, sizeof(int));
  if (e == cudaSuccess) e = cudaMemset(b->darena, 0, sizeof(double) * nD);
  if (e != cudaSuccess) {
    free_batch(b);
    return TSVDM_ECUDA;
  }
  b->width = b->min_cols >= 64 ? 64 : 32;
  *out = b;
  return TSVDM_OK;
}

tsvdm_status tsvdm_batch_destroy(tsvdm_batch b) {
  if (!b) return TSVDM_EINVAL;
  cudaStreamSynchronize(b->st);
  free_batch(b);
  return TSVDM_OK;
}

tsvdm_status tsvdm_batch_run(tsvdm_batch b, const tsvdm_batch_io *io) {
  if (!b || !io) return TSVDM_EINVAL;
  for (size_t i = 0; i < b->items.size(); ++i)
    if (!io[i].X || !io[i].M || !io[i].U || !io[i].S || !io[i].V) return TSVDM_EINVAL;
  tsvdm_status s = upload_rel_targets(b, io, false);
  if (s != TSVDM_OK) return s;
  return run_any(b, io, false);
}

tsvdm_status tsvdm_batch_capture(tsvdm_batch b, const tsvdm_batch_io *io) {
  if (!b || !io) return TSVDM_EINVAL;
  if (b->st == nullptr) return TSVDM_EINVAL;   // the legacy default stream cannot be captured
  for (size_t i = 0; i < b->items.size(); ++i)
    if (!io[i].X || !io[i].M || !io[i].U || !io[i].S || !io[i].V) return TSVDM_EINVAL;
  if (b->exec) {
    cudaGraphExecDestroy(b->exec);
    b->exec = nullptr;
  }
  if (b->graph) {
    cudaGraphDestroy(b->graph);
    b->graph = nullptr;
  }
  // Everything the graph reads from the host is uploaded before capture; the first, plain
  // run also settles every launch configuration (occupancy queries, shared-memory limits).
  tsvdm_status s0 = upload_rel_targets(b, io, true);
  if (s0 != TSVDM_OK) return s0;
  s0 = run_any(b, io, false);
  if (s0 != TSVDM_OK) return s0;
  CKB(cudaStreamSynchronize(b->st));
  CKB(cudaStreamBeginCapture(b->st, cudaStreamCaptureModeThreadLocal));
  tsvdm_status s = run_any(b, io, false);
  cudaGraph_t g = nullptr;
  cudaError_t e = cudaStreamEndCapture(b->st, &g);
  if (s != TSVDM_OK) {
    if (g) cudaGraphDestroy(g);
    return s;
  }
  CKB(e);
  b->graph = g;
  CKB(cudaGraphInstantiate(&b->exec, g, 0));
  return TSVDM_OK;
}

tsvdm_status tsvdm_batch_launch(tsvdm_batch b) {
  if (!b || !b->exec) return TSVDM_EINVAL;
  CKB(cudaGraphLaunch(b->exec, b->st));
  return TSVDM_OK;
}

tsvdm_status tsvdm_batch_status(tsvdm_batch b, int64_t *sweeps, int64_t *rotations) {
  if (!b) return TSVDM_EINVAL;
  std::vector<int> sw(b->total_slices);
  std::vector<long long> ro(b->total_slices);
  int s = 0;
  CKB(cudaMemcpyAsync(sw.data(), b->sweeps, sizeof(int) * sw.size(), cudaMemcpyDeviceToHost, b->st));
  CKB(cudaMemcpyAsync(ro.data(), b->rots, sizeof(long long) * ro.size(), cudaMemcpyDeviceToHost, b->st));
  CKB(cudaMemcpyAsync(&s, b->status, sizeof(int), cudaMemcpyDeviceToHost, b->st));
  CKB(cudaStreamSynchronize(b->st));
  int64_t a = 0, c = 0;
  for (size_t i = 0; i < sw.size(); ++i) {
    a += sw[i] > 0 ? sw[i] : 0;
    c += ro[i];
  }
  if (sweeps) *sweeps = a;
  if (rotations) *rotations = c;
  if (s) CKB(cudaMemsetAsync(b->status, 0, sizeof(int), b->st));
  if (s & ST_NONFINITE) return TSVDM_ENONFINITE;
  if (s & ST_TIMEOUT) return TSVDM_ETIMEOUT;
  if (s & ST_NOCONV) return TSVDM_ENOCONV;
  return TSVDM_OK;
}

tsvdm_status tsvdm_batch_graph_kernels(tsvdm_batch b, int64_t *kernels) {
  if (!b || !kernels || !b->graph) return TSVDM_EINVAL;
  size_t n = 0;
  CKB(cudaGraphGetNodes(b->graph, nullptr, &n));
  std::vector<cudaGraphNode_t> nodes(n);
  if (n) CKB(cudaGraphGetNodes(b->graph, nodes.data(), &n));
  int64_t k = 0;
  for (size_t i = 0; i < n; ++i) {
    cudaGraphNodeType t;
    CKB(cudaGraphNodeGetType(nodes[i], &t));
    if (t == cudaGraphNodeTypeKernel) ++k;
  }
  *kernels = k;
  return TSVDM_OK;
}

tsvdm_status tsvdm_batch_tune(tsvdm_batch b, const tsvdm_batch_io *io, int *choice) {
  if (!b || !io) return TSVDM_EINVAL;
  struct Cand { int width, cluster, stages, engine; };
  std::vector<Cand> cands;
  const int widths[2] = {32, 64};
  const int clusters[3] = {1, 2, 4};
  const int stages[2] = {2, 3};
  if (b->dtype == TSVDM_F32 && b->min_cols >= 64)     // tensor-core Gram / apply
    cands.push_back({64, 1, 0, JACOBI_TC});
  for (int w : widths) {
    if (w == 64 && b->min_cols < 64) continue;
    for (int c : clusters)
      for (int s : stages) cands.push_back({w, c, s, JACOBI_FMA});
  }
  tsvdm_status s0 = upload_rel_targets(b, io, false);
  if (s0 != TSVDM_OK) return s0;
  float best = 1e30f;
  Cand bc = {b->width, b->cluster, b->stages, b->engine};
  for (const Cand &c : cands) {
    b->width = c.width;
    b->cluster = c.cluster;
    b->stages = c.stages;
    b->engine = c.engine;
    b->clusters = 0;
    tsvdm_status s = run_any(b, io, true);
    if (s != TSVDM_OK) return s;
    CKB(cudaStreamSynchronize(b->st));
    float ms = 0.f;
    CKB(cudaEventElapsedTime(&ms, b->ev[0], b->ev[1]));
    if (ms < best) {
      best = ms;
      bc = c;
    }
  }
  b->width = bc.width;
  b->cluster = bc.cluster;
  b->stages = bc.stages;
  b->engine = bc.engine;
  b->last_jacobi_ms = best;
  if (choice) {
    choice[0] = bc.width;
    choice[1] = bc.cluster;
    choice[2] = bc.engine == JACOBI_TC ? 0 : (bc.stages == 0 ? 2 : bc.stages);
    choice[3] = (int)(best * 1000.f);
  }
  return TSVDM_OK;
}

}  // extern "C"
