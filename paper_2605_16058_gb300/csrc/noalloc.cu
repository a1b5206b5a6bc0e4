// Allocation-free entry point: the t-SVDM-II rank choice (the same device selection kernels
// that tsvdm_tolerance runs) with its scratch in a fixed, file-scope device array instead
// of a plan's workspace.
//
// Who needs it: callers that must not call cudaMalloc.  Examples are a process that hands
// all device memory to another allocator when it starts (a framework's caching pool), so
// a driver allocation would fail, and latency-bound services that forbid allocation on
// their request path because a driver allocation can synchronise the device and take
// milliseconds.  Such callers already hold the singular values and the output buffers.
//
// The scratch (about 2.1 MiB: one FP64 tail sum per singular value, the search's per-CTA
// partial sums and its state, plus a few FP64 scalars) is part of the library image:
// every GPU that loads the library holds it until the process exits.  Every call shares
// it and keeps the previous call's contents; the search state, which must start at zero,
// is cleared in stream order by each call.  Calls whose kernels overlap on the GPU
// (different streams, or several host threads) race on it; serialise them on one stream.
#include "common.cuh"

namespace {

constexpr int64_t NOALLOC_MAX_VALUES = 262144;      // sigma values (cols * nslices) per call
// tail sums (one per value), then at most 1024 CTAs x 16 partial sums, then the state
constexpr int64_t NOALLOC_SCRATCH_DOUBLES = NOALLOC_MAX_VALUES + 1024 * 16 + 32;

static __device__ __align__(256) double g_select_scratch[NOALLOC_SCRATCH_DOUBLES];
static __device__ __align__(256) double g_select_scal[tsvdm::SC_COUNT];

// Device addresses of the scratch on the current device.  In host code the array names
// are host-side stand-ins, not device addresses, so the kernels are given the looked-up
// pointers.  The lookup (which allocates nothing) runs on every call, so that a context
// created again after cudaDeviceReset is served at the module's new address; the first
// lookup on a device may load the module.
tsvdm_status scratch_for_current_device(void **scratch, double **scal) {
  if (cudaGetSymbolAddress(scratch, g_select_scratch) != cudaSuccess) return TSVDM_ECUDA;
  void *s = nullptr;
  if (cudaGetSymbolAddress(&s, g_select_scal) != cudaSuccess) return TSVDM_ECUDA;
  *scal = (double *)s;
  return TSVDM_OK;
}

}  // namespace

extern "C" tsvdm_status tsvdm_select_ranks_noalloc(const float *sigma, int64_t cols,
                                                   int64_t nslices, double eps, int32_t *ranks,
                                                   int64_t *offsets, double *summary,
                                                   void *stream) {
  if (!sigma || !ranks || !offsets) return TSVDM_EINVAL;
  if (cols < 1 || nslices < 1 || !(eps > 0.0 && eps < 1.0)) return TSVDM_EINVAL;
  if (cols > NOALLOC_MAX_VALUES || nslices > NOALLOC_MAX_VALUES ||
      cols * nslices > NOALLOC_MAX_VALUES)
    return TSVDM_ESCRATCH;
  if (tsvdm::select_workspace_bytes(cols, nslices) > sizeof(double) * NOALLOC_SCRATCH_DOUBLES)
    return TSVDM_ESCRATCH;
  void *scratch = nullptr;
  double *scal = nullptr;
  tsvdm_status s = scratch_for_current_device(&scratch, &scal);
  if (s != TSVDM_OK) return s;
  cudaStream_t st = (cudaStream_t)stream;
  // The kernels write every tail sum before reading it and write (do not accumulate) the
  // scalars they report; the search state is zeroed inside select_ranks.
  if (tsvdm::select_ranks<float>(sigma, (int)cols, (int)nslices, eps, scratch, scal, ranks,
                                 offsets, nullptr, st) != cudaSuccess)
    return TSVDM_ECUDA;
  if (summary) {
    const int idx[4] = {tsvdm::SC_TOTAL, tsvdm::SC_DISCARD, tsvdm::SC_TAU, tsvdm::SC_TOTRANK};
    for (int q = 0; q < 4; ++q)
      if (cudaMemcpyAsync(summary + q, scal + idx[q], sizeof(double), cudaMemcpyDeviceToDevice,
                          st) != cudaSuccess)
        return TSVDM_ECUDA;
  }
  return TSVDM_OK;
}
