// Allocation-free entry point: the t-SVDM-II rank choice (the same device selection kernel
// that tsvdm_tolerance runs) with its scratch in a fixed, file-scope device array
// instead of a plan's workspace.
//
// Who needs it: callers that must not call cudaMalloc.  Examples are a process that hands
// all device memory to another allocator when it starts (a framework's caching pool), so
// a driver allocation would fail, and latency-bound services that forbid allocation on
// their request path because a driver allocation can synchronise the device and take
// milliseconds.  Such callers already hold the singular values and the output buffers.
//
// The scratch (2 MiB: one FP64 tail sum per singular value, plus a few FP64 scalars) is
// part of the library image: every GPU that loads the library holds it until the process
// exits.  Every call shares it, so calls whose kernels overlap on the GPU (different
// streams, or several host threads) race on it; serialise them on one stream.
#include <mutex>

#include "common.cuh"

namespace {

constexpr int64_t NOALLOC_MAX_VALUES = 262144;      // sigma values (cols * nslices) per call
constexpr int MAX_DEVICES = 64;

static __device__ __align__(256) double g_select_scratch[NOALLOC_MAX_VALUES];
static __device__ __align__(256) double g_select_scal[tsvdm::SC_COUNT];

struct DeviceScratch {
  void *keys = nullptr;
  double *scal = nullptr;
  bool ready = false;
};
DeviceScratch g_scratch[MAX_DEVICES];
std::mutex g_scratch_mu;

// Device addresses of the scratch on the current device, looked up once per device with
// that device current.  (In host code the array names are host-side stand-ins, not device
// addresses, so the kernel must be given the looked-up pointers.)
tsvdm_status scratch_for_current_device(DeviceScratch *out) {
  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess) return TSVDM_ECUDA;
  if (dev < 0 || dev >= MAX_DEVICES) return TSVDM_ENOTSUP;
  std::lock_guard<std::mutex> lock(g_scratch_mu);
  DeviceScratch &d = g_scratch[dev];
  if (!d.ready) {
    void *k = nullptr, *s = nullptr;
    if (cudaGetSymbolAddress(&k, g_select_scratch) != cudaSuccess) return TSVDM_ECUDA;
    if (cudaGetSymbolAddress(&s, g_select_scal) != cudaSuccess) return TSVDM_ECUDA;
    d.keys = k;
    d.scal = (double *)s;
    d.ready = true;
  }
  *out = d;
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
  DeviceScratch d;
  tsvdm_status s = scratch_for_current_device(&d);
  if (s != TSVDM_OK) return s;
  cudaStream_t st = (cudaStream_t)stream;
  // Nothing needs clearing: the kernel writes every key before reading it and writes (does
  // not accumulate) the scalars it reports.
  if (tsvdm::select_ranks<float>(sigma, (int)cols, (int)nslices, eps, d.keys, d.scal, ranks,
                                 offsets, st) != cudaSuccess)
    return TSVDM_ECUDA;
  if (summary) {
    const int idx[4] = {tsvdm::SC_TOTAL, tsvdm::SC_DISCARD, tsvdm::SC_TAU, tsvdm::SC_TOTRANK};
    for (int q = 0; q < 4; ++q)
      if (cudaMemcpyAsync(summary + q, d.scal + idx[q], sizeof(double), cudaMemcpyDeviceToDevice,
                          st) != cudaSuccess)
        return TSVDM_ECUDA;
  }
  return TSVDM_OK;
}
