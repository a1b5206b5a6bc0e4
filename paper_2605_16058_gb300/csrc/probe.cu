// Peak-rate probes: the measured denominators of the roofline fractions the benchmark
// reports (the FP32 CUDA-core rate that bounds the slice SVDs' arithmetic, the FP64 rate of
// the all-FP64 path, and the TF32 / BF16 tensor-core rates of the TTMs).  Each probe is a
// kernel that does nothing but the unit's own instruction, back to back, on every SM.
#include <cuda_runtime.h>

#include "common.cuh"
#include "tc.cuh"

namespace tsvdm {
namespace {

constexpr int CHAINS = 8;             // independent FMA chains per thread

// FMA loop: CHAINS independent accumulators per thread, iters rounds of CHAINS FMAs.  The
// result is stored only when `sink` is set (never by the host), but the compiler cannot
// know that, so the loop is kept.
template <typename T>
__global__ void __launch_bounds__(256) fma_probe_kernel(int64_t iters, T a, T b, T *sink) {
  T acc[CHAINS];
#pragma unroll
  for (int c = 0; c < CHAINS; ++c) acc[c] = (T)(threadIdx.x + c);
  // 8 rounds per loop trip, so that the loop's own instructions take few issue slots
  for (int64_t it = 0; it < iters; it += 8) {
#pragma unroll
    for (int u = 0; u < 8; ++u)
#pragma unroll
      for (int c = 0; c < CHAINS; ++c) acc[c] = fma(acc[c], a, b);
  }
  T s = 0;
#pragma unroll
  for (int c = 0; c < CHAINS; ++c) s += acc[c];
  if (sink) sink[blockIdx.x * blockDim.x + threadIdx.x] = s;
}

// tcgen05 MMA loop: one CTA per SM, one thread issues `iters` M=128 x N=256 MMAs (K = 8
// TF32 or 16 BF16 each) from two zero-filled shared-memory tiles into TMEM, then waits
// (bounded) for their completion and frees the TMEM.
constexpr uint32_t PN = 256;
__global__ void __launch_bounds__(128, 1) mma_probe_kernel(int64_t iters, int bf16, int *status) {
  extern __shared__ __align__(1024) unsigned char smem_raw[];
  unsigned char *tiles =
      reinterpret_cast<unsigned char *>(((uintptr_t)smem_raw + 1023) & ~(uintptr_t)1023);
  __shared__ uint64_t bar;
  __shared__ uint32_t tmem;
  unsigned char *A = tiles, *B = tiles + 16384;           // [128 x 128 B], [256 x 128 B]
  for (int i = threadIdx.x; i < (16384 + 32768) / 16; i += blockDim.x)
    reinterpret_cast<uint4 *>(tiles)[i] = make_uint4(0, 0, 0, 0);
  if (threadIdx.x == 0) {
    tc::mbar_init(&bar, 1);
    tc::mbar_init_fence();
  }
  if (threadIdx.x < 32) tc::tmem_alloc_n<PN>(&tmem);
  tc::fence_proxy_async();
  tc::fence_before_sync();
  __syncthreads();
  tc::fence_after_sync();
  if (threadIdx.x == 0) {
    const uint32_t idesc = tc::instr_desc(bf16 ? 1u : 2u, 128, PN);
    for (int64_t it = 0; it < iters; ++it) {
      const uint32_t kk = (uint32_t)(it & 3);
      const uint64_t da = tc::smem_desc(A + kk * 32, 1024, 2);
      const uint64_t db = tc::smem_desc(B + kk * 32, 1024, 2);
      if (bf16)
        tc::mma_f16(tmem, da, db, idesc, it > 0 ? 1u : 0u);
      else
        tc::mma_tf32(tmem, da, db, idesc, it > 0 ? 1u : 0u);
    }
    tc::mma_commit(&bar);
    if (!tc::mbar_wait(&bar, 0, 1u << 26)) atomicOr(status, ST_TIMEOUT);
  }
  tc::fence_before_sync();
  __syncthreads();
  tc::fence_after_sync();
  if (threadIdx.x < 32) tc::tmem_dealloc_n<PN>(tmem);
}

}  // namespace
}  // namespace tsvdm

using namespace tsvdm;

extern "C" tsvdm_status tsvdm_probe_peak(int unit, int64_t iters, void *stream,
                                         double *tflops) {
  if (!tflops || iters < 1 || unit < TSVDM_PROBE_FP32_FMA || unit > TSVDM_PROBE_FP64_FMA)
    return TSVDM_EINVAL;
  cudaStream_t st = (cudaStream_t)stream;
  int dev = 0, sms = 0;
  if (cudaGetDevice(&dev) != cudaSuccess) return TSVDM_ECUDA;
  if (cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess)
    return TSVDM_ECUDA;
  int *status = nullptr;
  cudaEvent_t e0 = nullptr, e1 = nullptr;
  tsvdm_status ret = TSVDM_OK;
  double flops = 0.0;
  float ms = 0.f;
  const bool mma = unit == TSVDM_PROBE_TF32_MMA || unit == TSVDM_PROBE_BF16_MMA;
  // more shared memory than two CTAs can hold, so that every SM runs exactly one probe CTA
  const size_t smem = 120 * 1024;
  int grid = sms, per_sm = 0;
  if (cudaEventCreate(&e0) != cudaSuccess || cudaEventCreate(&e1) != cudaSuccess ||
      cudaMalloc(&status, sizeof(int)) != cudaSuccess ||
      cudaMemsetAsync(status, 0, sizeof(int), st) != cudaSuccess) {
    ret = TSVDM_ECUDA;
    goto done;
  }
  if (mma) {
    if (cudaFuncSetAttribute(mma_probe_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize,
                             (int)smem) != cudaSuccess) {
      ret = TSVDM_ECUDA;
      goto done;
    }
    flops = 2.0 * 128 * PN * (unit == TSVDM_PROBE_BF16_MMA ? 16 : 8) * (double)iters * grid;
  } else {
    auto f32 = fma_probe_kernel<float>;
    auto f64 = fma_probe_kernel<double>;
    if ((unit == TSVDM_PROBE_FP32_FMA
             ? cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, f32, 256, 0)
             : cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, f64, 256, 0)) !=
        cudaSuccess) {
      ret = TSVDM_ECUDA;
      goto done;
    }
    grid = sms * (per_sm > 0 ? per_sm : 1);
    iters = (iters + 7) / 8 * 8;
    flops = 2.0 * CHAINS * (double)iters * 256.0 * grid;
  }
  for (int rep = 0; rep < 2; ++rep) {      // the first launch warms up, the second is timed
    if (rep == 1) cudaEventRecord(e0, st);
    if (mma)
      mma_probe_kernel<<<grid, 128, smem, st>>>(iters, unit == TSVDM_PROBE_BF16_MMA, status);
    else if (unit == TSVDM_PROBE_FP32_FMA)
      fma_probe_kernel<float><<<grid, 256, 0, st>>>(iters, 0.999999f, 1e-7f, nullptr);
    else
      fma_probe_kernel<double><<<grid, 256, 0, st>>>(iters, 0.999999, 1e-7, nullptr);
    if (cudaGetLastError() != cudaSuccess) {
      ret = TSVDM_ECUDA;
      goto done;
    }
  }
  cudaEventRecord(e1, st);
  if (cudaEventSynchronize(e1) != cudaSuccess || cudaEventElapsedTime(&ms, e0, e1) != cudaSuccess) {
    ret = TSVDM_ECUDA;
    goto done;
  }
  {
    int s = 0;
    if (cudaMemcpy(&s, status, sizeof(int), cudaMemcpyDeviceToHost) != cudaSuccess) {
      ret = TSVDM_ECUDA;
      goto done;
    }
    if (s) {
      ret = TSVDM_ETIMEOUT;
      goto done;
    }
  }
  *tflops = flops / (ms * 1e-3) / 1e12;
done:
  if (status) cudaFree(status);
  if (e0) cudaEventDestroy(e0);
  if (e1) cudaEventDestroy(e1);
  return ret;
}
