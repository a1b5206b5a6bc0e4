// t-SVDM-II rank choice (Algorithm 2, steps 2-8) on the device.
//
// Input: each slice's singular values, sorted descending (cols x nslices).
//   v = every sigma^2 (FP64), sorted ascending by an LSD radix sort of order-preserving
//   keys: for FP32 the bits of sigma itself (sigma^2 of an FP32 value is exact in FP64,
//   so the order and the ties of sigma and sigma^2 agree), for FP64 the bits of sigma^2;
//   w = the running FP64 sums of v in sorted order (block-wide scans, fixed order);
//   J = #{l : w_l / sum(v) < eps^2} (w is non-decreasing, so this is the largest such l);
//   tau = v_J; rho_i = #{j : sigma_{j,i}^2 > tau} (values equal to tau are dropped);
//   offsets = exclusive prefix sum of rho (int64).
// The whole selection runs in one CTA of 1024 threads: the key count is n3 min(n1, n2)
// (a few hundred thousand at most for the workloads here), so it is latency-bound and a
// single CTA with block-wide scans keeps it deterministic.
#include "common.cuh"

namespace tsvdm {
namespace {

constexpr int ST = 1024;
constexpr int NW = ST / 32;

template <typename T> struct KeyOf;
template <> struct KeyOf<float> {
  using K = unsigned int;
  __device__ static K key(float s) { return __float_as_uint(s); }
  __device__ static double val(K k) {
    double s = (double)__uint_as_float(k);
    return s * s;
  }
};
template <> struct KeyOf<double> {
  using K = unsigned long long;
  __device__ static K key(double s) { return (K)__double_as_longlong(s * s); }
  __device__ static double val(K k) { return __longlong_as_double((long long)k); }
};

__device__ __forceinline__ unsigned lanemask_lt() {
  unsigned m;
  asm("mov.u32 %0, %%lanemask_lt;" : "=r"(m));
  return m;
}

// Block-wide inclusive scan of one double per thread, fixed order. Returns the inclusive
// value; *total receives the block sum.
__device__ double block_scan(double v, double *wsum, double *total) {
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
#pragma unroll
  for (int o = 1; o < 32; o <<= 1) {
    double u = __shfl_up_sync(0xffffffffu, v, o);
    if (lane >= o) v += u;
  }
  if (lane == 31) wsum[warp] = v;
  __syncthreads();
  if (warp == 0) {
    double x = wsum[lane];
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
      double u = __shfl_up_sync(0xffffffffu, x, o);
      if (lane >= o) x += u;
    }
    wsum[lane] = x;
  }
  __syncthreads();
  if (warp > 0) v += wsum[warp - 1];
  *total = wsum[NW - 1];
  __syncthreads();
  return v;
}

__device__ long long block_scan_ll(long long v, long long *wsum, long long *total) {
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
#pragma unroll
  for (int o = 1; o < 32; o <<= 1) {
    long long u = __shfl_up_sync(0xffffffffu, v, o);
    if (lane >= o) v += u;
  }
  if (lane == 31) wsum[warp] = v;
  __syncthreads();
  if (warp == 0) {
    long long x = wsum[lane];
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
      long long u = __shfl_up_sync(0xffffffffu, x, o);
      if (lane >= o) x += u;
    }
    wsum[lane] = x;
  }
  __syncthreads();
  if (warp > 0) v += wsum[warp - 1];
  *total = wsum[NW - 1];
  __syncthreads();
  return v;
}

template <typename T>
__device__ void select_body(const T *__restrict__ sig, int cols, int nslices, double eps,
                            void *kws, double *scal, int *ranks, int64_t *offsets) {
  using KO = KeyOf<T>;
  using K = typename KO::K;
  __shared__ int wc[NW * 256];
  __shared__ int base_off[256];
  __shared__ int tile_cnt[256];
  __shared__ double wsum[NW];
  __shared__ long long wsum_ll[NW];
  __shared__ K s_tau;
  __shared__ int s_has_tau;
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  const int64_t N = (int64_t)cols * nslices;
  K *buf0 = reinterpret_cast<K *>(kws);
  K *buf1 = buf0 + N;

  for (int64_t e = tid; e < N; e += ST) buf0[e] = KO::key(sig[e]);
  __syncthreads();

  // LSD radix sort, 8-bit digits, stable
  K *src = buf0, *dst = buf1;
  for (int pass = 0; pass < (int)sizeof(K); ++pass) {
    const int sh = 8 * pass;
    if (tid < 256) base_off[tid] = 0;
    __syncthreads();
    for (int64_t e = tid; e < N; e += ST) atomicAdd(&base_off[(int)((src[e] >> sh) & 255)], 1);
    __syncthreads();
    if (tid == 0) {
      int run = 0;
      for (int d = 0; d < 256; ++d) {
        int c = base_off[d];
        base_off[d] = run;
        run += c;
      }
    }
    __syncthreads();
    for (int64_t b0 = 0; b0 < N; b0 += ST) {
      const int64_t e = b0 + tid;
      const bool valid = e < N;
      const K key = valid ? src[e] : K(0);
      const int d = valid ? (int)((key >> sh) & 255) : 256;
      for (int x = tid; x < NW * 256; x += ST) wc[x] = 0;
      __syncthreads();
      const unsigned peers = __match_any_sync(0xffffffffu, d);
      const int rk = __popc(peers & lanemask_lt());
      if (valid && rk == 0) wc[warp * 256 + d] = __popc(peers);
      __syncthreads();
      if (tid < 256) {
        int run = 0;
        for (int w = 0; w < NW; ++w) {
          int c = wc[w * 256 + tid];
          wc[w * 256 + tid] = run;
          run += c;
        }
        tile_cnt[tid] = run;
      }
      __syncthreads();
      if (valid) dst[base_off[d] + wc[warp * 256 + d] + rk] = key;
      __syncthreads();
      if (tid < 256) base_off[tid] += tile_cnt[tid];
      __syncthreads();
    }
    K *t = src;
    src = dst;
    dst = t;
  }
  // src holds the keys in ascending order.

  // pass 1: total = w_N (same blocked scan as pass 2, so w_N == total exactly)
  double carry = 0.0, tot;
  for (int64_t b0 = 0; b0 < N; b0 += ST) {
    int64_t e = b0 + tid;
    double v = e < N ? KO::val(src[e]) : 0.0;
    block_scan(v, wsum, &tot);
    carry += tot;
  }
  const double total = carry;
  // pass 2: J = #{l : w_l / total < eps^2}
  const double eps2 = eps * eps;
  long long Jc = 0;
  carry = 0.0;
  if (total > 0.0) {
    for (int64_t b0 = 0; b0 < N; b0 += ST) {
      int64_t e = b0 + tid;
      double v = e < N ? KO::val(src[e]) : 0.0;
      double w = block_scan(v, wsum, &tot) + carry;
      carry += tot;
      int ok = (e < N) && (w / total < eps2);
      Jc += __syncthreads_count(ok);
    }
  }
  if (tid == 0) {
    if (total == 0.0) {
      s_has_tau = 1;          // an all-zero spectrum keeps nothing
      s_tau = ~K(0);
    } else if (Jc > 0) {
      s_has_tau = 1;
      s_tau = src[Jc - 1];
    } else {
      s_has_tau = 0;          // J = 0: nothing is discarded
      s_tau = K(0);
    }
  }
  __syncthreads();
  const bool has_tau = s_has_tau;
  const K tau = s_tau;
  // ranks: each slice's keys are in descending order -> binary search
  long long carry_ll = 0, tot_ll;
  double disc = 0.0;
  for (int b0 = 0; b0 < nslices; b0 += ST) {
    int i = b0 + tid;
    long long r = 0;
    if (i < nslices) {
      const T *s = sig + (int64_t)i * cols;
      if (!has_tau) {
        r = cols;
      } else if (total == 0.0) {
        r = 0;
      } else {
        int lo = 0, hi = cols;      // first j with key(s[j]) <= tau
        while (lo < hi) {
          int mid = (lo + hi) >> 1;
          if (KO::key(s[mid]) > tau) lo = mid + 1;
          else hi = mid;
        }
        r = lo;
      }
      for (int j = (int)r; j < cols; ++j) disc += KO::val(KO::key(s[j]));
      ranks[i] = (int)r;
    }
    long long incl = block_scan_ll(r, wsum_ll, &tot_ll);
    if (i < nslices) offsets[i] = carry_ll + incl - r;
    carry_ll += tot_ll;
  }
  // discarded sum (fixed-order block reduction)
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) disc += __shfl_xor_sync(0xffffffffu, disc, o);
  if (lane == 0) wsum[warp] = disc;
  __syncthreads();
  if (tid == 0) {
    double d = 0.0;
    for (int w = 0; w < NW; ++w) d += wsum[w];
    offsets[nslices] = carry_ll;
    scal[SC_TOTAL] = total;
    scal[SC_DISCARD] = total > 0.0 ? d : 0.0;
    scal[SC_TAU] = (has_tau && total > 0.0) ? KO::val(tau) : -1.0;
    scal[SC_TOTRANK] = (double)carry_ll;
  }
}

// t-SVDM-I truncation sums: total = sum of all sigma^2, discarded = sum over j >= k.
template <typename T>
__global__ void __launch_bounds__(ST) trunc_sums_kernel(const T *__restrict__ sig, int cols,
                                                        int nslices, int64_t k, double *scal) {
  __shared__ double wt[NW], wd[NW];
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  const int64_t N = (int64_t)cols * nslices;
  double t = 0.0, d = 0.0;
  for (int64_t e = tid; e < N; e += ST) {
    double v = (double)sig[e];
    v *= v;
    t += v;
    if ((e % cols) >= k) d += v;
  }
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) {
    t += __shfl_xor_sync(0xffffffffu, t, o);
    d += __shfl_xor_sync(0xffffffffu, d, o);
  }
  if (lane == 0) {
    wt[warp] = t;
    wd[warp] = d;
  }
  __syncthreads();
  if (tid == 0) {
    double a = 0.0, b = 0.0;
    for (int w = 0; w < NW; ++w) {
      a += wt[w];
      b += wd[w];
    }
    scal[SC_TOTAL] = a;
    scal[SC_DISCARD] = b;
  }
}

template <typename T>
__global__ void __launch_bounds__(ST, 1) select_kernel(const T *__restrict__ sig, int cols,
                                                       int nslices, double eps, void *kws,
                                                       double *scal, int *ranks,
                                                       int64_t *offsets) {
  select_body<T>(sig, cols, nslices, eps, kws, scal, ranks, offsets);
}

// One CTA per segment (one t-SVDM-II tensor of a batch).
template <typename T>
__global__ void __launch_bounds__(ST, 1) select_seg_kernel(const SelectSeg *segs) {
  const SelectSeg g = segs[blockIdx.x];
  select_body<T>(reinterpret_cast<const T *>(g.sig), g.cols, g.nslices, g.eps, g.keys, g.scal,
                 g.ranks, g.offsets);
}

}  // namespace

template <typename T>
cudaError_t select_segments(const SelectSeg *segs, int count, cudaStream_t st) {
  if (count <= 0) return cudaSuccess;
  select_seg_kernel<T><<<count, ST, 0, st>>>(segs);
  return cudaGetLastError();
}
template cudaError_t select_segments<float>(const SelectSeg *, int, cudaStream_t);
template cudaError_t select_segments<double>(const SelectSeg *, int, cudaStream_t);

template <typename T>
cudaError_t trunc_sums(const T *sig, int cols, int nslices, int64_t k, double *scal,
                       cudaStream_t st) {
  trunc_sums_kernel<T><<<1, ST, 0, st>>>(sig, cols, nslices, k, scal);
  return cudaGetLastError();
}
template cudaError_t trunc_sums<float>(const float *, int, int, int64_t, double *, cudaStream_t);
template cudaError_t trunc_sums<double>(const double *, int, int, int64_t, double *, cudaStream_t);

template <typename T>
cudaError_t select_ranks(const T *sig, int cols, int nslices, double eps, void *keys_ws,
                         double *scal, int *ranks, int64_t *offsets, cudaStream_t st) {
  select_kernel<T><<<1, ST, 0, st>>>(sig, cols, nslices, eps, keys_ws, scal, ranks, offsets);
  return cudaGetLastError();
}

template cudaError_t select_ranks<float>(const float *, int, int, double, void *, double *, int *,
                                         int64_t *, cudaStream_t);
template cudaError_t select_ranks<double>(const double *, int, int, double, void *, double *,
                                          int *, int64_t *, cudaStream_t);

}  // namespace tsvdm
