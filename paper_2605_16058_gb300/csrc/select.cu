// t-SVDM-II rank choice (Algorithm 2, steps 2-8) on the device.
//
// Input: each slice's singular values, sorted descending (cols x nslices).  Algorithm 2
// sorts all v = sigma^2 ascending, takes the running sums w, J = #{l : w_l < eps^2 sum(v)}
// (the largest such l, w being non-decreasing), tau = v_J, and keeps in slice i the
// rho_i = #{j : sigma_{j,i}^2 > tau} values above tau (so every copy of tau is dropped).
//
// The sort is not needed for tau.  With S(k) = the sum of all values whose key is below k
// (keys: the bits of sigma for FP32, of sigma^2 for FP64; both order like the values), the
// first copy of a value x is included in J exactly when (S(x) + x) / sum(v) < eps^2; the
// left side only grows with x, so tau is the largest present value x for which it holds.
// Here:
//   1. per slice, the FP64 sums of sigma^2 over each tail j..cols-1 (ascending order is the
//      tail of the descending slice), and their total;
//   2. a bisection over the key bits for the largest key k with (S(k) + val(k)) / sum(v)
//      < eps^2, where S(k) adds each slice's tail below k (binary search in the slice);
//   3. tau = the largest present key <= k; rho_i, the discarded sum and the offsets
//      (exclusive prefix sum of rho, int64) from one binary search per slice.
// All sums are FP64 in a fixed order, so a result is reproducible run to run; against the
// sorted running sum of Algorithm 2 it differs only by FP64 summation order.  One CTA per
// selection: the work is a few hundred slices times ~32 bisection steps of a binary search.
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

// Block-wide inclusive scan of one int64 per thread, fixed order; *total receives the
// block sum.
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

// Fixed-order block reduction of one double per thread (every thread gets the sum).
__device__ double block_sum(double v, double *wsum) {
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  if (lane == 0) wsum[warp] = v;
  __syncthreads();
  double t = 0.0;
  for (int w = 0; w < NW; ++w) t += wsum[w];
  __syncthreads();
  return t;
}

template <typename K>
__device__ K block_max(K v, K *wk) {
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) {
    const K u = __shfl_xor_sync(0xffffffffu, v, o);
    v = u > v ? u : v;
  }
  if (lane == 0) wk[warp] = v;
  __syncthreads();
  K t = wk[0];
  for (int w = 1; w < NW; ++w) t = wk[w] > t ? wk[w] : t;
  __syncthreads();
  return t;
}

// First index j of the descending slice s with key(s[j]) < k (cols if none).
template <typename T>
__device__ __forceinline__ int first_below(const T *s, int cols, typename KeyOf<T>::K k) {
  int lo = 0, hi = cols;
  while (lo < hi) {
    const int mid = (lo + hi) >> 1;
    if (KeyOf<T>::key(s[mid]) >= k) lo = mid + 1;
    else hi = mid;
  }
  return lo;
}

template <typename T>
__device__ void select_body(const T *__restrict__ sig, int cols, int nslices, double eps,
                            void *kws, double *scal, int *ranks, int64_t *offsets) {
  using KO = KeyOf<T>;
  using K = typename KO::K;
  // key of +inf: no finite singular value reaches it
  constexpr K KINF = sizeof(K) == 4 ? K(0x7f800000u) : K(0x7ff0000000000000ull);
  __shared__ double wsum[NW];
  __shared__ long long wsum_ll[NW];
  __shared__ K wkey[NW];
  const int tid = threadIdx.x;
  // tail[i * cols + j] = sum of sigma_{j',i}^2 for j' >= j (the cols - j smallest of slice i)
  double *tail = reinterpret_cast<double *>(kws);
  double part = 0.0;
  for (int i = tid; i < nslices; i += ST) {
    const T *s = sig + (int64_t)i * cols;
    double *t = tail + (int64_t)i * cols;
    double run = 0.0;
    for (int j = cols - 1; j >= 0; --j) {
      run += KO::val(KO::key(s[j]));
      t[j] = run;
    }
    part += run;
  }
  const double total = block_sum(part, wsum);
  const double eps2 = eps * eps;
  bool has_tau = false;
  K tau = K(0);
  if (total == 0.0) {
    has_tau = true;                  // an all-zero spectrum keeps nothing
    tau = ~K(0);
  } else if (eps2 >= 1.0) {
    // (the entry points take eps in (0, 1); this keeps the kernel exact for any eps)
    // w_N = sum(v) exactly, so eps^2 > 1 discards every value and eps^2 = 1 all but the
    // last one in sorted order: tau is the largest value, or the second largest counting
    // copies (decided here without any sum, so the boundary w_N is exact)
    K m1 = K(0);
    for (int i = tid; i < nslices; i += ST) {
      const K k0 = KO::key(sig[(int64_t)i * cols]);
      m1 = k0 > m1 ? k0 : m1;
    }
    m1 = block_max<K>(m1, wkey);
    if (eps2 > 1.0) {
      has_tau = true;
      tau = m1;
    } else {
      double copies = 0.0;
      K second = K(0);
      int found = 0;
      for (int i = tid; i < nslices; i += ST) {
        const T *s = sig + (int64_t)i * cols;
        const int c = first_below(s, cols, m1);         // copies of the largest value
        copies += (double)c;
        if (c < cols) {
          const K kc = KO::key(s[c]);
          if (!found || kc > second) second = kc;
          found = 1;
        }
      }
      copies = block_sum(copies, wsum);
      found = __syncthreads_or(found);
      second = block_max<K>(second, wkey);
      if (copies >= 2.0) {
        has_tau = true;
        tau = m1;
      } else {
        has_tau = found != 0;
        tau = second;
      }
    }
  } else if (eps2 > 0.0) {
    // largest key k with (S(k) + val(k)) / total < eps^2 (Algorithm 2's own comparison):
    // true at k = 0, false at +inf
    K lo = 0, hi = KINF;
    while (hi - lo > 1) {
      const K mid = lo + (hi - lo) / 2;
      double below = 0.0;
      for (int i = tid; i < nslices; i += ST) {
        const int c = first_below(sig + (int64_t)i * cols, cols, mid);
        if (c < cols) below += tail[(int64_t)i * cols + c];
      }
      const double S = block_sum(below, wsum);
      if ((S + KO::val(mid)) / total < eps2)
        lo = mid;
      else
        hi = mid;
    }
    // tau = the largest present key <= lo (none: J = 0, nothing is discarded)
    K best = K(0);
    int found = 0;
    for (int i = tid; i < nslices; i += ST) {
      const T *s = sig + (int64_t)i * cols;
      const int c = first_below(s, cols, lo + 1);       // first key <= lo
      if (c < cols) {
        const K kc = KO::key(s[c]);
        if (!found || kc > best) best = kc;
        found = 1;
      }
    }
    found = __syncthreads_or(found);
    best = block_max<K>(best, wkey);
    has_tau = found != 0;
    tau = best;
  }
  // ranks (values above tau), their offsets and the discarded sum
  long long carry_ll = 0, tot_ll;
  double disc = 0.0;
  for (int b0 = 0; b0 < nslices; b0 += ST) {
    const int i = b0 + tid;
    long long r = 0;
    if (i < nslices) {
      const T *s = sig + (int64_t)i * cols;
      if (!has_tau) {
        r = cols;
      } else if (total == 0.0) {
        r = 0;
      } else {
        r = tau == ~K(0) ? 0 : first_below(s, cols, tau + 1);   // first key <= tau
        if (r < cols) disc += tail[(int64_t)i * cols + r];
      }
      ranks[i] = (int)r;
    }
    long long incl = block_scan_ll(r, wsum_ll, &tot_ll);
    if (i < nslices) offsets[i] = carry_ll + incl - r;
    carry_ll += tot_ll;
  }
  const double d = block_sum(disc, wsum);
  if (tid == 0) {
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
