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
//   2. a search over the key bits for the largest key k with (S(k) + val(k)) / sum(v)
//      < eps^2, where S(k) adds each slice's tail below k (binary search in the slice);
//   3. tau = the largest present key <= k; rho_i, the discarded sum and the offsets
//      (exclusive prefix sum of rho, int64) from one binary search per slice.
// All sums are FP64 in a fixed order, so a result is reproducible run to run; against the
// sorted running sum of Algorithm 2 it differs only by FP64 summation order.
//
// One tensor (select_ranks) runs over the whole GPU: a warp per slice forms the tail sums,
// then each search launch splits the key interval into 16 and evaluates the 15 inner keys
// over all slices (CTAs take disjoint slice ranges; the last CTA to finish adds their
// partial sums in CTA order and narrows the interval, so no CTA ever waits for another),
// and one CTA finishes steps 3.  The tensors of a batch (select_segments) take one CTA each.
// Singular values that are NaN, infinite or negative (-0 counts as 0) make the selection
// report NaN sums, zero ranks and offsets, and the non-finite status bit.
#include <algorithm>

#include "common.cuh"

namespace tsvdm {
namespace {

constexpr int ST = 1024;
constexpr int NW = ST / 32;

template <typename T> struct KeyOf;
template <> struct KeyOf<float> {
  using K = unsigned int;
  static constexpr K KINF = 0x7f800000u;     // key of +inf: no finite value reaches it
  static constexpr int ROUNDS = 8;           // 16-way search rounds that narrow [0, KINF] to 1
  __device__ static K key(float s) { return __float_as_uint(fabsf(s)); }
  __device__ static double val(K k) {
    double s = (double)__uint_as_float(k);
    return s * s;
  }
};
template <> struct KeyOf<double> {
  using K = unsigned long long;
  static constexpr K KINF = 0x7ff0000000000000ull;
  static constexpr int ROUNDS = 16;
  __device__ static K key(double s) { return (K)__double_as_longlong(s * s); }
  __device__ static double val(K k) { return __longlong_as_double((long long)k); }
};

template <typename T>
__device__ __forceinline__ bool bad_value(T x) {
  return !(x >= T(0)) || isinf(x);      // NaN, negative or infinite (-0 passes)
}

// Block-wide inclusive scan of one int64 per thread, fixed order; *total receives the
// block sum.  (Blocks of ST threads.)
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
template <int NWARPS>
__device__ double block_sum(double v, double *wsum) {
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  if (lane == 0) wsum[warp] = v;
  __syncthreads();
  double t = 0.0;
  for (int w = 0; w < NWARPS; ++w) t += wsum[w];
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
    if (KeyOf<T>::key(__ldg(s + mid)) >= k) lo = mid + 1;
    else hi = mid;
  }
  return lo;
}

// Steps 3 of the selection, given the tail sums, the total and the search result `lo`
// (the largest key whose Algorithm 2 inequality holds; used when eps^2 in (0, 1)).
// One block of ST threads.
template <typename T>
__device__ void select_finish(const T *__restrict__ sig, int cols, int nslices, double eps2,
                              const double *tail, double total, typename KeyOf<T>::K lo,
                              bool bad, double *scal, int *ranks, int64_t *offsets,
                              int *status) {
  using KO = KeyOf<T>;
  using K = typename KO::K;
  __shared__ double wsum[NW];
  __shared__ long long wsum_ll[NW];
  __shared__ K wkey[NW];
  const int tid = threadIdx.x;
  if (bad) {
    for (int i = tid; i < nslices; i += ST) {
      ranks[i] = 0;
      offsets[i] = 0;
    }
    if (tid == 0) {
      offsets[nslices] = 0;
      scal[SC_TOTAL] = scal[SC_DISCARD] = scal[SC_TAU] = scal[SC_TOTRANK] = __longlong_as_double(
          0x7ff8000000000000ll);
      if (status) atomicOr(status, ST_NONFINITE);
    }
    return;
  }
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
      copies = block_sum<NW>(copies, wsum);
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
  const double d = block_sum<NW>(disc, wsum);
  if (tid == 0) {
    offsets[nslices] = carry_ll;
    scal[SC_TOTAL] = total;
    scal[SC_DISCARD] = total > 0.0 ? d : 0.0;
    scal[SC_TAU] = (has_tau && total > 0.0) ? KO::val(tau) : -1.0;
    scal[SC_TOTRANK] = (double)carry_ll;
  }
}

// The whole selection of one tensor in one block (a batch segment).
template <typename T>
__device__ void select_body(const T *__restrict__ sig, int cols, int nslices, double eps,
                            void *kws, double *scal, int *ranks, int64_t *offsets) {
  using KO = KeyOf<T>;
  using K = typename KO::K;
  __shared__ double wsum[NW];
  const int tid = threadIdx.x;
  // tail[i * cols + j] = sum of sigma_{j',i}^2 for j' >= j (the cols - j smallest of slice i)
  double *tail = reinterpret_cast<double *>(kws);
  double part = 0.0;
  int bad = 0;
  for (int i = tid; i < nslices; i += ST) {
    const T *s = sig + (int64_t)i * cols;
    double *t = tail + (int64_t)i * cols;
    double run = 0.0;
    for (int j = cols - 1; j >= 0; --j) {
      const T x = s[j];
      bad |= bad_value(x);
      run += KO::val(KO::key(x));
      t[j] = run;
    }
    part += run;
  }
  bad = __syncthreads_or(bad);
  const double total = block_sum<NW>(part, wsum);
  const double eps2 = eps * eps;
  K lo = 0, hi = KO::KINF;
  if (!bad && total != 0.0 && eps2 > 0.0 && eps2 < 1.0) {
    // largest key k with (S(k) + val(k)) / total < eps^2 (Algorithm 2's own comparison):
    // true at k = 0, false at +inf
    while (hi - lo > 1) {
      const K mid = lo + (hi - lo) / 2;
      double below = 0.0;
      for (int i = tid; i < nslices; i += ST) {
        const int c = first_below(sig + (int64_t)i * cols, cols, mid);
        if (c < cols) below += tail[(int64_t)i * cols + c];
      }
      const double S = block_sum<NW>(below, wsum);
      if ((S + KO::val(mid)) / total < eps2)
        lo = mid;
      else
        hi = mid;
    }
  }
  select_finish<T>(sig, cols, nslices, eps2, tail, total, lo, bad != 0, scal, ranks, offsets,
                   nullptr);
}

// ---------------------------------------------------------------- one tensor, whole GPU
// Search state after the tail sums (in the workspace, behind the tail sums and partials).
struct SelState {
  unsigned long long lo, hi;   // the search interval (keys)
  double total;                // sum of all sigma^2
  int bad;                     // a NaN, infinite or negative value was seen
  int search;                  // 1: eps^2 in (0, 1) and total > 0, the key search runs
  unsigned int arrive;         // CTAs finished with the current launch
  int pad[9];
};
constexpr int SEL_WARPS = 8;               // slices per tail CTA (a warp each)
constexpr int SEL_CAND = 16;               // key interval split per search launch
constexpr int SEL_SLICE_LANES = 256 / SEL_CAND;
constexpr int SEL_MAX_CTAS = 1024;

// Last-CTA detection: true in every thread of the CTA that finishes the launch last, after
// which it sees every other CTA's results.
__device__ __forceinline__ bool last_cta(SelState *st) {
  __shared__ int last;
  __threadfence();
  __syncthreads();
  if (threadIdx.x == 0) last = atomicAdd(&st->arrive, 1u) == gridDim.x - 1;
  __syncthreads();
  if (last) __threadfence();
  return last;
}

// 1. Tail sums, a warp per slice: the 32 lanes take contiguous chunks, sum them from the
// end, and the chunk sums are combined by a suffix scan across the lanes (fixed order).
template <typename T>
__global__ void __launch_bounds__(256) sel_tails_kernel(const T *__restrict__ sig, int cols,
                                                        int nslices, double eps2, double *tail,
                                                        SelState *st) {
  using KO = KeyOf<T>;
  __shared__ double wsum[SEL_WARPS];
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  const int i = blockIdx.x * SEL_WARPS + warp;
  int bad = 0;
  if (i < nslices) {
    const T *s = sig + (int64_t)i * cols;
    double *t = tail + (int64_t)i * cols;
    const int chunk = (cols + 31) / 32;
    const int j0 = min(lane * chunk, cols), j1 = min(j0 + chunk, cols);
    double csum = 0.0;
    for (int j = j1 - 1; j >= j0; --j) {
      const T x = s[j];
      bad |= bad_value(x);
      csum += KO::val(KO::key(x));
    }
    // inclusive suffix sums of the chunk sums (lane l: chunks l..31), then exclusive
    double incl = csum;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
      const double u = __shfl_down_sync(0xffffffffu, incl, o);
      if (lane + o < 32) incl += u;
    }
    double run = __shfl_down_sync(0xffffffffu, incl, 1);
    if (lane == 31) run = 0.0;
    for (int j = j1 - 1; j >= j0; --j) {
      run += KO::val(KO::key(s[j]));
      t[j] = run;
    }
  }
  if (__syncthreads_or(bad) && threadIdx.x == 0) atomicOr(&st->bad, 1);
  if (!last_cta(st)) return;
  // the total over the slices' tails, in slice order per thread, then a fixed tree
  double part = 0.0;
  for (int k = threadIdx.x; k < nslices; k += 256) part += tail[(int64_t)k * cols];
  const double total = block_sum<SEL_WARPS>(part, wsum);
  if (threadIdx.x == 0) {
    st->total = total;
    st->lo = 0;
    st->hi = KO::KINF;
    st->search = (total != 0.0 && eps2 > 0.0 && eps2 < 1.0 && !*(volatile int *)&st->bad) ? 1 : 0;
    st->arrive = 0;
  }
}

// 2. One 16-way search round: the keys c_1 < ... < c_15 inside (lo, hi) split it into 16
// (or lo + 1 .. hi - 1 when it is narrower); S(c_m) is summed over the CTAs' slice ranges
// (thread = candidate x slice lane, slices of a lane in increasing order, then the lanes in
// order, then the CTAs in order), and the last CTA keeps the sub-interval where Algorithm
// 2's inequality changes from true to false.
template <typename T>
__global__ void __launch_bounds__(256) sel_round_kernel(const T *__restrict__ sig, int cols,
                                                        int nslices, double eps2,
                                                        const double *tail, double *part,
                                                        SelState *st, int per_cta) {
  using KO = KeyOf<T>;
  using K = typename KO::K;
  __shared__ double red[SEL_CAND][SEL_SLICE_LANES + 1];
  __shared__ int holds[SEL_CAND];
  const K lo = (K)st->lo, hi = (K)st->hi;
  if (!st->search || hi - lo <= 1) return;      // uniform across the grid
  const K span = hi - lo;
  const int nc = span >= SEL_CAND ? SEL_CAND - 1 : (int)(span - 1);
  auto cand = [&](int m) -> K {                  // m = 1 .. nc
    if (span >= SEL_CAND) return lo + (span / SEL_CAND) * m + ((span % SEL_CAND) * m) / SEL_CAND;
    return lo + (K)m;
  };
  const int m = (threadIdx.x % SEL_CAND) + 1, sl = threadIdx.x / SEL_CAND;
  const int i0 = blockIdx.x * per_cta, i1 = min(i0 + per_cta, nslices);
  double acc = 0.0;
  if (m <= nc) {
    const K c = cand(m);
    for (int i = i0 + sl; i < i1; i += SEL_SLICE_LANES) {
      const int j = first_below(sig + (int64_t)i * cols, cols, c);
      if (j < cols) acc += tail[(int64_t)i * cols + j];
    }
  }
  red[m - 1][sl] = acc;
  __syncthreads();
  if (threadIdx.x < SEL_CAND) {
    double s = 0.0;
    for (int q = 0; q < SEL_SLICE_LANES; ++q) s += red[threadIdx.x][q];
    part[(int64_t)blockIdx.x * SEL_CAND + threadIdx.x] = s;
  }
  if (!last_cta(st)) return;
  if (threadIdx.x < SEL_CAND) {
    const int mm = threadIdx.x + 1;
    int h = 0;
    if (mm <= nc) {
      double S = 0.0;
      for (int b = 0; b < (int)gridDim.x; ++b) S += part[(int64_t)b * SEL_CAND + threadIdx.x];
      h = (S + KO::val(cand(mm))) / st->total < eps2;
    }
    holds[threadIdx.x] = h;
  }
  __syncthreads();
  if (threadIdx.x == 0) {
    // the inequality holds for c_1 .. c_q and fails from c_{q+1} on (it only grows with k)
    int q = 0;
    while (q < nc && holds[q]) ++q;
    st->lo = q > 0 ? (unsigned long long)cand(q) : (unsigned long long)lo;
    st->hi = q < nc ? (unsigned long long)cand(q + 1) : (unsigned long long)hi;
    st->arrive = 0;
  }
}

// 3. tau, ranks, offsets, discarded sum (one block).
template <typename T>
__global__ void __launch_bounds__(ST, 1) sel_finish_kernel(const T *__restrict__ sig, int cols,
                                                           int nslices, double eps2,
                                                           const double *tail, SelState *st,
                                                           double *scal, int *ranks,
                                                           int64_t *offsets, int *status) {
  using K = typename KeyOf<T>::K;
  select_finish<T>(sig, cols, nslices, eps2, tail, st->total, (K)st->lo, st->bad != 0, scal,
                   ranks, offsets, status);
}

template <typename T>
__global__ void __launch_bounds__(ST, 1) select_seg_kernel(const SelectSeg *segs) {
  const SelectSeg g = segs[blockIdx.x];
  select_body<T>(reinterpret_cast<const T *>(g.sig), g.cols, g.nslices, g.eps, g.keys, g.scal,
                 g.ranks, g.offsets);
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

}  // namespace

size_t select_workspace_bytes(int64_t cols, int64_t nslices) {
  const int64_t ctas = std::min<int64_t>((nslices + SEL_SLICE_LANES - 1) / SEL_SLICE_LANES,
                                         SEL_MAX_CTAS);
  return sizeof(double) * (size_t)(cols * nslices) +
         sizeof(double) * (size_t)(ctas * SEL_CAND) + sizeof(SelState);
}

int select_launches(bool fp64) { return 3 + (fp64 ? KeyOf<double>::ROUNDS : KeyOf<float>::ROUNDS); }

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

// ws: select_workspace_bytes(cols, nslices) bytes, 16-byte aligned: the tail sums, the
// search round's per-CTA partial sums, the search state (zeroed here, in stream order).
template <typename T>
cudaError_t select_ranks(const T *sig, int cols, int nslices, double eps, void *ws,
                         double *scal, int *ranks, int64_t *offsets, int *status,
                         cudaStream_t st) {
  if (cols < 1 || nslices < 1) return cudaErrorInvalidValue;
  const double eps2 = eps * eps;
  double *tail = reinterpret_cast<double *>(ws);
  const int ctas = (int)std::min<int64_t>(((int64_t)nslices + SEL_SLICE_LANES - 1) /
                                              SEL_SLICE_LANES,
                                          SEL_MAX_CTAS);
  const int per_cta = (nslices + ctas - 1) / ctas;
  double *part = tail + (int64_t)cols * nslices;
  SelState *state = reinterpret_cast<SelState *>(part + (int64_t)ctas * SEL_CAND);
  cudaError_t e = cudaMemsetAsync(state, 0, sizeof(SelState), st);
  if (e != cudaSuccess) return e;
  sel_tails_kernel<T><<<(nslices + SEL_WARPS - 1) / SEL_WARPS, 256, 0, st>>>(sig, cols, nslices,
                                                                            eps2, tail, state);
  if ((e = cudaGetLastError()) != cudaSuccess) return e;
  for (int r = 0; r < KeyOf<T>::ROUNDS; ++r) {
    sel_round_kernel<T><<<ctas, 256, 0, st>>>(sig, cols, nslices, eps2, tail, part, state,
                                              per_cta);
    if ((e = cudaGetLastError()) != cudaSuccess) return e;
  }
  sel_finish_kernel<T><<<1, ST, 0, st>>>(sig, cols, nslices, eps2, tail, state, scal, ranks,
                                         offsets, status);
  return cudaGetLastError();
}

template cudaError_t select_ranks<float>(const float *, int, int, double, void *, double *, int *,
                                         int64_t *, int *, cudaStream_t);
template cudaError_t select_ranks<double>(const double *, int, int, double, void *, double *,
                                          int *, int64_t *, int *, cudaStream_t);

}  // namespace tsvdm
