// Fast mode-3 transform by the orthonormal DCT-II (Sec. 2.2: the paper's transform, which
// it notes can be applied in O(n log n) instead of as a dense n x n product).
//
// For a mode-3 fiber x (length n, a power of two), with s_0 = sqrt(1/n), s_k = sqrt(2/n):
//   forward  y_k = s_k sum_t x_t cos(pi k (2t + 1) / (2n))        (y = M x)
//   inverse  x = M^T y                                            (DCT-III, M orthogonal)
// Forward, after Makhoul: v_t = x_{2t}, v_{n-1-t} = x_{2t+1}; V = FFT_n(v);
//   y_k = s_k Re(e^{-i pi k / (2n)} V_k).
// Inverse: V_k = e^{i pi k / (2n)} (y_k - i y_{n-k}) / (s_k n) (y_n = 0, the s_{n-k} = s_k
//   of k >= 1 taken out); v = n IFFT_n(V) / n; x_{2t} = Re v_t, x_{2t+1} = Re v_{n-1-t}.
// The FFT is a radix-2 decimation-in-frequency FFT in shared memory whose output is in
// bit-reversed order (read through __brev); its stages run in passes of up to four, each
// thread holding the 2^a values of one butterfly group in registers, so shared memory is
// read and written once per pass instead of once per stage.
//
// A CTA takes R consecutive rows of the (rows x n) column-major view (R fibers): the loads
// and stores of one t cover R consecutive floats.  Twiddles come from tables computed on
// the host in double precision.  HBM traffic: one read and one write of the tensor.
#include "common.cuh"

namespace tsvdm {
namespace {

template <typename T> struct Cx { T re, im; };

constexpr int DT = 256;

// Position of element i of a fiber in shared memory: one padding element after every 16
// (a complex value spans two banks, so 16 of them fill the 32 banks): the FFT passes, whose
// register groups gather elements 2^blo apart, then meet at most 2-way bank conflicts
// instead of up to 32-way.
__device__ __forceinline__ int pad(int i) { return i + (i >> 4); }

template <typename T>
__device__ __forceinline__ Cx<T> cmul(Cx<T> a, Cx<T> b) {
  return {a.re * b.re - a.im * b.im, a.re * b.im + a.im * b.re};
}

// One pass of A DIF stages s0 .. s0 + A - 1 on every fiber of the tile: group g of a fiber
// holds the indices base + (m << blo), m < 2^A, blo = L - s0 - A.  Stage s pairs index i with
// i + (n >> (s + 1)) and multiplies the difference by tw[(i mod h) << s], h = n >> (s + 1).
template <typename T, int A>
__device__ __forceinline__ void dif_pass(Cx<T> *buf, int ld, int R, int n, int L, int s0,
                                         const Cx<T> *tw) {
  constexpr int NM = 1 << A;
  const int blo = L - s0 - A;
  const int G = n >> A;
  for (int gi = threadIdx.x; gi < R * G; gi += DT) {
    const int r = gi / G, g = gi - r * G;
    const int lo = g & ((1 << blo) - 1), hi = g >> blo;
    const int base = lo | (hi << (blo + A));
    Cx<T> *f = buf + (int64_t)r * ld;
    Cx<T> v[NM];
#pragma unroll
    for (int m = 0; m < NM; ++m) v[m] = f[pad(base + (m << blo))];
#pragma unroll
    for (int st = 0; st < A; ++st) {
      const int s = s0 + st;
      const int h = n >> (s + 1);
      const int hm = 1 << (A - 1 - st);
#pragma unroll
      for (int m = 0; m < NM; ++m) {
        if (m & hm) continue;
        const int i = base + (m << blo);
        const Cx<T> a = v[m], b = v[m + hm];
        v[m] = {a.re + b.re, a.im + b.im};
        v[m + hm] = cmul<T>({a.re - b.re, a.im - b.im}, tw[(i & (h - 1)) << s]);
      }
    }
#pragma unroll
    for (int m = 0; m < NM; ++m) f[pad(base + (m << blo))] = v[m];
  }
}

__device__ __forceinline__ int brev(int k, int L) {
  return L > 0 ? (int)(__brev((unsigned)k) >> (32 - L)) : 0;
}

// tables (device): fw[n/2] forward FFT twiddles e^{-2 pi i m / n}, iw[n/2] their conjugates,
// post[n] = s_k e^{-i pi k / (2n)} (forward), pre[n] = e^{i pi k / (2n)} / (s_k n) (inverse)
template <typename T>
__global__ void __launch_bounds__(DT) dct_kernel(const T *__restrict__ X, int64_t P, int n,
                                                  int L, int R, bool inverse,
                                                  const Cx<T> *__restrict__ tab,
                                                  T *__restrict__ Y) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  Cx<T> *tw = reinterpret_cast<Cx<T> *>(smem_raw);                 // n/2 (max 1)
  Cx<T> *pp = tw + (n > 1 ? n / 2 : 1);                             // n
  Cx<T> *buf = pp + n;                                              // R x ld
  const int ld = pad(n) + 1;
  const int64_t r0 = (int64_t)blockIdx.x * R;
  const int64_t off = (int64_t)blockIdx.y * P * n;                  // batch of views
  const T *Xb = X + off;
  T *Yb = Y + off;
  const int nh = n > 1 ? n / 2 : 1;
  const Cx<T> *ftab = tab + (inverse ? nh : 0);
  const Cx<T> *ptab = tab + 2 * nh + (inverse ? n : 0);
  for (int i = threadIdx.x; i < nh; i += DT) tw[i] = ftab[i];
  for (int i = threadIdx.x; i < n; i += DT) pp[i] = ptab[i];
  // load (R consecutive rows per t)
  for (int idx = threadIdx.x; idx < R * n; idx += DT) {
    const int r = idx % R, t = idx / R;
    const int64_t row = r0 + r;
    const T x = row < P ? Xb[row + P * t] : T(0);
    if (!inverse) {
      const int j = (t & 1) ? n - 1 - (t >> 1) : (t >> 1);
      buf[(int64_t)r * ld + pad(j)] = {x, T(0)};
    } else {
      buf[(int64_t)r * ld + pad(t)] = {x, T(0)};
    }
  }
  __syncthreads();
  if (inverse) {
    // V_k and V_{n-k} from y_k and y_{n-k} (one thread per pair)
    const int np = n / 2 + 1;
    for (int idx = threadIdx.x; idx < R * np; idx += DT) {
      const int r = idx / np, k = idx - r * np;
      Cx<T> *f = buf + (int64_t)r * ld;
      const T yk = f[pad(k < n ? k : 0)].re;
      if (k == 0) {
        f[0] = {yk * pp[0].re, T(0)};
      } else if (2 * k == n) {
        f[pad(k)] = cmul<T>(pp[k], {yk, -yk});
      } else if (k < n) {
        const T ynk = f[pad(n - k)].re;
        f[pad(k)] = cmul<T>(pp[k], {yk, -ynk});
        f[pad(n - k)] = cmul<T>(pp[n - k], {ynk, -yk});
      }
    }
    __syncthreads();
  }
  // the FFT (forward or inverse by the twiddle table), in passes of up to four stages
  for (int s0 = 0; s0 < L;) {
    const int a = L - s0 >= 4 ? 4 : L - s0;
    switch (a) {
      case 4: dif_pass<T, 4>(buf, ld, R, n, L, s0, tw); break;
      case 3: dif_pass<T, 3>(buf, ld, R, n, L, s0, tw); break;
      case 2: dif_pass<T, 2>(buf, ld, R, n, L, s0, tw); break;
      default: dif_pass<T, 1>(buf, ld, R, n, L, s0, tw); break;
    }
    s0 += a;
    __syncthreads();
  }
  // output (bit-reversed FFT order), R consecutive rows per output index
  for (int idx = threadIdx.x; idx < R * n; idx += DT) {
    const int r = idx % R, k = idx / R;
    const int64_t row = r0 + r;
    if (row >= P) continue;
    const Cx<T> *f = buf + (int64_t)r * ld;
    T y;
    if (!inverse) {
      const Cx<T> v = f[pad(brev(k, L))];
      y = pp[k].re * v.re - pp[k].im * v.im;
    } else {
      const int j = (k & 1) ? n - 1 - (k >> 1) : (k >> 1);
      y = f[pad(brev(j, L))].re;
    }
    Yb[row + P * k] = y;
  }
}

}  // namespace

int dct_rows_per_cta(int n) {
  int R = 4096 / (n > 0 ? n : 1);
  return R < 1 ? 1 : (R > 32 ? 32 : R);
}

size_t dct_smem_bytes(int n, size_t cx_bytes) {
  const int R = dct_rows_per_cta(n);
  return cx_bytes * ((size_t)(n > 1 ? n / 2 : 1) + n + (size_t)R * (n + (n >> 4) + 1));
}

template <typename T>
cudaError_t dct_mode3(const T *X, int64_t P, int64_t n, int64_t batch, bool inverse,
                      const void *tables, T *Y, cudaStream_t st) {
  if (n < 1 || n > 4096 || (n & (n - 1)) != 0 || P < 1 || batch < 1) return cudaErrorInvalidValue;
  int L = 0;
  while ((1 << L) < n) ++L;
  const int R = dct_rows_per_cta((int)n);
  const size_t smem = dct_smem_bytes((int)n, sizeof(Cx<T>));
  auto kern = dct_kernel<T>;
  if (smem > 48 * 1024) {
    cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                         (int)smem);
    if (e != cudaSuccess) return e;
  }
  for (int64_t q0 = 0; q0 < batch; q0 += 65535) {          // grid.y limit
    const int64_t qn = batch - q0 < 65535 ? batch - q0 : 65535;
    dim3 grid((unsigned)((P + R - 1) / R), (unsigned)qn);
    kern<<<grid, DT, smem, st>>>(X + q0 * P * n, P, (int)n, L, R, inverse,
                                 reinterpret_cast<const Cx<T> *>(tables), Y + q0 * P * n);
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return e;
  }
  return cudaSuccess;
}

template cudaError_t dct_mode3<float>(const float *, int64_t, int64_t, int64_t, bool,
                                      const void *, float *, cudaStream_t);
template cudaError_t dct_mode3<double>(const double *, int64_t, int64_t, int64_t, bool,
                                       const void *, double *, cudaStream_t);

}  // namespace tsvdm
