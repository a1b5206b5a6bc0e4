/*
 * Plain FP64 CPU oracle for the star-M truncated tensor SVD (t-SVDM-I / t-SVDM-II).
 *
 * TEST INFRASTRUCTURE ONLY.  Nothing on the product path links, loads or calls this
 * file: only the test-suite, the smoke check and the CPU-baseline leg of the benchmark
 * use it.  It shares no code, header or constant with the CUDA library.
 *
 * What it computes (the definitions, written out with no blocking or reordering):
 *
 *   oracle_ttm3      mode-3 tensor-times-matrix, Sec. 2.1 (definition of the mode-k TTM):
 *                    Y(a,b,i) = sum_t M(i,t) X(a,b,t), summed in the order t = 0..n-1.
 *   oracle_svd       thin SVD of one m x p matrix by Hestenes one-sided Jacobi
 *                    (cyclic ordering i<j, Demmel-Veselic stopping rule), the per-slice
 *                    svd of Algorithm 1.  Singular values descending, ties kept in
 *                    original column order; each left vector's largest-magnitude entry
 *                    is made positive (the paper leaves signs free).
 *   oracle_svd_slices  the loop of Algorithm 1 over the n frontal slices, one slice at a
 *                    time per worker thread (slices are independent).
 *
 * Layout: everything column-major; frontal slice i of an m x p x n tensor starts at
 * offset i*m*p (Sec. 3, data layout).  An n x n matrix M has M(i,t) at M[i + n*t].
 */
#include <math.h>
#include <pthread.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

/* Y = X x_3 M, with X m x p x n and M J x n (so Y is m x p x J).  Only the output slices
 * listed in `which` (length nwhich) are formed; which == NULL means all J slices, written
 * at their own position.  With a list, output slice which[q] is written at position q. */
void oracle_ttm3(const double *X, int64_t m, int64_t p, int64_t n, const double *M,
                 int64_t J, const int64_t *which, int64_t nwhich, double *Y) {
  int64_t mp = m * p;
  int64_t nout = which ? nwhich : J;
  for (int64_t q = 0; q < nout; ++q) {
    int64_t i = which ? which[q] : q;
    double *y = Y + q * mp;
    for (int64_t e = 0; e < mp; ++e) {
      double acc = 0.0;
      for (int64_t t = 0; t < n; ++t) acc += M[i + J * t] * X[e + mp * t];
      y[e] = acc;
    }
  }
}

/* Hestenes one-sided Jacobi on the columns of W (rows x cols, rows >= cols), with the
 * rotations accumulated in Z (cols x cols, starts as the identity).  Returns the number
 * of sweeps taken, or -1 if `max_sweeps` sweeps still rotated. */
static int jacobi_columns(double *W, int64_t rows, int64_t cols, double *Z,
                          int max_sweeps, double tol) {
  for (int64_t a = 0; a < cols * cols; ++a) Z[a] = 0.0;
  for (int64_t a = 0; a < cols; ++a) Z[a + cols * a] = 1.0;
  for (int sweep = 1; sweep <= max_sweeps; ++sweep) {
    int rotated = 0;
    for (int64_t i = 0; i < cols - 1; ++i) {
      for (int64_t j = i + 1; j < cols; ++j) {
        double *wi = W + rows * i, *wj = W + rows * j;
        double alpha = 0.0, beta = 0.0, gamma = 0.0;
        for (int64_t r = 0; r < rows; ++r) {
          alpha += wi[r] * wi[r];
          beta += wj[r] * wj[r];
          gamma += wi[r] * wj[r];
        }
        if (!(fabs(gamma) > tol * sqrt(alpha * beta))) continue;
        rotated = 1;
        double zeta = (beta - alpha) / (2.0 * gamma);
        double t = (zeta >= 0.0 ? 1.0 : -1.0) / (fabs(zeta) + sqrt(1.0 + zeta * zeta));
        double c = 1.0 / sqrt(1.0 + t * t);
        double s = c * t;
        for (int64_t r = 0; r < rows; ++r) {
          double x = wi[r], y = wj[r];
          wi[r] = c * x - s * y;
          wj[r] = s * x + c * y;
        }
        double *zi = Z + cols * i, *zj = Z + cols * j;
        for (int64_t r = 0; r < cols; ++r) {
          double x = zi[r], y = zj[r];
          zi[r] = c * x - s * y;
          zj[r] = s * x + c * y;
        }
      }
    }
    if (!rotated) return sweep;
  }
  return -1;
}

/* Thin SVD of the m x p column-major matrix A:  A = U diag(S) V^T with U m x r, V p x r,
 * r = min(m,p).  A is not modified.  Returns sweeps taken (>0) or -1 (no convergence).
 * Wide matrices (m < p) are handled by factoring A^T and exchanging U and V. */
int oracle_svd(const double *A, int64_t m, int64_t p, double *U, double *S, double *V,
               int max_sweeps) {
  int wide = m < p;
  int64_t rows = wide ? p : m, cols = wide ? m : p;  /* the matrix W that is rotated */
  double *W = (double *)malloc(sizeof(double) * rows * cols);
  double *Z = (double *)malloc(sizeof(double) * cols * cols);
  double *nrm = (double *)malloc(sizeof(double) * cols);
  int64_t *ord = (int64_t *)malloc(sizeof(int64_t) * cols);
  for (int64_t a = 0; a < m; ++a)
    for (int64_t b = 0; b < p; ++b) {
      double v = A[a + m * b];
      if (wide) W[b + rows * a] = v; else W[a + rows * b] = v;
    }
  double tol = (double)rows * ldexp(1.0, -53);
  int sweeps = jacobi_columns(W, rows, cols, Z, max_sweeps, tol);

  /* sigma_j = ||w_j||, then order by sigma descending; a stable insertion sort keeps
   * equal values in their original column order. */
  for (int64_t j = 0; j < cols; ++j) {
    double acc = 0.0;
    for (int64_t r = 0; r < rows; ++r) acc += W[r + rows * j] * W[r + rows * j];
    nrm[j] = sqrt(acc);
    ord[j] = j;
  }
  for (int64_t a = 1; a < cols; ++a) {
    int64_t key = ord[a];
    int64_t b = a - 1;
    while (b >= 0 && nrm[ord[b]] < nrm[key]) { ord[b + 1] = ord[b]; --b; }
    ord[b + 1] = key;
  }
  /* left vectors of W are w_j / sigma_j (zero when sigma_j = 0); right vectors are Z's
   * columns.  For a wide A, A's left vectors are Z's columns and its right vectors are
   * W's normalised columns. */
  int64_t ulen = wide ? cols : rows, vlen = wide ? rows : cols;
  for (int64_t q = 0; q < cols; ++q) {
    int64_t j = ord[q];
    double sg = nrm[j];
    S[q] = sg;
    double *u = U + ulen * q, *v = V + vlen * q;
    const double *wcol = W + rows * j, *zcol = Z + cols * j;
    for (int64_t r = 0; r < rows; ++r) {
      double w = sg > 0.0 ? wcol[r] / sg : 0.0;
      if (wide) v[r] = w; else u[r] = w;
    }
    for (int64_t r = 0; r < cols; ++r) {
      if (wide) u[r] = zcol[r]; else v[r] = zcol[r];
    }
    /* sign: make the largest-magnitude entry of the left vector positive (first such
     * entry on ties); if the left vector is zero, use the right vector instead. */
    const double *ref = u;
    int64_t rlen = ulen;
    double best = 0.0;
    int64_t arg = -1;
    for (int64_t r = 0; r < rlen; ++r)
      if (fabs(ref[r]) > best) { best = fabs(ref[r]); arg = r; }
    if (arg < 0) {
      ref = v; rlen = vlen;
      for (int64_t r = 0; r < rlen; ++r)
        if (fabs(ref[r]) > best) { best = fabs(ref[r]); arg = r; }
    }
    if (arg >= 0 && ref[arg] < 0.0) {
      for (int64_t r = 0; r < ulen; ++r) u[r] = -u[r];
      for (int64_t r = 0; r < vlen; ++r) v[r] = -v[r];
    }
  }
  free(W); free(Z); free(nrm); free(ord);
  return sweeps;
}

typedef struct {
  const double *A; int64_t m, p, n; double *U, *S, *V; int max_sweeps; int *sweeps;
  int64_t next; pthread_mutex_t lock;
} slice_job;

static void *slice_worker(void *arg) {
  slice_job *job = (slice_job *)arg;
  int64_t r = job->m < job->p ? job->m : job->p;
  for (;;) {
    pthread_mutex_lock(&job->lock);
    int64_t i = job->next++;
    pthread_mutex_unlock(&job->lock);
    if (i >= job->n) break;
    job->sweeps[i] = oracle_svd(job->A + i * job->m * job->p, job->m, job->p,
                                job->U + i * job->m * r, job->S + i * r,
                                job->V + i * job->p * r, job->max_sweeps);
  }
  return NULL;
}

/* Algorithm 1's loop: thin SVD of each of the n frontal slices of A (m x p x n).
 * U m x r x n, S r x n, V p x r x n.  sweeps[i] receives slice i's sweep count (-1 when
 * it did not converge).  Slices are spread over `threads` worker threads. */
void oracle_svd_slices(const double *A, int64_t m, int64_t p, int64_t n, double *U,
                       double *S, double *V, int max_sweeps, int *sweeps, int threads) {
  slice_job job = {A, m, p, n, U, S, V, max_sweeps, sweeps, 0, PTHREAD_MUTEX_INITIALIZER};
  if (threads < 1) threads = 1;
  if (threads > 256) threads = 256;
  pthread_t tid[256];
  for (int a = 0; a < threads; ++a) pthread_create(&tid[a], NULL, slice_worker, &job);
  for (int a = 0; a < threads; ++a) pthread_join(tid[a], NULL);
}
