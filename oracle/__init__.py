"""Plain FP64 CPU oracle for the star-M truncated tensor SVD.

TEST INFRASTRUCTURE ONLY: the test-suite, the smoke check and the benchmark's CPU-baseline
leg are the only callers.  The CUDA library never imports, links or calls anything here,
and this package imports nothing from the CUDA library.

Every function states the passage of the paper (arXiv 2605.16058, "High-Performance
star-M SVD for Big Data Compression") that it writes out.  Heavy loops (the mode-3 TTM
and the per-slice Jacobi SVD) live in ``tsvdm_oracle.c``; the rest is NumPy in float64.
Tensors are NumPy arrays of shape (m, p, n) indexed X[a, b, t]; they are handed to C in
column-major (Fortran) order, so frontal slice t is contiguous, as in Sec. 3.

Readings of the paper used here (where it is silent or ambiguous):
  * the primary factors are the transform-domain ("hat") Uhat, Shat, Vhat (Fig. 1,
    Algorithm 2 output); original-domain factors are those mapped back by M^{-1};
  * Algorithm 2 compares w_J / ||S||_F^2 < eps^2 strictly, tau = v_J is a sigma^2 value,
    and rho_i counts sigma^2 > tau strictly, so every value equal to tau is discarded;
  * J = 0 (no admissible index) discards nothing; an all-zero tensor keeps nothing and
    reports relative error 0;
  * the reported relative error is sqrt(discarded sigma^2 / ||S||_F^2), Algorithm 2's
    own normalisation, equal to the relative reconstruction error for any nonzero
    multiple of an orthogonal M;
  * the truncation loss used for differentiation is the transform-domain relative error
    sqrt(sum of discarded sigma^2) / ||X||_F, equal to the original-domain error when M
    is orthogonal (Sec. 2.3);
  * the Cayley form of an orthogonal M is M(A) = (I+W)^{-1}(I-W) M0 with W = A^T - A;
  * a d-way tensor (d > 3) takes one matrix M_k along every mode k >= 3 (the order-d star-M
    product of Sec. 2.1); its frontal slices are all trailing index combinations, in
    column-major order (i3 fastest), and t-SVDM-I/II treat them as one set of slices.

Parity unpinned: the paper's compression-ratio and error values on its real datasets
(NCEP/NCAR reanalysis, NekRS Taylor-Green vortex, MoVO2 X-ray volume) cannot be pinned,
because those datasets are not available; only the storage formula behind them is.
"""
from __future__ import annotations

import ctypes
import math
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "tsvdm_oracle.c")
_SO = os.path.join(_HERE, "_tsvdm_oracle.so")
_lock = threading.Lock()
_lib = None

MAX_SWEEPS = 60


def build_oracle(force: bool = False) -> str:
    """Compile the C part of the oracle with gcc into oracle/_tsvdm_oracle.so."""
    if force or not os.path.exists(_SO) or os.path.getmtime(_SO) < os.path.getmtime(_SRC):
        tmp = _SO + ".%d.tmp" % os.getpid()
        subprocess.check_call(["gcc", "-O2", "-fPIC", "-shared", "-std=c99", "-o", tmp,
                               _SRC, "-lm", "-lpthread"])
        os.replace(tmp, _SO)
    return _SO


def _get():
    global _lib
    with _lock:
        if _lib is None:
            lib = ctypes.CDLL(build_oracle())
            i64, dp, ip = ctypes.c_int64, ctypes.POINTER(ctypes.c_double), ctypes.POINTER(ctypes.c_int64)
            lib.oracle_ttm3.argtypes = [dp, i64, i64, i64, dp, i64, ip, i64, dp]
            lib.oracle_ttm3.restype = None
            lib.oracle_svd.argtypes = [dp, i64, i64, dp, dp, dp, ctypes.c_int]
            lib.oracle_svd.restype = ctypes.c_int
            lib.oracle_svd_slices.argtypes = [dp, i64, i64, i64, dp, dp, dp, ctypes.c_int,
                                              ctypes.POINTER(ctypes.c_int), ctypes.c_int]
            lib.oracle_svd_slices.restype = None
            _lib = lib
    return _lib


def _dp(a):
    return a.ctypes.data_as(ctypes.POINTER(ctypes.c_double))


def _f64(a):
    return np.asfortranarray(np.asarray(a, dtype=np.float64))


def default_threads() -> int:
    return max(1, os.cpu_count() or 1)


# --------------------------------------------------------------------------------------
# Sec. 2.1: mode-3 TTM
# --------------------------------------------------------------------------------------
def ttm3(X, M, which=None):
    """Y = X x_3 M (Sec. 2.1): Y(:,:,i) = sum_t M[i,t] X(:,:,t).  M is J x n.

    ``which`` optionally lists the output slices to form (returned in that order)."""
    X = _f64(X)
    M = _f64(M)
    if X.ndim == 2:
        X = X[:, :, None]
    m, p, n = X.shape
    J = M.shape[0]
    assert M.shape[1] == n
    if which is None:
        Y = np.zeros((m, p, J), dtype=np.float64, order="F")
        _get().oracle_ttm3(_dp(X), m, p, n, _dp(M), J, None, 0, _dp(Y))
    else:
        w = np.ascontiguousarray(np.asarray(which, dtype=np.int64))
        Y = np.zeros((m, p, len(w)), dtype=np.float64, order="F")
        _get().oracle_ttm3(_dp(X), m, p, n, _dp(M), J,
                           w.ctypes.data_as(ctypes.POINTER(ctypes.c_int64)), len(w), _dp(Y))
    return Y


# --------------------------------------------------------------------------------------
# Algorithm 1: slice-wise thin SVD (Hestenes one-sided Jacobi per slice)
# --------------------------------------------------------------------------------------
def svd(A, max_sweeps=MAX_SWEEPS):
    """Thin SVD of one matrix: returns U (m x r), S (r,), V (p x r), sweeps."""
    A = _f64(A)
    m, p = A.shape
    r = min(m, p)
    U = np.zeros((m, r), order="F")
    S = np.zeros(r)
    V = np.zeros((p, r), order="F")
    sw = _get().oracle_svd(_dp(A), m, p, _dp(U), _dp(S), _dp(V), max_sweeps)
    return U, S, V, sw


def svd_slices(Ahat, max_sweeps=MAX_SWEEPS, threads=None):
    """Algorithm 1's loop over frontal slices: U (m,r,n), S (r,n), V (p,r,n), sweeps (n,)."""
    Ahat = _f64(Ahat)
    if Ahat.ndim == 2:
        Ahat = Ahat[:, :, None]
    m, p, n = Ahat.shape
    r = min(m, p)
    U = np.zeros((m, r, n), order="F")
    S = np.zeros((r, n), order="F")
    V = np.zeros((p, r, n), order="F")
    sweeps = np.zeros(n, dtype=np.int32)
    _get().oracle_svd_slices(_dp(Ahat), m, p, n, _dp(U), _dp(S), _dp(V), max_sweeps,
                             sweeps.ctypes.data_as(ctypes.POINTER(ctypes.c_int)),
                             threads or default_threads())
    return U, S, V, sweeps


def data_transform(X):
    """Sec. 2.2's data-driven M: the transposed matrix of left singular vectors of the mode-3
    unfolding A_(3) (n3 x n1 n2; row t is frontal slice t), by decreasing singular value,
    each vector with its largest-magnitude entry positive.  The SVD is LAPACK's (a library
    routine as one step).  Returns (M, sigma)."""
    X = _f64(X)
    n3 = X.shape[2]
    A3 = X.reshape(-1, n3, order="F").T
    W, sig, _ = np.linalg.svd(A3, full_matrices=True)
    for j in range(W.shape[1]):
        i = int(np.argmax(np.abs(W[:, j])))
        if W[i, j] < 0:
            W[:, j] = -W[:, j]
    return W.T.copy(), sig


def ttm_mode(X, M, mode):
    """Y = X x_mode M for a d-way X (Sec. 2.1's mode-k product; mode is 0-based):
    Y(.., i, ..) = sum_t M[i,t] X(.., t, ..).  Each trailing index combination is one
    mode-3 product of the (leading dims) x 1 x n_mode view, done by ttm3's loops."""
    X = _f64(X)
    M = _f64(M)
    shp = X.shape
    lead = int(np.prod(shp[:mode], dtype=np.int64))
    tail = int(np.prod(shp[mode + 1:], dtype=np.int64))
    X3 = X.reshape((lead, shp[mode], tail), order="F")
    Y3 = np.empty((lead, M.shape[0], tail), order="F")
    for q in range(tail):
        Y3[:, :, q] = ttm3(np.asfortranarray(X3[:, None, :, q]), M)[:, 0, :]
    return Y3.reshape(shp[:mode] + (M.shape[0],) + shp[mode + 1:], order="F")


def dway_transform(X, Ms):
    """Ahat = X x_3 M_3 x_4 M_4 ... for a d-way X and the list Ms = [M_3, M_4, ...]."""
    Y = _f64(X)
    for j, M in enumerate(Ms):
        Y = ttm_mode(Y, M, 2 + j)
    return Y


def to_slices(Y):
    """n1 x n2 x n3 x ... x nd -> n1 x n2 x (n3 ... nd), slice index i3 + n3 i4 + ..."""
    return Y.reshape((Y.shape[0], Y.shape[1], -1), order="F")


def _transform(X, M):
    """The forward transform of Algorithm 1: ttm3 for a 3-way X and one M; for a d-way X
    and a list of matrices (one per mode >= 3), all of them, viewed as frontal slices."""
    if isinstance(M, (list, tuple)):
        return to_slices(dway_transform(X, M))
    return ttm3(X, M)


def full_tsvdm(X, M, threads=None, max_sweeps=MAX_SWEEPS):
    """Algorithm 1: Ahat = X x_3 M, then the thin SVD of every frontal slice of Ahat.  For a
    d-way X, M is the list of per-mode matrices and the slices run over all trailing index
    combinations."""
    Ahat = _transform(X, M)
    U, S, V, sweeps = svd_slices(Ahat, max_sweeps=max_sweeps, threads=threads)
    return dict(Ahat=Ahat, U=U, S=S, V=V, sweeps=sweeps)


# --------------------------------------------------------------------------------------
# Sec. 3.3 (t-SVDM-I) and Fig. 1: uniform rank k per slice
# --------------------------------------------------------------------------------------
def fixed_rank(X, M, k, threads=None, max_sweeps=MAX_SWEEPS):
    """t-SVDM-I: keep the leading k triplets of every transformed slice (hat domain).

    rel_err is sqrt(sum of discarded sigma^2 / sum of all sigma^2), the normalisation of
    Algorithm 2 (||S||_F^2); by Eckart-Young (Sec. 2.3) it equals ||X - X_k||_F / ||X||_F
    whenever M is a nonzero multiple of an orthogonal matrix."""
    X = _f64(X)
    full = full_tsvdm(X, M, threads=threads, max_sweeps=max_sweeps)
    r = full["S"].shape[0]
    if not (1 <= k <= r):
        raise ValueError("k must satisfy 1 <= k <= min(n1, n2)")
    S = full["S"]
    discarded = float(np.sum(S[k:, :] ** 2))
    total = float(np.sum(S ** 2))
    return dict(U=full["U"][:, :k, :].copy(order="F"), S=S[:k, :].copy(order="F"),
                V=full["V"][:, :k, :].copy(order="F"), Ahat=full["Ahat"], S_all=S,
                sweeps=full["sweeps"], discarded=discarded, total=total,
                rel_err=math.sqrt(discarded / total) if total > 0 else 0.0)


# --------------------------------------------------------------------------------------
# Algorithm 2: t-SVDM-II rank choice from a global error tolerance
# --------------------------------------------------------------------------------------
def select_ranks(S, eps):
    """Algorithm 2 steps 2-8 on the singular values S (r x n, any order within a slice).

    Returns dict(ranks (n,), J (1-based count of discarded values, 0 = none), tau
    (sigma^2 threshold, -inf when J = 0), total = ||S||_F^2, discarded = sum of the
    sigma^2 that are not kept)."""
    S = np.asarray(S, dtype=np.float64)
    if S.ndim == 1:
        S = S[:, None]
    r, n = S.shape
    v = np.sort((S * S).reshape(-1, order="F"), kind="stable")   # step 3: ascending
    w = np.cumsum(v)                                             # step 4: w_k = sum v_1..v_k
    total = float(w[-1]) if w.size else 0.0                      # ||S||_F^2 = sum of v
    if total == 0.0:
        # all singular values are zero: nothing carries energy, keep nothing
        return dict(ranks=np.zeros(n, dtype=np.int64), J=int(v.size), tau=0.0,
                    total=0.0, discarded=0.0)
    eps2 = float(eps) * float(eps)
    ok = np.nonzero(w / total < eps2)[0]                         # step 5
    J = int(ok[-1]) + 1 if ok.size else 0
    tau = float(v[J - 1]) if J > 0 else -math.inf                # step 6
    S2 = S * S
    ranks = np.sum(S2 > tau, axis=0).astype(np.int64)            # step 8
    discarded = float(np.sum(np.where(S2 > tau, 0.0, S2)))
    return dict(ranks=ranks, J=J, tau=tau, total=total, discarded=discarded)


def offsets_from_ranks(ranks):
    ranks = np.asarray(ranks, dtype=np.int64)
    off = np.zeros(len(ranks) + 1, dtype=np.int64)
    off[1:] = np.cumsum(ranks)
    return off


def tolerance(X, M, eps, threads=None, max_sweeps=MAX_SWEEPS):
    """t-SVDM-II (Algorithm 2, 'truncate' strategy of Sec. 3.4): full t-SVDM, global
    threshold, then the leading rho_i hat-domain triplets of slice i packed without
    padding (slice i's columns at offsets[i] .. offsets[i+1])."""
    X = _f64(X)
    full = full_tsvdm(X, M, threads=threads, max_sweeps=max_sweeps)
    sel = select_ranks(full["S"], eps)
    ranks = sel["ranks"]
    off = offsets_from_ranks(ranks)
    tot = int(off[-1])
    m, r, n = full["U"].shape
    p = full["V"].shape[0]
    U = np.zeros((m, tot), order="F")
    S = np.zeros(tot)
    V = np.zeros((p, tot), order="F")
    for i in range(n):
        a, b = off[i], off[i + 1]
        U[:, a:b] = full["U"][:, : b - a, i]
        S[a:b] = full["S"][: b - a, i]
        V[:, a:b] = full["V"][:, : b - a, i]
    tot2 = sel["total"]
    return dict(ranks=ranks, offsets=off, U=U, S=S, V=V, S_all=full["S"],
                Ahat=full["Ahat"], sweeps=full["sweeps"], J=sel["J"], tau=sel["tau"],
                total=tot2, discarded=sel["discarded"],
                rel_err=math.sqrt(sel["discarded"] / tot2) if tot2 > 0 else 0.0)


# --------------------------------------------------------------------------------------
# Reconstruction (Sec. 2.1 star-M product; Sec. 2.2 map back by M^{-1})
# --------------------------------------------------------------------------------------
def reconstruct(U, S, V, Minv, k=None, offsets=None):
    """X_k = (U_i diag(S_i) V_i^T per slice) x_3 M^{-1}.

    Uniform rank: U (m,k,n), S (k,n), V (p,k,n).  Variable rank: packed U (m,total),
    S (total,), V (p,total) with ``offsets`` (n+1).  For a d-way tensor Minv is the list of
    per-mode inverses [M_3^{-1}, M_4^{-1}, ...] and the result is m x p x n3 x ... x nd."""
    if isinstance(Minv, (list, tuple)):
        dims = tuple(_f64(Mi).shape[0] for Mi in Minv)
        eye = np.eye(int(np.prod(dims)))
        Ak = reconstruct(U, S, V, eye, k=k, offsets=offsets)        # slice products only
        Ak = Ak.reshape(Ak.shape[:2] + dims, order="F")
        for j, Mi in enumerate(Minv):
            Ak = ttm_mode(Ak, Mi, 2 + j)
        return Ak
    Minv = _f64(Minv)
    n = Minv.shape[0]
    if offsets is None:
        U = np.asarray(U, dtype=np.float64)
        m, p = U.shape[0], np.asarray(V).shape[0]
        Ak = np.zeros((m, p, n), order="F")
        for i in range(n):
            Ak[:, :, i] = (U[:, :, i] * S[None, :, i]) @ np.asarray(V)[:, :, i].T
    else:
        U = np.asarray(U, dtype=np.float64)
        V = np.asarray(V, dtype=np.float64)
        S = np.asarray(S, dtype=np.float64)
        m, p = U.shape[0], V.shape[0]
        Ak = np.zeros((m, p, n), order="F")
        for i in range(n):
            a, b = int(offsets[i]), int(offsets[i + 1])
            Ak[:, :, i] = (U[:, a:b] * S[None, a:b]) @ V[:, a:b].T
    return ttm3(Ak, Minv)


def frob(X) -> float:
    X = np.asarray(X, dtype=np.float64)
    return math.sqrt(float(np.sum(X * X)))


def rel_err_direct(X, Xk) -> float:
    xn = frob(X)
    return frob(np.asarray(X, dtype=np.float64) - Xk) / xn if xn > 0 else 0.0


def original_domain(F, Minv):
    """Map a hat-domain factor (m x k x n) or diagonal block (k x n) back by M^{-1} (for a
    d-way tensor: the list of per-mode inverses, n = n3 ... nd slices)."""
    F = np.asarray(F, dtype=np.float64)
    if isinstance(Minv, (list, tuple)):
        dims = tuple(_f64(Mi).shape[0] for Mi in Minv)
        G = F[:, None, :] if F.ndim == 2 else F
        G = G.reshape(G.shape[:2] + dims, order="F")
        for j, Mi in enumerate(Minv):
            G = ttm_mode(G, Mi, 2 + j)
        G = to_slices(G)
        return G[:, 0, :] if F.ndim == 2 else G
    if F.ndim == 2:
        return ttm3(F[:, None, :], Minv)[:, 0, :]
    return ttm3(F, Minv)


# --------------------------------------------------------------------------------------
# Truncation loss and its gradient (differentiable extension of t-SVDM-I)
# --------------------------------------------------------------------------------------
def loss_and_grad(X, M, k, threads=None):
    """L(X, M) = sqrt(E) / ||X||_F with E = sum_i sum_{j>k} sigma_j(Ahat_i)^2, Ahat = X x_3 M.

    dE/dAhat_i = 2 R_i with R_i = Ahat_i - U_k S_k V_k^T (first-order perturbation of the
    singular values, valid when sigma_k > sigma_{k+1}).  With Ahat_(mat) = X_(mat) M^T:
      dL/dX = (R x_3 M^T) / (sqrt(E) ||X||) - L X / ||X||^2
      dL/dM = R_(mat)^T X_(mat) / (sqrt(E) ||X||)          (n x n)
    where X_(mat) is the (m p) x n column-major view."""
    X = _f64(X)
    M = _f64(M)
    m, p, n = X.shape
    fr = fixed_rank(X, M, k, threads=threads)
    Ahat = fr["Ahat"]
    R = np.zeros_like(Ahat, order="F")
    for i in range(n):
        R[:, :, i] = Ahat[:, :, i] - (fr["U"][:, :, i] * fr["S"][None, :, i]) @ fr["V"][:, :, i].T
    E = float(np.sum(R * R))
    xn = frob(X)
    L = math.sqrt(E) / xn
    if E == 0.0:
        return dict(loss=0.0, dX=np.zeros_like(X), dM=np.zeros_like(M), E=0.0, R=R, fr=fr)
    scale = 1.0 / (math.sqrt(E) * xn)
    dX = ttm3(R, M.T) * scale - (L / (xn * xn)) * X
    Rm = R.reshape(m * p, n, order="F")
    Xm = X.reshape(m * p, n, order="F")
    dM = (Rm.T @ Xm) * scale
    return dict(loss=L, dX=dX, dM=dM, E=E, R=R, fr=fr)


def cayley(A, M0):
    """Cayley-parametrised orthogonal transform: W = A^T - A (skew),
    Q = (I + W)^{-1} (I - W), M = Q M0."""
    A = np.asarray(A, dtype=np.float64)
    n = A.shape[0]
    W = A.T - A
    I = np.eye(n)
    Q = np.linalg.solve(I + W, I - W)
    return Q @ np.asarray(M0, dtype=np.float64), Q, W


def cayley_grad(A, M0, dM):
    """Chain rule through cayley(): dL/dQ = dL/dM M0^T;
    dL/dW = -(I+W)^{-T} dL/dQ (Q+I)^T;  dL/dA = (dL/dW)^T - dL/dW."""
    A = np.asarray(A, dtype=np.float64)
    n = A.shape[0]
    _, Q, W = cayley(A, M0)
    I = np.eye(n)
    dQ = np.asarray(dM) @ np.asarray(M0, dtype=np.float64).T
    dW = -np.linalg.solve((I + W).T, dQ @ (Q + I).T)
    return dW.T - dW


def adam_step(param, grad, m1, m2, t, lr=1e-3, b1=0.9, b2=0.999, eps=1e-8):
    """One Adam update (Kingma & Ba, Algorithm 1), in place; t is the 1-based step."""
    m1[...] = b1 * m1 + (1.0 - b1) * grad
    m2[...] = b2 * m2 + (1.0 - b2) * grad * grad
    mh = m1 / (1.0 - b1 ** t)
    vh = m2 / (1.0 - b2 ** t)
    param[...] = param - lr * mh / (np.sqrt(vh) + eps)
    return param


# --------------------------------------------------------------------------------------
# Storage bookkeeping (Sec. 3.4 variable-rank format; compression ratios of Sec. 4)
# --------------------------------------------------------------------------------------
def compression_ratio_fixed(m, p, n, k) -> float:
    """Input entries m p n over the t-SVDM-I factors' entries n k (m + p + 1)."""
    return (m * p) / (k * (m + p + 1.0))


def compression_ratio_variable(m, p, ranks, with_sigma=True) -> float:
    """Input entries over sum_i rho_i (m + p [+ 1]) for the variable-rank format."""
    ranks = np.asarray(ranks)
    n = len(ranks)
    per = m + p + (1 if with_sigma else 0)
    tot = float(np.sum(ranks)) * per
    return (m * p * n) / tot if tot > 0 else math.inf
