"""Seeded synthetic inputs shaped like the paper's workloads (Sec. 4).

This module generates inputs only: it holds none of the method's arithmetic, imports
nothing else from this package, and serves both the CUDA path and the FP64 oracle.
Everything is drawn on the host in float64 with ``numpy.random.default_rng`` (PCG64) in
the order documented per function, then cast.  Tensors are (n1, n2, n3) arrays in
column-major (Fortran) order: frontal slice t is contiguous.

Workloads (the paper's datasets are not available; these stand in for them):
  * ``cp_tensor``      sum of R rank-1 terms 2^(-r/4) a_r o b_r o c_r plus Gaussian noise
                       (the 64x48x16 smoke case and the uneven batch);
  * ``climate``        spatial Gaussian random fields with power spectrum |k|^-3, evolved
                       along mode 3 as AR(1) with rho = 0.95 (stands in for the NCEP/NCAR
                       air-temperature reanalysis of Sec. 4.1);
  * ``cfd``            40 travelling waves with k^-5/3 amplitudes and a cosine spanwise
                       profile plus 1e-4 relative noise (stands in for the Taylor-Green
                       vortex DNS of Sec. 4.2);
  * ``crystal``        Gaussian peaks on a shared lattice with log-normal intensities and a
                       slice-dependent drift (stands in for the MoVO2 X-ray diffuse
                       scattering volume of Sec. 4.3).
Transforms: the orthonormal DCT-II (Sec. 2.2) and Haar-random orthogonal matrices.
"""
from __future__ import annotations

import math

import numpy as np


def dct2_matrix(n: int) -> np.ndarray:
    """Orthonormal DCT-II as an n x n matrix, row i = frequency i:
    M[i, t] = sqrt((2 - [i == 0]) / n) * cos(pi * (2t + 1) * i / (2n))."""
    i = np.arange(n, dtype=np.float64)[:, None]
    t = np.arange(n, dtype=np.float64)[None, :]
    M = np.cos(math.pi * (2.0 * t + 1.0) * i / (2.0 * n)) * math.sqrt(2.0 / n)
    M[0, :] = math.sqrt(1.0 / n)
    return np.asfortranarray(M)


def haar_orthogonal(n: int, rng: np.random.Generator) -> np.ndarray:
    """Haar-distributed orthogonal matrix: QR of an n x n N(0,1) matrix (drawn row-major),
    with Q's columns multiplied by sign(diag R)."""
    G = rng.standard_normal((n, n))
    Q, R = np.linalg.qr(G)
    d = np.sign(np.diag(R))
    d[d == 0] = 1.0
    return np.asfortranarray(Q * d[None, :])


def cp_tensor(n1, n2, n3, R, rng, noise_rel=1e-3, dtype=np.float64):
    """X = sum_{r=1..R} 2^(-r/4) a_r o b_r o c_r  +  N(0, s^2) noise.

    Draw order: for r = 1..R, a_r (n1), b_r (n2), c_r (n3) ~ N(0,1), each normalised to
    unit length; then the noise tensor (n1*n2*n3 draws, column-major order) scaled to
    s = noise_rel * ||X_clean||_F / sqrt(n1 n2 n3)."""
    A = np.empty((n1, R))
    B = np.empty((n2, R))
    C = np.empty((n3, R))
    for r in range(R):
        a = rng.standard_normal(n1)
        b = rng.standard_normal(n2)
        c = rng.standard_normal(n3)
        A[:, r] = a / np.linalg.norm(a)
        B[:, r] = b / np.linalg.norm(b)
        C[:, r] = c / np.linalg.norm(c)
    sig = 2.0 ** (-np.arange(1, R + 1, dtype=np.float64) / 4.0)
    KR = (A[:, None, :] * B[None, :, :]).reshape(n1 * n2, R, order="F")   # a_r (x) b_r
    Xm = KR @ (C * sig[None, :]).T                                       # (n1 n2) x n3
    X = Xm.reshape(n1, n2, n3, order="F")
    if noise_rel > 0:
        s = noise_rel * np.linalg.norm(Xm) / math.sqrt(Xm.size)
        X = X + s * rng.standard_normal(n1 * n2 * n3).reshape(n1, n2, n3, order="F")
    return np.asfortranarray(X.astype(dtype, copy=False))


def smoke_case(seed=0):
    """64 x 48 x 16 float64, R = 12 CP terms with 1e-3 relative noise, DCT-II_16, k = 8."""
    rng = np.random.default_rng(seed)
    X = cp_tensor(64, 48, 16, 12, rng, noise_rel=1e-3, dtype=np.float64)
    return dict(X=X, M=dct2_matrix(16), k=8)


def _grf_slice(rng, n1, n2, amp):
    w = rng.standard_normal((n1, n2))
    f = np.fft.irfft2(np.fft.rfft2(w) * amp, s=(n1, n2))
    f -= f.mean()
    sd = f.std()
    return f / sd if sd > 0 else f


def climate(shape=(1024, 512, 365), seed=1, rho=0.95, dtype=np.float32):
    """Climate-shaped tensor: each frontal slice is a periodic Gaussian random field with
    isotropic power |k|^-3 (amplitude |k|^-1.5, k = 0 removed, unit variance); along
    mode 3, X_t = rho X_{t-1} + sqrt(1 - rho^2) xi_t with xi_t independent fields.
    Draw order: white noise for X_0, then for xi_1 .. xi_{n3-1}, each (n1, n2) row-major."""
    n1, n2, n3 = shape
    rng = np.random.default_rng(seed)
    kx = np.fft.fftfreq(n1) * n1
    ky = np.fft.rfftfreq(n2) * n2
    kk = np.sqrt(kx[:, None] ** 2 + ky[None, :] ** 2)
    amp = np.zeros_like(kk)
    amp[kk > 0] = kk[kk > 0] ** -1.5
    X = np.empty((n1, n2, n3), dtype=dtype, order="F")
    cur = _grf_slice(rng, n1, n2, amp)
    X[:, :, 0] = cur
    q = math.sqrt(1.0 - rho * rho)
    for t in range(1, n3):
        cur = rho * cur + q * _grf_slice(rng, n1, n2, amp)
        X[:, :, t] = cur
    return X


def cfd(shape=(2048, 256, 512), seed=3, waves=40, noise_rel=1e-4, dtype=np.float32):
    """CFD-shaped tensor (grid x snapshots x spanwise modes):
    X[x, t, z] = sum_w k_w^(-5/3) sin(k_w x_i - om_w t_j + phi_w) cos(pi q_w (z + 1/2) / n3)
    with x_i = 2 pi i / n1, t_j = 2 pi j / n2.
    Draw order: k_w ~ U[1, 64] (waves), om_w ~ U[0, 2pi), phi_w ~ U[0, 2pi),
    q_w ~ U{0..63}; then noise N(0,1), one (n1*n2) column-major block per z,
    scaled to noise_rel * ||X_clean||_F / sqrt(numel)."""
    n1, n2, n3 = shape
    rng = np.random.default_rng(seed)
    k = rng.uniform(1.0, 64.0, waves)
    om = rng.uniform(0.0, 2 * math.pi, waves)
    ph = rng.uniform(0.0, 2 * math.pi, waves)
    q = rng.integers(0, 64, waves)
    xi = 2 * math.pi * np.arange(n1) / n1
    tj = 2 * math.pi * np.arange(n2) / n2
    F = np.empty((n1 * n2, waves))
    for w in range(waves):
        F[:, w] = (k[w] ** (-5.0 / 3.0) *
                   np.sin(k[w] * xi[:, None] - om[w] * tj[None, :] + ph[w])).reshape(-1, order="F")
    Cz = np.cos(math.pi * q[None, :] * (np.arange(n3)[:, None] + 0.5) / n3)   # n3 x waves
    FtF = F.T @ F
    clean_sq = float(np.sum((Cz @ FtF) * Cz))          # ||X_clean||_F^2
    s = noise_rel * math.sqrt(clean_sq) / math.sqrt(n1 * n2 * n3)
    X = np.empty((n1, n2, n3), dtype=dtype, order="F")
    for z in range(n3):
        col = F @ Cz[z] + s * rng.standard_normal(n1 * n2)
        X[:, :, z] = col.reshape(n1, n2, order="F")
    return X


def crystal(shape=(512, 256, 128), lattice=(20, 10), seed=4, dtype=np.float32):
    """Crystallography-shaped tensor: each frontal slice s is a sum of isotropic Gaussian
    peaks at the sites of a shared La x Lb lattice (spacing n1/La, n2/Lb, offset half a
    spacing), widths ~ U[1, 3] px, base intensities exp(1.5 N(0,1)) (log-normal), and a
    slice-dependent drift I_{p,s} = I_p exp(0.3 sin(2 pi s / n3 + theta_p)),
    theta_p ~ U[0, 2pi).  Draw order: widths, base-intensity normals, theta (each P)."""
    n1, n2, n3 = shape
    La, Lb = lattice
    P = La * Lb
    rng = np.random.default_rng(seed)
    width = rng.uniform(1.0, 3.0, P)
    base = np.exp(1.5 * rng.standard_normal(P))
    theta = rng.uniform(0.0, 2 * math.pi, P)
    da, db = n1 / La, n2 / Lb
    xs = (np.arange(P) // Lb) * da + da / 2
    ys = (np.arange(P) % Lb) * db + db / 2
    gx = np.arange(n1, dtype=np.float64)
    gy = np.arange(n2, dtype=np.float64)
    G = np.empty((n1 * n2, P))
    for pk in range(P):
        ex = np.exp(-((gx - xs[pk]) ** 2) / (2 * width[pk] ** 2))
        ey = np.exp(-((gy - ys[pk]) ** 2) / (2 * width[pk] ** 2))
        G[:, pk] = np.outer(ex, ey).reshape(-1, order="F")
    s = np.arange(n3, dtype=np.float64)
    I = base[:, None] * np.exp(0.3 * np.sin(2 * math.pi * s[None, :] / n3 + theta[:, None]))
    X = (G @ I).reshape(n1, n2, n3, order="F")
    return np.asfortranarray(X.astype(dtype, copy=False))


def batch_shapes(count=64, seed=2):
    """Shapes of the uneven batch: n1 ~ U{128..1024}, n2 ~ U{64..512}, n3 ~ U{8..128}
    (inclusive integers), drawn in that order per tensor."""
    rng = np.random.default_rng(seed)
    out = []
    for _ in range(count):
        n1 = int(rng.integers(128, 1025))
        n2 = int(rng.integers(64, 513))
        n3 = int(rng.integers(8, 129))
        out.append((n1, n2, n3))
    return out


def batch_item(idx, shape, seed=2, dtype=np.float32):
    """Tensor ``idx`` of the uneven batch: CP tensor with R = min(n1, n2) // 4 and 1e-3
    noise, a Haar orthogonal M, t-SVDM-I (k = 16) for even idx, t-SVDM-II (eps = 1e-3)
    for odd idx.  Drawn from default_rng([seed, idx]): CP data first, then M."""
    n1, n2, n3 = shape
    rng = np.random.default_rng([seed, idx])
    X = cp_tensor(n1, n2, n3, max(1, min(n1, n2) // 4), rng, noise_rel=1e-3, dtype=dtype)
    M = haar_orthogonal(n3, rng)
    if idx % 2 == 0:
        return dict(X=X, M=M, mode="fixed", k=16)
    return dict(X=X, M=M, mode="tol", eps=1e-3)
