"""Input generators: the DCT-II matrix and Haar matrices against SciPy / orthogonality,
seeded determinism, and the documented shapes and structure of each workload."""
import numpy as np
import scipy.fft

from paper_2605_16058_gb300 import synth


def test_dct_matrix_equals_scipy_orthonormal_dct2():
    for n in (1, 2, 7, 16, 365):
        assert np.allclose(synth.dct2_matrix(n), scipy.fft.dct(np.eye(n), type=2, norm="ortho", axis=0),
                           atol=1e-13)
        M = synth.dct2_matrix(n)
        assert np.linalg.norm(M @ M.T - np.eye(n)) < 1e-12


def test_haar_orthogonal():
    rng = np.random.default_rng(0)
    Q = synth.haar_orthogonal(40, rng)
    assert np.linalg.norm(Q.T @ Q - np.eye(40)) < 1e-12


def test_generators_are_seeded_and_shaped():
    a = synth.smoke_case()["X"]
    b = synth.smoke_case()["X"]
    assert a.shape == (64, 48, 16) and a.dtype == np.float64 and np.array_equal(a, b)
    c = synth.climate(shape=(32, 16, 9))
    assert c.shape == (32, 16, 9) and c.dtype == np.float32 and c.flags.f_contiguous
    assert np.allclose(c[:, :, 0].std(), 1.0, atol=1e-5)
    d = synth.cfd(shape=(64, 16, 8))
    assert d.shape == (64, 16, 8)
    e = synth.crystal(shape=(40, 20, 6), lattice=(4, 2))
    assert e.shape == (40, 20, 6) and np.all(e >= 0)
    shapes = synth.batch_shapes()
    assert len(shapes) == 64
    assert all(128 <= s[0] <= 1024 and 64 <= s[1] <= 512 and 8 <= s[2] <= 128 for s in shapes)
    it = synth.batch_item(1, (130, 70, 9))
    assert it["mode"] == "tol" and it["X"].shape == (130, 70, 9)


def test_crystal_is_low_cp_rank():
    X = synth.crystal(shape=(40, 20, 12), lattice=(2, 2), dtype=np.float64)
    s = np.linalg.svd(X.reshape(-1, 12, order="F"), compute_uv=False)
    assert s[4] < 1e-10 * s[0]          # 4 peaks -> mode-3 unfolding has rank <= 4


def test_climate_field_has_the_documented_statistics():
    """Along mode 3 an AR(1) process with coefficient rho (lag-1 correlation rho); within
    a slice a Gaussian random field whose power falls as |k|^-3."""
    X = synth.climate(shape=(64, 64, 400), seed=3, rho=0.95, dtype=np.float64)
    lag1 = np.corrcoef(X[:, :, :-1].reshape(-1), X[:, :, 1:].reshape(-1))[0, 1]
    assert abs(lag1 - 0.95) < 0.02
    S = synth.climate(shape=(256, 256, 1), seed=5, dtype=np.float64)[:, :, 0]
    P = np.abs(np.fft.fft2(S)) ** 2
    k = np.fft.fftfreq(256) * 256
    kk = np.sqrt(k[:, None] ** 2 + k[None, :] ** 2)
    shells = np.arange(2, 60)
    radial = [P[(kk >= s) & (kk < s + 1)].mean() for s in shells]
    slope = np.polyfit(np.log(shells + 0.5), np.log(radial), 1)[0]
    assert abs(slope + 3.0) < 0.25


def test_cfd_without_noise_has_one_spanwise_mode_per_wave():
    """X[:, :, z] = sum over waves of a fixed field times cos(pi q_w (z + 1/2) / n3): the
    mode-3 unfolding has rank <= the number of waves."""
    D = synth.cfd(shape=(64, 16, 24), waves=5, noise_rel=0.0, dtype=np.float64)
    s = np.linalg.svd(D.reshape(-1, 24, order="F"), compute_uv=False)
    assert s[5] < 1e-12 * s[0]
