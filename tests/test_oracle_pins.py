"""Pins for the FP64 oracle: each test checks the oracle against something other than
itself (LAPACK through NumPy, SciPy's DCT, closed forms, hand-worked examples from
Algorithm 2, the paper's printed compression ratios, finite differences)."""
import math
import os

import numpy as np
import pytest
import scipy.fft

import oracle
from paper_2605_16058_gb300 import synth

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


def _proj_diff(U1, U2):
    return np.linalg.norm(U1 @ U1.T - U2 @ U2.T)


# ---------------------------------------------------------------- TTM (Sec. 2.1)
def test_ttm_equals_scipy_dct_along_mode3():
    rng = np.random.default_rng(10)
    X = rng.standard_normal((7, 5, 13))
    got = oracle.ttm3(X, synth.dct2_matrix(13))
    want = scipy.fft.dct(X, type=2, norm="ortho", axis=2)
    assert np.max(np.abs(got - want)) < 1e-13


def test_ttm_identity_permutation_and_rectangular():
    rng = np.random.default_rng(11)
    X = rng.standard_normal((4, 3, 6))
    assert np.array_equal(oracle.ttm3(X, np.eye(6)), X)
    perm = rng.permutation(6)
    P = np.eye(6)[perm]                       # (P x)_i = x_perm[i]
    assert np.array_equal(oracle.ttm3(X, P), X[:, :, perm])
    M = rng.standard_normal((2, 6))           # J = 2 output slices
    Y = oracle.ttm3(X, M)
    assert Y.shape == (4, 3, 2)
    assert np.allclose(Y[1, 2, 1], sum(M[1, t] * X[1, 2, t] for t in range(6)), atol=1e-14)
    sub = oracle.ttm3(X, M, which=[1])
    assert np.array_equal(sub[:, :, 0], Y[:, :, 1])


# ---------------------------------------------------------------- slice SVD (Alg. 1)
@pytest.mark.parametrize("m,p,rank", [(40, 25, None), (25, 40, None), (33, 33, None),
                                      (30, 20, 6), (1, 9, None), (9, 1, None), (17, 12, 0)])
def test_svd_matches_lapack(m, p, rank):
    rng = np.random.default_rng(m * 100 + p)
    A = rng.standard_normal((m, p))
    if rank is not None:
        A = rng.standard_normal((m, rank)) @ rng.standard_normal((rank, p)) if rank else np.zeros((m, p))
    U, S, V, sweeps = oracle.svd(A)
    assert sweeps > 0
    r = min(m, p)
    Ul, Sl, Vlt = np.linalg.svd(A, full_matrices=False)
    smax = max(Sl[0], 1e-300)
    assert np.max(np.abs(S - Sl)) <= 1e-12 * smax + 1e-300
    assert np.all(np.diff(S) <= 0)                               # descending
    recon = (U * S[None, :]) @ V.T
    assert np.linalg.norm(recon - A) <= 1e-13 * max(np.linalg.norm(A), 1e-300)
    nz = S > 1e-10 * smax
    if nz.any():
        assert np.linalg.norm(U[:, nz].T @ U[:, nz] - np.eye(nz.sum())) < 1e-13
        # subspace check against LAPACK only where the spectrum has a gap
        for k in range(1, r):
            if S[k - 1] - S[k] > 1e-6 * smax and S[k - 1] > 1e-10 * smax:
                assert _proj_diff(U[:, :k], Ul[:, :k]) < 1e-10
                assert _proj_diff(V[:, :k], Vlt[:k].T) < 1e-10
    assert np.linalg.norm(V.T @ V - np.eye(r)) < 1e-13 or not nz.all()
    # sign rule: largest-magnitude entry of each nonzero left vector is positive
    for j in np.nonzero(nz)[0]:
        a = int(np.argmax(np.abs(U[:, j])))
        assert U[a, j] > 0


def test_svd_known_closed_form():
    # [[3, 0], [4, 5]] has singular values sqrt(45) and sqrt(5)
    U, S, V, _ = oracle.svd(np.array([[3.0, 0.0], [4.0, 5.0]]))
    assert np.allclose(S, [math.sqrt(45), math.sqrt(5)], rtol=0, atol=1e-14)
    # a diagonal matrix with unsorted entries: singular values are |d| sorted
    U, S, V, _ = oracle.svd(np.diag([1.0, -7.0, 3.0]))
    assert np.array_equal(S, [7.0, 3.0, 1.0])
    assert np.allclose(np.abs(U), np.abs(np.eye(3)[:, [1, 2, 0]]))


def test_svd_sweep_cap_reports_nonconvergence():
    rng = np.random.default_rng(5)
    A = rng.standard_normal((30, 20))
    _, _, _, sw = oracle.svd(A, max_sweeps=1)
    assert sw == -1


def test_slices_equal_single_svd_per_slice():
    rng = np.random.default_rng(6)
    A = rng.standard_normal((12, 9, 5))
    U, S, V, sweeps = oracle.svd_slices(A, threads=3)
    for i in range(5):
        u, s, v, _ = oracle.svd(A[:, :, i])
        assert np.array_equal(S[:, i], s)
        assert np.array_equal(U[:, :, i], u)


# ---------------------------------------------------------------- star-M identities
def test_orthogonality_in_star_m_sense():
    """U^T *M U = I for orthonormal M reduces to Uhat_i^T Uhat_i = I per slice."""
    c = synth.smoke_case()
    full = oracle.full_tsvdm(c["X"], c["M"])
    for i in range(16):
        u, v = full["U"][:, :, i], full["V"][:, :, i]
        assert np.linalg.norm(u.T @ u - np.eye(u.shape[1])) < 1e-13
        assert np.linalg.norm(v.T @ v - np.eye(v.shape[1])) < 1e-13
    # and in the original domain: the facewise product of U^T and U mapped back is I*M
    M = c["M"]
    Ut = oracle.original_domain(full["U"], M.T)
    # (U^T * U)^ = Uhat_i^T Uhat_i = I for each slice -> the tensor identity
    hat = oracle.ttm3(Ut, M)
    assert np.allclose(hat, full["U"], atol=1e-13)


def test_full_rank_reconstruction_is_exact():
    c = synth.smoke_case()
    r = 48
    res = oracle.fixed_rank(c["X"], c["M"], r)
    Xk = oracle.reconstruct(res["U"], res["S"], res["V"], c["M"].T)
    assert oracle.rel_err_direct(c["X"], Xk) < 5e-14
    assert res["rel_err"] == 0.0


@pytest.mark.parametrize("k", [1, 4, 8, 11])
def test_eckart_young_truncation_error(k):
    c = synth.smoke_case()
    res = oracle.fixed_rank(c["X"], c["M"], k)
    Xk = oracle.reconstruct(res["U"], res["S"], res["V"], c["M"].T)
    direct = np.sum((c["X"] - Xk) ** 2)
    assert abs(direct - res["discarded"]) <= 1e-12 * np.sum(c["X"] ** 2)
    assert abs(oracle.rel_err_direct(c["X"], Xk) - res["rel_err"]) < 1e-12


def test_eckart_young_with_scaled_orthogonal_m():
    """M = c Q: singular values scale by c, the reconstruction (with M^{-1} = Q^T / c)
    is unchanged, and the error equals sqrt(sum discarded sigma^2) / c."""
    c = synth.smoke_case()
    Q = c["M"]
    scale = 2.5
    base = oracle.fixed_rank(c["X"], Q, 5)
    res = oracle.fixed_rank(c["X"], scale * Q, 5)
    assert np.allclose(res["S"], scale * base["S"], rtol=1e-13)
    Xk = oracle.reconstruct(res["U"], res["S"], res["V"], Q.T / scale)
    err2 = np.sum((c["X"] - Xk) ** 2)
    assert abs(err2 - res["discarded"] / scale ** 2) <= 1e-12 * np.sum(c["X"] ** 2)


def test_identity_m_is_slicewise_matrix_svd():
    rng = np.random.default_rng(7)
    X = rng.standard_normal((10, 8, 4))
    full = oracle.full_tsvdm(X, np.eye(4))
    for i in range(4):
        assert np.allclose(full["S"][:, i], np.linalg.svd(X[:, :, i], compute_uv=False),
                           rtol=0, atol=1e-13)


def test_n3_equal_one_is_matrix_svd():
    rng = np.random.default_rng(8)
    X = rng.standard_normal((9, 6, 1))
    full = oracle.full_tsvdm(X, np.array([[1.0]]))
    assert np.allclose(full["S"][:, 0], np.linalg.svd(X[:, :, 0], compute_uv=False), atol=1e-13)


def test_cp_rank_bound_without_noise():
    """A CP tensor with R = 12 terms has transformed slices of rank <= 12."""
    rng = np.random.default_rng(0)
    X = synth.cp_tensor(64, 48, 16, 12, rng, noise_rel=0.0)
    M = synth.dct2_matrix(16)
    full = oracle.full_tsvdm(X, M)
    smax = full["S"].max()
    assert np.all(full["S"][12:, :] < 1e-12 * smax)
    res = oracle.fixed_rank(X, M, 12)
    Xk = oracle.reconstruct(res["U"], res["S"], res["V"], M.T)
    assert oracle.rel_err_direct(X, Xk) < 1e-13


# ---------------------------------------------------------------- Algorithm 2
def _read_alg2():
    rows = []
    with open(os.path.join(GOLDEN, "alg2_worked_example.txt")) as f:
        for line in f:
            if line.startswith("#") or not line.strip():
                continue
            case, sig, eps, J, tau, ranks = [x.strip() for x in line.split("|")]
            slices = [[float(v) for v in s.split()] for s in sig.split(";")]
            rows.append((case, np.array(slices).T, float(eps), int(J), float(tau),
                         [int(v) for v in ranks.split()]))
    return rows


@pytest.mark.parametrize("row", _read_alg2(), ids=lambda r: "%s-eps%g" % (r[0], r[2]))
def test_alg2_worked_examples(row):
    case, S, eps, J, tau, ranks = row
    sel = oracle.select_ranks(S, eps)
    assert sel["J"] == J
    if J == 0:
        assert sel["tau"] == -math.inf
    else:
        assert math.isclose(sel["tau"], tau, rel_tol=1e-12)      # tau is a sigma^2 value
    assert list(sel["ranks"]) == ranks


def test_alg2_on_prescribed_spectra_end_to_end():
    """Build X whose transformed slices have chosen singular values (Haar factors), run
    the whole t-SVDM-II oracle, and compare ranks with the hand-worked example A."""
    rng = np.random.default_rng(12)
    M = synth.dct2_matrix(3)
    spectra = np.array([[10, 3, 1], [5, 2, 0.5], [4, 0.3, 0.1]], dtype=float).T
    n1, n2 = 6, 4
    Ahat = np.zeros((n1, n2, 3))
    for i in range(3):
        P = synth.haar_orthogonal(n1, rng)[:, :3]
        Q = synth.haar_orthogonal(n2, rng)[:, :3]
        Ahat[:, :, i] = (P * spectra[:, i]) @ Q.T
    X = np.einsum("abi,it->abt", Ahat, M)          # X = Ahat x_3 M^T
    for eps, want in [(0.2, [2, 1, 1]), (0.1, [2, 2, 1]), (0.05, [3, 2, 1])]:
        res = oracle.tolerance(X, M, eps)
        assert list(res["ranks"]) == want
        assert np.allclose(res["S_all"][:3], spectra, atol=1e-13)
        Xk = oracle.reconstruct(res["U"], res["S"], res["V"], M.T, offsets=res["offsets"])
        assert abs(oracle.rel_err_direct(X, Xk) - res["rel_err"]) < 1e-12
        assert res["rel_err"] < eps


def test_alg2_invariants_random_spectra():
    rng = np.random.default_rng(13)
    S = np.sort(np.exp(rng.standard_normal((20, 30)) * 2.0), axis=0)[::-1]
    prev = None
    for eps in [1e-4, 1e-3, 1e-2, 0.05, 0.1, 0.3, 0.6, 0.9]:
        sel = oracle.select_ranks(S, eps)
        total = np.sum(S ** 2)
        assert sel["discarded"] / total < eps ** 2                 # error bound holds
        kept = np.concatenate([S[: sel["ranks"][i], i] ** 2 for i in range(S.shape[1])])
        if kept.size:                                              # maximality
            assert (sel["discarded"] + kept.min()) / total >= eps ** 2
        if prev is not None:
            assert np.all(sel["ranks"] <= prev)                    # monotone in eps
        prev = sel["ranks"]
        sel2 = oracle.select_ranks(2.0 * S, eps)                   # M -> 2M
        assert np.array_equal(sel2["ranks"], sel["ranks"])


def test_alg2_degenerate_cases():
    S = np.zeros((4, 3))
    sel = oracle.select_ranks(S, 0.1)
    assert list(sel["ranks"]) == [0, 0, 0]
    rng = np.random.default_rng(14)
    X = np.zeros((5, 4, 3))
    res = oracle.tolerance(X, synth.dct2_matrix(3), 0.1)
    assert list(res["ranks"]) == [0, 0, 0] and res["rel_err"] == 0.0
    S = np.array([[1.0], [0.0]])          # exact-zero singular values are discarded first
    sel = oracle.select_ranks(S, 0.5)
    assert list(sel["ranks"]) == [1]


# ---------------------------------------------------------------- storage (Sec. 3.4, 4)
def test_compression_ratio_variable_hand_worked():
    """The variable-rank storage count of Sec. 3.4 by hand: three 3 x 2 slices (18 input
    entries) with ranks 1, 0, 2 keep three triplets of 3 + 2 (+ 1 singular value)
    entries; uniform ranks give the t-SVDM-I ratio; keeping nothing is unbounded."""
    assert oracle.compression_ratio_variable(3, 2, [1, 0, 2]) == 18 / 18
    assert oracle.compression_ratio_variable(3, 2, [1, 0, 2], with_sigma=False) == 18 / 15
    assert oracle.compression_ratio_variable(4, 5, [2, 1]) == 40 / 30      # 3 x (4 + 5 + 1)
    for m, p, n, k in [(73, 144, 5, 1), (253, 253, 3, 20), (300, 400, 2, 150)]:
        v = oracle.compression_ratio_variable(m, p, [k] * n)
        assert abs(v - oracle.compression_ratio_fixed(m, p, n, k)) <= 1e-12 * v
    assert oracle.compression_ratio_variable(3, 2, [0, 0]) == float("inf")


def test_compression_ratios_match_paper():
    with open(os.path.join(GOLDEN, "compression_ratios.txt")) as f:
        for line in f:
            if line.startswith("#") or not line.strip():
                continue
            name, m, p, k, ratio, digits = [x.strip() for x in line.split("|")]
            cr = oracle.compression_ratio_fixed(int(m), int(p), 1, int(k))
            assert round(cr, int(digits)) == float(ratio), name


# ---------------------------------------------------------------- gradient and Cayley
def _fd_instance():
    X = synth.crystal(shape=(32, 24, 8), lattice=(3, 2), seed=4, dtype=np.float64)
    return X


def test_gradient_wrt_x_matches_central_differences():
    X = _fd_instance()
    M = synth.dct2_matrix(8)
    k = 2
    g = oracle.loss_and_grad(X, M, k)
    S = g["fr"]["S_all"]
    assert np.all(S[k - 1] - S[k] > 1e-6 * S[0])                  # a gap at k
    rng = np.random.default_rng(15)
    h = 1e-3
    for _ in range(4):
        D = rng.standard_normal(X.shape)
        D /= np.linalg.norm(D)                                     # unit direction, step h
        lp = oracle.loss_and_grad(X + h * D, M, k)["loss"]
        lm = oracle.loss_and_grad(X - h * D, M, k)["loss"]
        fd = (lp - lm) / (2 * h)
        an = float(np.sum(g["dX"] * D))
        assert abs(fd - an) <= 1e-3 * max(abs(an), 1e-3 * g["loss"])


def test_gradient_wrt_m_matches_central_differences():
    X = _fd_instance()
    M = synth.dct2_matrix(8)
    k = 2
    g = oracle.loss_and_grad(X, M, k)
    rng = np.random.default_rng(16)
    h = 1e-3
    for _ in range(4):
        D = rng.standard_normal(M.shape)
        D /= np.linalg.norm(D)
        lp = oracle.loss_and_grad(X, M + h * D, k)["loss"]
        lm = oracle.loss_and_grad(X, M - h * D, k)["loss"]
        fd = (lp - lm) / (2 * h)
        an = float(np.sum(g["dM"] * D))
        assert abs(fd - an) <= 1e-3 * max(abs(an), 1e-3 * g["loss"])


def test_gradient_matches_dense_svd_autograd():
    torch = pytest.importorskip("torch")
    X = _fd_instance()
    M = synth.dct2_matrix(8)
    k = 2
    g = oracle.loss_and_grad(X, M, k)
    Xt = torch.tensor(X, dtype=torch.float64, requires_grad=True)
    Mt = torch.tensor(M, dtype=torch.float64, requires_grad=True)
    Ahat = torch.einsum("abt,it->abi", Xt, Mt)
    s = torch.linalg.svdvals(Ahat.permute(2, 0, 1))               # (n, r)
    E = torch.sum(s[:, k:] ** 2)
    L = torch.sqrt(E) / torch.linalg.norm(Xt)
    L.backward()
    assert abs(L.item() - g["loss"]) < 1e-12
    assert np.allclose(Xt.grad.numpy(), g["dX"], rtol=1e-8, atol=1e-10)
    assert np.allclose(Mt.grad.numpy(), g["dM"], rtol=1e-8, atol=1e-10)


def test_cayley_is_orthogonal_and_starts_at_m0():
    n = 6
    M0 = synth.dct2_matrix(n)
    Mz, _, _ = oracle.cayley(np.zeros((n, n)), M0)
    assert np.array_equal(Mz, M0)
    rng = np.random.default_rng(17)
    A = 0.3 * rng.standard_normal((n, n))
    M, Q, W = oracle.cayley(A, M0)
    assert np.allclose(W, -W.T)
    assert np.linalg.norm(M.T @ M - np.eye(n)) < 1e-13
    # closed form for n = 2: W = [[0, -w], [w, 0]] gives the rotation by angle 2 atan(w)
    w = 0.4
    A2 = np.array([[0.0, w], [0.0, 0.0]])          # W = A^T - A = [[0, -w], [w, 0]]
    M2, _, _ = oracle.cayley(A2, np.eye(2))
    th = 2 * math.atan(w)
    assert np.allclose(M2, [[math.cos(th), math.sin(th)], [-math.sin(th), math.cos(th)]], atol=1e-14)


def test_cayley_gradient_matches_central_differences():
    n = 8
    X = _fd_instance()
    M0 = synth.dct2_matrix(n)
    rng = np.random.default_rng(18)
    A = 0.05 * rng.standard_normal((n, n))
    k = 2

    def loss(Ap):
        return oracle.loss_and_grad(X, oracle.cayley(Ap, M0)[0], k)["loss"]

    M, _, _ = oracle.cayley(A, M0)
    dM = oracle.loss_and_grad(X, M, k)["dM"]
    dA = oracle.cayley_grad(A, M0, dM)
    h = 1e-3
    for _ in range(3):
        D = rng.standard_normal((n, n))
        D /= np.linalg.norm(D)
        fd = (loss(A + h * D) - loss(A - h * D)) / (2 * h)
        an = float(np.sum(dA * D))
        assert abs(fd - an) <= 1e-3 * max(abs(an), 1e-3)


def test_adam_step_first_update_is_lr_times_sign():
    p = np.array([1.0, -2.0, 0.5])
    g = np.array([0.3, -4.0, 0.0])
    m1 = np.zeros(3)
    m2 = np.zeros(3)
    oracle.adam_step(p, g, m1, m2, 1, lr=1e-3)
    # first step: mhat = g, vhat = g^2, update = lr * g / (|g| + eps)
    assert np.allclose(p, [1.0 - 1e-3, -2.0 + 1e-3, 0.5], atol=1e-10)


def test_rel_err_is_scale_free_for_multiples_of_orthogonal_m():
    c = synth.smoke_case()
    a = oracle.fixed_rank(c["X"], c["M"], 6)
    b = oracle.fixed_rank(c["X"], 3.0 * c["M"], 6)
    assert abs(a["rel_err"] - b["rel_err"]) < 1e-13
    Xk = oracle.reconstruct(b["U"], b["S"], b["V"], c["M"].T / 3.0)
    assert abs(oracle.rel_err_direct(c["X"], Xk) - b["rel_err"]) < 1e-12


# ---------------------------------------------------------------- d-way tensors
def _dway_case(dims, seed):
    rng = np.random.default_rng(seed)
    X = rng.standard_normal(dims)
    Ms = [synth.haar_orthogonal(n, rng) for n in dims[2:]]
    return X, Ms


def test_dway_transform_equals_kronecker_mode3():
    """Modes 3 and 4 (and 5) transformed one after the other equal one mode-3 product of
    the flattened trailing modes with the Kronecker product M_5 (x) M_4 (x) M_3 (column-major
    flattening puts i3 fastest): a different computation of the same operator."""
    for dims in [(5, 4, 3, 2), (4, 3, 2, 3, 2)]:
        X, Ms = _dway_case(dims, 11)
        K = Ms[0]
        for M in Ms[1:]:
            K = np.kron(M, K)
        got = oracle.to_slices(oracle.dway_transform(X, Ms))
        want = np.einsum("it,abt->abi", K, oracle.to_slices(X))
        assert np.max(np.abs(got - want)) <= 1e-13 * np.max(np.abs(want))


def test_dway_mode_product_against_einsum():
    X, Ms = _dway_case((4, 3, 5, 2), 12)
    got = oracle.ttm_mode(X, Ms[0], 2)
    want = np.einsum("it,abtq->abiq", Ms[0], X)
    assert np.max(np.abs(got - want)) <= 1e-13 * np.max(np.abs(want))
    got = oracle.ttm_mode(X, Ms[1], 3)
    want = np.einsum("iq,abtq->abti", Ms[1], X)
    assert np.max(np.abs(got - want)) <= 1e-13 * np.max(np.abs(want))


def test_dway_with_trivial_last_mode_is_the_3way_decomposition():
    X, Ms = _dway_case((12, 9, 5), 13)
    X4 = X[:, :, :, None]
    a = oracle.fixed_rank(X4, [Ms[0], np.ones((1, 1))], 4)
    b = oracle.fixed_rank(X, Ms[0], 4)
    assert np.max(np.abs(a["S"] - b["S"])) <= 1e-12 * b["S"].max()
    assert abs(a["rel_err"] - b["rel_err"]) <= 1e-12


def test_dway_eckart_young_and_reconstruction():
    """Orthogonal M_k: the d-way transform is orthogonal, so the reported relative error
    (discarded sigma^2) equals the direct reconstruction error, for t-SVDM-I and II."""
    X, Ms = _dway_case((10, 8, 3, 4), 14)
    Minv = [M.T for M in Ms]
    f = oracle.fixed_rank(X, Ms, 3)
    Xk = oracle.reconstruct(f["U"], f["S"], f["V"], Minv)
    assert Xk.shape == X.shape
    assert abs(oracle.rel_err_direct(X, Xk) - f["rel_err"]) <= 1e-12
    t = oracle.tolerance(X, Ms, 0.3)
    Xt = oracle.reconstruct(t["U"], t["S"], t["V"], Minv, offsets=t["offsets"])
    assert abs(oracle.rel_err_direct(X, Xt) - t["rel_err"]) <= 1e-12
    assert t["rel_err"] < 0.3
    # full rank reproduces X
    r = min(X.shape[:2])
    g = oracle.fixed_rank(X, Ms, r)
    Xr = oracle.reconstruct(g["U"], g["S"], g["V"], Minv)
    assert oracle.rel_err_direct(X, Xr) <= 1e-12


def test_dway_original_domain_factors_rebuild_x():
    """Original-domain factors (each mapped back by the per-mode inverses) rebuild X_k with
    the d-way star-M product, i.e. the transform of their facewise product."""
    X, Ms = _dway_case((7, 6, 2, 3), 15)
    Minv = [M.T for M in Ms]
    f = oracle.fixed_rank(X, Ms, 6)
    Xk = oracle.reconstruct(f["U"], f["S"], f["V"], Minv)
    U = oracle.original_domain(f["U"], Minv)
    # U x_3 M_3 x_4 M_4 returns the hat-domain factor
    back = oracle.to_slices(oracle.dway_transform(U.reshape((7, 6, 2, 3), order="F"), Ms))
    assert np.max(np.abs(back - f["U"])) <= 1e-13
    assert oracle.rel_err_direct(X, Xk) <= 1e-12


# ---------------------------------------------------------------- data-driven M
def test_data_transform_diagonalises_the_mode3_gram():
    """M's rows are the left singular vectors of A_(3): M is orthogonal and
    M A_(3) A_(3)^T M^T = diag(sigma^2), decreasing (with M^T in place of M the product is
    not diagonal, so a transposition fails here); the transformed slices carry the
    energies sigma_i^2."""
    rng = np.random.default_rng(41)
    X = synth.cp_tensor(20, 15, 9, 6, rng, noise_rel=0.3)
    M, sig = oracle.data_transform(X)
    assert np.max(np.abs(M @ M.T - np.eye(9))) <= 1e-12
    A3 = X.reshape(-1, 9, order="F").T
    D = M @ (A3 @ A3.T) @ M.T
    assert np.max(np.abs(D - np.diag(np.diag(D)))) <= 1e-10 * np.max(np.abs(D))
    assert np.allclose(np.diag(D), sig ** 2, rtol=1e-10)
    assert np.all(np.diff(np.diag(D)) <= 0)
    Ahat = oracle.ttm3(X, M)
    energies = np.array([np.sum(Ahat[:, :, i] ** 2) for i in range(9)])
    assert np.allclose(energies, sig ** 2, rtol=1e-10)
    for j in range(9):                              # sign rule
        assert M[j, np.argmax(np.abs(M[j]))] > 0
