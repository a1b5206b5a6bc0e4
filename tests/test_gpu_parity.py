"""CUDA path (through the C ABI) against the FP64 oracle, element by element, on seeded
inputs that span several tiles with ragged tails.

Tolerances (stated per precision):
  singular values   |s_gpu - s_oracle| <= 1e-5 sigma_max (FP32), 1e-12 sigma_max (FP64)
  subspaces         ||U_k U_k^T - U~_k U~_k^T||_F <= 1e-4 where the gap at k exceeds
                    g(p) sigma_max (FP32) / 1e-6 sigma_max (FP64) (no sign ambiguity): FP32
                    rotations leave the columns errors of about c u sigma_max, so the
                    projector carries c u sigma_max / gap, with c growing like sqrt(p) (p
                    columns; measured c = 7 at p = 500, a 1.03e-4 projector at a gap of
                    4e-3 sigma_max); g(p) = 4e-4 sqrt(p) keeps that model at half the bar
  relative error    |rel_gpu - rel_oracle| <= 1e-5 (FP32), 1e-12 (FP64)
  t-SVDM-II ranks   exact, except slices holding a sigma^2 within 1e-6 relative of tau
  TTM               max |Y - Y_oracle| <= 2e-6 max|Y| (FP32), 1e-13 max|Y| (FP64)
"""
import numpy as np
import pytest

import oracle
from paper_2605_16058_gb300 import synth

from helpers import np_lib, proj_diff, t_lib

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")


def _need_gpu():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")


@pytest.fixture(scope="module", autouse=True)
def _lib():
    _need_gpu()
    from paper_2605_16058_gb300 import build
    build.build()


def _plan(n1, n2, n3, dt, orthogonal=True):
    from paper_2605_16058_gb300.tsvdm import Plan
    return Plan(n1, n2, n3, dtype=dt, orthogonal=orthogonal)


TOL = {torch.float32: dict(sig=1e-5, proj=1e-4, gap=4e-4, rel=1e-5, ttm=2e-6),
       torch.float64: dict(sig=1e-12, proj=1e-9, gap=1e-6, rel=1e-12, ttm=1e-13)}


def _rand(shape, seed, dtype=np.float64):
    return np.random.default_rng(seed).standard_normal(shape).astype(dtype)


# ---------------------------------------------------------------- TTM
@pytest.mark.parametrize("dt", [torch.float32, torch.float64])
@pytest.mark.parametrize("shape", [(37, 29, 19), (130, 3, 70), (1, 1, 1), (5, 7, 129)])
def test_ttm_forward_and_inverse(dt, shape):
    n1, n2, n3 = shape
    X = _rand(shape, 1)
    M = synth.haar_orthogonal(n3, np.random.default_rng(2)) * 1.5
    plan = _plan(n1, n2, n3, dt)
    Xd, Md = t_lib(X, dtype=dt), t_lib(M, dtype=dt)
    Y = plan.transform(Xd, Md)
    want = oracle.ttm3(X.astype(np.float32) if dt == torch.float32 else X,
                       M.astype(np.float32) if dt == torch.float32 else M)
    got = np_lib(Y)
    assert np.max(np.abs(got - want)) <= TOL[dt]["ttm"] * max(np.max(np.abs(want)), 1e-30) * (n3 ** 0.5)
    Xb = np_lib(plan.transform(Y, Md, inverse=True))     # M^{-1} = M^T / c^2
    assert np.max(np.abs(Xb - X)) <= 50 * TOL[dt]["ttm"] * np.max(np.abs(X)) * n3 ** 0.5


# ---------------------------------------------------------------- t-SVDM-I
CASES_I = [
    ("smoke", None, torch.float64, 8),
    ("tall", (100, 37, 5), torch.float32, 6),
    ("wide", (37, 100, 5), torch.float32, 6),
    ("tiles", (200, 130, 3), torch.float32, 20),
    ("tall64", (150, 70, 4), torch.float64, 10),
    ("one_slice", (33, 20, 1), torch.float32, 20),
    ("rankdef", (80, 40, 3), torch.float32, 4),
    # 16 column blocks (a ragged last one): 14 of the 15 rounds of a sweep are cross sweeps
    ("blocks16", (520, 500, 2), torch.float32, 40),
    # 60 columns exactly zero in every slice: pairs that never rotate, rank 80
    ("zerocols", (150, 140, 2), torch.float32, 12),
]


def _case_input(name, shape, seed=3):
    if name == "smoke":
        c = synth.smoke_case()
        return c["X"], c["M"]
    n1, n2, n3 = shape
    rng = np.random.default_rng(seed)
    if name == "rankdef":
        X = synth.cp_tensor(n1, n2, n3, 5, rng, noise_rel=0.0)
    else:
        X = synth.cp_tensor(n1, n2, n3, min(n1, n2) // 2, rng, noise_rel=1e-2)
    if name == "zerocols":
        X[:, 40:100, :] = 0.0
    return X, synth.dct2_matrix(n3)


def _gap(dt, p):
    """Relative gap above which subspaces are compared (see the module docstring)."""
    return TOL[dt]["gap"] * (np.sqrt(p) if dt == torch.float32 else 1.0)


def _compare_factors(dt, S_o, U_o, V_o, S_g, U_g, V_g, k):
    tol = TOL[dt]
    n3 = S_o.shape[1]
    gap = _gap(dt, S_o.shape[0])
    for i in range(n3):
        so, sg = S_o[:, i], S_g[:, i]
        smax = max(so[0], 1e-300)
        assert np.max(np.abs(so[:k] - sg[:k])) <= tol["sig"] * smax, (i, so[:k], sg[:k])
        for kk in range(1, k + 1):
            gap_next = so[kk - 1] - (so[kk] if kk < len(so) else 0.0)
            if gap_next > gap * smax and so[kk - 1] > gap * smax:
                assert proj_diff(U_o[:, :kk, i], U_g[:, :kk, i]) <= tol["proj"], (i, kk)
                assert proj_diff(V_o[:, :kk, i], V_g[:, :kk, i]) <= tol["proj"], (i, kk)


def _fixed_rank_case(name, shape, dt, k, engine=None, angles=None, vectors=None):
    X, M = _case_input(name, shape)
    n1, n2, n3 = X.shape
    if dt == torch.float32:
        X = X.astype(np.float32).astype(np.float64)
        M = M.astype(np.float32).astype(np.float64)
    ref = oracle.fixed_rank(X, M, k)
    plan = _plan(n1, n2, n3, dt)
    if engine is not None:
        plan.set_engine(engine)
    if angles is not None:
        plan.set_angle_precision(angles)
    if vectors is not None:
        plan.set_vectors(vectors)
    out = plan.fixed_rank(t_lib(X, dtype=dt), t_lib(M, dtype=dt), k)
    U_g, S_g, V_g = np_lib(out["U"]), np_lib(out["S"]), np_lib(out["V"])
    assert U_g.shape == (n1, k, n3) and S_g.shape == (k, n3) and V_g.shape == (n2, k, n3)
    full = oracle.svd_slices(ref["Ahat"])
    _compare_factors(dt, ref["S_all"], full[0], full[2], S_g, U_g, V_g, k)
    assert abs(out["rel_err"] - ref["rel_err"]) <= TOL[dt]["rel"]
    # left vectors orthonormal per slice
    for i in range(n3):
        nz = S_g[:, i] > 1e-6 * max(S_g[0, i], 1e-300)
        u = U_g[:, nz, i]
        assert np.linalg.norm(u.T @ u - np.eye(u.shape[1])) < (1e-4 if dt == torch.float32 else 1e-10)


@pytest.mark.parametrize("name,shape,dt,k", CASES_I, ids=[c[0] for c in CASES_I])
def test_fixed_rank_matches_oracle(name, shape, dt, k):
    _fixed_rank_case(name, shape, dt, k)


# Both engines of the Jacobi products on every FP32 case: "tc" forced also on slices
# narrower than a 64-column block pair (padding columns) and on row counts that are not a
# multiple of 4 (the unvectorised load path), "fma" on slices the automatic choice sends
# to the tensor cores; each with the rotation test and angle in FP64 (the default) and in
# FP32 (the opt-in setting).
CASES_ENGINE = [c for c in CASES_I if c[2] == torch.float32]


@pytest.mark.parametrize("angles", ["fp64", "fp32"])
@pytest.mark.parametrize("engine", ["tc", "fma"])
@pytest.mark.parametrize("name,shape,dt,k", CASES_ENGINE, ids=[c[0] for c in CASES_ENGINE])
def test_fixed_rank_each_engine(name, shape, dt, k, engine, angles):
    _fixed_rank_case(name, shape, dt, k, engine, angles)


# Two passes (singular values first, then the kept triplets' other side from the slices):
# every t-SVDM-I case, FP32 and FP64, tall and wide (both sides of the second pass).
@pytest.mark.parametrize("name,shape,dt,k", CASES_I, ids=[c[0] for c in CASES_I])
def test_fixed_rank_second_pass(name, shape, dt, k):
    _fixed_rank_case(name, shape, dt, k, vectors="second_pass")


# The second pass's product Z = A^T U_k on both engines for FP32 slices: the tensor cores
# (tall slices, K-major 16-byte loads, N = the kept count in multiples of 16) and the
# CUDA-core tiled product (the FMA engine, and every wide slice).
@pytest.mark.parametrize("engine", ["tc", "fma"])
@pytest.mark.parametrize("name,shape,dt,k", CASES_ENGINE, ids=[c[0] for c in CASES_ENGINE])
def test_fixed_rank_second_pass_each_engine(name, shape, dt, k, engine):
    _fixed_rank_case(name, shape, dt, k, engine, vectors="second_pass")


def test_engine_argument_errors():
    from paper_2605_16058_gb300 import native as N
    p64 = _plan(8, 8, 2, torch.float64)
    with pytest.raises(N.TsvdmError) as e:
        p64.set_engine("tc")
    assert e.value.status == N.ENOTSUP
    p32 = _plan(8, 8, 2, torch.float32)
    with pytest.raises(N.TsvdmError) as e:
        N.tsvdm_plan_set_engine(p32.handle, 7)
    assert e.value.status == N.EINVAL


@pytest.mark.parametrize("dt", [torch.float32, torch.float64])
def test_reconstruct_matches_oracle(dt):
    X, M = _case_input("tall", (100, 37, 5))
    n1, n2, n3 = X.shape
    k = 7
    plan = _plan(n1, n2, n3, dt)
    Md = t_lib(M, dtype=dt)
    out = plan.fixed_rank(t_lib(X, dtype=dt), Md, k)
    Xk = np_lib(plan.reconstruct(out["U"], out["S"], out["V"], Md, k=k))
    U, S, V = np_lib(out["U"]), np_lib(out["S"]), np_lib(out["V"])
    want = oracle.reconstruct(U, S, V, M.T)
    assert np.max(np.abs(Xk - want)) <= 1e-5 * np.max(np.abs(want)) * (1 if dt == torch.float32 else 1e-7)
    # Eckart-Young: the direct error equals the reported one
    direct = oracle.rel_err_direct(X, Xk)
    assert abs(direct - out["rel_err"]) <= (2e-5 if dt == torch.float32 else 1e-11)


@pytest.mark.parametrize("engine", ["tc", "fma"])
@pytest.mark.parametrize("flat", [False, True])
def test_reconstruct_packed_each_engine(engine, flat):
    """Back-transform of packed t-SVDM-II factors (ranks vary per slice) over several
    128 x 256 output tiles with ragged edges, both engines of the slice products, against
    the oracle's reconstruction of the same factors.  flat: X nearly constant along mode 3,
    so the DCT leaves almost all energy in slice 0 and the other slices get rank 0."""
    rng = np.random.default_rng(17)
    n1, n2, n3 = 300, 270, 4
    if flat:
        A = synth.cp_tensor(n1, n2, 1, 40, rng, noise_rel=1e-2)[:, :, 0]
        X = A[:, :, None] * np.ones(n3) + 1e-6 * rng.standard_normal((n1, n2, n3))
    else:
        X = synth.cp_tensor(n1, n2, n3, 40, rng, noise_rel=1e-2)
    X = X.astype(np.float32).astype(np.float64)
    M = synth.dct2_matrix(n3).astype(np.float32).astype(np.float64)
    plan = _plan(n1, n2, n3, torch.float32)
    plan.set_engine(engine)
    Md = t_lib(M, dtype=torch.float32)
    out = plan.tolerance(t_lib(X, dtype=torch.float32), Md, 0.05)
    ranks = out["ranks"].cpu().numpy()
    if flat:
        assert ranks[0] > 0 and (ranks[1:] == 0).all()
    offs = out["offsets"]
    Xk = np_lib(plan.reconstruct(out["U"], out["S"], out["V"], Md, offsets=offs))
    want = oracle.reconstruct(np_lib(out["U"]), np_lib(out["S"]), np_lib(out["V"]), M.T,
                              offsets=offs.cpu().numpy())
    assert np.max(np.abs(Xk - want)) <= 1e-5 * np.max(np.abs(want))
    assert abs(oracle.rel_err_direct(X, Xk) - out["rel_err"]) <= 2e-5


def test_original_domain_factors():
    X, M = _case_input("tall", (60, 30, 6))
    n1, n2, n3 = X.shape
    k = 5
    plan = _plan(n1, n2, n3, torch.float64)
    Md = t_lib(M, dtype=torch.float64)
    hat = plan.fixed_rank(t_lib(X, dtype=torch.float64), Md, k)
    org = plan.fixed_rank(t_lib(X, dtype=torch.float64), Md, k, original_domain=True)
    for key in ("U", "S", "V"):
        assert np.allclose(oracle.original_domain(np_lib(hat[key]), M.T), np_lib(org[key]), atol=1e-12)


# ---------------------------------------------------------------- t-SVDM-II
def _tie_slices(S, tau, rel=1e-6):
    if not np.isfinite(tau) or tau <= 0:
        return set()
    near = np.abs(S * S - tau) <= rel * tau
    return set(np.nonzero(near.any(axis=0))[0])


@pytest.mark.parametrize("angles", ["fp64", "fp32"])
@pytest.mark.parametrize("dt,shape,eps", [(torch.float64, (64, 48, 16), 0.05),
                                          (torch.float32, (90, 60, 12), 0.02),
                                          (torch.float32, (40, 70, 9), 0.1),
                                          (torch.float32, (300, 200, 20), 0.03),
                                          (torch.float64, (50, 30, 7), 1e-9)])
@pytest.mark.parametrize("vectors", ["accumulate", "second_pass"])
def test_tolerance_matches_oracle(dt, shape, eps, angles, vectors):
    """t-SVDM-II at the stated tolerances: ranks exact (ties aside), the relative error
    within 1e-5 (FP32) / 1e-12 (FP64) of the oracle's, packed singular values within
    1e-5 / 1e-12 of the slice's largest, packed subspaces by projector."""
    n1, n2, n3 = shape
    rng = np.random.default_rng(7)
    X = synth.cp_tensor(n1, n2, n3, min(n1, n2) // 3, rng, noise_rel=1e-2)
    M = synth.dct2_matrix(n3)
    if dt == torch.float32:
        X = X.astype(np.float32).astype(np.float64)
        M = M.astype(np.float32).astype(np.float64)
    ref = oracle.tolerance(X, M, eps)
    plan = _plan(n1, n2, n3, dt)
    plan.set_angle_precision(angles)
    plan.set_vectors(vectors)
    out = plan.tolerance(t_lib(X, dtype=dt), t_lib(M, dtype=dt), eps)
    ranks = out["ranks"].cpu().numpy()
    off = out["offsets"].cpu().numpy()
    assert off[0] == 0 and np.array_equal(np.diff(off), ranks) and off[-1] == out["total_rank"]
    ties = _tie_slices(ref["S_all"], ref["tau"])
    for i in range(n3):
        if i not in ties:
            assert ranks[i] == ref["ranks"][i], (i, ranks[i], ref["ranks"][i])
    assert abs(out["rel_err"] - ref["rel_err"]) <= TOL[dt]["rel"]
    assert out["rel_err"] < eps or out["total_rank"] == n3 * min(n1, n2)
    # packed factors: slice i's columns hold its leading rho_i triplets
    U = out["U"].cpu().double().numpy().T
    S = out["S"].cpu().double().numpy()
    V = out["V"].cpu().double().numpy().T
    full = oracle.svd_slices(ref["Ahat"])
    for i in range(n3):
        a, b = off[i], off[i + 1]
        if b == a:
            continue
        smax = ref["S_all"][0, i]
        assert np.max(np.abs(S[a:b] - ref["S_all"][: b - a, i])) <= TOL[dt]["sig"] * max(smax, 1e-300)
        kk = b - a
        so = ref["S_all"][:, i]
        if so[kk - 1] - (so[kk] if kk < len(so) else 0.0) > _gap(dt, min(n1, n2)) * smax:
            assert proj_diff(full[0][:, :kk, i], U[:, a:b]) <= TOL[dt]["proj"]
            assert proj_diff(full[2][:, :kk, i], V[:, a:b]) <= TOL[dt]["proj"]


def test_tolerance_ranks_equal_algorithm2_on_gpu_sigma():
    """Integer decision taken in FP64 on both sides: Algorithm 2 of the oracle applied to
    the GPU's own singular values reproduces the GPU's ranks exactly."""
    n1, n2, n3 = 120, 80, 24
    X = synth.climate(shape=(n1, n2, n3), seed=5)
    M = synth.dct2_matrix(n3)
    plan = _plan(n1, n2, n3, torch.float32)
    for eps in (1e-3, 1e-2, 5e-2, 0.2):
        out = plan.tolerance(t_lib(X), t_lib(M, dtype=torch.float32), eps)
        f = plan.fixed_rank(t_lib(X), t_lib(M, dtype=torch.float32), min(n1, n2), rel_err=False)
        S_gpu = np_lib(f["S"])
        sel = oracle.select_ranks(S_gpu, eps)
        assert np.array_equal(out["ranks"].cpu().numpy(), sel["ranks"])


# ---------------------------------------------------------------- status paths
def test_sweep_cap_reports_nonconvergence():
    from paper_2605_16058_gb300 import native
    X = _rand((64, 40, 3), 9, np.float32)
    plan = _plan(64, 40, 3, torch.float32)
    plan.set_jacobi(0.0, 1)
    out = plan.fixed_rank(t_lib(X), t_lib(np.eye(3), dtype=torch.float32), 4, raise_on_error=False)
    assert out["status"] == native.ENOCONV
    plan.set_jacobi(0.0, 0)
    out = plan.fixed_rank(t_lib(X), t_lib(np.eye(3), dtype=torch.float32), 4)
    assert out["status"] == native.OK


def test_angle_precision_and_wait_limit_argument_errors():
    from paper_2605_16058_gb300 import native as N
    p = _plan(8, 8, 2, torch.float32)
    with pytest.raises(N.TsvdmError) as e:
        N.tsvdm_plan_set_vectors(p.handle, 5)
    assert e.value.status == N.EINVAL
    with pytest.raises(N.TsvdmError) as e:
        N.tsvdm_plan_set_angle_precision(p.handle, 2)
    assert e.value.status == N.EINVAL
    with pytest.raises(N.TsvdmError) as e:
        p.set_wait_limit(-1)
    assert e.value.status == N.EINVAL
    with pytest.raises(N.TsvdmError) as e:
        p.set_wait_limit(1 << 32)
    assert e.value.status == N.EINVAL


def test_bounded_wait_runs_out_and_plan_recovers():
    """A tensor-core Jacobi whose scheduler waits are limited to one poll: one slice of
    64 columns gives one block pair per sweep, so the other workers of the GPU find no
    work and their idle wait runs out.  The kernel stops every worker and returns by
    itself; the call reports TSVDM_ETIMEOUT.  With the default bound restored the same
    plan, and a fresh plan, give the oracle's result."""
    from paper_2605_16058_gb300 import native
    rng = np.random.default_rng(11)
    X = synth.cp_tensor(1024, 64, 1, 20, rng, noise_rel=1e-2).astype(np.float32).astype(np.float64)
    M = np.ones((1, 1))
    Xd, Md = t_lib(X, dtype=torch.float32), t_lib(M, dtype=torch.float32)
    plan = _plan(1024, 64, 1, torch.float32)
    plan.set_engine("tc")
    plan.set_wait_limit(1)
    out = plan.fixed_rank(Xd, Md, 8, raise_on_error=False)
    assert out["status"] == native.ETIMEOUT
    assert plan.last_status() == native.OK           # the status word was read and cleared
    ref = oracle.fixed_rank(X, M, 8)
    plan.set_wait_limit(0)
    for p in (plan, _plan(1024, 64, 1, torch.float32)):
        p.set_engine("tc")
        got = p.fixed_rank(Xd, Md, 8)
        assert got["status"] == native.OK
        S = np_lib(got["S"])
        assert np.max(np.abs(S - ref["S"])) <= 1e-5 * ref["S"].max()


def test_nonfinite_input_is_reported():
    from paper_2605_16058_gb300 import native
    X = _rand((32, 20, 2), 10, np.float32)
    X[3, 4, 1] = np.nan
    plan = _plan(32, 20, 2, torch.float32)
    out = plan.fixed_rank(t_lib(X), t_lib(np.eye(2), dtype=torch.float32), 3, raise_on_error=False)
    assert out["status"] == native.ENONFINITE


def test_host_buffers_match_device_buffers():
    from paper_2605_16058_gb300 import native
    X, M = _case_input("tall", (70, 50, 6))
    Xf = X.astype(np.float32)
    plan = _plan(70, 50, 6, torch.float32)
    dev = plan.fixed_rank(t_lib(Xf), t_lib(M, dtype=torch.float32), 5)
    Xh = t_lib(Xf, device="cpu").pin_memory()
    Mh = t_lib(M, device="cpu", dtype=torch.float32)
    U = torch.empty(6, 5, 70).pin_memory()
    S = torch.empty(6, 5)
    V = torch.empty(6, 5, 50)
    err, st = native.tsvdm_fixed_rank(plan.handle, Xh, Mh, 5, U, S, V, 0, True)
    assert st == native.OK
    assert torch.equal(S, dev["S"].cpu()) and torch.equal(U, dev["U"].cpu())
    assert err == dev["rel_err"]


def test_zero_tensor_tolerance_keeps_nothing():
    plan = _plan(20, 10, 4, torch.float32)
    out = plan.tolerance(torch.zeros(4 * 10 * 20, device="cuda"), t_lib(synth.dct2_matrix(4), dtype=torch.float32), 0.1)
    assert out["total_rank"] == 0 and out["rel_err"] == 0.0


def test_argument_errors():
    from paper_2605_16058_gb300 import native
    plan = _plan(20, 10, 4, torch.float32, orthogonal=False)
    X = torch.zeros(800, device="cuda")
    M = torch.eye(4, device="cuda")
    with pytest.raises(native.TsvdmError) as e:
        plan.tolerance(X, M, 0.1)
    assert e.value.status == native.ENOTORTHO
    with pytest.raises(native.TsvdmError) as e:
        plan.fixed_rank(X, M, 11)
    assert e.value.status == native.EINVAL


# ---------------------------------------------------------------- data-driven M
@pytest.mark.parametrize("dt,shape,engine", [(torch.float64, (60, 40, 12), None),
                                             (torch.float32, (200, 130, 24), None),
                                             (torch.float32, (200, 130, 24), "fma"),
                                             (torch.float32, (36, 20, 200), None)])
def test_data_transform_matches_oracle(dt, shape, engine):
    """M from the library's Jacobi SVD of the mode-3 Gram against LAPACK's SVD of the
    unfolding: orthogonal, diagonalising the mode-3 Gram, the same rows (sign rule) where
    the singular values are well separated, and the same t-SVDM-I error.  FP32 Grams run on
    the tensor cores (n3 = 200: two bands of 128 rows, 256 padded columns) or, with the FMA
    engine, on the CUDA cores."""
    rng = np.random.default_rng(43)
    n1, n2, n3 = shape
    X = synth.cp_tensor(n1, n2, n3, 8, rng, noise_rel=0.2)
    if dt == torch.float32:
        X = X.astype(np.float32).astype(np.float64)
    Mo, sig = oracle.data_transform(X)
    plan = _plan(n1, n2, n3, dt)
    if engine is not None:
        plan.set_engine(engine)     # the mode-3 Gram on the CUDA cores
    Xd = t_lib(X, dtype=dt)
    Mg = np_lib(plan.data_transform(Xd))
    tol = 1e-10 if dt == torch.float64 else 2e-5
    assert np.max(np.abs(Mg @ Mg.T - np.eye(n3))) <= tol
    A3 = X.reshape(-1, n3, order="F").T
    G = A3 @ A3.T
    D = Mg @ G @ Mg.T
    assert np.max(np.abs(D - np.diag(np.diag(D)))) <= 10 * tol * np.max(np.abs(G))
    s2 = sig ** 2
    for j in range(n3):
        gap = min(abs(s2[j] - s2[j - 1]) if j > 0 else np.inf,
                  abs(s2[j] - s2[j + 1]) if j + 1 < n3 else np.inf)
        if gap > 1e-2 * s2[0]:
            assert np.max(np.abs(Mg[j] - Mo[j])) <= 100 * tol * s2[0] / gap, j
    k = 5
    out = plan.fixed_rank(Xd, t_lib(Mg, dtype=dt), k)
    ref = oracle.fixed_rank(X, Mo, k)
    assert abs(out["rel_err"] - ref["rel_err"]) <= (1e-5 if dt == torch.float32 else 1e-9)


def test_data_transform_host_buffers_and_errors():
    from paper_2605_16058_gb300 import native as N
    rng = np.random.default_rng(44)
    X = synth.cp_tensor(30, 20, 6, 4, rng, noise_rel=0.2)
    plan = _plan(30, 20, 6, torch.float64)
    dev = np_lib(plan.data_transform(t_lib(X, dtype=torch.float64)))
    host = torch.empty(6, 6, dtype=torch.float64)
    N.tsvdm_data_transform(plan.handle, t_lib(X, dtype=torch.float64).cpu(), host)
    assert np.array_equal(np_lib(host), dev)
    from paper_2605_16058_gb300.tsvdm import Plan
    p4 = Plan.dway((10, 8, 3, 2), dtype=torch.float64)
    with pytest.raises(N.TsvdmError) as e:
        p4.data_transform(torch.zeros(2, 3, 8, 10, dtype=torch.float64, device="cuda"),
                          out=torch.empty(6, 6, dtype=torch.float64, device="cuda"))
    assert e.value.status == N.ENOTSUP
