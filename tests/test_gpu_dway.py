"""d-way tensors (the order-d star-M product: one transform matrix per mode >= 3, slices =
all trailing index combinations) through the C ABI against the FP64 oracle: transforms,
t-SVDM-I, t-SVDM-II, reconstruction and original-domain factors, for 4-way and 5-way
tensors (tall and wide slices, ragged sizes), FP64 and FP32 plans.

Tolerances as in test_gpu_parity: sigma within 1e-5 sigma_max (FP32) / 1e-12 (FP64) of
the tensor's largest singular value, subspaces 1e-4 / 1e-9 where the gap exceeds
1e-3 / 1e-6 sigma_max, relative errors 1e-5 / 1e-12, transforms 2e-6 / 1e-13 of max|Y|
times sqrt(n) per mode."""
import numpy as np
import pytest

import oracle
from paper_2605_16058_gb300 import synth

from helpers import np_lib, proj_diff, t_lib

pytestmark = pytest.mark.gpu
torch = pytest.importorskip("torch")

TOL = {torch.float32: dict(sig=1e-5, proj=1e-4, gap=1e-3, rel=1e-5, ttm=2e-6),
       torch.float64: dict(sig=1e-12, proj=1e-9, gap=1e-6, rel=1e-12, ttm=1e-13)}


@pytest.fixture(scope="module", autouse=True)
def _lib():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2605_16058_gb300 import build
    build.build()


def _case(dims, dt, seed=5):
    rng = np.random.default_rng(seed)
    X = synth.cp_tensor(dims[0], dims[1], int(np.prod(dims[2:])), 6, rng, noise_rel=1e-2)
    X = X.reshape(dims, order="F")
    Ms = [synth.dct2_matrix(dims[2])] + [synth.haar_orthogonal(n, rng) for n in dims[3:]]
    if dt == torch.float32:
        X = X.astype(np.float32).astype(np.float64)
        Ms = [M.astype(np.float32).astype(np.float64) for M in Ms]
    return X, Ms


def _plan(dims, dt, prec=None):
    from paper_2605_16058_gb300.tsvdm import Plan
    return Plan.dway(dims, dtype=dt, prec=prec)


def _mbuf(Ms, dt):
    from paper_2605_16058_gb300.tsvdm import Plan
    return Plan.concat([t_lib(M, dtype=dt) for M in Ms])


# (dims, dtype, TTM precision): the BF16x3 case runs every per-mode TTM on the tensor
# cores (and its 12 slices of 66 columns through the tensor-core Jacobi)
CASES = [((40, 30, 5, 3), torch.float64, None), ((40, 30, 5, 3), torch.float32, None),
         ((24, 50, 3, 2, 4), torch.float32, None), ((130, 66, 4, 3), torch.float32, "bf16x3")]


@pytest.mark.parametrize("dims,dt,prec", [c for c in CASES if c[2] is None])
def test_dway_transform_forward_and_inverse(dims, dt, prec):
    X, Ms = _case(dims, dt)
    plan = _plan(dims, dt, prec)
    Mb = _mbuf(Ms, dt)
    Y = plan.transform(t_lib(X, dtype=dt), Mb)
    want = oracle.dway_transform(X, Ms)
    got = np_lib(Y)
    assert got.shape == want.shape
    scale = np.max(np.abs(want)) * np.sqrt(max(dims[2:])) * (len(dims) - 2)
    assert np.max(np.abs(got - want)) <= TOL[dt]["ttm"] * scale
    Xb = np_lib(plan.transform(Y, Mb, inverse=True))       # M_k^{-1} = M_k^T (orthogonal)
    assert np.max(np.abs(Xb - X)) <= 50 * TOL[dt]["ttm"] * scale


@pytest.mark.parametrize("dims,dt,prec", CASES)
def test_dway_fixed_rank_and_reconstruct(dims, dt, prec):
    X, Ms = _case(dims, dt)
    k = 5
    tol = TOL[dt]
    plan = _plan(dims, dt, prec)
    Mb = _mbuf(Ms, dt)
    out = plan.fixed_rank(t_lib(X, dtype=dt), Mb, k)
    ref = oracle.fixed_rank(X, Ms, k)
    S_g, U_g, V_g = np_lib(out["S"]), np_lib(out["U"]), np_lib(out["V"])
    N = int(np.prod(dims[2:]))
    assert S_g.shape == (k, N) and U_g.shape == (dims[0], k, N) and V_g.shape == (dims[1], k, N)
    smax = ref["S_all"].max()
    assert np.max(np.abs(S_g - ref["S"])) <= tol["sig"] * smax
    full = oracle.svd_slices(ref["Ahat"])
    for i in range(N):
        so = ref["S_all"][:, i]
        for kk in range(1, k + 1):
            gap = so[kk - 1] - (so[kk] if kk < len(so) else 0.0)
            if gap > tol["gap"] * smax and so[kk - 1] > tol["gap"] * smax:
                assert proj_diff(full[0][:, :kk, i], U_g[:, :kk, i]) <= tol["proj"], (i, kk)
                assert proj_diff(full[2][:, :kk, i], V_g[:, :kk, i]) <= tol["proj"], (i, kk)
    assert abs(out["rel_err"] - ref["rel_err"]) <= tol["rel"]
    # back-transform over every trailing mode; Eckart-Young: direct error = reported error
    Xk = np_lib(plan.reconstruct(out["U"], out["S"], out["V"], Mb, k=k)).reshape(dims, order="F")
    want = oracle.reconstruct(U_g, S_g, V_g, [M.T for M in Ms])
    # BF16x3 mode products carry ~2^-17 relative error per term (the split drops the
    # lo*lo product and rounds the lo part), and the back-transform applies one per mode
    rec = {None: 1e-5, "bf16x3": 5e-5}[prec] * (1 if dt == torch.float32 else 1e-7)
    assert np.max(np.abs(Xk - want)) <= rec * np.max(np.abs(want))
    assert abs(oracle.rel_err_direct(X, Xk) - out["rel_err"]) <= (2e-5 if dt == torch.float32 else 1e-11)


@pytest.mark.parametrize("dims,dt,prec", CASES)
def test_dway_tolerance(dims, dt, prec):
    X, Ms = _case(dims, dt)
    eps = 0.05
    plan = _plan(dims, dt, prec)
    Mb = _mbuf(Ms, dt)
    out = plan.tolerance(t_lib(X, dtype=dt), Mb, eps)
    ref = oracle.tolerance(X, Ms, eps)
    ranks = out["ranks"].cpu().numpy()
    tau = ref["tau"]
    near = np.zeros(ranks.shape[0], dtype=bool)
    if np.isfinite(tau) and tau > 0:
        near = (np.abs(ref["S_all"] ** 2 - tau) <= 1e-6 * tau).any(axis=0)
    assert np.array_equal(ranks[~near], ref["ranks"][~near])
    assert out["rel_err"] < eps
    assert abs(out["rel_err"] - ref["rel_err"]) <= TOL[dt]["rel"]
    offs = out["offsets"]
    Xk = np_lib(plan.reconstruct(out["U"], out["S"], out["V"], Mb, offsets=offs)).reshape(dims, order="F")
    assert abs(oracle.rel_err_direct(X, Xk) - out["rel_err"]) <= (2e-5 if dt == torch.float32 else 1e-11)


def test_dway_original_domain_factors():
    dims, dt = (36, 28, 4, 3), torch.float64
    X, Ms = _case(dims, dt)
    k = 4
    plan = _plan(dims, dt)
    Mb = _mbuf(Ms, dt)
    hat = plan.fixed_rank(t_lib(X, dtype=dt), Mb, k)
    org = plan.fixed_rank(t_lib(X, dtype=dt), Mb, k, original_domain=True)
    Minv = [M.T for M in Ms]
    for key in ("U", "V", "S"):
        want = oracle.original_domain(np_lib(hat[key]), Minv)
        assert np.max(np.abs(np_lib(org[key]) - want)) <= 1e-12 * max(np.max(np.abs(want)), 1e-300)


def test_dway_order3_plan_equals_plain_plan():
    from paper_2605_16058_gb300.tsvdm import Plan
    X, Ms = _case((30, 20, 6), torch.float64)
    a = Plan.dway((30, 20, 6), dtype=torch.float64)
    b = Plan(30, 20, 6, dtype=torch.float64)
    Xd, Md = t_lib(X, dtype=torch.float64), t_lib(Ms[0], dtype=torch.float64)
    fa, fb = a.fixed_rank(Xd, Md, 4), b.fixed_rank(Xd, Md, 4)
    assert torch.equal(fa["S"], fb["S"]) and torch.equal(fa["U"], fb["U"])


def test_dway_argument_errors():
    from paper_2605_16058_gb300 import native as N
    for dims in [(4, 4), (4, 4, 2, 2, 2, 2, 2, 2, 2), (4, 4, 0, 2), (4, -1, 2, 2)]:
        with pytest.raises(N.TsvdmError) as e:
            N.tsvdm_plan_create_dway(dims, N.F64, N.P_FP64, True)
        assert e.value.status == N.EINVAL
    dims, dt = (12, 10, 3, 2), torch.float64
    X, Ms = _case(dims, dt)
    plan = _plan(dims, dt)
    Mb = _mbuf(Ms, dt)
    f = plan.fixed_rank(t_lib(X, dtype=dt), Mb, 2)
    with pytest.raises(N.TsvdmError) as e:
        plan.backward(t_lib(X, dtype=dt), Mb, 2, f["U"], f["S"], f["V"])
    assert e.value.status == N.ENOTSUP
