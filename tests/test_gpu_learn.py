"""Differentiable path against the FP64 oracle: truncation loss and its gradients
(dL/dX, dL/dM), the Cayley map and its adjoint, Adam, the autograd wrapper, and a short
learned-transform run whose loss must decrease.

Tolerances: FP64 plans 1e-9 relative; FP32 plans 1e-4 relative (the residual
R = Ahat - U S V^T is formed in FP32 from a loss of a few percent, so its relative
accuracy is about u / L ~ 1e-5)."""
import numpy as np
import pytest

import oracle
from paper_2605_16058_gb300 import synth

from helpers import np_lib, t_lib

pytestmark = pytest.mark.gpu
torch = pytest.importorskip("torch")


@pytest.fixture(scope="module", autouse=True)
def _lib():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2605_16058_gb300 import build
    build.build()


def _rel(a, b):
    return float(np.linalg.norm(a - b) / max(np.linalg.norm(b), 1e-300))


@pytest.mark.parametrize("dt,case,tol,engine", [(torch.float64, "smoke", 1e-9, None),
                                                (torch.float32, "crystal", 1e-4, None),
                                                (torch.float32, "crystal", 1e-4, "fma"),
                                                (torch.float64, "crystal", 1e-9, None)])
def test_backward_matches_oracle(dt, case, tol, engine):
    """FP32 dL/dM: tensor-core A^T B (default engine) and the CUDA-core split-K product
    (FMA engine)."""
    from paper_2605_16058_gb300.tsvdm import Plan
    if case == "smoke":
        c = synth.smoke_case()
        X, M, k = c["X"], c["M"], c["k"]
    else:
        X = synth.crystal(shape=(32, 24, 8), lattice=(3, 2), dtype=np.float64)
        M, k = synth.dct2_matrix(8), 2
    if dt == torch.float32:
        X = X.astype(np.float32).astype(np.float64)
        M = M.astype(np.float32).astype(np.float64)
    n1, n2, n3 = X.shape
    plan = Plan(n1, n2, n3, dtype=dt)
    if engine is not None:
        plan.set_engine(engine)
    Xd, Md = t_lib(X, dtype=dt), t_lib(M, dtype=dt)
    f = plan.fixed_rank(Xd, Md, k)
    dX, dM = torch.empty_like(Xd), torch.empty_like(Md)
    loss = plan.backward(Xd, Md, k, f["U"], f["S"], f["V"], 1.0, dX, dM, "host")
    g = oracle.loss_and_grad(X, M, k)
    assert abs(loss - g["loss"]) <= tol * g["loss"]
    assert _rel(np_lib(dX), g["dX"]) <= tol * 10
    assert _rel(np_lib(dM), g["dM"]) <= tol * 10
    # upstream scalar scales both gradients
    dX2, dM2 = torch.empty_like(Xd), torch.empty_like(Md)
    plan.backward(Xd, Md, k, f["U"], f["S"], f["V"], -2.5, dX2, dM2, None)
    # dX = alpha (R x3 M^T) + beta X: where the two terms cancel, scaling them by dL moves
    # the rounding by an ulp of each term, so the comparison has an absolute floor.
    assert torch.allclose(dX2, -2.5 * dX, rtol=1e-5, atol=1e-6 * float(dX.abs().max()) * 2.5)


@pytest.mark.parametrize("dt", [torch.float32, torch.float64])
def test_cayley_and_adjoint_match_oracle(dt):
    from paper_2605_16058_gb300 import native as N
    n = 24
    rng = np.random.default_rng(21)
    A = 0.1 * rng.standard_normal((n, n))
    M0 = synth.dct2_matrix(n)
    dM = rng.standard_normal((n, n))
    dtc = N.F32 if dt == torch.float32 else N.F64
    Ad, M0d, dMd = t_lib(A, dtype=dt), t_lib(M0, dtype=dt), t_lib(dM, dtype=dt)
    M, Z, Q = torch.empty_like(Ad), torch.empty_like(Ad), torch.empty_like(Ad)
    work = torch.empty(3 * n * n, dtype=dt, device="cuda")
    N.tsvdm_cayley(n, dtc, Ad, M0d, M, Z, Q, work)
    Mo, Qo, Wo = oracle.cayley(A, M0)
    tol = 1e-5 if dt == torch.float32 else 1e-12
    assert np.max(np.abs(np_lib(M) - Mo)) <= tol
    Mn = np_lib(M)
    assert np.linalg.norm(Mn.T @ Mn - np.eye(n)) <= 10 * tol
    dA = torch.empty_like(Ad)
    N.tsvdm_cayley_backward(n, dtc, M0d, Z, Q, dMd, dA, work)
    want = oracle.cayley_grad(A, M0, dM)
    assert _rel(np_lib(dA), want) <= 10 * tol


def test_adam_matches_oracle():
    from paper_2605_16058_gb300 import native as N
    rng = np.random.default_rng(22)
    p = rng.standard_normal(1000)
    po, m1o, m2o = p.copy(), np.zeros(1000), np.zeros(1000)
    pd = torch.tensor(p, device="cuda")
    m1, m2 = torch.zeros_like(pd), torch.zeros_like(pd)
    for t in range(1, 6):
        g = rng.standard_normal(1000)
        oracle.adam_step(po, g, m1o, m2o, t, lr=1e-2)
        N.tsvdm_adam(1000, N.F64, pd, torch.tensor(g, device="cuda"), m1, m2, t, 1e-2)
    assert np.max(np.abs(pd.cpu().numpy() - po)) <= 1e-13


def test_autograd_function_gradients():
    from paper_2605_16058_gb300.tsvdm import Plan, TruncationLoss
    X = synth.crystal(shape=(32, 24, 8), lattice=(3, 2), dtype=np.float64)
    M = synth.dct2_matrix(8)
    plan = Plan(32, 24, 8, dtype=torch.float64)
    Xd = t_lib(X, dtype=torch.float64).requires_grad_(True)
    Md = t_lib(M, dtype=torch.float64).requires_grad_(True)
    L = TruncationLoss.apply(Xd, Md, plan, 2)
    (3.0 * L).backward()
    g = oracle.loss_and_grad(X, M, 2)
    assert abs(L.item() - g["loss"]) <= 1e-10
    assert _rel(np_lib(Xd.grad), 3.0 * g["dX"]) <= 1e-8
    # only the gradient that is asked for (M fixed), and the loss alone under no_grad
    Xe = t_lib(X, dtype=torch.float64).requires_grad_(True)
    Me = t_lib(M, dtype=torch.float64)
    Le = TruncationLoss.apply(Xe, Me, plan, 2)
    Le.backward()
    assert abs(Le.item() - g["loss"]) <= 1e-10
    assert _rel(np_lib(Xe.grad), g["dX"]) <= 1e-8 and Me.grad is None
    with torch.no_grad():
        L0 = TruncationLoss.apply(t_lib(X, dtype=torch.float64), Me, plan, 2)
    assert abs(L0.item() - g["loss"]) <= 1e-10
    assert _rel(np_lib(Md.grad), 3.0 * g["dM"]) <= 1e-8


def test_learned_transform_lowers_the_loss_and_matches_oracle_first_step():
    from paper_2605_16058_gb300.learn import CayleyTrainer
    X = synth.crystal(shape=(64, 48, 16), lattice=(4, 3), dtype=np.float64)
    M0 = synth.dct2_matrix(16)
    k = 3
    tr = CayleyTrainer(t_lib(X, dtype=torch.float64), t_lib(M0, dtype=torch.float64),
                       X.shape, k, lr=1e-3)
    losses, ms = tr.train(20)
    # oracle: the same first step (A = 0 -> M = M0, Adam's first update)
    g0 = oracle.loss_and_grad(X, M0, k)
    assert abs(losses[0] - g0["loss"]) <= 1e-9 * g0["loss"]
    dA = oracle.cayley_grad(np.zeros((16, 16)), M0, g0["dM"])
    A1 = np.zeros((16, 16))
    oracle.adam_step(A1, dA, np.zeros_like(A1), np.zeros_like(A1), 1, lr=1e-3)
    M1 = oracle.cayley(A1, M0)[0]
    g1 = oracle.loss_and_grad(X, M1, k)
    assert abs(losses[1] - g1["loss"]) <= 1e-8 * g1["loss"]
    assert losses[-1] < losses[0]


@pytest.mark.parametrize("dt,tol", [(torch.float64, 1e-10), (torch.float32, 1e-4)])
def test_warm_start_matches_cold_start(dt, tol):
    """A sequence of slightly different transforms (the situation of learned-M training):
    the warm-started decomposition equals the cold one (sigma, rank-k subspaces, relative
    error) and needs fewer Jacobi sweeps."""
    from paper_2605_16058_gb300.tsvdm import Plan
    X = synth.crystal(shape=(96, 70, 12), lattice=(4, 3), dtype=np.float64)
    n1, n2, n3 = X.shape
    k = 4
    rng = np.random.default_rng(31)
    M0 = synth.dct2_matrix(n3)
    warm, cold = Plan(n1, n2, n3, dtype=dt), Plan(n1, n2, n3, dtype=dt)
    warm.set_warm_start(True)
    Xd = t_lib(X, dtype=dt)
    sw_w, sw_c = [], []
    for it in range(4):
        A = 1e-3 * it * rng.standard_normal((n3, n3))
        M = oracle.cayley(A, M0)[0]
        Md = t_lib(M, dtype=dt)
        fw, fc = warm.fixed_rank(Xd, Md, k), cold.fixed_rank(Xd, Md, k)
        sw_w.append(warm.stats()[0])
        sw_c.append(cold.stats()[0])
        Sw, Sc = np_lib(fw["S"]), np_lib(fc["S"])
        assert np.max(np.abs(Sw - Sc)) <= tol * Sc.max()
        assert abs(fw["rel_err"] - fc["rel_err"]) <= tol
        Uw, Uc = np_lib(fw["U"]), np_lib(fc["U"])
        for i in range(n3):
            s_all = np.sort(np.linalg.svd(
                np.einsum("it,abt->abi", M, X)[:, :, i], compute_uv=False))[::-1]
            if s_all[k - 1] - s_all[k] > 1e-3 * s_all[0]:
                P = lambda u: u @ u.T
                assert np.linalg.norm(P(Uw[:, :, i]) - P(Uc[:, :, i])) <= 100 * tol
    assert sum(sw_w[1:]) < sum(sw_c[1:])          # warm starts converge in fewer sweeps
    # a new call of set_warm_start makes the next decomposition cold again
    warm.set_warm_start(True)
    warm.fixed_rank(Xd, Md, k)
    assert warm.stats()[0] == cold.stats()[0]


def test_learned_transform_with_warm_start_tracks_cold_training():
    from paper_2605_16058_gb300.learn import CayleyTrainer
    X = synth.crystal(shape=(64, 48, 16), lattice=(4, 3), dtype=np.float64)
    M0 = synth.dct2_matrix(16)
    args = (t_lib(X, dtype=torch.float64), t_lib(M0, dtype=torch.float64), X.shape, 3)
    cold = CayleyTrainer(*args, lr=1e-3)
    warm = CayleyTrainer(*args, lr=1e-3, warm_start=True)
    lc, _ = cold.train(10)
    lw, _ = warm.train(10)
    assert max(abs(a - b) / a for a, b in zip(lc, lw)) <= 1e-9
