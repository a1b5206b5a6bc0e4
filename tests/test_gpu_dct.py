"""The fast orthonormal DCT-II transform (tsvdm_plan_set_transform, TSVDM_TRANSFORM_DCT2)
through the C ABI against the FP64 oracle's dense transform by the same matrix.

Tolerances: transforms within 2e-6 max|Y| (FP32; an FFT's rounding grows like log2(n) u,
below the dense product's sqrt(n) u) and 1e-12 max|Y| (FP64; the oracle's DCT matrix is
itself formed with cosines of arguments up to pi n, accurate to ~1e-13 at n = 512);
decompositions at the stated parity tolerances of the dense plans (singular values 1e-5 /
1e-12 of sigma_max, relative errors 1e-5 / 1e-12, t-SVDM-II ranks exact)."""
import numpy as np
import pytest

import oracle
from paper_2605_16058_gb300 import synth

from helpers import np_lib, t_lib

pytestmark = pytest.mark.gpu
torch = pytest.importorskip("torch")

TTM_TOL = {torch.float32: 2e-6, torch.float64: 1e-12}


@pytest.fixture(scope="module", autouse=True)
def _lib():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2605_16058_gb300 import build
    build.build()


def _plan(n1, n2, n3, dt, orthogonal=True):
    from paper_2605_16058_gb300.tsvdm import Plan
    return Plan(n1, n2, n3, dtype=dt, orthogonal=orthogonal)


@pytest.mark.parametrize("dt", [torch.float32, torch.float64])
@pytest.mark.parametrize("shape", [(37, 29, 1), (37, 29, 2), (5, 7, 16), (130, 3, 128),
                                   (33, 17, 512), (3, 2, 4096)])
def test_fast_dct_matches_dense_transform(dt, shape):
    """Forward (DCT-II) and inverse (its transpose), rows not a multiple of a CTA's tile."""
    n1, n2, n3 = shape
    X = np.random.default_rng(3).standard_normal(shape)
    M = synth.dct2_matrix(n3)
    if dt == torch.float32:
        X = X.astype(np.float32).astype(np.float64)
    plan = _plan(n1, n2, n3, dt)
    plan.set_transform("dct2")
    Md = t_lib(M, dtype=dt)
    Y = plan.transform(t_lib(X, dtype=dt), Md)
    want = oracle.ttm3(X, M)
    got = np_lib(Y)
    assert np.max(np.abs(got - want)) <= TTM_TOL[dt] * np.max(np.abs(want))
    back = np_lib(plan.transform(t_lib(want, dtype=dt), Md, inverse=True))
    assert np.max(np.abs(back - X)) <= TTM_TOL[dt] * np.max(np.abs(X)) * 4


@pytest.mark.parametrize("dt", [torch.float32, torch.float64])
def test_fast_dct_decompositions_match_oracle(dt):
    """t-SVDM-I and t-SVDM-II through the fast transform equal the oracle's with the dense
    DCT-II, and the reconstruction inverts through DCT-III."""
    n1, n2, n3, k, eps = 120, 70, 16, 6, 0.05
    rng = np.random.default_rng(8)
    X = synth.cp_tensor(n1, n2, n3, 20, rng, noise_rel=1e-2)
    M = synth.dct2_matrix(n3)
    if dt == torch.float32:
        X = X.astype(np.float32).astype(np.float64)
    sig_tol, rel_tol = (1e-5, 1e-5) if dt == torch.float32 else (1e-12, 1e-12)
    plan = _plan(n1, n2, n3, dt)
    plan.set_transform("dct2")
    Xd, Md = t_lib(X, dtype=dt), t_lib(M, dtype=dt)
    out = plan.fixed_rank(Xd, Md, k)
    ref = oracle.fixed_rank(X, M, k)
    S = np_lib(out["S"])
    assert np.max(np.abs(S - ref["S"])) <= sig_tol * ref["S"].max()
    assert abs(out["rel_err"] - ref["rel_err"]) <= rel_tol
    Xk = np_lib(plan.reconstruct(out["U"], out["S"], out["V"], Md, k=k))
    assert abs(oracle.rel_err_direct(X, Xk) - ref["rel_err"]) <= 10 * rel_tol
    tol = plan.tolerance(Xd, Md, eps)
    tref = oracle.tolerance(X, M, eps)
    assert np.array_equal(tol["ranks"].cpu().numpy(), tref["ranks"])
    assert abs(tol["rel_err"] - tref["rel_err"]) <= rel_tol


def test_fast_dct_dway():
    """A 4-way tensor: one DCT-II per trailing mode, equal to the oracle's mode products."""
    from paper_2605_16058_gb300.tsvdm import Plan
    dims = (20, 12, 8, 4)
    X = np.random.default_rng(9).standard_normal(dims)
    Ms = [synth.dct2_matrix(d) for d in dims[2:]]
    plan = Plan.dway(dims, dtype=torch.float64)
    plan.set_transform("dct2")
    Mcat = Plan.concat([t_lib(M, dtype=torch.float64) for M in Ms])
    Y = np_lib(plan.transform(t_lib(X, dtype=torch.float64), Mcat))
    want = oracle.dway_transform(X, Ms)
    assert np.max(np.abs(Y - want)) <= 1e-12 * np.max(np.abs(want))


def test_fast_dct_argument_errors():
    from paper_2605_16058_gb300 import native as N
    for shape, orth, kind, status in [((8, 8, 12), True, "dct2", N.ENOTSUP),
                                      ((8, 8, 16), False, "dct2", N.EINVAL),
                                      ((8, 8, 16), True, 7, N.EINVAL)]:
        plan = _plan(*shape, torch.float32, orthogonal=orth)
        with pytest.raises(N.TsvdmError) as e:
            plan.set_transform(kind)
        assert e.value.status == status
    plan = _plan(8, 8, 16, torch.float32)
    plan.set_transform("dct2")
    plan.set_transform("dense")
