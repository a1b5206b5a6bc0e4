"""Tensor-core (tcgen05 + TMEM, TMA-fed) mode-3 TTM in BF16x3 and TF32 against the FP64
oracle.  Error model: each product of the BF16x3 split carries a relative error below
2^-15 and of TF32 below 2^-10, so |Y - Y_oracle| <= c u sum_t |X(:,t)| |B(t,:)| with the
stated u; the bound is checked element by element."""
import numpy as np
import pytest

import oracle
from paper_2605_16058_gb300 import synth

from helpers import np_lib, t_lib

pytestmark = pytest.mark.gpu
torch = pytest.importorskip("torch")

U_EFF = {"bf16x3": 2.0 ** -15, "tf32": 2.0 ** -10}


@pytest.fixture(scope="module", autouse=True)
def _lib():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2605_16058_gb300 import build
    build.build()


@pytest.mark.parametrize("prec", ["bf16x3", "tf32"])
@pytest.mark.parametrize("shape", [(32, 29, 19), (8, 16, 70), (4, 33, 129), (16, 16, 256),
                                   (12, 40, 300), (40, 25, 365), (8, 64, 512), (260, 2, 16)])
def test_tc_ttm_matches_oracle(prec, shape):
    from paper_2605_16058_gb300.tsvdm import Plan
    n1, n2, n3 = shape
    rng = np.random.default_rng(n3)
    X = rng.standard_normal(shape).astype(np.float32).astype(np.float64)
    M = (synth.haar_orthogonal(n3, rng) * 0.7).astype(np.float32).astype(np.float64)
    plan = Plan(n1, n2, n3, dtype=torch.float32, prec=prec)
    Xd, Md = t_lib(X, dtype=torch.float32), t_lib(M, dtype=torch.float32)
    Y = np_lib(plan.transform(Xd, Md))
    want = oracle.ttm3(X, M)
    bound = 4 * U_EFF[prec] * np.einsum("abt,it->abi", np.abs(X), np.abs(M)) + 1e-30
    assert np.all(np.abs(Y - want) <= bound), np.max(np.abs(Y - want) / bound)
    Xb = np_lib(plan.transform(plan.transform(Xd, Md), Md, inverse=True))
    bound2 = 8 * U_EFF[prec] * np.einsum("abt,it->abi", np.abs(want), np.abs(M.T)) / 0.49 + 1e-30
    assert np.all(np.abs(Xb - X) <= bound2 + 4 * U_EFF[prec] * np.abs(X))


@pytest.mark.parametrize("prec", ["bf16x3", "tf32"])
def test_tc_fixed_rank_close_to_oracle(prec):
    from paper_2605_16058_gb300.tsvdm import Plan
    rng = np.random.default_rng(3)
    X = synth.cp_tensor(96, 40, 24, 20, rng, noise_rel=1e-2).astype(np.float32).astype(np.float64)
    M = synth.dct2_matrix(24).astype(np.float32).astype(np.float64)
    ref = oracle.fixed_rank(X, M, 6)
    plan = Plan(96, 40, 24, dtype=torch.float32, prec=prec)
    out = plan.fixed_rank(t_lib(X, dtype=torch.float32), t_lib(M, dtype=torch.float32), 6)
    S = np_lib(out["S"])
    tol = 1e-5 if prec == "bf16x3" else 2e-3
    assert np.max(np.abs(S - ref["S"])) <= tol * ref["S"].max()
    assert abs(out["rel_err"] - ref["rel_err"]) <= (1e-5 if prec == "bf16x3" else 2e-3)
