"""Planted mistakes in the oracle.

Each test plants one plausible mistake in the FP64 oracle, on the CPU and only for the
length of the test (pytest's monkeypatch). It then checks that one of the oracle's pins
(tests/test_oracle_pins.py) fails. This is the evidence that the pins constrain every part
of the oracle that the GPU path is compared with.

The mistakes are the usual ones:
- a transposed operand;
- a dropped or flipped term;
- a wrong inequality or an off-by-one in Algorithm 2;
- a sign convention changed on one side only.
"""
import math

import numpy as np
import pytest

import oracle
import test_oracle_pins as pins


def _fails(fn, *args):
    """True when the pin's own assertion rejects the planted mistake (any other error
    propagates, so a broken plant cannot pass for a caught one)."""
    try:
        fn(*args)
    except AssertionError:
        return True
    return False


# ---------------------------------------------------------------- transform (Sec. 2.1)
def test_transposed_transform_is_caught(monkeypatch):
    real = oracle.ttm3
    monkeypatch.setattr(oracle, "ttm3", lambda X, M, which=None: real(
        X, np.ascontiguousarray(np.asarray(M).T), which))
    assert _fails(pins.test_ttm_equals_scipy_dct_along_mode3)


def test_transposed_mode_product_is_caught(monkeypatch):
    real = oracle.ttm_mode
    monkeypatch.setattr(oracle, "ttm_mode", lambda X, M, mode: real(
        X, np.ascontiguousarray(np.asarray(M).T), mode))
    assert _fails(pins.test_dway_transform_equals_kronecker_mode3)


# ---------------------------------------------------------------- slice SVD (Alg. 1)
def test_sign_flipped_on_one_side_is_caught(monkeypatch):
    real = oracle.svd

    def svd(A, *a, **kw):
        U, S, V, sweeps = real(A, *a, **kw)
        U = U.copy()
        U[:, 0] = -U[:, 0]                 # left vector flipped, right one not
        return U, S, V, sweeps

    monkeypatch.setattr(oracle, "svd", svd)
    assert _fails(pins.test_svd_matches_lapack, 40, 25, None)


# ---------------------------------------------------------------- Algorithm 2
def _alg2(S, eps, strict=True, ties_kept=False, descending=False, shift=0):
    """Algorithm 2 steps 2-8 with one optional planted mistake:
    strict=False     w_l / sum <= eps^2 instead of <;
    ties_kept        rho counts sigma^2 >= tau (copies of tau kept);
    descending       v sorted descending instead of ascending;
    shift            tau taken from position J + shift (an off-by-one)."""
    S = np.asarray(S, dtype=np.float64)
    if S.ndim == 1:
        S = S[:, None]
    v = np.sort((S * S).reshape(-1, order="F"), kind="stable")
    if descending:
        v = v[::-1]
    w = np.cumsum(v)
    total = float(w[-1]) if w.size else 0.0
    n = S.shape[1]
    if total == 0.0:
        return dict(ranks=np.zeros(n, dtype=np.int64), J=int(v.size), tau=0.0, total=0.0,
                    discarded=0.0)
    e2 = float(eps) ** 2
    ok = np.nonzero(w / total < e2 if strict else w / total <= e2)[0]
    J = int(ok[-1]) + 1 if ok.size else 0
    if J > 0:
        J = min(max(J + shift, 1), v.size)
    tau = float(v[J - 1]) if J > 0 else -math.inf
    S2 = S * S
    keep = S2 >= tau if ties_kept else S2 > tau
    return dict(ranks=np.sum(keep, axis=0).astype(np.int64), J=J, tau=tau, total=total,
                discarded=float(np.sum(np.where(keep, 0.0, S2))))


def _golden_failures(monkeypatch, **mistake):
    monkeypatch.setattr(oracle, "select_ranks", lambda S, eps: _alg2(S, eps, **mistake))
    return [row[0] for row in pins._read_alg2() if _fails(pins.test_alg2_worked_examples, row)]


def test_algorithm2_copy_without_mistake_passes_the_golden_cases(monkeypatch):
    # the copy above is faithful, so the failures below come from the planted mistakes
    assert _golden_failures(monkeypatch) == []


@pytest.mark.parametrize("mistake,case", [
    (dict(strict=False), "C"),             # "<=" at the exact boundary of case C
    (dict(ties_kept=True), "B"),           # copies of tau kept in case B
    (dict(descending=True), "A"),          # running sums of the largest values first
    (dict(shift=1), "A"),                  # tau one position too far
    (dict(shift=-1), "A"),                 # tau one position too early
])
def test_algorithm2_mistakes_are_caught_by_the_golden_cases(monkeypatch, mistake, case):
    assert case in _golden_failures(monkeypatch, **mistake)


# ---------------------------------------------------------------- truncation error
def test_missing_square_root_in_the_error_is_caught(monkeypatch):
    real = oracle.fixed_rank

    def fixed_rank(*a, **kw):
        res = dict(real(*a, **kw))
        res["rel_err"] = res["rel_err"] ** 2          # discarded / total without the root
        return res

    monkeypatch.setattr(oracle, "fixed_rank", fixed_rank)
    assert _fails(pins.test_eckart_young_truncation_error, 4)


# ---------------------------------------------------------------- gradients (backward)
def test_flipped_norm_term_in_dx_is_caught(monkeypatch):
    real = oracle.loss_and_grad

    def loss_and_grad(X, M, k, *a, **kw):
        g = dict(real(X, M, k, *a, **kw))
        xn2 = float(np.sum(np.asarray(X, dtype=np.float64) ** 2))
        g["dX"] = g["dX"] + 2.0 * (g["loss"] / xn2) * np.asarray(X)   # + L X / |X|^2
        return g

    monkeypatch.setattr(oracle, "loss_and_grad", loss_and_grad)
    assert _fails(pins.test_gradient_wrt_x_matches_central_differences)


def test_transposed_dm_is_caught(monkeypatch):
    real = oracle.loss_and_grad

    def loss_and_grad(*a, **kw):
        g = dict(real(*a, **kw))
        g["dM"] = g["dM"].T.copy()
        return g

    monkeypatch.setattr(oracle, "loss_and_grad", loss_and_grad)
    assert _fails(pins.test_gradient_wrt_m_matches_central_differences)


def test_cayley_factors_swapped_is_caught(monkeypatch):
    def cayley(A, M0):
        A = np.asarray(A, dtype=np.float64)
        n = A.shape[0]
        W = A.T - A
        I = np.eye(n)
        Q = np.linalg.solve(I - W, I + W)             # (I - W)^{-1} (I + W): the inverse map
        return Q @ np.asarray(M0, dtype=np.float64), Q, W

    monkeypatch.setattr(oracle, "cayley", cayley)
    assert _fails(pins.test_cayley_is_orthogonal_and_starts_at_m0)


# ---------------------------------------------------------------- back-transform (Sec. 2.2)
def test_reconstruction_through_the_transposed_inverse_is_caught(monkeypatch):
    real = oracle.reconstruct

    def reconstruct(U, S, V, Minv, k=None, offsets=None):
        if not isinstance(Minv, (list, tuple)):
            Minv = np.ascontiguousarray(np.asarray(Minv).T)    # M instead of M^{-1}
        return real(U, S, V, Minv, k=k, offsets=offsets)

    monkeypatch.setattr(oracle, "reconstruct", reconstruct)
    assert _fails(pins.test_full_rank_reconstruction_is_exact)


def test_original_domain_factor_missing_a_mode_is_caught(monkeypatch):
    real = oracle.original_domain

    def original_domain(F, Minv):
        if isinstance(Minv, (list, tuple)):                    # the last mode left out
            Minv = list(Minv[:-1]) + [np.eye(np.asarray(Minv[-1]).shape[0])]
        return real(F, Minv)

    monkeypatch.setattr(oracle, "original_domain", original_domain)
    assert _fails(pins.test_dway_original_domain_factors_rebuild_x)


# ---------------------------------------------------------------- data-driven M (Sec. 2.2)
def test_data_driven_transform_transposed_is_caught(monkeypatch):
    real = oracle.data_transform

    def data_transform(X):
        M, sig = real(X)
        return M.T.copy(), sig                                 # columns, not rows

    monkeypatch.setattr(oracle, "data_transform", data_transform)
    assert _fails(pins.test_data_transform_diagonalises_the_mode3_gram)


# ---------------------------------------------------------------- storage count (Sec. 3.4)
def test_variable_ratio_without_slice_count_is_caught(monkeypatch):
    def cr(m, p, ranks, with_sigma=True):           # the n of the input entries dropped
        tot = float(np.sum(ranks)) * (m + p + (1 if with_sigma else 0))
        return (m * p) / tot if tot > 0 else math.inf

    monkeypatch.setattr(oracle, "compression_ratio_variable", cr)
    assert _fails(pins.test_compression_ratio_variable_hand_worked)


def test_variable_ratio_without_sigma_entries_is_caught(monkeypatch):
    real = oracle.compression_ratio_variable
    monkeypatch.setattr(oracle, "compression_ratio_variable",
                        lambda m, p, ranks, with_sigma=True: real(m, p, ranks, False))
    assert _fails(pins.test_compression_ratio_variable_hand_worked)
