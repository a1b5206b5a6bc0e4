"""Allocation-free t-SVDM-II rank choice (tsvdm_select_ranks_noalloc) against the
existing entry point tsvdm_tolerance, through the C ABI, on two calls in a row.

The allocation-free entry point serves callers that must not call cudaMalloc (a process
whose device memory is all handed to another allocator, or a request path that forbids
driver allocations); it keeps its scratch in a fixed array inside the library.
Ranks and offsets are integers and must match exactly; the reported error within 1e-12.
"""
import ctypes

import numpy as np
import pytest

from paper_2605_16058_gb300 import synth

from helpers import t_lib

pytestmark = pytest.mark.gpu
torch = pytest.importorskip("torch")


@pytest.fixture(scope="module", autouse=True)
def _lib():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2605_16058_gb300 import build
    build.build()


def _noalloc(sig, cols, nslices, eps, ranks, offsets, summary):
    from paper_2605_16058_gb300 import native
    st = torch.cuda.current_stream().cuda_stream
    return native.lib().tsvdm_select_ranks_noalloc(
        ctypes.c_void_p(sig.data_ptr()), cols, nslices, float(eps),
        ctypes.c_void_p(ranks.data_ptr()), ctypes.c_void_p(offsets.data_ptr()),
        ctypes.c_void_p(summary.data_ptr()) if summary is not None else None,
        ctypes.c_void_p(st))


def test_noalloc_selection_matches_tsvdm_tolerance_twice():
    from paper_2605_16058_gb300 import native
    from paper_2605_16058_gb300.tsvdm import Plan
    n1, n2, n3 = 120, 80, 24
    X = synth.climate(shape=(n1, n2, n3), seed=6)
    M = synth.dct2_matrix(n3)
    plan = Plan(n1, n2, n3, dtype=torch.float32)
    Xd, Md = t_lib(X), t_lib(M, dtype=torch.float32)
    full = plan.fixed_rank(Xd, Md, n2, rel_err=False)      # sigma, descending per slice
    sig = full["S"].contiguous()                            # (n3, r) = r x n3 column-major
    for eps in (2e-2, 2e-2, 1e-3):                          # two identical calls, then another
        ref = plan.tolerance(Xd, Md, eps)
        ranks = torch.full((n3,), -1, dtype=torch.int32, device="cuda")
        offs = torch.full((n3 + 1,), -1, dtype=torch.int64, device="cuda")
        summ = torch.zeros(4, dtype=torch.float64, device="cuda")
        assert _noalloc(sig, n2, n3, eps, ranks, offs, summ) == native.OK
        torch.cuda.synchronize()
        assert torch.equal(ranks, ref["ranks"])
        assert torch.equal(offs, ref["offsets"])
        total, disc, tau, totrank = summ.cpu().tolist()
        assert int(totrank) == ref["total_rank"]
        assert abs(np.sqrt(disc / total) - ref["rel_err"]) <= 1e-12


def test_noalloc_rejects_sizes_beyond_its_scratch():
    from paper_2605_16058_gb300 import native
    sig = torch.zeros(4, device="cuda")
    ranks = torch.zeros(4, dtype=torch.int32, device="cuda")
    offs = torch.zeros(5, dtype=torch.int64, device="cuda")
    assert _noalloc(sig, 1024, 300, 0.1, ranks, offs, None) == native.ESCRATCH
    assert _noalloc(sig, 4, 1, 1.5, ranks, offs, None) == native.EINVAL


def _spectra():
    """Singular values (cols x nslices, descending per slice) whose squares and running
    sums are exact in FP64 (small integers: ties, zeros, exact boundaries), plus random
    ones."""
    out = [np.array([[3, 3, 2], [3, 2, 2], [2, 2, 2], [1, 0, 1]], dtype=np.float64),
           np.array([[5, 4], [1, 4], [1, 0], [0, 0]], dtype=np.float64),
           np.array([[2], [1], [1], [1]], dtype=np.float64),
           np.array([[7, 1, 1, 1]], dtype=np.float64),
           # golden case C: at eps = 0.25 the running sum meets eps^2 sum(v) exactly
           np.array([[1, 3], [1, 2], [0, 1]], dtype=np.float64)]
    rng = np.random.default_rng(40)
    for _ in range(6):
        cols, ns = int(rng.integers(1, 40)), int(rng.integers(1, 30))
        S = np.exp(rng.normal(0.0, 2.0, (cols, ns))).astype(np.float32).astype(np.float64)
        out.append(-np.sort(-S, axis=0))
    big = rng.integers(0, 6, (300, 40)).astype(np.float64)        # many ties
    out.append(-np.sort(-big, axis=0))
    return out


@pytest.mark.parametrize("eps", [0.05, 0.25, 0.5, 0.75, 0.999])
def test_noalloc_selection_matches_algorithm2_on_exact_spectra(eps):
    """Ranks, offsets, the total rank and tau equal Algorithm 2 (the oracle's sort and
    cumulative sum) exactly; the discarded energy to FP64 summation order."""
    import oracle
    from paper_2605_16058_gb300 import native
    for S in _spectra():
        cols, ns = S.shape
        want = oracle.select_ranks(S, eps)
        sig = torch.tensor(np.ascontiguousarray(S.T).astype(np.float32), device="cuda")
        ranks = torch.full((ns,), -1, dtype=torch.int32, device="cuda")
        offs = torch.full((ns + 1,), -1, dtype=torch.int64, device="cuda")
        summ = torch.zeros(4, dtype=torch.float64, device="cuda")
        assert _noalloc(sig, cols, ns, eps, ranks, offs, summ) == native.OK
        torch.cuda.synchronize()
        assert np.array_equal(ranks.cpu().numpy(), want["ranks"]), (S.T, eps)
        assert np.array_equal(offs.cpu().numpy(), oracle.offsets_from_ranks(want["ranks"]))
        total, disc, tau, totrank = summ.cpu().tolist()
        assert int(totrank) == int(np.sum(want["ranks"]))
        assert abs(total - want["total"]) <= 1e-13 * want["total"]
        assert abs(disc - want["discarded"]) <= 1e-13 * want["total"]
        if want["J"] > 0:
            assert tau == want["tau"]
        else:
            assert tau == -1.0


def test_noalloc_invalid_values_are_reported_and_minus_zero_is_zero():
    """-0 is a zero singular value (same result as +0); a NaN, an infinity or a negative
    value makes the call report NaN in the summary with every rank and offset 0; the next
    call on valid values is unaffected."""
    from paper_2605_16058_gb300 import native
    S = np.array([[4.0, 3.0], [2.0, 1.0], [1.0, 0.0], [0.0, 0.0]])
    cols, ns = S.shape

    def run(Sm, eps=0.3):
        sig = torch.tensor(np.ascontiguousarray(Sm.T).astype(np.float32), device="cuda")
        ranks = torch.full((ns,), -1, dtype=torch.int32, device="cuda")
        offs = torch.full((ns + 1,), -1, dtype=torch.int64, device="cuda")
        summ = torch.zeros(4, dtype=torch.float64, device="cuda")
        assert _noalloc(sig, cols, ns, eps, ranks, offs, summ) == native.OK
        torch.cuda.synchronize()
        return ranks.cpu().numpy(), offs.cpu().numpy(), summ.cpu().numpy()

    r0, o0, s0 = run(S)
    Sm = S.copy()
    Sm[3, 0] = -0.0
    Sm[2, 1] = -0.0
    r1, o1, s1 = run(Sm)
    assert np.array_equal(r0, r1) and np.array_equal(o0, o1) and np.array_equal(s0, s1)
    for bad in (np.nan, np.inf, -1.0):
        Sb = S.copy()
        Sb[2, 1] = bad
        rb, ob, sb = run(Sb)
        assert np.all(np.isnan(sb)) and not rb.any() and not ob.any(), bad
    r2, o2, s2 = run(S)
    assert np.array_equal(r0, r2) and np.array_equal(o0, o2) and np.array_equal(s0, s2)
