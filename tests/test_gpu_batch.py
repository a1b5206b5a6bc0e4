"""Batched launch of tensors with uneven shapes (t-SVDM-I and t-SVDM-II mixed, Haar M):
every tensor against the FP64 oracle; the CUDA-graph replay reproduces the plain run
bit for bit; the autotuner returns one of its candidates and keeps results valid."""
import numpy as np
import pytest

import oracle
from paper_2605_16058_gb300 import synth

from helpers import np_lib, proj_diff, t_lib

pytestmark = pytest.mark.gpu
torch = pytest.importorskip("torch")

SHAPES = [(130, 70, 9), (64, 100, 5), (200, 64, 7), (96, 96, 4), (150, 80, 6), (70, 140, 3)]


@pytest.fixture(scope="module", autouse=True)
def _lib():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2605_16058_gb300 import build
    build.build()


def _make():
    from paper_2605_16058_gb300 import native as N
    items, descs, ios, keep = [], [], [], []
    for idx, shape in enumerate(SHAPES):
        it = synth.batch_item(idx, shape, seed=9)
        n1, n2, n3 = shape
        r = min(n1, n2)
        X = it["X"].astype(np.float64)
        M = it["M"].astype(np.float32).astype(np.float64)
        Xd, Md = t_lib(X, dtype=torch.float32), t_lib(M, dtype=torch.float32)
        if it["mode"] == "fixed":
            k = min(it["k"], r)
            d = N.BatchDesc(n1, n2, n3, 0, k, 0.0)
            U = torch.zeros(n3, k, n1, device="cuda")
            S = torch.zeros(n3, k, device="cuda")
            V = torch.zeros(n3, k, n2, device="cuda")
            ranks = offs = None
        else:
            d = N.BatchDesc(n1, n2, n3, 1, 0, it["eps"])
            cap = n3 * r
            U = torch.zeros(cap, n1, device="cuda")
            S = torch.zeros(cap, device="cuda")
            V = torch.zeros(cap, n2, device="cuda")
            ranks = torch.zeros(n3, dtype=torch.int32, device="cuda")
            offs = torch.zeros(n3 + 1, dtype=torch.int64, device="cuda")
        rel = torch.zeros(1, dtype=torch.float64, device="cuda")
        ptr = lambda t: None if t is None else t.data_ptr()
        ios.append(N.BatchIO(Xd.data_ptr(), Md.data_ptr(), U.data_ptr(), S.data_ptr(), V.data_ptr(),
                             ptr(ranks), ptr(offs), rel.data_ptr()))
        keep.append(dict(X=X, M=M, Xd=Xd, Md=Md, U=U, S=S, V=V, ranks=ranks, offs=offs, rel=rel,
                         mode=it["mode"], k=d.k, eps=d.eps, shape=shape))
        descs.append(d)
    return descs, ios, keep


def _check(keep):
    for t in keep:
        n1, n2, n3 = t["shape"]
        if t["mode"] == "fixed":
            ref = oracle.fixed_rank(t["X"], t["M"], t["k"])
            S = np_lib(t["S"])
            smax = ref["S_all"].max()
            assert np.max(np.abs(S - ref["S"])) <= 1e-5 * smax
            U = np_lib(t["U"])
            for i in range(n3):
                so = ref["S_all"][:, i]
                kk = t["k"]
                if so[kk - 1] - so[kk] > 1e-2 * smax:      # u_eff sigma_max / gap
                    assert proj_diff(U[:, :kk, i], ref["U"][:, :, i]) <= 1e-4
            assert abs(t["rel"].item() - ref["rel_err"]) <= 1e-5
        else:
            ref = oracle.tolerance(t["X"], t["M"], t["eps"])
            ranks = t["ranks"].cpu().numpy()
            rel = t["rel"].item()
            assert rel < t["eps"]
            assert abs(rel - ref["rel_err"]) <= 1e-5                      # matched error
            tau = ref["tau"]
            near = np.zeros(n3, dtype=bool)
            if np.isfinite(tau) and tau > 0:                              # ties at tau
                near = (np.abs(ref["S_all"] ** 2 - tau) <= 1e-6 * tau).any(axis=0)
            for i in range(n3):
                if not near[i]:
                    assert ranks[i] == ref["ranks"][i]
            off = t["offs"].cpu().numpy()
            assert np.array_equal(np.diff(off), ranks)


@pytest.mark.parametrize("prec", ["fp32", "bf16x3"])
def test_batch_run_graph_replay_and_autotuner(prec):
    from paper_2605_16058_gb300 import native as N
    descs, ios, keep = _make()
    stream = torch.cuda.Stream()            # graphs are captured on a non-default stream
    torch.cuda.synchronize()
    b = N.tsvdm_batch_create(descs, N.F32, N.PRECISIONS[prec], stream)
    try:
        N.tsvdm_batch_run(b, ios)
        torch.cuda.synchronize()
        st, sweeps, rots = N.tsvdm_batch_status(b)
        assert st == N.OK and sweeps > 0
        _check(keep)
        first = [(t["S"].clone(), t["U"].clone(), t["rel"].clone()) for t in keep]
        for t in keep:                                   # wipe the outputs, replay the graph
            t["S"].zero_(); t["U"].zero_(); t["rel"].zero_()
        N.tsvdm_batch_capture(b, ios)
        assert N.tsvdm_batch_graph_kernels(b) >= len(keep) + 4   # TTMs, Jacobi, selection, ...
        for t in keep:
            t["S"].zero_(); t["U"].zero_(); t["rel"].zero_()
        torch.cuda.synchronize()
        N.tsvdm_batch_launch(b)
        N.tsvdm_batch_launch(b)
        torch.cuda.synchronize()
        for t, (S0, U0, r0) in zip(keep, first):
            assert torch.equal(t["S"], S0) and torch.equal(t["U"], U0) and torch.equal(t["rel"], r0)
        choice = N.tsvdm_batch_tune(b, ios)
        assert choice["width"] in (32, 64) and choice["cluster"] in (1, 2, 3, 4)
        assert choice["stages"] in (0, 2, 3) and choice["jacobi_ms"] > 0   # 0: tensor cores
        N.tsvdm_batch_run(b, ios)
        torch.cuda.synchronize()
        _check(keep)
    finally:
        N.tsvdm_batch_destroy(b)


def test_batch_capture_needs_a_non_default_stream():
    from paper_2605_16058_gb300 import native as N
    descs, ios, keep = _make()
    b = N.tsvdm_batch_create(descs[:1], N.F32, N.P_FP32, 0)
    try:
        with pytest.raises(N.TsvdmError) as e:
            N.tsvdm_batch_capture(b, ios[:1])
        assert e.value.status == N.EINVAL
        with pytest.raises(N.TsvdmError) as e:            # nothing captured
            N.tsvdm_batch_graph_kernels(b)
        assert e.value.status == N.EINVAL
    finally:
        N.tsvdm_batch_destroy(b)


def test_batch_rejects_bad_descriptors():
    from paper_2605_16058_gb300 import native as N
    with pytest.raises(N.TsvdmError):
        N.tsvdm_batch_create([N.BatchDesc(10, 8, 2, 0, 9, 0.0)], N.F32, N.P_FP32)   # k > r
    with pytest.raises(N.TsvdmError):
        N.tsvdm_batch_create([N.BatchDesc(10, 8, 2, 1, 0, 1.5)], N.F32, N.P_FP32)   # eps
