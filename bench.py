#!/usr/bin/env python
"""Throughput of the star-M truncated t-SVD hot path on one GB300 (or N replicas).

Workload (default): t-SVDM-II (Algorithm 2) of the climate-shaped tensor 1024 x 512 x 365
FP32 (spatial |k|^-3 Gaussian random fields evolved as AR(1), rho = 0.95, seed 1), M = the
orthonormal 365 x 365 DCT-II, relative tolerance eps = 1e-2.  One step = one C-ABI call
tsvdm_tolerance: mode-3 TTM, batched one-sided Jacobi SVD of the 365 slices, the global
sigma^2 sort / FP64 prefix sum / rank choice, and packing of the variable-rank factors.

Printed: ONE JSON line (rank 0).  `value` = input GB/s with X resident in HBM; `e2e` =
the same call given pinned HOST buffers (host->device copy of X and device->host copy of
ranks, offsets and the packed factors inside the timed region).  The input (765 MB) is
larger than L2 (129 MB), so no L2 flush is needed between steps.

--impl reference times the FP64 CPU oracle on the host cores (a bounded sample of the
same workload: the TTM and SVD of as many slices as there are cores, per step).
With torchrun and N > 1 each rank runs an independent replica (weak scaling, no
collective on the data path); the step time is the max over ranks.
"""
from __future__ import annotations

import argparse
import json
import math
import os
import statistics
import subprocess
import sys
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "t-SVDM input GB/s and slices/s at matched rel. error vs FP64; fwd+bwd ms/step"
WORKLOADS = {
    # name: (shape, eps, description)
    "climate": ((1024, 512, 365), 1e-2,
                "t-SVDM-II climate-shaped 1024x512x365 FP32, DCT-II, eps=1e-2"),
    # d-way (order-4) form of the climate tensor: 73 x 5 trailing modes (365 slices), one
    # DCT-II per mode (the same data as "climate", viewed as 4-way)
    "climate-4way": ((1024, 512, 73, 5), 1e-2,
                     "t-SVDM-II climate-shaped 1024x512x73x5 FP32 (4-way), DCT-II per trailing "
                     "mode, eps=1e-2"),
    "climate-304": ((1024, 512, 304), 1e-2,
                    "t-SVDM-II climate-shaped 1024x512x304 FP32, DCT-II, eps=1e-2"),
    "climate-128": ((1024, 512, 128), 1e-2,
                    "t-SVDM-II climate-shaped 1024x512x128 FP32, DCT-II, eps=1e-2"),
    "climate-medium": ((1024, 512, 48), 1e-2,
                       "t-SVDM-II climate-shaped 1024x512x48 FP32, DCT-II, eps=1e-2"),
    "climate-small": ((256, 128, 64), 1e-2,
                      "t-SVDM-II climate-shaped 256x128x64 FP32, DCT-II, eps=1e-2"),
    # 64 uneven CP tensors (n1 128..1024, n2 64..512, n3 8..128), Haar M, even t-SVDM-I
    # k=16 / odd t-SVDM-II eps=1e-3, one graph-captured batch (see run_batch_bench)
    "batch": (None, None, "64 uneven tensors, t-SVDM-I k=16 / t-SVDM-II eps=1e-3, Haar M, "
                          "one CUDA-graph batch"),
    "batch-small": (None, None, "8 uneven tensors (first 8 of the 64-tensor batch), graph"),
    # the mode-3 TTM alone (component benchmark of the transform, tensor cores)
    "ttm": ((1024, 512, 365), None, "mode-3 TTM alone, 1024x512x365 FP32 X, 365x365 M"),
    # the fast orthonormal DCT-II along mode 3 alone, CFD shape (power-of-two n3)
    "dct": ((2048, 256, 512), None, "fast mode-3 DCT-II alone, 2048x256x512 FP32"),
}
FP32_LANES_PER_SM = 128
SMS = 152


def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=5)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--workload", default="climate", choices=sorted(WORKLOADS))
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-e2e", action="store_true")
    ap.add_argument("--no-learned", action="store_true")
    ap.add_argument("--angles", default="fp64", choices=["fp64", "fp32"],
                    help="arithmetic of the slice SVDs' rotation test and angle")
    ap.add_argument("--vectors", default="second_pass", choices=["accumulate", "second_pass"],
                    help="singular vectors in one pass, or the kept ones in a second pass "
                         "(Sec. 3.4's compute-efficient strategy, the default here)")
    ap.add_argument("--quick", action="store_true",
                    help="skip the other configurations (all-FP64 GPU path, CFD, batch, "
                         "the 64x48x16 FP64 case)")
    ap.add_argument("--prec", default="bf16x3", choices=["fp32", "tf32", "bf16x3"],
                    help="TTM arithmetic (the slice SVDs run in FP32 in every mode)")
    ap.add_argument("--fp64-compare", action="store_true",
                    help="batch workload: also time the all-FP64 GPU path on the same inputs")
    return ap.parse_args()


_PROBED = {}


def probe_peaks():
    """Measured FP32 / FP64 CUDA-core and TF32 / BF16 tensor-core rates of this GPU
    (tsvdm_probe_peak: kernels that run only the unit's own instruction on every SM; best
    of three launches each, in TFLOP/s)."""
    if _PROBED:
        return _PROBED
    from paper_2605_16058_gb300 import native as N
    for name, unit, iters in [("fp32_fma", N.PROBE_FP32_FMA, 1 << 20),
                              ("tf32_mma", N.PROBE_TF32_MMA, 1 << 19),
                              ("bf16_mma", N.PROBE_BF16_MMA, 1 << 19),
                              ("fp64_fma", N.PROBE_FP64_FMA, 1 << 13)]:
        _PROBED[name] = max(N.tsvdm_probe_peak(unit, iters) for _ in range(3))
    return _PROBED


def fp32_peak_tflops():
    """The FP32 CUDA-core peak (measured by the probe once the library is loaded on a GPU)."""
    if _PROBED:
        return _PROBED["fp32_fma"], "measured on this GPU (FP32 FMA-loop probe, tsvdm_probe_peak)"
    pk, _ = peaks()
    return (SMS * FP32_LANES_PER_SM * 2 * pk.get("sm_max_mhz", 2070.0) * 1e6 / 1e12,
            "derived: 152 SMs x 128 FP32 lanes x 2 x max SM clock")


def peaks():
    p = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(p):
        with open(p) as f:
            d = json.load(f)
        return d, "measured"
    return {"hbm_gbs": 6800.0, "bf16_tflops": 1900.0, "sm_max_mhz": 2070.0}, "fallback"


class Clocks:
    """nvidia-smi samples during the timed region."""
    Q = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
         "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
         "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_index):
        self.idx = gpu_index
        self.proc = None
        try:
            self.proc = subprocess.Popen(["nvidia-smi", "--query-gpu=" + self.Q,
                                          "--format=csv,noheader,nounits", "-lms", "200",
                                          "-i", str(gpu_index)],
                                         stdout=subprocess.PIPE, stderr=subprocess.DEVNULL,
                                         text=True)
        except Exception:
            self.proc = None

    def stop(self):
        if self.proc is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        self.proc.terminate()
        try:
            out, _ = self.proc.communicate(timeout=5)
        except Exception:
            self.proc.kill()
            out, _ = self.proc.communicate()
        sm, smax, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for line in out.strip().splitlines():
            f = [x.strip() for x in line.split(",")]
            if len(f) < 9:
                continue
            try:
                sm.append(float(f[1]))
                smax.append(float(f[2]))
            except ValueError:
                continue
            for n, v in zip(names, f[5:9]):
                if v.lower().startswith("active"):
                    reasons.add(n)
        return {"sm_mhz": statistics.median(sm) if sm else None,
                "sm_max_mhz": max(smax) if smax else None,
                "reasons": sorted(reasons), "samples": len(sm)}


def max_over_ranks(x, dist, device):
    """The largest of the ranks' values of x (the slowest rank sets the job's time); x
    itself when there is one rank (dist is None)."""
    if dist is None:
        return x
    import torch
    t = torch.tensor([float(x)], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def jacobi_traffic_per_slice():
    """DRAM bytes per slice of the Jacobi kernel from the committed ncu summary, or None
    when the kernel source changed since those counters were taken."""
    import hashlib
    prof = os.path.join(ROOT, "profiles", "jacobi_tc_kernel_climate_1024x512x128.md")
    src = os.path.join(ROOT, "paper_2605_16058_gb300", "csrc", "jacobi.cu")
    try:
        txt = open(prof).read()
        sha = hashlib.sha1(open(src, "rb").read()).hexdigest()
    except OSError:
        return None
    vals = dict(l.split(":", 1) for l in txt.splitlines()
                if l.startswith(("dram_bytes_per_slice:", "jacobi_source_sha1:")))
    if vals.get("jacobi_source_sha1", "").strip() != sha:
        return None
    return float(vals["dram_bytes_per_slice"])


def spread(n, count):
    """`count` slice indices spread evenly over 0 .. n-1 (both ends included)."""
    import numpy as np
    return sorted(set(int(round(x)) for x in np.linspace(0, n - 1, max(1, min(count, n)))))


def cpu_sample(X, M, which, threads):
    """The oracle (FP64, as it stands) on a bounded sample: TTM + SVD of the slices
    `which`, spread over `threads` worker threads.  Returns the time and the oracle's
    U (m x r x len(which)) and singular values (r x len(which))."""
    import oracle
    t0 = time.perf_counter()
    A = oracle.ttm3(X, M, which=list(which))
    U, S, V, _ = oracle.svd_slices(A, threads=threads)
    return time.perf_counter() - t0, U, S


def batch_inputs(count):
    """Seeded inputs of the uneven batch (first `count` of the 64 shapes)."""
    from paper_2605_16058_gb300 import synth
    shapes = synth.batch_shapes()[:count]
    return [(sh, synth.batch_item(i, sh)) for i, sh in enumerate(shapes)]


def batch_measure(args, local, count, fp64_compare):
    """All `count` tensors of the batch in one CUDA graph (TTMs, one persistent Jacobi launch
    over every slice, grouped finalize/selection, emission), autotuned; returns the figures
    of the replay (and of the all-FP64 graph on the same inputs when fp64_compare)."""
    import numpy as np
    import torch
    from paper_2605_16058_gb300 import build, native as N

    build.build()
    torch.cuda.set_device(local)
    items = batch_inputs(count)
    stream = torch.cuda.Stream()

    def make(dtype, prec):
        tdt = torch.float32 if dtype == N.F32 else torch.float64
        descs, ios, keep = [], [], []
        for idx, (sh, it) in enumerate(items):
            n1, n2, n3 = sh
            r = min(n1, n2)
            X = torch.from_numpy(np.ascontiguousarray(it["X"].transpose(2, 1, 0))).to(tdt).cuda()
            M = torch.from_numpy(np.ascontiguousarray(it["M"].T)).to(tdt).cuda()
            if it["mode"] == "fixed":
                descs.append(N.BatchDesc(n1, n2, n3, 0, it["k"], 0.0))
                U = torch.empty(n3, it["k"], n1, dtype=tdt, device="cuda")
                S = torch.empty(n3, it["k"], dtype=tdt, device="cuda")
                V = torch.empty(n3, it["k"], n2, dtype=tdt, device="cuda")
                rk = of = None
            else:
                descs.append(N.BatchDesc(n1, n2, n3, 1, 0, it["eps"]))
                U = torch.empty(n3 * r, n1, dtype=tdt, device="cuda")
                S = torch.empty(n3 * r, dtype=tdt, device="cuda")
                V = torch.empty(n3 * r, n2, dtype=tdt, device="cuda")
                rk = torch.empty(n3, dtype=torch.int32, device="cuda")
                of = torch.empty(n3 + 1, dtype=torch.int64, device="cuda")
            rel = torch.zeros(1, dtype=torch.float64, device="cuda")
            p = lambda t: None if t is None else t.data_ptr()
            ios.append(N.BatchIO(X.data_ptr(), M.data_ptr(), U.data_ptr(), S.data_ptr(),
                                 V.data_ptr(), p(rk), p(of), rel.data_ptr()))
            keep.append((X, M, U, S, V, rk, of, rel))
        torch.cuda.synchronize()
        b = N.tsvdm_batch_create(descs, dtype, prec, stream)
        return b, ios, keep

    def timed(b, steps, warmup):
        for _ in range(warmup):
            N.tsvdm_batch_launch(b)
        torch.cuda.synchronize()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        for _ in range(steps):
            N.tsvdm_batch_launch(b)
        e1.record(stream)
        torch.cuda.synchronize()
        return e0.elapsed_time(e1) / steps

    in_bytes = sum(sh[0] * sh[1] * sh[2] * 4 for sh, _ in items)
    nslices = sum(sh[2] for sh, _ in items)
    b, ios, keep = make(N.F32, N.PRECISIONS[args.prec])
    choice = N.tsvdm_batch_tune(b, ios)
    N.tsvdm_batch_capture(b, ios)
    clk = Clocks(local)
    ms = timed(b, args.steps, max(3, args.warmup))
    clocks = clk.stop()
    st, sweeps, rots = N.tsvdm_batch_status(b)
    alg, mp_sum = 0.0, 0.0
    for sh, _ in items:
        m_, p_ = max(sh[0], sh[1]), min(sh[0], sh[1])
        alg += sh[2] * 3.0 * m_ * p_ * (p_ - 1)       # dots of one sweep, every slice
        mp_sum += sh[2] * (m_ + p_)
    mean_sw = sweeps / nslices
    # algorithmic flops: dots of every executed sweep (mean sweeps per slice) plus
    # 6 (m + p) per applied rotation (slice-averaged m + p)
    alg_flops = alg * mean_sw + rots * 6.0 * mp_sum / nslices
    fp32_peak, fp32_src = fp32_peak_tflops()
    rels = [float(k[7].item()) for k in keep]
    out = {
        "ms_per_step": ms, "value": in_bytes / (ms * 1e-3) / 1e9, "unit": "GB/s",
        "slices_per_s": nslices / (ms * 1e-3), "tensors": len(items), "slices": nslices,
        "input_bytes": in_bytes, "status": int(st), "jacobi_sweeps_mean": mean_sw,
        "autotuned": choice,
        "max_rel_err_tol_items": max(r for (sh, it), r in zip(items, rels) if it["mode"] == "tol"),
        "roofline": {"bound": "alu", "kernel": "jacobi", "unit": "TFLOP/s", "peak": fp32_peak,
                     "peak_source": fp32_src, "kernel_ms": choice["jacobi_ms"],
                     "algorithmic_flops": alg_flops,
                     "achieved": alg_flops / (choice["jacobi_ms"] * 1e-3) / 1e12},
        "clocks": clocks, "gpu_launches": N.tsvdm_batch_graph_kernels(b) * args.steps,
    }
    out["roofline"]["frac"] = out["roofline"]["achieved"] / fp32_peak
    N.tsvdm_batch_destroy(b)
    if fp64_compare:
        b64, ios64, keep64 = make(N.F64, N.P_FP64)
        N.tsvdm_batch_run(b64, ios64)
        N.tsvdm_batch_capture(b64, ios64)
        ms64 = timed(b64, 1, 0)
        rels64 = [float(k[7].item()) for k in keep64]
        out["fp64_gpu"] = {"ms_per_step": ms64, "speedup_of_fp32_batch": ms64 / ms,
                           "max_abs_rel_err_diff": max(abs(a - c) for a, c in zip(rels, rels64))}
        N.tsvdm_batch_destroy(b64)
        del keep64
    del keep
    torch.cuda.empty_cache()
    return out


def run_batch_bench(args, world, rank, local):
    """The batch workload as the benchmark's line (input GB/s of one graph replay)."""
    count = 64 if args.workload == "batch" else 8
    b = batch_measure(args, local, count, args.fp64_compare)
    line = {
        "metric": METRIC, "value": b["value"], "unit": "GB/s", "n_gpus": 1,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": b["ms_per_step"],
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f32",
        "data": "synthetic", "slices_per_s": b["slices_per_s"], "ttm_precision": args.prec,
        "config": {"workload": WORKLOADS[args.workload][2], "tensors": b["tensors"],
                   "slices": b["slices"], "input_bytes": b["input_bytes"], "status": b["status"],
                   "jacobi_sweeps_mean": b["jacobi_sweeps_mean"], "autotuned": b["autotuned"],
                   "max_rel_err_tol_items": b["max_rel_err_tol_items"]},
        "roofline": b["roofline"], "clocks": b["clocks"], "gpu_launches": b["gpu_launches"],
    }
    if "fp64_gpu" in b:
        line["fp64_gpu_ms_per_step"] = b["fp64_gpu"]["ms_per_step"]
        line["speedup_vs_fp64_gpu"] = b["fp64_gpu"]["speedup_of_fp32_batch"]
    print(json.dumps(line), flush=True)


def run_ttm_bench(args, local):
    """The forward mode-3 TTM alone: input GB/s of Y = X x_3 M in the chosen precision,
    with its HBM roofline (2 P n + n^2 elements moved) and, for BF16x3, tensor work."""
    import numpy as np
    import torch
    from paper_2605_16058_gb300 import build, synth
    from paper_2605_16058_gb300.tsvdm import Plan
    build.build()
    torch.cuda.set_device(local)
    (n1, n2, n3), _, desc = WORKLOADS[args.workload]
    g = torch.Generator(device="cuda").manual_seed(7)
    X = torch.randn(n3, n2, n1, device="cuda", generator=g)
    M = torch.from_numpy(synth.haar_orthogonal(n3, np.random.default_rng(7))
                         .astype(np.float32)).cuda()
    Y = torch.empty_like(X)
    fast = args.workload == "dct"
    plan = Plan(n1, n2, n3, dtype=torch.float32, prec="fp32" if fast else args.prec)
    if fast:
        plan.set_transform("dct2")
    for _ in range(max(3, args.warmup)):
        plan.transform(X, M, out=Y)
    torch.cuda.synchronize()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record()
    for _ in range(args.steps):
        plan.transform(X, M, out=Y)
    e1.record()
    torch.cuda.synchronize()
    ms = e0.elapsed_time(e1) / args.steps
    P = n1 * n2
    byts = (2 * P * n3 + n3 * n3) * 4
    pk, src = peaks()
    gbs = byts / (ms * 1e-3) / 1e9
    line = {"metric": "mode-3 %s input GB/s" % ("DCT-II" if fast else "TTM"),
            "value": P * n3 * 4 / (ms * 1e-3) / 1e9,
            "unit": "GB/s", "n_gpus": 1, "steps": args.steps, "warmup": args.warmup,
            "ms_per_step": ms, "higher_is_better": True, "dtype": "f32",
            "ttm_precision": "fft-fp32" if fast else args.prec, "data": "synthetic",
            "config": {"workload": desc},
            "roofline": {"bound": "hbm", "achieved": gbs, "peak": pk["hbm_gbs"], "unit": "GB/s",
                         "frac": gbs / pk["hbm_gbs"], "peak_source": "of " + src}}
    print(json.dumps(line), flush=True)
    plan.close()


def run_reference(args, wl):
    import numpy as np
    import oracle
    from paper_2605_16058_gb300 import synth
    shape, eps, desc = wl if wl[0] else ((None, None, None), None, wl[2])
    n1, n2 = shape[0], shape[1]
    cores = os.cpu_count() or 1
    if n1 is None:                       # batch: sample slices of the first tensor
        (n1, n2, n3), it = batch_inputs(1)[0]
        X, M = it["X"], it["M"]
    else:
        n3 = int(np.prod(shape[2:]))
        X = synth.climate(shape=(n1, n2, n3), seed=1)
        # d-way: the transform of every trailing mode equals one mode-3 product of the
        # flattened trailing modes with the Kronecker product of the per-mode matrices
        M = synth.dct2_matrix(shape[2])
        for d in shape[3:]:
            M = np.kron(synth.dct2_matrix(d), M)
    ns = min(cores, n3)
    oracle.build_oracle()
    for _ in range(max(0, args.warmup)):
        A = oracle.ttm3(X, M, which=[0])
    which = spread(n3, ns)
    times = [cpu_sample(X, M, which, cores)[0] for _ in range(args.steps)]
    t = statistics.mean(times)
    bytes_per_slice = n1 * n2 * 4
    gbs = ns * bytes_per_slice / t / 1e9
    line = {
        "impl": "reference", "metric": METRIC, "value": gbs, "unit": "GB/s", "n_gpus": args.gpus,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": t * 1e3,
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
        "data": "synthetic", "slices_per_s": ns / t,
        "config": {"workload": desc, "sample": "TTM + one-sided Jacobi SVD of %d of the %d "
                   "slices per step (spread over the spectrum)" % (ns, n3)},
        "cpu_baseline": {"value": gbs, "unit": "GB/s", "cores": cores, "kind": "oracle",
                         "sample": "%d slices of %dx%d per step" % (ns, n1, n2)},
        "e2e": {"value": gbs, "unit": "GB/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }
    print(json.dumps(line), flush=True)


def matched_error(plan, X, M, ranks, which, S_o, r):
    """The north star's "matched" test on the oracle's sample: over the sampled slices, the
    relative truncation error at the GPU's ranks from the GPU's singular values against the
    same from the oracle's (FP64 TTM + Jacobi SVD of each slice), within 1e-5."""
    import numpy as np
    from paper_2605_16058_gb300 import native
    full = plan.fixed_rank(X, M, r, rel_err=False)
    S_g = full["S"].double().cpu().numpy().T          # r x n3
    rk = ranks.cpu().numpy()
    dg = tg = do = to = 0.0
    for q, i in enumerate(which):
        dg += float(np.sum(S_g[rk[i]:, i] ** 2))
        tg += float(np.sum(S_g[:, i] ** 2))
        do += float(np.sum(S_o[rk[i]:, q] ** 2))
        to += float(np.sum(S_o[:, q] ** 2))
    eg, eo = float(np.sqrt(dg / tg)), float(np.sqrt(do / to))
    smax = float(S_g.max())
    return {"sample_slices": len(which), "rel_err_gpu": eg, "rel_err_oracle": eo,
            "abs_diff": abs(eg - eo), "tol": 1e-5, "matched": abs(eg - eo) <= 1e-5,
            "max_sigma_err_over_sigma_max": float(max(
                np.max(np.abs(S_g[:, i] - S_o[:, q])) for q, i in enumerate(which)) / smax)}


def fp64_climate(Xh, Mh, shape, eps, ms_mixed, rel_mixed, stream):
    """The all-FP64 GPU path (FP64 TTM, FP64 Jacobi, FP64 selection) on the same climate
    input: one timed call (several seconds), against the mixed-precision step."""
    import torch
    from paper_2605_16058_gb300 import native
    from paper_2605_16058_gb300.tsvdm import Plan
    n1, n2, n3 = shape
    r = min(n1, n2)
    X = Xh.double().cuda()
    M = Mh.double().cuda()
    plan = Plan(n1, n2, n3, dtype=torch.float64, orthogonal=True, stream=stream)
    cap = n3 * r
    ranks = torch.empty(n3, dtype=torch.int32, device="cuda")
    offs = torch.empty(n3 + 1, dtype=torch.int64, device="cuda")
    U = torch.empty(cap, n1, dtype=torch.float64, device="cuda")
    S = torch.empty(cap, dtype=torch.float64, device="cuda")
    V = torch.empty(cap, n2, dtype=torch.float64, device="cuda")
    torch.cuda.synchronize()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    tot, rel, st = native.tsvdm_tolerance(plan.handle, X, M, eps, ranks, offs, U, S, V, cap)
    e1.record(stream)
    torch.cuda.synchronize()
    ms = e0.elapsed_time(e1)
    sweeps, _ = native.tsvdm_plan_stats(plan.handle)
    plan.close()
    del X, M, U, S, V
    torch.cuda.empty_cache()
    return {"ms_per_step": ms, "value": n1 * n2 * n3 * 4 / (ms * 1e-3) / 1e9, "unit": "GB/s",
            "input": "the same FP32 climate tensor, cast to FP64", "rel_err": rel,
            "total_rank": int(tot), "status": int(st), "jacobi_sweeps_mean": sweeps / n3,
            "speedup_of_mixed": ms / ms_mixed, "rel_err_diff_vs_mixed": abs(rel - rel_mixed),
            "timing": "one call (CUDA events), after the mixed-precision runs"}


def cfd_measure(args, stream):
    """CFD-shaped 2048 x 256 x 512 FP32, DCT-II, t-SVDM-I k = 32, with the BF16x3 and TF32
    tensor-core TTMs (FP32 Jacobi), against the all-FP64 GPU run on the same data and the
    FP64 oracle on sampled slices: time, TTM roofline, error per output."""
    import numpy as np
    import torch
    from paper_2605_16058_gb300 import native, synth
    from paper_2605_16058_gb300.tsvdm import Plan
    n1, n2, n3, k = 2048, 256, 512, 32
    P = n1 * n2
    Xn = synth.cfd(shape=(n1, n2, n3), seed=3)
    Mn = synth.dct2_matrix(n3).astype(np.float32)
    X = torch.from_numpy(np.ascontiguousarray(Xn.transpose(2, 1, 0))).cuda()
    M = torch.from_numpy(np.ascontiguousarray(Mn.T)).cuda()
    cores = os.cpu_count() or 1
    which = spread(n3, cores)
    t_o, U_o, S_o = cpu_sample(Xn, Mn.astype(np.float64), which, cores)
    pk, src = peaks()
    pr = probe_peaks()
    out = {"workload": "CFD-shaped 2048x256x512 FP32 (40 travelling waves, 1e-4 noise), "
                       "DCT-II, t-SVDM-I k=32", "oracle_sample_slices": len(which)}
    res = {}
    for prec in ("bf16x3", "tf32", "dct2", "fp64"):
        dt = torch.float64 if prec == "fp64" else torch.float32
        Xp, Mp = (X.double(), M.double()) if prec == "fp64" else (X, M)
        plan = Plan(n1, n2, n3, dtype=dt, prec="fp32" if prec == "dct2" else prec,
                    orthogonal=True, stream=stream)
        if prec == "dct2":
            plan.set_transform("dct2")        # the fast DCT-II kernel instead of the TTM
        U = torch.empty(n3, k, n1, dtype=dt, device="cuda")
        S = torch.empty(n3, k, dtype=dt, device="cuda")
        V = torch.empty(n3, k, n2, dtype=dt, device="cuda")
        steps, warm = (1, 0) if prec == "fp64" else (args.steps, max(3, args.warmup))
        for _ in range(warm):
            native.tsvdm_fixed_rank(plan.handle, Xp, Mp, k, U, S, V, 0, True)
        native.tsvdm_plan_profile(plan.handle, 1)
        torch.cuda.synchronize()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        stage = []
        e0.record(stream)
        for _ in range(steps):
            rel, st = native.tsvdm_fixed_rank(plan.handle, Xp, Mp, k, U, S, V, 0, True)
            stage.append(native.tsvdm_plan_profile_read(plan.handle)[0])
        e1.record(stream)
        torch.cuda.synchronize()
        ms = e0.elapsed_time(e1) / steps
        ttm_ms = statistics.mean(s_["ttm"] for s_ in stage)
        jac_ms = statistics.mean(s_["jacobi"] for s_ in stage)
        d = {"ms_per_step": ms, "value": P * n3 * 4 / (ms * 1e-3) / 1e9, "unit": "GB/s",
             "slices_per_s": n3 / (ms * 1e-3), "rel_err": rel, "status": int(st),
             "ttm_ms": ttm_ms, "jacobi_ms": jac_ms, "steps": steps}
        byts = (2 * P * n3 + n3 * n3) * (8 if prec == "fp64" else 4)
        d["ttm_hbm"] = {"achieved": byts / (ttm_ms * 1e-3) / 1e9, "peak": pk["hbm_gbs"],
                        "unit": "GB/s", "frac": byts / (ttm_ms * 1e-3) / 1e9 / pk["hbm_gbs"],
                        "peak_source": "of " + src}
        if prec in ("bf16x3", "tf32"):
            terms = 3 if prec == "bf16x3" else 1
            flops = terms * 2.0 * P * n3 * n3
            peak = pr["bf16_mma"] if prec == "bf16x3" else pr["tf32_mma"]
            d["ttm_tensor"] = {"achieved": flops / (ttm_ms * 1e-3) / 1e12, "peak": peak,
                               "unit": "TFLOP/s", "frac": flops / (ttm_ms * 1e-3) / 1e12 / peak,
                               "flops": flops, "peak_source": "measured on this GPU (%s MMA "
                               "probe)" % ("BF16" if prec == "bf16x3" else "TF32"),
                               "note": "BF16x3 counts its three BF16 products"}
        Sg = S.double().cpu().numpy().T           # k x n3
        Ug = U.double().cpu().numpy().transpose(2, 1, 0)   # n1 x k x n3
        smax = float(Sg.max())
        sig_err = max(float(np.max(np.abs(Sg[:, i] - S_o[:k, q]))) for q, i in enumerate(which))
        pd, npd = 0.0, 0
        for q, i in enumerate(which):
            if S_o[k - 1, q] - S_o[k, q] > 1e-2 * smax:
                a, b = U_o[:, :k, q], Ug[:, :, i]
                pd = max(pd, float(np.linalg.norm(a @ a.T - b @ b.T)))
                npd += 1
        d["vs_oracle"] = {"sigma_max_abs_err_over_sigma_max": sig_err / smax,
                          "U_projector_max_diff": pd if npd else None,
                          "U_projector_slices": npd,
                          "note": "projectors of the rank-k subspace where the gap at k "
                                  "exceeds 1e-2 sigma_max"}
        res[prec] = (d, Sg)
        plan.close()
        del U, S, V
        torch.cuda.empty_cache()
    S64 = res["fp64"][1]
    for prec in ("bf16x3", "tf32", "dct2", "fp64"):
        d, Sg = res[prec]
        if prec != "fp64":
            d["vs_fp64_gpu"] = {"rel_err_diff": abs(d["rel_err"] - res["fp64"][0]["rel_err"]),
                                "sigma_max_abs_err_over_sigma_max":
                                    float(np.max(np.abs(Sg - S64)) / S64.max()),
                                "speedup": res["fp64"][0]["ms_per_step"] / d["ms_per_step"]}
        out[prec] = d
    return out


def config0_measure():
    """The 64 x 48 x 16 FP64 t-SVDM-I case (k = 8, DCT-II): GPU call time (median of 20
    after 3 warm-ups) and error, the oracle single-threaded beside it."""
    import numpy as np
    import torch
    import oracle
    from paper_2605_16058_gb300 import synth
    from paper_2605_16058_gb300.tsvdm import Plan
    c = synth.smoke_case()
    Xn, Mn, k = c["X"], c["M"], c["k"]
    n1, n2, n3 = Xn.shape
    X = torch.from_numpy(np.ascontiguousarray(Xn.transpose(2, 1, 0))).cuda()
    M = torch.from_numpy(np.ascontiguousarray(np.asarray(Mn).T)).cuda()
    plan = Plan(n1, n2, n3, dtype=torch.float64)
    for _ in range(3):
        out = plan.fixed_rank(X, M, k)
    ts = []
    for _ in range(20):
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record()
        out = plan.fixed_rank(X, M, k)
        e1.record()
        torch.cuda.synchronize()
        ts.append(e0.elapsed_time(e1))
    plan.close()
    to = []
    for _ in range(3):
        t0 = time.perf_counter()
        ref = oracle.fixed_rank(Xn, Mn, k, threads=1)
        to.append((time.perf_counter() - t0) * 1e3)
    return {"workload": "64x48x16 FP64 CP tensor (12 terms), DCT-II, t-SVDM-I k=8",
            "gpu_ms": statistics.median(ts), "rel_err_gpu": out["rel_err"],
            "oracle_ms_single_thread": statistics.median(to), "rel_err_oracle": ref["rel_err"],
            "rel_err_diff": abs(out["rel_err"] - ref["rel_err"]),
            "timing": "GPU: CUDA events around the call (it synchronises for rel_err)"}


def main():
    args = parse()
    wl = WORKLOADS[args.workload]
    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    if args.impl == "reference":
        if rank == 0:
            run_reference(args, wl)
        return
    if args.workload.startswith("batch"):
        run_batch_bench(args, world, rank, local)
        return
    if args.workload in ("ttm", "dct"):
        run_ttm_bench(args, local)
        return

    import numpy as np
    import torch
    from paper_2605_16058_gb300 import build, native, synth
    from paper_2605_16058_gb300.tsvdm import Plan

    build.build()
    torch.cuda.set_device(local)
    dist = None
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl", device_id=torch.device("cuda", local))
    probes = probe_peaks()

    shape, eps, desc = wl
    n1, n2 = shape[0], shape[1]
    n3 = int(np.prod(shape[2:]))
    r = min(n1, n2)
    Xn = synth.climate(shape=(n1, n2, n3), seed=1)   # d-way: the same field, trailing modes split
    stream = torch.cuda.current_stream()
    if len(shape) == 3:
        Mn = synth.dct2_matrix(n3)
        Mh = torch.from_numpy(np.ascontiguousarray(Mn.T.astype(np.float32))).pin_memory()
        plan = Plan(n1, n2, n3, dtype=torch.float32, prec=args.prec, orthogonal=True,
                    stream=stream)
        plan.set_angle_precision(args.angles)
        plan.set_vectors(args.vectors)
        msizes = [n3]
    else:
        # one DCT-II per trailing mode, concatenated; the CPU baseline uses the equivalent
        # mode-3 transform by their Kronecker product
        msizes = list(shape[2:])
        Ms = [synth.dct2_matrix(d) for d in msizes]
        Mh = torch.cat([torch.from_numpy(np.ascontiguousarray(Mk.T.astype(np.float32))).reshape(-1)
                        for Mk in Ms]).pin_memory()
        Mn = Ms[0]
        for Mk in Ms[1:]:
            Mn = np.kron(Mk, Mn)
        plan = Plan.dway(shape, dtype=torch.float32, prec=args.prec, orthogonal=True,
                         stream=stream)
    Xh = torch.from_numpy(np.ascontiguousarray(Xn.transpose(2, 1, 0))).pin_memory()
    X = Xh.cuda()
    M = Mh.cuda()
    cap = n3 * r
    ranks = torch.empty(n3, dtype=torch.int32, device="cuda")
    offs = torch.empty(n3 + 1, dtype=torch.int64, device="cuda")
    U = torch.empty(cap, n1, device="cuda")
    S = torch.empty(cap, device="cuda")
    V = torch.empty(cap, n2, device="cuda")

    def step():
        return native.tsvdm_tolerance(plan.handle, X, M, eps, ranks, offs, U, S, V, cap)

    for _ in range(max(3, args.warmup)):
        tot, rel, st = step()
    native.tsvdm_plan_profile(plan.handle, 1)
    clk = Clocks(local)
    if dist:
        dist.barrier()
    torch.cuda.synchronize()
    e0 = torch.cuda.Event(enable_timing=True)
    e1 = torch.cuda.Event(enable_timing=True)
    stage_ms = []
    launches = 0
    e0.record(stream)
    for _ in range(args.steps):
        tot, rel, st = step()
        ms, nl = native.tsvdm_plan_profile_read(plan.handle)
        stage_ms.append(ms)
        launches += nl
    e1.record(stream)
    torch.cuda.synchronize()
    if dist:
        dist.barrier()
    clocks = clk.stop()
    ms_step = max_over_ranks(e0.elapsed_time(e1) / args.steps, dist, "cuda")
    ranks_timed = ranks.clone()
    sweeps, rots = native.tsvdm_plan_stats(plan.handle)
    native.tsvdm_plan_profile(plan.handle, 0)
    in_bytes = n1 * n2 * n3 * 4
    value = world * in_bytes / (ms_step * 1e-3) / 1e9
    slices_s = world * n3 / (ms_step * 1e-3)

    # the other vector strategy on the same plan and input (one timed call after one warm-up)
    other = "accumulate" if args.vectors == "second_pass" else "second_pass"
    alt = None
    if len(shape) == 3 and not args.quick:
        plan.set_vectors(other)
        step()
        torch.cuda.synchronize()
        a0, a1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        a0.record(stream)
        tot_a, rel_a, _ = step()
        a1.record(stream)
        torch.cuda.synchronize()
        alt = {"vectors": other, "ms_per_step": a0.elapsed_time(a1), "rel_err": rel_a,
               "total_rank": int(tot_a)}
        plan.set_vectors(args.vectors)
        step()

    # end to end through the C ABI with pinned host buffers
    e2e = None
    if not args.no_e2e:
        Uh = torch.empty(cap, n1).pin_memory()
        Sh = torch.empty(cap).pin_memory()
        Vh = torch.empty(cap, n2).pin_memory()
        rh = torch.empty(n3, dtype=torch.int32).pin_memory()
        oh = torch.empty(n3 + 1, dtype=torch.int64).pin_memory()
        native.tsvdm_tolerance(plan.handle, Xh, Mh, eps, rh, oh, Uh, Sh, Vh, cap)
        torch.cuda.synchronize()
        if dist:
            dist.barrier()
        t0 = time.perf_counter()
        for _ in range(args.steps):
            tot_h, _, _ = native.tsvdm_tolerance(plan.handle, Xh, Mh, eps, rh, oh, Uh, Sh, Vh, cap)
        torch.cuda.synchronize()
        te = max_over_ranks((time.perf_counter() - t0) / args.steps, dist, "cuda")
        d2h = tot_h * (n1 + n2 + 1) * 4 + n3 * 4 + (n3 + 1) * 8
        e2e = {"value": world * in_bytes / te / 1e9, "unit": "GB/s",
               "h2d_bytes_per_step": in_bytes + M.numel() * 4, "d2h_bytes_per_step": int(d2h),
               "ms_per_step": te * 1e3}

    # back-transform of the packed t-SVDM-II factors to the original domain (per-slice
    # U S V^T, then x3 M^{-1}): CUDA events around the C-ABI call on the plan's stream.
    # Algorithmic bytes: the factors read once, the n1 x n2 x n3 result written once.
    native.tsvdm_plan_profile(plan.handle, 0)
    Xk = torch.empty_like(X)
    plan.reconstruct(U, S, V, M, offsets=offs, out=Xk)
    torch.cuda.synchronize()
    r0 = torch.cuda.Event(enable_timing=True)
    r1 = torch.cuda.Event(enable_timing=True)
    r0.record(stream)
    for _ in range(3):
        plan.reconstruct(U, S, V, M, offsets=offs, out=Xk)
    r1.record(stream)
    torch.cuda.synchronize()
    rec_ms = r0.elapsed_time(r1) / 3
    rec_bytes = (int(tot) * (n1 + n2 + 1) + n1 * n2 * n3 + M.numel()) * 4
    rec_rel = float(((Xk - X).pow(2).sum(dtype=torch.float64) /
                     X.pow(2).sum(dtype=torch.float64)).sqrt())
    del Xk

    # data-driven M (Sec. 2.2: transposed left singular vectors of the mode-3 unfolding):
    # its upfront cost, and the t-SVDM-II result it gives on the same data and eps
    data_m = None
    if len(shape) == 3:
        Md = torch.empty(n3, n3, device="cuda")
        plan.data_transform(X, out=Md)                      # first call sets up its plan
        torch.cuda.synchronize()
        d0, d1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        d0.record(stream)
        plan.data_transform(X, out=Md)
        d1.record(stream)
        torch.cuda.synchronize()
        tot_d, rel_d, _ = native.tsvdm_tolerance(plan.handle, X, Md, eps, ranks, offs, U, S, V, cap)
        data_m = {"transform_ms": d0.elapsed_time(d1), "total_rank": int(tot_d),
                  "rel_err": rel_d, "total_rank_dct": int(tot),
                  "compression_ratio": n1 * n2 * n3 / max(int(tot_d) * (n1 + n2 + 1), 1),
                  "compression_ratio_dct": n1 * n2 * n3 / max(int(tot) * (n1 + n2 + 1), 1)}
        del Md

    # roofline of the dominant kernel (batched Jacobi), live CUDA-event duration
    jac_ms = statistics.mean(s["jacobi"] for s in stage_ms)
    m_, p_ = max(n1, n2), min(n1, n2)
    alg_flops = sweeps * 3.0 * m_ * p_ * (p_ - 1) + rots * 6.0 * (m_ + p_)
    pk, src = peaks()
    fp32_peak, fp32_src = fp32_peak_tflops()
    achieved = alg_flops / (jac_ms * 1e-3) / 1e12
    ttm_ms = statistics.mean(s["ttm"] for s in stage_ms)
    # one read and one write of the tensor per transformed mode (plus each matrix)
    ttm_gbs = sum(2 * n1 * n2 * n3 * 4 + d * d * 4 for d in msizes) / (ttm_ms * 1e-3) / 1e9
    stages = {k: round(statistics.mean(s[k] for s in stage_ms), 3) for k in native.STAGES}

    line = {
        "metric": METRIC, "value": value, "unit": "GB/s", "n_gpus": world, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": ms_step, "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None, "dtype": "f32", "data": "synthetic",
        "slices_per_s": slices_s, "ttm_precision": args.prec,
        "config": {"workload": desc, "parallelism": "replicas" if world > 1 else "single",
                   "l2": "input %.0f MB%s" % (n1 * n2 * n3 * 4 / 1e6, " > 129 MB L2, no flush"
                                               if n1 * n2 * n3 * 4 > 129e6 else ""), "total_rank": int(tot),
                   "rel_err": rel, "status": int(st),
                   "jacobi_sweeps_mean": sweeps / n3, "jacobi_rotations": int(rots)},
        "roofline": {"bound": "alu", "kernel": "jacobi", "achieved": achieved,
                     "peak": fp32_peak, "unit": "TFLOP/s", "frac": achieved / fp32_peak,
                     "traffic": (None if jacobi_traffic_per_slice() is None
                                 else jacobi_traffic_per_slice() * n3),
                     "traffic_note": "ncu dram bytes per slice (1024x512x128 capture) x slices",
                     "peak_source": fp32_src,
                     "note": "classical one-sided Jacobi flop count (3 m p (p-1) per sweep + "
                             "6 (m + p) per rotation) against the FP32 CUDA-core peak; the "
                             "Gram and rotation apply run as split products on tcgen05, the "
                             "inner Gram sweeps on the CUDA cores",
                     "algorithmic_flops": alg_flops, "kernel_ms": jac_ms},
        "stages_ms": stages,
        "ttm_roofline": {"bound": "hbm", "achieved": ttm_gbs, "peak": pk["hbm_gbs"],
                         "unit": "GB/s", "frac": ttm_gbs / pk["hbm_gbs"],
                         "peak_source": "of %s" % src},
        "gpu_launches": int(launches),
        "vectors": args.vectors, "angles": args.angles, "other_vectors": alt,
        "clocks": clocks,
        "e2e": e2e,
        "data_driven_m": data_m,
        "reconstruct": {"ms": rec_ms, "rel_err": rec_rel,
                        "slice_product_flops": 2.0 * n1 * n2 * int(tot),
                        "roofline": {"bound": "hbm",
                                     "achieved": rec_bytes / (rec_ms * 1e-3) / 1e9,
                                     "peak": pk["hbm_gbs"], "unit": "GB/s",
                                     "frac": rec_bytes / (rec_ms * 1e-3) / 1e9 / pk["hbm_gbs"],
                                     "algorithmic_bytes": rec_bytes,
                                     "peak_source": "of %s" % src}},
    }
    if not args.no_learned:
        # fwd+bwd of the learned Cayley transform: crystal-shaped 512x256x128 FP32, k = 16,
        # 50 Adam steps at lr 1e-3 (every step: Cayley, t-SVDM-I, backward, adjoint, Adam)
        from paper_2605_16058_gb300.learn import CayleyTrainer
        cs = (512, 256, 128)
        Xc = synth.crystal(shape=cs, seed=4)
        Xcd = torch.from_numpy(np.ascontiguousarray(Xc.transpose(2, 1, 0))).cuda()
        M0 = torch.from_numpy(np.ascontiguousarray(synth.dct2_matrix(cs[2]).T.astype(np.float32))).cuda()
        runs = {}
        for warm in (False, True):
            tr = CayleyTrainer(Xcd, M0, cs, 16, lr=1e-3, warm_start=warm)
            tr.train(3, record=False)                    # warm-up (3 steps, then restart)
            tr = CayleyTrainer(Xcd, M0, cs, 16, lr=1e-3, warm_start=warm)
            runs[warm] = tr.train(50)
        (lc, ms_c), (lw, ms_w) = runs[False], runs[True]
        split = tr.part_split(5)
        # compressibility at a matched tolerance: t-SVDM-II of the crystal tensor with the
        # learned transform and with DCT-II (the starting point), eps = 1e-2
        Ml = tr.current_transform()
        pc = Plan(*cs, dtype=torch.float32, prec=args.prec, orthogonal=True)
        crs = {}
        for name, Mx in (("learned", Ml), ("dct2", M0)):
            oc = pc.tolerance(Xcd, Mx, 1e-2)
            crs[name] = {"total_rank": int(oc["total_rank"]), "rel_err": oc["rel_err"],
                         "compression_ratio": cs[0] * cs[1] * cs[2] /
                         max(int(oc["total_rank"]) * (cs[0] + cs[1] + 1), 1)}
        pc.close()
        line["learned_m"] = {"workload": "crystal-shaped 512x256x128 FP32, Cayley(DCT-II), "
                                         "k=16, 50 Adam steps lr=1e-3; slice SVDs warm-started "
                                         "from the previous step's right vectors",
                             "fwd_bwd_ms_per_step": ms_w, "step_split_ms": split,
                             "tsvdm2_eps_1e-2": crs, "loss_first": lw[0],
                             "loss_last": lw[-1], "cold_start_ms_per_step": ms_c,
                             "cold_start_loss_last": lc[-1]}
    line["peaks_measured"] = dict(
        {k + "_tflops": v for k, v in probes.items()},
        how="tsvdm_probe_peak: FP32/FP64 FMA loops (8 chains per thread, full occupancy) and "
            "tcgen05 kind::tf32 / kind::f16 M=128 N=256 MMA loops (one CTA per SM); best of 3")
    if rank == 0 and world == 1 and not args.no_cpu_baseline:
        cores = os.cpu_count() or 1
        which = spread(n3, cores)
        ns = len(which)
        tcpu, U_o, S_o = cpu_sample(Xn, Mn, which, cores)
        cgbs = ns * n1 * n2 * 4 / tcpu / 1e9
        line["cpu_baseline"] = {"value": cgbs, "unit": "GB/s", "cores": cores, "kind": "oracle",
                                "sample": "FP64 TTM + one-sided Jacobi SVD of %d of the %d "
                                          "slices spread over the spectrum (%.1f s)"
                                          % (ns, n3, tcpu)}
        if len(shape) == 3:
            line["matched"] = matched_error(plan, X, M, ranks_timed, which, S_o, r)
    if rank == 0 and world == 1 and not args.quick and len(shape) == 3:
        line["fp64_gpu"] = fp64_climate(Xh, Mh, (n1, n2, n3), eps, ms_step, rel, stream)
        line["cfd"] = cfd_measure(args, stream)
        line["batch"] = batch_measure(args, local, 64, True)
        line["config0"] = config0_measure()
    if rank == 0:
        print(json.dumps(line), flush=True)
    plan.close()
    if dist:
        dist.destroy_process_group()


if __name__ == "__main__":
    main()
