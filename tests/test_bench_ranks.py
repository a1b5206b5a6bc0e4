"""The benchmark's multi-rank host logic, on CPU. Under torchrun the bench runs one
independent replica per GPU (there is no data-path collective):
- the job's time is the slowest rank's time, every rank reduced to it (checked with world
  size 2 over gloo);
- with one rank the reduction is the value itself;
- the reference arm runs and prints on rank 0 alone."""
import importlib.util
import os
import socket
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _bench():
    spec = importlib.util.spec_from_file_location("bench_under_test",
                                                  os.path.join(ROOT, "bench.py"))
    mod = importlib.util.module_from_spec(spec)
    spec.loader.exec_module(mod)
    return mod


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank_main(rank, world, port, queue):
    import torch.distributed as dist
    dist.init_process_group("gloo", init_method="tcp://127.0.0.1:%d" % port, rank=rank,
                            world_size=world)
    try:
        b = _bench()
        mine = 1.5 + rank                           # rank 1 is the slow one
        queue.put((rank, b.max_over_ranks(mine, dist, "cpu")))
        dist.barrier()
    finally:
        dist.destroy_process_group()


def test_slowest_rank_time_over_gloo_world_two():
    import torch.multiprocessing as mp
    ctx = mp.get_context("spawn")
    queue = ctx.SimpleQueue()
    port = _free_port()
    procs = [ctx.Process(target=_rank_main, args=(r, 2, port, queue)) for r in range(2)]
    for p in procs:
        p.start()
    for p in procs:
        p.join(timeout=120)
    assert all(p.exitcode == 0 for p in procs), [p.exitcode for p in procs]
    got = sorted(queue.get() for _ in range(2))
    assert got == [(0, 2.5), (1, 2.5)]


def test_one_rank_reduction_is_the_value_itself():
    assert _bench().max_over_ranks(3.25, None, "cuda") == 3.25


def test_reference_arm_runs_on_rank_zero_only(monkeypatch, capsys):
    b = _bench()
    calls = []
    monkeypatch.setattr(b, "run_reference", lambda args, wl: calls.append(wl[2]))
    monkeypatch.setattr(sys, "argv", ["bench.py", "--impl", "reference", "--gpus", "2",
                                      "--steps", "3", "--warmup", "3"])
    monkeypatch.setenv("WORLD_SIZE", "2")
    monkeypatch.setenv("LOCAL_RANK", "1")
    monkeypatch.setenv("RANK", "1")
    b.main()
    assert calls == [] and capsys.readouterr().out == ""
    monkeypatch.setenv("LOCAL_RANK", "0")
    monkeypatch.setenv("RANK", "0")
    b.main()
    assert len(calls) == 1
