"""The N > 1 host logic of bench.py on CPU with two gloo ranks: each rank
searches its own instance (weak scaling, no data-path collective), and the
job's work is the sum over ranks while its time is the slowest rank's."""
import os
import socket

import numpy as np
import pytest
import torch
import torch.distributed as dist
import torch.multiprocessing as mp


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _worker(rank, world, port, out):
    import bench
    dist.init_process_group("gloo", init_method=f"tcp://127.0.0.1:{port}", rank=rank,
                            world_size=world)
    try:
        work, secs = bench.reduce_over_ranks([10.0 * (rank + 1), 1.0], 2.0 + rank, "cpu", world)
        inst = bench.rank_instance(2, rank)
        out.put((rank, work, secs, inst.motif, inst.ascii[:64].tobytes()))
    finally:
        dist.destroy_process_group()


def test_two_rank_weak_scaling_totals():
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_worker, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    res = sorted(q.get(timeout=120) for _ in procs)
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    for rank, work, secs, _, _ in res:
        assert work == [30.0, 2.0] and secs == 3.0
    assert res[0][3] != res[1][3] and res[0][4] != res[1][4]  # different instances


def test_single_process_totals_are_local():
    import bench
    work, secs = bench.reduce_over_ranks([5.0, 7.0], 1.5, "cpu", 1)
    assert work == [5.0, 7.0] and secs == 1.5


def test_reference_arm_runs_on_rank0_only(monkeypatch):
    import argparse

    import bench
    monkeypatch.setenv("RANK", "1")
    args = argparse.Namespace(config=2, steps=1, warmup=0, ref_sample=10)
    assert bench.run_reference(args) == 0  # returns at once, without oracle work


def test_reference_arm_line_on_cpu():
    """The reference arm (the oracle on the host's cores) prints one JSON line
    with the contract's keys; each step is the bounded sample it times."""
    import json
    import os
    import subprocess
    import sys
    root = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
    env = dict(os.environ, RANK="0", WORLD_SIZE="1")
    out = subprocess.run([sys.executable, os.path.join(root, "bench.py"), "--impl", "reference",
                          "--steps", "1", "--warmup", "3", "--ref-trials", "1", "--ref-cands", "2"],
                         capture_output=True, text=True, timeout=300, env=env, cwd=root)
    assert out.returncode == 0, out.stderr[-2000:]
    line = json.loads(out.stdout.strip().splitlines()[-1])
    assert line["impl"] == "reference" and line["unit"] == "scores/s"
    assert line["value"] > 0 and line["higher_is_better"] is True
    assert 0 < line["ms_per_step"] < line["ms_per_search_extrapolated"]
    assert line["cpu_baseline"]["kind"] == "oracle" and line["cpu_baseline"]["value"] == line["value"]
    assert line["e2e"]["h2d_bytes_per_step"] == 0 and line["e2e"]["value"] == line["value"]
    assert line["config"]["config_index"] == 5 and line["steps"] == 1 and line["warmup"] == 3
