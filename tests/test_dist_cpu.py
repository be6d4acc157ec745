"""The multi-process path of bench.py on CPU: two ranks over gloo.

A run on N GPUs is N independent replicas of the workload (no collective
on the data path); the only cross-rank steps are the barriers around the
timed region and the reductions that form the whole-job number: the
slowest rank's time and the sum of the units all ranks processed.  These
tests run those steps with world size 2 on the host, and launch the
reference arm under torchrun to check that rank 0 alone prints its line.
"""
import json
import multiprocessing as mp
import os
import socket
import subprocess
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank_main(rank, world, port, q):
    os.environ.update(RANK=str(rank), LOCAL_RANK=str(rank), WORLD_SIZE=str(world),
                      MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), BENCH_BACKEND="gloo")
    sys.path.insert(0, ROOT)
    import bench
    import torch.distributed as dist
    w, r, local = bench.dist_init()
    bench.barrier(w)
    # rank k took (k + 1) * 1.5 s for (k + 1) * 100 units
    slowest = bench.max_over_ranks(w, (r + 1) * 1.5, "cpu")
    total = bench.sum_over_ranks(w, (r + 1) * 100.0, "cpu")
    rate = bench.whole_job_rate(w, (r + 1) * 100.0, (r + 1) * 1.5, "cpu")
    bench.barrier(w)
    dist.destroy_process_group()
    q.put((r, w, local, slowest, total, rate))


def test_two_ranks_gloo_reductions():
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_rank_main, args=(k, 2, port, q)) for k in range(2)]
    for p in procs:
        p.start()
    out = sorted(q.get(timeout=120) for _ in procs)
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    assert [o[:3] for o in out] == [(0, 2, 0), (1, 2, 1)]
    for _, _, _, slowest, total, rate in out:
        assert slowest == 3.0          # the max over ranks, seen by every rank
        assert total == 300.0          # 100 + 200 units
        assert rate == 100.0           # 300 units / 3 s


def test_single_rank_needs_no_process_group():
    sys.path.insert(0, ROOT)
    import bench
    env = {k: os.environ.pop(k) for k in ("WORLD_SIZE", "RANK", "LOCAL_RANK") if k in os.environ}
    try:
        assert bench.dist_init() == (1, 0, 0)
        assert bench.max_over_ranks(1, 2.5, "cpu") == 2.5
        assert bench.whole_job_rate(1, 10.0, 4.0, "cpu") == 2.5
    finally:
        os.environ.update(env)


def test_reference_arm_under_torchrun_prints_once(orc):
    """--impl reference with two ranks: rank 0 times the CPU reference and
    prints one JSON line; rank 1 exits 0 without work."""
    cmd = [sys.executable, "-m", "torch.distributed.run", "--nnodes=1", "--nproc-per-node", "2",
           "--master-addr", "127.0.0.1", "--master-port", str(_free_port()),
           os.path.join(ROOT, "bench.py"), "--impl", "reference", "--gpus", "2",
           "--steps", "1", "--warmup", "0"]
    res = subprocess.run(cmd, cwd=ROOT, capture_output=True, text=True, timeout=300)
    assert res.returncode == 0, res.stderr[-2000:]
    lines = [ln for ln in res.stdout.splitlines() if ln.startswith("{")]
    assert len(lines) == 1
    d = json.loads(lines[0])
    assert d["impl"] == "reference" and d["n_gpus"] == 2 and d["value"] > 0
    assert d["cpu_baseline"]["kind"] == "oracle"
    assert d["e2e"]["h2d_bytes_per_step"] == 0
