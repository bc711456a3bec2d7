"""The multi-rank host logic of bench.py on the CPU: two gloo ranks.

With N GPUs the bench runs N independent replicas (the path has no data
exchange between GPUs), times each rank's steps, and reports the units all
ranks processed over the slowest rank's time.  Here two processes stand in
for the ranks: the barrier, the maximum over ranks and the whole-job value
are checked against their definitions.
"""
import os
import socket

import pytest

torch = pytest.importorskip("torch")
dist = pytest.importorskip("torch.distributed")
mp = pytest.importorskip("torch.multiprocessing")


def free_port() -> int:
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def rank_main(rank: int, world: int, port: int, out):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank), WORLD_SIZE=str(world),
                      LOCAL_RANK=str(rank))
    import bench

    w, r, local = bench.dist_env()
    dist.init_process_group("gloo", init_method="env://")
    try:
        bench.barrier(w)
        local_ms = 10.0 + 5.0 * r                  # rank 1 is the slower one
        mx = bench.max_over_ranks(local_ms, w)
        value, t_ms = bench.aggregate_value(1000.0, 4, w, local_ms)
        out.put((r, w, local, mx, value, t_ms))
        bench.barrier(w)
    finally:
        dist.destroy_process_group()


def test_two_ranks_report_whole_job_throughput():
    world = 2
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = free_port()
    procs = [ctx.Process(target=rank_main, args=(r, world, port, q)) for r in range(world)]
    for p in procs:
        p.start()
    for p in procs:
        p.join(timeout=120)
        assert p.exitcode == 0
    res = sorted(q.get(timeout=10) for _ in range(world))
    for r, (rank, w, local, mx, value, t_ms) in enumerate(res):
        assert rank == r and w == world and local == r
        assert mx == 15.0 and t_ms == 15.0
        # 1000 units per step, 4 steps, on each of 2 ranks, over the slowest rank's 15 ms
        assert value == pytest.approx(1000.0 * 4 * 2 / 0.015)


def test_one_rank_needs_no_process_group():
    import bench

    assert bench.max_over_ranks(3.5, 1) == 3.5
    value, t_ms = bench.aggregate_value(10.0, 2, 1, 4.0)
    assert t_ms == 4.0 and value == pytest.approx(10.0 * 2 / 0.004)


def test_gpus_flag_starts_one_rank_per_gpu():
    """bench.py --gpus N started without torchrun starts the N ranks itself."""
    import json
    import subprocess
    import sys

    import bench

    cmd = bench.replica_command(["--gpus", "2"], 2, 12345)
    assert cmd[1:4] == ["-m", "torch.distributed.run", "--nnodes=1"] and "--nproc-per-node=2" in cmd
    assert cmd[cmd.index("--master-addr") + 1] == "127.0.0.1" and cmd[-2:] == ["--gpus", "2"]
    env = {k: v for k, v in os.environ.items() if k not in ("WORLD_SIZE", "RANK", "LOCAL_RANK")}
    res = subprocess.run([sys.executable, bench.__file__, "--gpus", "2", "--launcher-check"], capture_output=True,
                         text=True, timeout=180, env=env)
    assert res.returncode == 0, res.stderr
    lines = [json.loads(l) for l in res.stdout.splitlines() if l.startswith("{")]
    assert sorted((d["rank"], d["world"], d["local_rank"]) for d in lines) == [(0, 2, 0), (1, 2, 1)]


def test_gpus_flag_must_match_the_world_size(monkeypatch):
    import bench

    monkeypatch.setenv("WORLD_SIZE", "3")
    assert bench.main(["--gpus", "2", "--launcher-check"]) == 2
