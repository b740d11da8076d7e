"""The benchmark's multi-process path on CPU (gloo, world size 2).

Every unit of the path is independent, so ranks run replicas with no data-path
collective; what crosses ranks is the timing (the slowest rank sets the job's
time) and, in the reference arm, the rule that rank 0 alone works and prints.
"""
from __future__ import annotations

import contextlib
import io
import json
import multiprocessing as mp
import os
import socket
import sys

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _free_port() -> int:
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _reduce_worker(rank: int, world: int, port: int, q) -> None:
    sys.path.insert(0, ROOT)
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank),
                      WORLD_SIZE=str(world))
    import torch.distributed as dist
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        import bench
        t_max = bench.reduce_over_ranks(1.5 + rank, world, "max")
        b_sum = bench.reduce_over_ranks(100.0 * (rank + 1), world, "sum")
        q.put((rank, t_max, b_sum))
    finally:
        dist.destroy_process_group()


def _reference_worker(rank: int, world: int, q) -> None:
    sys.path.insert(0, ROOT)
    os.environ.update(RANK=str(rank), WORLD_SIZE=str(world), LOCAL_RANK=str(rank))
    import bench
    sys.argv = ["bench.py", "--impl", "reference", "--workload", "ellipsoids128", "--steps", "1",
                "--warmup", "0", "--cpu-budget", "0.3", "--gpus", str(world)]
    out = io.StringIO()
    with contextlib.redirect_stdout(out):
        bench.main()
    q.put((rank, out.getvalue()))


def _run(target, args_of, world):
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    ps = [ctx.Process(target=target, args=args_of(r) + (q,)) for r in range(world)]
    for p in ps:
        p.start()
    res = [q.get(timeout=300) for _ in ps]
    for p in ps:
        p.join(timeout=60)
        assert p.exitcode == 0
    return sorted(res)


def test_max_time_and_summed_units_over_two_ranks():
    port = _free_port()
    res = _run(_reduce_worker, lambda r: (r, 2, port), 2)
    # both ranks see the slowest rank's time and the job's total units
    assert res == [(0, 2.5, 300.0), (1, 2.5, 300.0)]


def test_one_process_needs_no_group():
    sys.path.insert(0, ROOT)
    import bench
    assert bench.reduce_over_ranks(3.25, 1, "max") == 3.25
    assert bench.reduce_over_ranks(7, 1, "sum") == 7.0


def test_reference_arm_rank0_alone_prints_one_line():
    res = _run(_reference_worker, lambda r: (r, 2), 2)
    (r0, out0), (r1, out1) = res
    assert out1 == ""
    lines = [ln for ln in out0.splitlines() if ln.strip()]
    assert len(lines) == 1
    d = json.loads(lines[0])
    assert d["impl"] == "reference" and d["n_gpus"] == 2 and d["value"] > 0
    assert d["cpu_baseline"]["kind"] == "oracle"
    assert d["e2e"]["h2d_bytes_per_step"] == 0
