"""The multi-rank logic of bench.py on CPU with world_size 2 over gloo: the
max-over-ranks timing, the whole-job rate, and the reference arm printing on
rank 0 only.  (Each rank reconstructs its own scan: replicas, no data-path
collective.)"""
import contextlib
import io
import multiprocessing as mp
import os
import socket
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _free_port():
    with contextlib.closing(socket.socket(socket.AF_INET, socket.SOCK_STREAM)) as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _worker(rank, world, port, q):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank), WORLD_SIZE=str(world),
                      LOCAL_RANK=str(rank))
    sys.path.insert(0, ROOT)
    import torch.distributed as dist
    import bench
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        w, r, l = bench.rank_env()
        slow = bench.max_over_ranks(dist, 10.0 + 5.0 * rank, device="cpu")
        rate = bench.aggregate_rate(1000, w, slow / 1e3)
        dist.barrier()
        q.put((r, w, l, slow, rate))
    finally:
        dist.destroy_process_group()


def test_max_over_ranks_and_rate_with_two_gloo_ranks():
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_worker, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    out = sorted(q.get(timeout=120) for _ in procs)
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    assert [o[0] for o in out] == [0, 1] and all(o[1] == 2 for o in out)
    for r, w, l, slow, rate in out:
        assert slow == 15.0                       # the slower rank's time on every rank
        assert rate == pytest.approx(1000 * 2 / 0.015)


def test_single_process_needs_no_group():
    sys.path.insert(0, ROOT)
    import bench
    assert bench.max_over_ranks(None, 3.5) == 3.5
    assert bench.aggregate_rate(10, 1, 2.0) == 5.0


def test_reference_arm_prints_on_rank_zero_only(monkeypatch):
    sys.path.insert(0, ROOT)
    import bench
    monkeypatch.setenv("RANK", "1")
    monkeypatch.setenv("WORLD_SIZE", "2")
    buf = io.StringIO()
    with contextlib.redirect_stdout(buf):
        bench.run_reference(type("A", (), dict(steps=1, warmup=0, gpus=2))())
    assert buf.getvalue() == ""
