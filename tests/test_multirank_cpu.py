"""The N > 1 host path of bench.py on CPU: two gloo ranks, max-over-ranks timing and the
whole-job throughput (each rank evaluates its own batch; no data-path collective)."""
import os
import socket

import pytest

torch = pytest.importorskip("torch")
import torch.distributed as dist  # noqa: E402
import torch.multiprocessing as mp  # noqa: E402


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _worker(rank, world, port, out):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank), WORLD_SIZE=str(world))
    import bench

    dist.init_process_group("gloo", rank=rank, world_size=world)
    r, w, _ = bench.dist_env()
    ms = bench.max_over_ranks(100.0 + 50.0 * r, dist, "cpu")  # rank 1 is slower
    val = bench.job_throughput(w, 16384, ms / 5)
    out.put((r, w, ms, val))
    dist.destroy_process_group()


def test_two_rank_gloo_max_and_throughput():
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
    assert [r[0] for r in res] == [0, 1] and all(r[1] == 2 for r in res)
    assert all(r[2] == 150.0 for r in res)  # the max, on every rank
    assert all(abs(r[3] - 2 * 16384 / 0.030) < 1e-6 for r in res)
