"""The N > 1 host path on CPU with two gloo ranks: bench.py's max-over-ranks timing and
whole-job throughput (each rank evaluates its own batch; no data-path collective), and
replicas: each rank's own library instance builds a bitwise identical core."""
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


def _replica_worker(rank, world, port, out):
    """One rank of a replicated run: its own library instance (operator, host-built core),
    its own seeded batch; the only exchange is the test's comparison of the results."""
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank), WORLD_SIZE=str(world))
    import hashlib

    import numpy as np

    import bench
    import paper_2605_28475_gb300 as W

    dist.init_process_group("gloo", rank=rank, world_size=world)
    km = lm = 3
    h = W.wef_create(km, lm, 1.0)
    try:
        sizes = W.wef_sizes(h)
        R = W.wef_core_build(h, 10, 10)
        flops = W.wef_flops(h, W.WEF_RADIAL_FP32)
    finally:
        W.wef_destroy(h)
    bench.KMAX = bench.LMAX = km
    f = bench.inputs(64, seed=3 + rank)  # the bench's per-rank seed
    got = [None] * world
    dist.all_gather_object(got, (tuple(sizes), hashlib.sha256(np.ascontiguousarray(R).tobytes()).hexdigest(), flops,
                                 hashlib.sha256(np.ascontiguousarray(f).tobytes()).hexdigest()))
    out.put((rank, got))
    dist.destroy_process_group()


def test_two_rank_gloo_replicas():
    """Two gloo ranks each create the operator and build its core on the host: the replicas
    are bitwise identical (the core needs no broadcast), while each rank's seeded batch is
    its own (weak scaling: every rank evaluates different cells)."""
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_replica_worker, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    res = sorted(q.get(timeout=300) for _ in procs)
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    for _, got in res:
        (s0, c0, fl0, f0), (s1, c1, fl1, f1) = got
        assert s0 == s1 and c0 == c1 and fl0 == fl1  # identical operator and core on both ranks
        assert f0 != f1  # per-rank batches
