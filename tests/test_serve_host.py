"""Host-side logic of the request loop: the arena allocator, the Poisson generator, batch
packing and the scheduling loop (driven with a fake server whose batches finish at once)."""
import numpy as np
import pytest

torch = pytest.importorskip("torch")

from paper_2605_28475_gb300 import serve  # noqa: E402


def test_arena_first_fit_and_merge():
    a = serve.Arena(4096, "cpu")
    x = a.alloc(1000)
    y = a.alloc(1000)
    z = a.alloc(1000)
    assert x == (0, 1024) and y == (1024, 1024) and z == (2048, 1024)
    assert a.alloc(2000) is None
    a.release(*y)
    assert a.alloc(1100) is None  # fragment too small
    a.release(*x)
    assert a.free[0] == (0, 2048)  # merged with the neighbour
    w = a.alloc(2000)
    assert w == (0, 2048)
    a.release(*w)
    a.release(*z)
    assert a.free == [(0, 4096)]


def test_poisson_requests_seeded():
    mk = lambda sh, n, s: np.zeros((n, 1))  # noqa: E731
    r1 = serve.poisson_requests(50.0, 2.0, [(8, 8), (12, 12)], 4096, seed=3, make_cells=mk)
    r2 = serve.poisson_requests(50.0, 2.0, [(8, 8), (12, 12)], 4096, seed=3, make_cells=mk)
    assert [(r.arrival, r.shape, r.f.shape[0]) for r in r1] == [(r.arrival, r.shape, r.f.shape[0]) for r in r2]
    assert 60 < len(r1) < 140
    assert all(1 <= r.f.shape[0] <= 4096 for r in r1)
    assert all(0 <= r.arrival < 2.0 for r in r1)
    assert sorted(r1) == r1


def test_pack_batch_caps():
    mk = lambda n, sh=(8, 8), t=0.0: serve.Request(t, 0, sh, np.zeros((n, 1)))  # noqa: E731
    w = [mk(100), mk(50, (12, 12)), mk(300), mk(200), mk(10)]
    # oldest shape only, in arrival order, up to the cell cap
    assert [r.f.shape[0] for r in serve.pack_batch(w, 450)] == [100, 300]
    assert [r.f.shape[0] for r in serve.pack_batch(w, 10_000)] == [100, 300, 200, 10]
    # estimated-time cap: 1 ms per cell, 0.35 s per batch
    cost = {(8, 8): 1e-3, (12, 12): 5e-3}
    assert [r.f.shape[0] for r in serve.pack_batch(w, 10_000, cost, 0.35)] == [100]
    # the oldest request goes alone even if it exceeds both caps
    assert [r.f.shape[0] for r in serve.pack_batch([mk(5000)] + w, 450, cost, 0.35)] == [5000]
    assert serve.pack_batch([], 450) == []
    # size-aware admission: overdue requests (waiting > 0.5 s at now = 1 s) first, in arrival
    # order, then the others by increasing estimated time
    w2 = [mk(100, t=0.2), mk(50, (12, 12), 0.8), mk(300, t=0.9), mk(10, t=0.95), mk(200, t=0.3)]
    got = serve.pack_batch(w2, 10_000, cost, 10.0, mixed=True, now=1.0, max_wait_s=0.5)
    assert [r.f.shape[0] for r in got] == [100, 200, 10, 50, 300]
    # mixed batches (ragged evaluation): every shape, still in arrival order and within the caps
    assert [r.f.shape[0] for r in serve.pack_batch(w, 450, mixed=True)] == [100, 50, 300]
    assert [r.f.shape[0] for r in serve.pack_batch(w, 10_000, cost, 0.5, mixed=True)] == [100, 50]


class _FakeServer:
    """The interface run() drives, with batches that finish at the next poll: it packs the
    same batches as the real server (pack_batch), refuses requests above a cell limit, and
    has `slots` batches in flight at most."""

    def __init__(self, max_cells_ever, slots=2, max_batch_cells=64):
        self.max_cells_ever, self.slots, self.max_batch_cells = max_cells_ever, slots, max_batch_cells
        self.in_flight, self.completed, self.rejected, self.batches = [], [], [], 0

    def fits_ever(self, r):
        return r.f.shape[0] <= self.max_cells_ever

    def try_launch(self, waiting, now):
        if len(self.in_flight) >= self.slots or not waiting:
            return False
        chosen = serve.pack_batch(waiting, self.max_batch_cells)
        ids = {id(r) for r in chosen}
        waiting[:] = [r for r in waiting if id(r) not in ids]
        for r in chosen:
            r.admitted = now
        self.in_flight.append(chosen)
        self.batches += 1
        return True

    def poll(self, now_fn):
        t, n = now_fn(), 0
        for batch in self.in_flight:
            for r in batch:
                r.done = t
                self.completed.append(r)
                n += 1
        self.in_flight = []
        return n

    def wait(self, timeout):
        if timeout:
            __import__("time").sleep(min(timeout, 1e-3))

    def idle(self):
        return not self.in_flight


def test_run_loop_accounts_for_every_request():
    """Every request is completed or rejected exactly once, in its shape's batches, never
    before it arrived; the summary counts agree with the server's records."""
    mk = lambda sh, n, s: np.zeros((n, 1))  # noqa: E731
    reqs = serve.poisson_requests(400.0, 0.25, [(8, 8), (12, 12)], 100, seed=4, make_cells=mk)
    srv = _FakeServer(max_cells_ever=80)
    out = serve.run(srv, reqs)
    assert out["requests"] == len(reqs) == out["completed"] + out["rejected"]
    assert {id(r) for r in srv.completed}.isdisjoint({id(r) for r in srv.rejected})
    assert all(r.f.shape[0] > 80 for r in srv.rejected) and all(r.f.shape[0] <= 80 for r in srv.completed)
    assert all(r.arrival <= r.admitted <= r.done for r in srv.completed)
    assert out["cells"] == sum(r.f.shape[0] for r in srv.completed)
    assert out["p50_ms"] is not None and out["p50_ms"] <= out["p99_ms"]
    assert out["batches"] == srv.batches <= out["completed"]
    # latency by request size: small (<= 64 cells) and large (>= 1024 cells, none here)
    assert out["small"]["requests"] == sum(1 for r in srv.completed if r.f.shape[0] <= 64)
    assert out["large"]["requests"] == 0 and out["large"]["p50_ms"] is None


def test_pin_requests():
    """Set-up of a request stream: every request's cells copied into one pinned buffer, each
    with a pinned output of the same shape."""
    if not torch.cuda.is_available():
        pytest.skip("pinned host memory needs a CUDA driver")
    reqs = [serve.Request(0.0, i, (1, 1), np.full((i + 1, 2, 4), float(i))) for i in range(3)]
    fin, fout = serve.pin_requests(reqs)
    assert fin.is_pinned() and fout.is_pinned() and fin.numel() == 2 * 4 * 6
    for i, r in enumerate(reqs):
        assert tuple(r.f.shape) == (i + 1, 2, 4) and bool((r.f == float(i)).all()) and r.out.shape == r.f.shape
