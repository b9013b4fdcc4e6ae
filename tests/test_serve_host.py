"""Host-side logic of the request loop: the arena allocator and the Poisson generator."""
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
