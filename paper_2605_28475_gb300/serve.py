"""Continuous-batching request loop for Q(f, f) evaluations (host orchestration only).

Requests (a batch of cells of one (Kmax, Lmax) operator) arrive over time.  Each is
admitted as soon as a stream slot and enough of a fixed device arena are free: its
coefficients are copied into the arena (device-resident from then on), its evaluation
is launched through the C ABI on the slot's stream, and it completes when the
slot's event fires.  Requests that arrive while others are on the GPU are admitted
in the same way, so their kernels overlap on the device.  Requests larger than the
whole arena are rejected.  Nothing here computes: every evaluation is a wef_evaluate
call.
"""
import heapq
import math
import time
from dataclasses import dataclass, field

import numpy as np

from . import PRECISIONS, wef_evaluate, wef_workspace_size


class Arena:
    """First-fit allocator over one pre-allocated device buffer (no per-request cudaMalloc)."""

    def __init__(self, nbytes, device):
        import torch

        self.buf = torch.empty(int(nbytes), dtype=torch.uint8, device=device)
        self.base = self.buf.data_ptr()
        self.size = int(nbytes)
        self.free = [(0, self.size)]  # sorted (offset, length)

    def alloc(self, n):
        n = (int(n) + 255) // 256 * 256
        for i, (o, ln) in enumerate(self.free):
            if ln >= n:
                if ln == n:
                    self.free.pop(i)
                else:
                    self.free[i] = (o + n, ln - n)
                return o, n
        return None

    def release(self, o, n):
        self.free.append((o, n))
        self.free.sort()
        merged = []
        for a, ln in self.free:
            if merged and merged[-1][0] + merged[-1][1] == a:
                merged[-1] = (merged[-1][0], merged[-1][1] + ln)
            else:
                merged.append((a, ln))
        self.free = merged

    def ptr(self, o):
        return self.base + o


@dataclass(order=True)
class Request:
    arrival: float
    rid: int = field(compare=False)
    shape: tuple = field(compare=False)
    f: np.ndarray = field(compare=False, repr=False)
    admitted: float = field(default=math.nan, compare=False)
    done: float = field(default=math.nan, compare=False)
    q: object = field(default=None, compare=False, repr=False)


class Server:
    """ops: {(kmax, lmax): Operator with an uploaded core}."""

    def __init__(self, ops, arena_bytes, nslots=8, precision="tf32", device="cuda:0", keep_results=False):
        import torch

        self.torch = torch
        self.ops = ops
        self.prec = PRECISIONS[precision]
        self.dev = torch.device(device)
        self.arena = Arena(arena_bytes, self.dev)
        self.streams = [torch.cuda.Stream(self.dev) for _ in range(nslots)]
        self.slot_busy = [None] * nslots  # (request, event, allocations)
        self.keep = keep_results
        self.completed = []
        self.rejected = []

    def _need(self, req):
        km, lm = req.shape
        n = req.f.shape[0]
        N = (km + 1) * (lm + 1) ** 2
        ws = wef_workspace_size(self.ops[req.shape].h, n, self.prec)
        return [n * N * 8, n * N * 8, max(ws, 256)]

    def fits_ever(self, req):
        return sum((b + 255) // 256 * 256 for b in self._need(req)) <= self.arena.size

    def try_admit(self, req, now):
        """Admit `req` into a free slot if the arena has room; returns True on success."""
        torch = self.torch
        slot = next((i for i, b in enumerate(self.slot_busy) if b is None), None)
        if slot is None:
            return False
        allocs = []
        for nb in self._need(req):
            a = self.arena.alloc(nb)
            if a is None:
                for o, ln in allocs:
                    self.arena.release(o, ln)
                return False
            allocs.append(a)
        (fo, _), (qo, _), (wo, wn) = allocs
        st = self.streams[slot]
        n = req.f.shape[0]
        fdev = self.arena.ptr(fo)
        qdev = self.arena.ptr(qo)
        host = torch.from_numpy(req.f.reshape(-1))
        # pinned staging keeps the copy asynchronous on the slot's stream
        pinned = host.pin_memory()
        dst = torch.empty(0, dtype=torch.float64, device=self.dev).set_(
            self.arena.buf.untyped_storage(), fo // 8, (pinned.numel(),))
        with torch.cuda.stream(st):
            dst.copy_(pinned, non_blocking=True)
            wef_evaluate(self.ops[req.shape].h, fdev, qdev, n, self.prec, self.arena.ptr(wo), wn, st.cuda_stream)
            ev = torch.cuda.Event()
            ev.record(st)
        req.admitted = now
        self.slot_busy[slot] = (req, ev, allocs, pinned)
        return True

    def poll(self, now_fn):
        """Complete every request whose event has fired; returns how many completed."""
        torch = self.torch
        k = 0
        for i, b in enumerate(self.slot_busy):
            if b is None:
                continue
            req, ev, allocs, _pinned = b
            if ev.query():
                req.done = now_fn()
                if self.keep:
                    km, lm = req.shape
                    n = req.f.shape[0]
                    N = (km + 1) * (lm + 1) ** 2
                    qo = allocs[1][0]
                    req.q = torch.empty(0, dtype=torch.float64, device=self.dev).set_(
                        self.arena.buf.untyped_storage(), qo // 8, (n * N,)).clone().reshape(n, km + 1, -1)
                for o, ln in allocs:
                    self.arena.release(o, ln)
                self.slot_busy[i] = None
                self.completed.append(req)
                k += 1
        return k

    def idle(self):
        return all(b is None for b in self.slot_busy)


def poisson_requests(rate, duration, shapes, max_cells, seed, make_cells):
    """Seeded Poisson arrivals over [0, duration): sizes log-uniform in [1, max_cells],
    shape uniform over `shapes`.  make_cells(shape, n, seed) draws the coefficients."""
    rng = np.random.Generator(np.random.PCG64(seed))
    t, rid, out = 0.0, 0, []
    while True:
        t += rng.exponential(1.0 / rate)
        if t >= duration:
            break
        n = int(np.clip(np.round(np.exp(rng.uniform(0.0, np.log(max_cells)))), 1, max_cells))
        shape = shapes[rng.integers(len(shapes))]
        out.append(Request(t, rid, shape, make_cells(shape, n, seed * 1000003 + rid)))
        rid += 1
    return out


def run(server, requests, time_limit=None):
    """Replay `requests` (arrival times in seconds from now) through `server`;
    returns a summary with p50/p99 arrival-to-completion latency and throughput."""
    pending = list(requests)
    heapq.heapify(pending)
    waiting = []  # arrived, not yet admitted (FIFO)
    t0 = time.perf_counter()
    now = lambda: time.perf_counter() - t0  # noqa: E731
    last_arrival = requests[-1].arrival if requests else 0.0
    while pending or waiting or not server.idle():
        t = now()
        while pending and pending[0].arrival <= t:
            r = heapq.heappop(pending)
            if server.fits_ever(r):
                waiting.append(r)
            else:
                server.rejected.append(r)
        while waiting and server.try_admit(waiting[0], now()):
            waiting.pop(0)
        server.poll(now)
        if time_limit is not None and t > time_limit + last_arrival:
            break
        if not waiting and pending and server.idle():
            dt = pending[0].arrival - now()
            if dt > 0:
                time.sleep(min(dt, 0.002))
    wall = now()
    lat = np.array([r.done - r.arrival for r in server.completed])
    cells = int(sum(r.f.shape[0] for r in server.completed))
    return {
        "requests": len(requests),
        "completed": len(server.completed),
        "rejected": len(server.rejected),
        "cells": cells,
        "wall_s": wall,
        "cells_per_s": cells / wall if wall > 0 else 0.0,
        "p50_ms": float(np.percentile(lat, 50) * 1e3) if lat.size else None,
        "p99_ms": float(np.percentile(lat, 99) * 1e3) if lat.size else None,
        "mean_queue_ms": float(np.mean([r.admitted - r.arrival for r in server.completed]) * 1e3) if lat.size else None,
    }
