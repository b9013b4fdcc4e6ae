"""Continuous-batching request loop for Q(f, f) evaluations (host orchestration only).

Requests (a batch of cells of one (Kmax, Lmax) operator) arrive over time and wait in
a FIFO.  Whenever one of the stream slots is free, the scheduler takes the shape of
the oldest waiting request and packs every waiting request of that shape (in arrival
order, up to a cell cap, an estimated GPU time per batch and what the device arena can
hold) into one batch: their
coefficients are copied into one contiguous arena region (device-resident from then
on) and evaluated by a single wef_evaluate call on the slot's stream.  Requests that
arrive while batches are on the GPU join the next batch of their shape, and batches
on different slots overlap on the device.  Requests larger than the whole arena are
rejected.  Nothing here computes: every evaluation is a wef_evaluate call.
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

    def view(self, o, n_doubles):
        import torch

        return torch.empty(0, dtype=torch.float64, device=self.buf.device).set_(self.buf.untyped_storage(), o // 8,
                                                                                 (int(n_doubles),))


@dataclass(order=True)
class Request:
    arrival: float
    rid: int = field(compare=False)
    shape: tuple = field(compare=False)
    f: np.ndarray = field(compare=False, repr=False)
    admitted: float = field(default=math.nan, compare=False)
    done: float = field(default=math.nan, compare=False)
    q: object = field(default=None, compare=False, repr=False)


def _n_per_cell(shape):
    km, lm = shape
    return (km + 1) * (lm + 1) ** 2


def pack_batch(waiting, max_cells, cost_per_cell=None, max_batch_s=None):
    """Requests of the oldest waiting request's shape, in arrival order, while the batch
    stays within `max_cells` cells and (if costs are given) `max_batch_s` seconds of
    estimated GPU time.  The oldest request is always taken, whatever its size."""
    if not waiting:
        return []
    shape = waiting[0].shape
    c = None if cost_per_cell is None else cost_per_cell.get(shape)
    chosen, cells = [], 0
    for r in waiting:
        if r.shape != shape:
            continue
        n = r.f.shape[0]
        if chosen and (cells + n > max_cells or (c is not None and max_batch_s is not None and (cells + n) * c > max_batch_s)):
            break
        chosen.append(r)
        cells += n
    return chosen


class Server:
    """ops: {(kmax, lmax): Operator with an uploaded core}."""

    def __init__(self, ops, arena_bytes, nslots=8, precision="tf32", device="cuda:0", max_batch_cells=16384,
                 keep_results=False, cost_per_cell=None, max_batch_s=None):
        import torch

        self.torch = torch
        self.ops = ops
        self.prec = PRECISIONS[precision]
        self.dev = torch.device(device)
        self.arena = Arena(arena_bytes, self.dev)
        self.streams = [torch.cuda.Stream(self.dev) for _ in range(nslots)]
        self.slot_busy = [None] * nslots  # (requests, event, allocations, q offset)
        self.max_batch_cells = int(max_batch_cells)
        self.cost_per_cell = cost_per_cell  # {shape: estimated seconds per cell}
        self.max_batch_s = max_batch_s
        self.keep = keep_results
        self.completed = []
        self.rejected = []
        self.batches = 0

    def _bytes(self, shape, ncells):
        N = _n_per_cell(shape)
        ws = wef_workspace_size(self.ops[shape].h, ncells, self.prec)
        return [ncells * N * 8, ncells * N * 8, max(ws, 256)]

    def fits_ever(self, req):
        return sum((b + 255) // 256 * 256 for b in self._bytes(req.shape, req.f.shape[0])) <= self.arena.size

    def _alloc(self, sizes):
        allocs = []
        for nb in sizes:
            a = self.arena.alloc(nb)
            if a is None:
                for o, ln in allocs:
                    self.arena.release(o, ln)
                return None
            allocs.append(a)
        return allocs

    def try_launch(self, waiting, now):
        """Pack waiting requests of the oldest request's shape into one batch on a free slot.
        Removes the launched requests from `waiting`; returns True if a batch was launched."""
        torch = self.torch
        slot = next((i for i, b in enumerate(self.slot_busy) if b is None), None)
        if slot is None or not waiting:
            return False
        shape = waiting[0].shape
        chosen = pack_batch(waiting, self.max_batch_cells, self.cost_per_cell, self.max_batch_s)
        cells = sum(r.f.shape[0] for r in chosen)
        allocs = self._alloc(self._bytes(shape, cells))
        while allocs is None and len(chosen) > 1:  # shrink the batch to what memory allows
            cells -= chosen.pop().f.shape[0]
            allocs = self._alloc(self._bytes(shape, cells))
        if allocs is None:
            return False
        ids = {id(r) for r in chosen}
        waiting[:] = [r for r in waiting if id(r) not in ids]
        (fo, _), (qo, _), (wo, wn) = allocs
        N = _n_per_cell(shape)
        st = self.streams[slot]
        staging = []
        with torch.cuda.stream(st):
            off = 0
            for r in chosen:
                n = r.f.shape[0]
                pinned = torch.from_numpy(r.f.reshape(-1)).pin_memory()
                self.arena.view(fo + off * N * 8, n * N).copy_(pinned, non_blocking=True)
                staging.append(pinned)
                r.admitted = now
                off += n
            try:
                wef_evaluate(self.ops[shape].h, self.arena.ptr(fo), self.arena.ptr(qo), cells, self.prec,
                             self.arena.ptr(wo), wn, st.cuda_stream)
            except Exception:
                # the evaluation was refused or failed to launch: once the work already
                # queued on the slot has finished, return the memory to the arena and the
                # requests to the front of the queue
                st.synchronize()
                for o, ln in allocs:
                    self.arena.release(o, ln)
                waiting[:0] = chosen
                raise
            ev = torch.cuda.Event()
            ev.record(st)
        self.slot_busy[slot] = (chosen, ev, allocs, staging)
        self.batches += 1
        return True

    def poll(self, now_fn):
        """Complete every batch whose event has fired; returns how many requests completed."""
        k = 0
        for i, b in enumerate(self.slot_busy):
            if b is None:
                continue
            chosen, ev, allocs, _staging = b
            if not ev.query():
                continue
            t = now_fn()
            qo = allocs[1][0]
            off = 0
            for r in chosen:
                n = r.f.shape[0]
                N = _n_per_cell(r.shape)
                r.done = t
                if self.keep:
                    km, lm = r.shape
                    r.q = self.arena.view(qo + off * N * 8, n * N).clone().reshape(n, km + 1, -1)
                off += n
                self.completed.append(r)
                k += 1
            for o, ln in allocs:
                self.arena.release(o, ln)
            self.slot_busy[i] = None
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
    waiting = []  # arrived, not yet launched (FIFO)
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
        server.poll(now)
        while server.try_launch(waiting, now()):
            pass
        if time_limit is not None and t > time_limit + last_arrival:
            break
        if not waiting and pending and server.idle():
            dt = pending[0].arrival - now()
            if dt > 0:
                time.sleep(min(dt, 0.002))
        elif not server.idle():
            time.sleep(0.0002)
    wall = now()
    lat = np.array([r.done - r.arrival for r in server.completed])
    cells = int(sum(r.f.shape[0] for r in server.completed))
    return {
        "requests": len(requests),
        "completed": len(server.completed),
        "rejected": len(server.rejected),
        "batches": server.batches,
        "cells": cells,
        "wall_s": wall,
        "cells_per_s": cells / wall if wall > 0 else 0.0,
        "p50_ms": float(np.percentile(lat, 50) * 1e3) if lat.size else None,
        "p99_ms": float(np.percentile(lat, 99) * 1e3) if lat.size else None,
        "mean_queue_ms": float(np.mean([r.admitted - r.arrival for r in server.completed]) * 1e3) if lat.size else None,
    }
