"""Continuous-batching request loop for Q(f, f) evaluations (host orchestration only).

Requests (a batch of cells of one (Kmax, Lmax) operator) arrive over time and wait in a
FIFO.  Whenever one of the stream slots is free, the scheduler packs waiting requests, in
arrival order (or, with size-aware admission, overdue ones first and then the cheapest),
up to a cell cap, an estimated GPU time per batch and what the device arena can hold, into
one batch.  On the radial-first and FP64 paths a batch mixes requests of
every shape and runs as one wef_evaluate_ragged call (each cell tagged with its operator
and its position in the batch); on the tensor-core paths a batch holds one shape and runs
as one wef_evaluate call.  Per batch, on the slot's stream: the requests' coefficients are
copied from (pinned) host memory into one arena region, evaluated, and every request's Q
is copied back into its host output before the batch's completion event, so a request is
complete when its result is in host memory.  Requests that arrive while batches are on the
GPU join the next batch, and batches on different slots overlap on the device.  Requests
larger than the whole arena are rejected.  Completions are waited for by one helper thread
per batch in flight (blocking-sync events), so the scheduler sleeps until the next arrival
or completion instead of polling.  Nothing here computes: every evaluation is a library call.
"""
import heapq
import math
import queue
import threading
import time
from dataclasses import dataclass, field

import numpy as np

from . import (PRECISIONS, WEF_FP64, WEF_RADIAL_FP32, wef_evaluate, wef_evaluate_ragged, wef_ragged_workspace_size,
               wef_workspace_size)


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

    def view(self, o, n, dtype=None):
        """n elements of `dtype` (default float64) starting at byte offset o."""
        import torch

        dtype = torch.float64 if dtype is None else dtype
        size = torch.empty(0, dtype=dtype).element_size()
        return torch.empty(0, dtype=dtype, device=self.buf.device).set_(self.buf.untyped_storage(), o // size, (int(n),))


@dataclass(order=True)
class Request:
    """f: the request's cells [n, K, NQ] (numpy, or a CPU tensor, ideally pinned); out: where
    its Q is delivered (a CPU float64 tensor of f's shape, ideally pinned; allocated at
    completion if None)."""
    arrival: float
    rid: int = field(compare=False)
    shape: tuple = field(compare=False)
    f: object = field(compare=False, repr=False)
    out: object = field(default=None, compare=False, repr=False)
    admitted: float = field(default=math.nan, compare=False)
    done: float = field(default=math.nan, compare=False)

    @property
    def q(self):
        return self.out


def _n_per_cell(shape):
    km, lm = shape
    return (km + 1) * (lm + 1) ** 2


def _cost(r, cost_per_cell):
    return 0.0 if cost_per_cell is None else cost_per_cell.get(r.shape, 0.0) * r.f.shape[0]


def pack_batch(waiting, max_cells, cost_per_cell=None, max_batch_s=None, mixed=False, now=None, max_wait_s=None):
    """Waiting requests in arrival order (of the first candidate's shape only, unless `mixed`)
    while the batch stays within `max_cells` cells and (if costs are given) `max_batch_s`
    seconds of estimated GPU time.  The first candidate is always taken, whatever its size.
    With `max_wait_s` (size-aware admission): requests waiting longer than that come first,
    in arrival order, then the others by increasing estimated GPU time."""
    if not waiting:
        return []
    seq = waiting
    if max_wait_s is not None and now is not None:
        late = [r for r in waiting if now - r.arrival > max_wait_s]
        fresh = sorted((r for r in waiting if now - r.arrival <= max_wait_s), key=lambda r: _cost(r, cost_per_cell))
        seq = late + fresh
    shape = seq[0].shape
    chosen, cells, est = [], 0, 0.0
    for r in seq:
        if r.shape != shape and not mixed:
            continue
        n = r.f.shape[0]
        c = _cost(r, cost_per_cell)
        if chosen and (cells + n > max_cells or (max_batch_s is not None and est + c > max_batch_s)):
            break
        chosen.append(r)
        cells += n
        est += c
    return chosen


def _host(x):
    import torch

    return x if isinstance(x, torch.Tensor) else torch.from_numpy(np.ascontiguousarray(x))


def pin_requests(requests):
    """Copy every request's cells into one pinned host buffer and give each request a pinned
    output of the same size (set-up, before serving: no page-locking on the launch path)."""
    import torch

    total = sum(int(np.prod(r.f.shape)) for r in requests)
    fin = torch.empty(total, dtype=torch.float64).pin_memory()
    fout = torch.empty(total, dtype=torch.float64).pin_memory()
    o = 0
    for r in requests:
        n = int(np.prod(r.f.shape))
        fin[o:o + n].copy_(_host(r.f).reshape(-1))
        r.f = fin[o:o + n].view(tuple(r.f.shape))
        r.out = fout[o:o + n].view(tuple(r.f.shape))
        o += n
    return fin, fout


class Server:
    """ops: {(kmax, lmax): Operator with an uploaded core}.  ragged (default: on for the
    radial-first and FP64 paths) packs requests of every shape into one batch."""

    def __init__(self, ops, arena_bytes, nslots=8, precision="rf32", device="cuda:0", max_batch_cells=16384,
                 keep_results=False, cost_per_cell=None, max_batch_s=None, ragged=None, max_wait_s=None):
        import torch

        self.torch = torch
        self.ops = ops
        self.shapes = list(ops.keys())
        self.shape_index = {sh: i for i, sh in enumerate(self.shapes)}
        self.handles = [ops[sh].h for sh in self.shapes]
        self.prec = PRECISIONS[precision] if isinstance(precision, str) else int(precision)
        self.ragged = (self.prec in (WEF_RADIAL_FP32, WEF_FP64)) if ragged is None else bool(ragged)
        self.dev = torch.device(device)
        self.arena = Arena(arena_bytes, self.dev)
        self.streams = [torch.cuda.Stream(self.dev) for _ in range(nslots)]
        self.slot_busy = [None] * nslots  # (requests, allocations)
        self.staging = [None] * nslots  # pinned per-slot buffers for the batch's cell tags
        self.max_batch_cells = int(max_batch_cells)
        self.cost_per_cell = cost_per_cell  # {shape: estimated seconds per cell}
        self.max_batch_s = max_batch_s
        self.max_wait_s = max_wait_s  # size-aware admission bound (None: arrival order)
        self.keep = keep_results  # results are always delivered to Request.out; kept for compatibility
        self.completed = []
        self.rejected = []
        self.batches = 0
        self.batch_log = []  # the requests of every launched batch
        self._done = queue.Queue()
        self._ready = []

    def _bytes(self, reqs):
        """Arena bytes of a batch: f, Q, (ragged) per-cell tags, workspace."""
        cells = sum(r.f.shape[0] for r in reqs)
        vals = sum(r.f.shape[0] * _n_per_cell(r.shape) for r in reqs)
        if self.ragged:
            ws = wef_ragged_workspace_size(self.handles, cells, self.prec)
            return [vals * 8, vals * 8, cells * 12 + 256, max(ws, 256)]
        ws = wef_workspace_size(self.ops[reqs[0].shape].h, cells, self.prec)
        return [vals * 8, vals * 8, max(ws, 256)]

    def fits_ever(self, req):
        return sum((b + 255) // 256 * 256 for b in self._bytes([req])) <= self.arena.size

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

    def _tags(self, slot, chosen, cells):
        """Pinned host arrays of a batch: the offset (int64) of every cell, then its operator
        index (int32), so that both device arrays are naturally aligned."""
        torch = self.torch
        st = self.staging[slot]
        if st is None or st.numel() < cells * 12:
            st = self.staging[slot] = torch.empty(max(cells, self.max_batch_cells, 4096) * 12,
                                                  dtype=torch.uint8).pin_memory()
        offs = st[:cells * 8].view(torch.int64).numpy()
        ids = st[cells * 8:cells * 12].view(torch.int32).numpy()
        c = v = 0
        for r in chosen:
            n, N = r.f.shape[0], _n_per_cell(r.shape)
            ids[c:c + n] = self.shape_index[r.shape]
            offs[c:c + n] = v + N * np.arange(n, dtype=np.int64)
            c += n
            v += n * N
        return st[:cells * 12]

    def try_launch(self, waiting, now):
        """Pack waiting requests into one batch on a free slot.  Removes the launched
        requests from `waiting`; returns True if a batch was launched."""
        torch = self.torch
        slot = next((i for i, b in enumerate(self.slot_busy) if b is None), None)
        if slot is None or not waiting:
            return False
        chosen = pack_batch(waiting, self.max_batch_cells, self.cost_per_cell, self.max_batch_s, mixed=self.ragged,
                            now=now, max_wait_s=self.max_wait_s)
        allocs = self._alloc(self._bytes(chosen))
        while allocs is None and len(chosen) > 1:  # shrink the batch to what memory allows
            chosen.pop()
            allocs = self._alloc(self._bytes(chosen))
        if allocs is None:
            return False
        ids = {id(r) for r in chosen}
        waiting[:] = [r for r in waiting if id(r) not in ids]
        cells = sum(r.f.shape[0] for r in chosen)
        vals = sum(r.f.shape[0] * _n_per_cell(r.shape) for r in chosen)
        fo, qo = allocs[0][0], allocs[1][0]
        wo, wn = allocs[-1]
        st = self.streams[slot]
        with torch.cuda.stream(st):
            v = 0
            for r in chosen:
                n = r.f.shape[0] * _n_per_cell(r.shape)
                self.arena.view(fo + 8 * v, n).copy_(_host(r.f).reshape(-1), non_blocking=True)
                r.admitted = now
                v += n
            try:
                if self.ragged:
                    to = allocs[2][0]
                    self.arena.view(to, cells * 12, torch.uint8).copy_(self._tags(slot, chosen, cells),
                                                                       non_blocking=True)
                    wef_evaluate_ragged(self.handles, self.arena.ptr(to + 8 * cells), self.arena.ptr(to),
                                        self.arena.ptr(fo), self.arena.ptr(qo), cells, self.prec,
                                        self.arena.ptr(wo), wn, st.cuda_stream)
                else:
                    wef_evaluate(self.ops[chosen[0].shape].h, self.arena.ptr(fo), self.arena.ptr(qo), cells,
                                 self.prec, self.arena.ptr(wo), wn, st.cuda_stream)
            except Exception:
                # the evaluation was refused or failed to launch: once the work already
                # queued on the slot has finished, return the memory to the arena and the
                # requests to the front of the queue
                st.synchronize()
                for o, ln in allocs:
                    self.arena.release(o, ln)
                waiting[:0] = chosen
                raise
            # deliver every request's Q to its host output, then mark the batch done
            v = 0
            for r in chosen:
                n = r.f.shape[0] * _n_per_cell(r.shape)
                if r.out is None:
                    r.out = torch.empty(tuple(r.f.shape), dtype=torch.float64)
                r.out.reshape(-1).copy_(self.arena.view(qo + 8 * v, n), non_blocking=True)
                v += n
            ev = torch.cuda.Event(blocking=True)
            ev.record(st)
        self.slot_busy[slot] = (chosen, allocs)
        self.batches += 1
        self.batch_log.append(list(chosen))
        threading.Thread(target=self._waiter, args=(slot, ev), daemon=True).start()
        return True

    def _waiter(self, slot, ev):
        ev.synchronize()
        self._done.put(slot)

    def wait(self, timeout):
        """Block until a batch completes or `timeout` seconds pass (None: until a completion)."""
        if self.idle():
            if timeout:
                time.sleep(timeout)
            return
        try:
            self._ready.append(self._done.get(timeout=timeout))
        except queue.Empty:
            pass

    def poll(self, now_fn):
        """Complete every batch whose results are in host memory; returns how many requests completed."""
        while True:
            try:
                self._ready.append(self._done.get_nowait())
            except queue.Empty:
                break
        k = 0
        for slot in self._ready:
            chosen, allocs = self.slot_busy[slot]
            t = now_fn()
            for r in chosen:
                r.done = t
                self.completed.append(r)
                k += 1
            for o, ln in allocs:
                self.arena.release(o, ln)
            self.slot_busy[slot] = None
        self._ready = []
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


def _percentiles(lat_s):
    lat = np.asarray(lat_s)
    if not lat.size:
        return {"requests": 0, "p50_ms": None, "p99_ms": None}
    return {"requests": int(lat.size), "p50_ms": float(np.percentile(lat, 50) * 1e3),
            "p99_ms": float(np.percentile(lat, 99) * 1e3)}


def run(server, requests, time_limit=None, small_cells=64, large_cells=1024):
    """Replay `requests` (arrival times in seconds from now) through `server`; returns a
    summary with p50/p99 arrival-to-completion latency (result in host memory), the same for
    small (<= small_cells) and large (>= large_cells) requests, and throughput."""
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
        if pending and pending[0].arrival <= now():
            continue
        if waiting and server.idle():
            continue  # memory freed by the completions just polled
        server.wait(max(pending[0].arrival - now(), 0.0) if pending else None)
    wall = now()
    lat = np.array([r.done - r.arrival for r in server.completed])
    cells = int(sum(r.f.shape[0] for r in server.completed))
    out = {
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
    out["small"] = _percentiles([r.done - r.arrival for r in server.completed if r.f.shape[0] <= small_cells])
    out["large"] = _percentiles([r.done - r.arrival for r in server.completed if r.f.shape[0] >= large_cells])
    return out
