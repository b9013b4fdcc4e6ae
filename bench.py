"""Benchmark: batched Q(f, f) cell-evaluations per second on GB300.

Workload (one step = one pass of the whole hot path over one batch): hard spheres
(gamma = 1), Kmax = Lmax = 12, 16384 cells, each cell a seeded two-Maxwellian
mixture projected onto the basis; core from the library's own quadrature.
The batch (288 MB of f in, 288 MB of Q out) is larger than the 129 MB L2, so no
flush is needed between steps.

    python bench.py [--gpus N] [--steps K] [--warmup W] [--precision rf32|tf32|bf16|fp64] [--impl ours|reference]

The headline is the mixed-precision radial-first path (radial contraction in FP32 with
FP32 accumulation, the Gaunt reduction and the conservation projection in FP64).  The
same run also times the angular-first paths (plain FP64; FP64 angular coupling with the
radial stage on the tcgen05 tensor cores in BF16 or TF32) with the same protocol and
reports them under "variants" with the speedup over plain FP64.
Prints one JSON line (rank 0).  Under torchrun every rank evaluates its own batch
(weak scaling, no data-path collective); the barrier and the max over ranks of
the timed region are the only collectives.
"""
import argparse
import functools
import json
import os
import queue
import statistics
import subprocess
import sys
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

KMAX = LMAX = 12
GAMMA = 1.0
NCELLS = 16384
METRIC = "Q(f,f) cell-evals/s at K=L=12"
PEAKS_FILE = os.path.join(ROOT, "MEASURED_PEAKS.json")
# FP64 FMA pipe: 2 DFMA lanes per SM per clock on GB300 (measured: 1.20 TFLOP/s at
# 1987 MHz with full warps), x 152 SMs x 2 flops x 2070 MHz maximum clock.
FP64_PEAK_TFLOPS = 152 * 2 * 2 * 2.070e9 / 1e12
# DRAM bytes (read + write) of one launch of the dominant kernel at the default workload
# (K=L=12, 16384 cells), from a one-pass ncu capture of the timed step's launch
# (dram__bytes_read.sum 215.83 MB + dram__bytes_write.sum 278.35 MB; command and reading in
# profiles/rf_kernel_13_traffic_kl12_16384cells.md).  Re-capture whenever the kernel changes.
TRAFFIC_BYTES = {"rf32": 494.18e6}
TRAFFIC_NOTE = ("captured with the kernel version of this file's commit (FP64 accumulators in tensor memory, two "
                "CTAs per SM, 24 MB L2 tile groups, J = 3, packed FP32x2 stages); shared-memory accumulators moved "
                "486.7 MB, 48 MB tile groups 728.7 MB")
# arithmetic types of each path: FP64 reductions and projection, plus the radial products
DTYPES = {"fp64": "f64", "bf16": "f64+bf16", "tf32": "f64+tf32", "rf32": "f64+f32", "rftc": "f64+f32+3xtf32"}


def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=5)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--precision", default="rf32", choices=["fp64", "bf16", "tf32", "rf32", "rftc"])
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--ncells", type=int, default=NCELLS)
    ap.add_argument("--kl", type=int, default=KMAX, help="Kmax = Lmax of the main workload (default 12)")
    ap.add_argument("--cpu-sample-rows", type=int, default=None,
                    help="output rows of each sampled cell the CPU oracle evaluates (default: all N)")
    ap.add_argument("--cpu-sample-cells", type=int, default=4)
    ap.add_argument("--workload", default="kl12",
                    choices=["kl12", "maxwell4", "hs8", "ragged", "serve", "baselines", "rk4", "core"],
                    help="kl12: hard spheres K=L=12 x 16384 cells (default); maxwell4: one Maxwell cell at "
                         "K=L=4; hs8: hard spheres K=L=8 x 4096 cells; ragged: VHS, 32768 cells with "
                         "(Kmax, Lmax) drawn from {6,8,10,12,16}; serve: Poisson request stream; baselines: "
                         "factorised vs naive-COO vs dense tensor at K=L=8; rk4: device RK4 and linearized "
                         "products at K=L=12; core: GPU vs host assembly of the core at K=L=12")
    ap.add_argument("--duration", type=float, default=60.0, help="serve: seconds of arrivals")
    ap.add_argument("--serve-slots", type=int, default=16, help="serve: stream slots (batches in flight)")
    ap.add_argument("--serve-batch-ms", type=float, default=20.0, help="serve: estimated GPU time cap per batch")
    ap.add_argument("--serve-max-wait-ms", type=float, default=100.0,
                    help="serve: size-aware admission bound (0: arrival order)")
    ap.add_argument("--variants", default="all", choices=["all", "none"],
                    help="kl12: also time the other precisions (all) or only --precision (none)")
    return ap.parse_args()


def max_over_ranks(ms_local, dist, device=None):
    """The timed region's duration as the max over ranks (every rank gets it)."""
    if dist is None:
        return ms_local
    import torch

    t = torch.tensor([float(ms_local)], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    dist.barrier()
    return float(t.item())


def job_throughput(world, ncells_per_rank, ms_step):
    """Whole-job cells/s: all ranks' cells divided by the (max over ranks) step time."""
    return world * ncells_per_rank / (ms_step / 1e3)


def dist_env():
    rank = int(os.environ.get("RANK", "0"))
    world = int(os.environ.get("WORLD_SIZE", "1"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return rank, world, local


def inputs(ncells, seed):
    import wef_inputs as wi

    return wi.two_maxwellians(KMAX, LMAX, ncells, seed=seed, pool=min(1024, ncells))


@functools.lru_cache(maxsize=None)
def cpu_model():
    """The host CPU's model name (lscpu, else /proc/cpuinfo, else the machine type)."""
    try:
        out = subprocess.run(["lscpu"], capture_output=True, text=True, timeout=10).stdout
        for line in out.splitlines():
            if line.strip().startswith("Model name:"):
                return line.split(":", 1)[1].strip()
    except (OSError, subprocess.SubprocessError):
        pass
    try:
        with open("/proc/cpuinfo") as fh:
            for line in fh:
                if line.startswith("model name"):
                    return line.split(":", 1)[1].strip()
    except OSError:
        pass
    import platform

    return platform.machine()


REFERENCE_STEP_ROWS = 384  # output rows per reference-arm step: a few seconds of CPU work


def sample_rows_of(rows):
    """Output rows per sampled cell for the CPU oracle: all N by default, at most N."""
    N = (KMAX + 1) * (LMAX + 1) ** 2
    return N if rows is None or rows <= 0 else min(int(rows), N)


def cpu_baseline(sample_cells, sample_rows=None, seed=3, with_angular_first=False, R=None, f=None):
    """The oracle (dense FP64 CPU contraction) timed on a bounded sample of the workload:
    `sample_cells` cells and `sample_rows` of the N output rows (default all), scaled to
    cells/s.  R, f: the workload's own core and cells (the sample is f's first cells); by
    default a random stand-in core (the timing does not depend on the values) and fresh
    two-Maxwellian cells.  Returns (line object, Q and the sums of |terms| of the sampled
    cells and rows, the rows).  With `with_angular_first`, also the paper's factorised
    contraction in numpy (a CPU comparison point, reported inside the object)."""
    import wef_inputs as wi
    from oracle import dense, gaunt

    K, NQ = KMAX + 1, (LMAX + 1) ** 2
    N = K * NQ
    sample_rows = sample_rows_of(sample_rows)
    if R is None:
        R = wi.random_core(len(gaunt.channels(LMAX)), KMAX, seed=11)
    fs = (wi.two_maxwellians(KMAX, LMAX, sample_cells, seed=seed) if f is None else f[:sample_cells])
    fs = np.asarray(fs).reshape(sample_cells, -1)
    op = dense.DenseOperator(KMAX, LMAX, dense.conservation_zeroing(R, LMAX))
    rows = np.sort(np.random.default_rng(seed).choice(N, sample_rows, replace=False))
    t0 = time.perf_counter()
    Qo, T = op.evaluate_rows_with_terms(fs, rows)
    dt = time.perf_counter() - t0
    value = sample_cells * (sample_rows / N) / dt
    out = {
        "value": value,
        "unit": "cells/s",
        "cores": os.cpu_count(),
        "cpu_model": cpu_model(),
        "kind": "oracle",
        "sample": f"{sample_cells} cells x {sample_rows} of {N} output rows (dense C slices, Q and its sums of "
        f"|terms|), {dt:.1f} s; numpy BLAS threads default (all {os.cpu_count()} host cores)",
    }
    if with_angular_first:
        out["angular_first"] = cpu_angular_first()
        try:  # a comparison figure only: its failure must not cost the benchmark line
            out["angular_first_all_cores"] = cpu_angular_first_all_cores()
        except Exception as e:  # noqa: BLE001
            out["angular_first_all_cores"] = {"error": f"{type(e).__name__}: {e}"}
    return out, (Qo, T, rows)


ERROR_EPS = 2.0 ** -10  # cancellation floor of the per-cell error, relative to the sums of |terms|


def error_vs_oracle(Q, Qo, T):
    """Per-cell error of Q [cells, rows] against the oracle: max_a |Q - Qo| over the cell's
    rows divided by max(max_a |Qo|, ERROR_EPS * max_a T) (the infinity norm of the cell,
    guarded against cancellation), reported as max and median over the cells, with the
    plain per-cell relative error beside it."""
    d = np.max(np.abs(Q - Qo), axis=1)
    qn = np.max(np.abs(Qo), axis=1)
    g = d / np.maximum(np.maximum(qn, ERROR_EPS * np.max(T, axis=1)), 1e-300)
    r = d / np.maximum(qn, 1e-300)
    return {"max": float(np.max(g)), "median": float(np.median(g)), "plain_rel_max": float(np.max(r)),
            "plain_rel_median": float(np.median(r))}


def cpu_angular_first(sample_cells=32, seed=3):
    """The paper's factorised angular-first contraction (Sec. 4.5.4) in plain numpy on the
    host, timed on `sample_cells` cells: a CPU comparison point for the factorisation."""
    import wef_inputs as wi
    from oracle import angular_first, gaunt

    R = wi.random_core(len(gaunt.channels(LMAX)), KMAX, seed=11)
    f = wi.two_maxwellians(KMAX, LMAX, sample_cells, seed=seed)
    sl = angular_first.slices(LMAX)
    t0 = time.perf_counter()
    angular_first.evaluate(KMAX, LMAX, R, f, sl=sl)
    dt = time.perf_counter() - t0
    return {"value": sample_cells / dt, "unit": "cells/s", "cores": 1, "cpu_model": cpu_model(),
            "kind": "angular-first numpy (Sec. 4.5.4)",
            "sample": f"{sample_cells} cells, {dt:.1f} s; numpy einsum without BLAS: one thread"}


def _angular_first_worker(barrier, results, seed, cells):
    """One process of cpu_angular_first_all_cores: set-up, wait for every process, evaluate."""
    import wef_inputs as wi
    from oracle import angular_first, gaunt

    R = wi.random_core(len(gaunt.channels(LMAX)), KMAX, seed=11)
    f = wi.two_maxwellians(KMAX, LMAX, cells, seed=seed)
    sl = angular_first.slices(LMAX)
    barrier.wait(timeout=600)
    t0 = time.perf_counter()
    angular_first.evaluate(KMAX, LMAX, R, f, sl=sl)
    results.put((cells, t0, time.perf_counter()))


def cpu_angular_first_all_cores(cells_per_process=24, seed=3, processes=None, time_limit_s=300.0):
    """The same numpy angular-first contraction on every host core (or on `processes`
    cores): one spawned process per core, each on its own cells, released together by a
    barrier; throughput = all cells over the wall time from the first start to the last
    finish."""
    import multiprocessing as mp

    n = processes or os.cpu_count() or 1
    ctx = mp.get_context("spawn")
    barrier, results = ctx.Barrier(n), ctx.Queue()
    procs = [ctx.Process(target=_angular_first_worker, args=(barrier, results, seed + i, cells_per_process))
             for i in range(n)]
    for p in procs:
        p.start()
    got, deadline = [], time.monotonic() + time_limit_s
    try:
        while len(got) < n:
            try:
                got.append(results.get(timeout=1.0))
            except queue.Empty:
                if time.monotonic() > deadline:
                    raise RuntimeError(f"not finished within {time_limit_s:.0f} s")
                # a process that has exited without its result will never send it
                if any(p.exitcode not in (None, 0) for p in procs):
                    raise RuntimeError("a worker process failed")
    finally:
        for p in procs:
            p.join(timeout=5 if len(got) == n else 0)
            if p.is_alive():
                p.terminate()
                p.join(timeout=5)
    cells = sum(g[0] for g in got)
    wall = max(g[2] for g in got) - min(g[1] for g in got)
    return {"value": cells / wall, "unit": "cells/s", "cores": n, "cpu_model": cpu_model(),
            "kind": "angular-first numpy (Sec. 4.5.4), one process per core",
            "sample": f"{n} processes x {cells_per_process} cells, {wall:.1f} s wall from first start to last finish"}


class ClockSampler:
    """nvidia-smi samples of SM clock, power and throttle reasons while running."""

    FIELDS = "clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,clocks_event_reasons.hw_slowdown," \
             "clocks_event_reasons.hw_thermal_slowdown,clocks_event_reasons.sw_thermal_slowdown," \
             "clocks_event_reasons.sw_power_cap"

    def __init__(self, index):
        self.index = index
        self.proc = None

    def __enter__(self):
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", "-i", str(self.index), f"--query-gpu={self.FIELDS}", "--format=csv,noheader,nounits",
                 "-lms", "200"], stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
        except OSError:
            self.proc = None
        return self

    def __exit__(self, *a):
        self.lines = []
        if self.proc is not None:
            self.proc.terminate()
            out, _ = self.proc.communicate(timeout=10)
            self.lines = [ln for ln in out.splitlines() if ln.strip()]

    def summary(self):
        sm, mx, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for ln in getattr(self, "lines", []):
            p = [x.strip() for x in ln.split(",")]
            try:
                sm.append(float(p[0]))
                mx.append(float(p[1]))
            except (ValueError, IndexError):
                continue
            for n, v in zip(names, p[4:8]):
                if v.lower() == "active":
                    reasons.add(n)
        if not sm:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["unsampled"]}
        return {"sm_mhz": statistics.median(sm), "sm_max_mhz": max(mx), "reasons": sorted(reasons), "samples": len(sm)}


def fp64_probe():
    """Live FP64 FMA pipe throughput from the package's probe utility (None if not built)."""
    exe = os.path.join(ROOT, "paper_2605_28475_gb300", "_build", "fp64_peak")
    if not os.path.exists(exe):
        return None
    try:
        out = subprocess.run([exe], capture_output=True, text=True, timeout=120)
        return json.loads(out.stdout.strip().splitlines()[-1]) if out.returncode == 0 else None
    except (OSError, ValueError, subprocess.TimeoutExpired, IndexError):
        return None


def run_reference(args, rank, world):
    """The reference arm: the oracle (dense FP64 CPU contraction) on the host cores, W warm-up
    and K timed steps, each step a bounded sample of the workload (`--cpu-sample-cells`
    cells x `--cpu-sample-rows` output rows); rank 0 only (no GPU work)."""
    if rank != 0:
        return
    rows = args.cpu_sample_rows or REFERENCE_STEP_ROWS  # per step; the headline's sample takes all rows
    for _ in range(args.warmup):
        cpu_baseline(args.cpu_sample_cells, rows)
    t0 = time.perf_counter()
    samples = [cpu_baseline(args.cpu_sample_cells, rows)[0] for _ in range(max(args.steps, 1))]
    dt = time.perf_counter() - t0
    cells_per_step = args.cpu_sample_cells * sample_rows_of(rows) / ((KMAX + 1) * (LMAX + 1) ** 2)
    value = cells_per_step * len(samples) / dt
    cb = dict(samples[-1])
    cb["value"] = value
    cb["sample"] = f"{len(samples)} steps of " + cb["sample"]
    line = {
        "impl": "reference", "metric": METRIC, "value": value, "unit": "cells/s", "n_gpus": args.gpus,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1e3 * dt / len(samples), "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
        "config": {"workload": f"hard spheres, Kmax=Lmax={KMAX}, two-Maxwellian cells (bounded CPU sample per step)"},
        "cpu_baseline": cb, "e2e": {"value": value, "unit": "cells/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }
    print(json.dumps(line), flush=True)


# ------------------------------------------------------------------ further workloads
def _line(metric, value, unit, ms, args, world, dtype, workload, hib=True, **kw):
    d = {"metric": metric, "value": value, "unit": unit, "n_gpus": world, "steps": args.steps, "warmup": args.warmup,
         "ms_per_step": ms, "higher_is_better": hib, "scaling": "weak", "vs_baseline": None, "dtype": dtype,
         "data": "synthetic", "config": {"workload": workload}}
    d.update(kw)
    return d


def _time_steps(step, steps, warmup, stream, torch):
    for _ in range(warmup):
        step()
    torch.cuda.synchronize()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    for _ in range(steps):
        step()
    e1.record(stream)
    torch.cuda.synchronize()
    return e0.elapsed_time(e1) / steps


def bench_small(args, W, torch, dev, world, kind):
    """maxwell4: one perturbed-Maxwellian cell, Maxwell molecules, K=L=4, FP64 (latency);
    hs8: 4096 two-Maxwellian cells, hard spheres, K=L=8, FP64 (cells/s)."""
    import wef_inputs as wi

    if kind == "maxwell4":
        km, gamma, n, f_host = 4, 0.0, 1, wi.perturbed_maxwellian(4, 4, 1, seed=1)
    else:
        km, gamma, n, f_host = 8, 1.0, 4096, wi.two_maxwellians(8, 8, 4096, seed=2, pool=1024)
    op = W.Operator(km, km, gamma)
    op.upload_core(op.build_core(device=True))
    f = torch.from_numpy(f_host).to(dev)
    q = torch.empty_like(f)
    st = torch.cuda.current_stream(dev)
    ws = op.workspace(n, 0, dev)
    step = lambda: W.wef_evaluate(op.h, f.data_ptr(), q.data_ptr(), n, 0, ws.data_ptr(), ws.numel(), st.cuda_stream)  # noqa: E731
    ms = _time_steps(step, max(args.steps, 20), args.warmup, st, torch)
    fp64_flops, _ = W.wef_flops(op.h, 0)
    wl = ("Maxwell molecules, Kmax=Lmax=4, 1 perturbed-Maxwellian cell, FP64" if kind == "maxwell4" else
          "hard spheres, Kmax=Lmax=8, 4096 two-Maxwellian cells, FP64")
    if kind == "maxwell4":
        # device latency: 50 evaluations captured back to back in one CUDA graph, replayed
        reps = 50
        g = torch.cuda.CUDAGraph()
        with torch.cuda.graph(g):
            cs = torch.cuda.current_stream(dev).cuda_stream
            for _ in range(reps):
                W.wef_evaluate(op.h, f.data_ptr(), q.data_ptr(), n, 0, ws.data_ptr(), ws.numel(), cs)
        for _ in range(3):
            g.replay()
        torch.cuda.synchronize(dev)
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(st)
        for _ in range(max(args.steps, 5)):
            g.replay()
        e1.record(st)
        torch.cuda.synchronize(dev)
        dev_us = e0.elapsed_time(e1) * 1e3 / (max(args.steps, 5) * reps)
        # what a caller sees: one synchronous call (launch from Python + wait), median
        wall = []
        for _ in range(200):
            t0 = time.perf_counter()
            step()
            st.synchronize()
            wall.append(time.perf_counter() - t0)
        return _line("Q(f,f) latency, 1 cell, K=L=4", dev_us, "us", dev_us / 1e3, args, world, "f64", wl, hib=False,
                     fp64_flops_per_cell=fp64_flops, latency_note="device time per evaluation (graph of 50 back-to-back "
                     "evaluations, replayed)", sync_call_us_median=1e6 * statistics.median(wall),
                     queued_call_us=ms * 1e3, gpu_launches=2 * reps * max(args.steps, 5))
    return _line("Q(f,f) cell-evals/s at K=L=8", n / (ms / 1e3), "cells/s", ms, args, world, "f64", wl,
                 roofline={"bound": "alu", "achieved": fp64_flops * n / (ms / 1e3) / 1e12, "peak": FP64_PEAK_TFLOPS,
                           "unit": "TFLOP/s", "frac": fp64_flops * n / (ms / 1e3) / 1e12 / FP64_PEAK_TFLOPS,
                           "note": "whole step (re-tiling + contraction)"})


def bench_baselines(args, W, torch, dev, world):
    """Factorised vs unfactorised on the same GPU (Sec. 4.5), hard spheres, Kmax=Lmax=8,
    two-Maxwellian cells, core from the library quadrature: plain FP64 (angular-first),
    radial-first (FP32 radial, FP64 reduction), naive COO loop (FP64) and dense tensor
    (cuBLAS FP64 GEMMs over the assembled N^3 tensor)."""
    import wef_inputs as wi

    km = 8
    op = W.Operator(km, km, 1.0)
    op.upload_core(op.build_core(device=True))
    st = torch.cuda.current_stream(dev)
    n_fact, n_dense = 4096, 256
    f_host = wi.two_maxwellians(km, km, n_fact, seed=2, pool=1024)
    f = torch.from_numpy(f_host).to(dev)
    q = torch.empty_like(f)
    res = {}
    for name, prec in (("fp64", 0), ("rf32", W.PRECISIONS["rf32"])):
        ws = op.workspace(n_fact, prec, dev)
        step = lambda: W.wef_evaluate(op.h, f.data_ptr(), q.data_ptr(), n_fact, prec, ws.data_ptr(), ws.numel(), st.cuda_stream)  # noqa: E731,B023
        res[name] = n_fact / (_time_steps(step, max(args.steps, 5), args.warmup, st, torch) / 1e3)
    ws = torch.empty(max(W.wef_workspace_size(op.h, n_fact, 0), 256), dtype=torch.uint8, device=dev)
    step = lambda: W.wef_naive_evaluate(op.h, f.data_ptr(), q.data_ptr(), n_fact, ws.data_ptr(), ws.numel(), st.cuda_stream)  # noqa: E731
    res["naive_coo"] = n_fact / (_time_steps(step, max(args.steps, 3), args.warmup, st, torch) / 1e3)
    C = torch.empty(W.wef_dense_tensor_size(op.h) // 8, dtype=torch.float64, device=dev)
    W.wef_dense_assemble(op.h, C.data_ptr(), C.numel() * 8, st.cuda_stream)
    wsd = torch.empty(W.wef_dense_workspace_size(op.h, n_dense), dtype=torch.uint8, device=dev)
    fd = f[:n_dense].contiguous()
    qd = torch.empty_like(fd)
    step = lambda: W.wef_dense_evaluate(op.h, C.data_ptr(), fd.data_ptr(), qd.data_ptr(), n_dense, wsd.data_ptr(), wsd.numel(), st.cuda_stream)  # noqa: E731
    res["dense"] = n_dense / (_time_steps(step, 3, 2, st, torch) / 1e3)
    N, K, rfp = op.N, km + 1, W.PRECISIONS["rf32"]
    n_sym = W.wef_flops(op.h, rfp)[0] / (2 * K)  # symmetrised Gaunt entries (2K FP64 flops each there)
    return _line("Q(f,f) cell-evals/s at K=L=8, factorised vs unfactorised (FP64)", res["fp64"], "cells/s", None, args,
                 world, "f64", f"hard spheres, Kmax=Lmax=8, two-Maxwellian cells ({n_fact} per batch; dense: {n_dense}), "
                 f"core from the library quadrature",
                 cells_per_s=res, speedup_vs_dense={k: v / res["dense"] for k, v in res.items()},
                 flops_per_cell={"dense": 2.0 * N**3, "naive_coo": n_sym * 2.0 * (K**3 + K**2 + K),
                                 "fp64": W.wef_flops(op.h, 0)[0], "rf32_fp64": W.wef_flops(op.h, rfp)[0],
                                 "rf32_fp32": W.wef_flops(op.h, rfp)[1]})


def bench_rk4(args, W, torch, dev, world, ncells=16384, nrk=4):
    """Time integration on the device: RK4 steps of df/dt = Q(f, f) for every cell (four
    evaluations per step), hard spheres, Kmax=Lmax=12, two-Maxwellian cells; and linearized
    products L d at per-cell base states (three evaluations each)."""
    import wef_inputs as wi

    op = W.Operator(KMAX, LMAX, GAMMA)
    op.upload_core(op.build_core(device=True))
    f0 = torch.from_numpy(inputs(ncells, seed=3)).to(dev)
    f = f0.clone()
    d = torch.from_numpy(wi.random_cells(KMAX, LMAX, ncells, seed=9)).to(dev)
    st = torch.cuda.current_stream(dev)
    prec = W.PRECISIONS[args.precision]
    step = lambda: op.integrate(f, 1e-3, nrk, precision=prec)  # noqa: E731
    ms = _time_steps(step, args.steps, args.warmup, st, torch)
    out = torch.empty_like(d)
    lstep = lambda: op.linearized_apply(f0, d, out, precision=prec)  # noqa: E731
    ms_l = _time_steps(lstep, args.steps, args.warmup, st, torch)
    dtype = DTYPES[args.precision]
    return _line("RK4 cell-steps/s at K=L=12", ncells * nrk / (ms / 1e3), "cell-steps/s", ms, args, world, dtype,
                 f"hard spheres, Kmax=Lmax=12, {ncells} two-Maxwellian cells, {nrk} RK4 steps (dt=1e-3) per timed "
                 f"step, {args.precision} evaluations",
                 evaluations_per_s=4 * ncells * nrk / (ms / 1e3),
                 linearized_products_per_s=ncells / (ms_l / 1e3))


def bench_core(args, W, torch, dev, world):
    """Assembly of the kinematic core (Sec. 4.3, Appendix A-B) at Kmax=Lmax=12, hard spheres,
    paddings 20/20: on the GPU (FP64) against the host builder on all host cores."""
    op = W.Operator(KMAX, LMAX, GAMMA)
    op.build_core(device=True)  # warm-up (context, module load)
    t = []
    for _ in range(max(1, min(args.steps, 3))):
        torch.cuda.synchronize(dev)
        t0 = time.perf_counter()
        Rd = op.build_core(device=True)
        t.append(time.perf_counter() - t0)
    t0 = time.perf_counter()
    Rh = op.build_core()
    th = time.perf_counter() - t0
    sec = statistics.median(t)
    K = KMAX + 1
    # radial points x channels x K^3 FMAs (the dominant contraction), 2 flops each
    return _line("core assembly seconds at K=L=12", sec, "s", sec * 1e3, args, world, "f64",
                 "hard spheres, Kmax=Lmax=12, 616 channels, paddings 20/20, GPU assembly (median of runs) vs the host "
                 "builder on all host cores", hib=False, host_seconds=th, host_cores=os.cpu_count(),
                 max_rel_diff=float(np.max(np.abs(Rd - Rh)) / np.max(np.abs(Rh))), K=K)


def bench_ragged(args, W, torch, dev, world, ncells=32768, seed=4):
    """VHS gamma=0.5, ncells cells with (Kmax, Lmax) drawn independently from {6,8,10,12,16},
    grouped by shape; one persistent TF32 launch replayed from a CUDA graph, autotuned."""
    import wef_inputs as wi

    vals = [6, 8, 10, 12, 16]
    rng = np.random.Generator(np.random.PCG64(seed))
    draws = rng.integers(0, 5, (ncells, 2))
    shapes = [(vals[a], vals[b]) for a in range(5) for b in range(5)]
    counts = [int(np.sum((draws[:, 0] == a) & (draws[:, 1] == b))) for a in range(5) for b in range(5)]
    ops, fs = [], []
    real = os.environ.get("WEF_BENCH_QUADRATURE_CORES") == "1"
    for i, ((km, lm), n) in enumerate(zip(shapes, counts)):
        op = W.Operator(km, lm, 0.5)
        R = op.build_core(device=True) if real else wi.random_core(op.n_channels, km, seed=100 + i)
        op.upload_core(R)
        ops.append(op)
        fs.append(wi.two_maxwellians(km, lm, n, seed=200 + i, pool=min(256, max(n, 1))).reshape(-1))
    f = torch.from_numpy(np.concatenate(fs)).to(dev)
    q = torch.empty_like(f)
    plan = W.wef_plan_create([o.h for o in ops], counts, W.WEF_MIXED_TF32, 0)
    ws = torch.empty(W.wef_plan_workspace_size(plan), dtype=torch.uint8, device=dev)
    st = torch.cuda.current_stream(dev)
    g = W.wef_plan_autotune(plan, f.data_ptr(), q.data_ptr(), ws.data_ptr(), ws.numel(), st.cuda_stream)
    step = lambda: W.wef_plan_graph_launch(plan, f.data_ptr(), q.data_ptr(), ws.data_ptr(), ws.numel(), st.cuda_stream)  # noqa: E731
    ms = _time_steps(step, args.steps, args.warmup, st, torch)
    W.wef_plan_status(plan)
    flops = sum(W.wef_flops(o.h, W.WEF_MIXED_TF32)[0] * n for o, n in zip(ops, counts))
    achieved = flops / (ms / 1e3) / 1e12
    W.wef_plan_destroy(plan)
    # the same ragged batch through a radial-first plan (one persistent launch per shape on
    # autotuned concurrent streams, graph-replayed), for comparison
    rplan = W.wef_plan_create([o.h for o in ops], counts, W.WEF_RADIAL_FP32, 0)
    rws = torch.empty(W.wef_plan_workspace_size(rplan), dtype=torch.uint8, device=dev)
    rg = W.wef_plan_autotune(rplan, f.data_ptr(), q.data_ptr(), rws.data_ptr(), rws.numel(), st.cuda_stream)
    rstep = lambda: W.wef_plan_graph_launch(rplan, f.data_ptr(), q.data_ptr(), rws.data_ptr(), rws.numel(), st.cuda_stream)  # noqa: E731
    rms = _time_steps(rstep, args.steps, args.warmup, st, torch)
    W.wef_plan_destroy(rplan)
    # the same batch through wef_evaluate_ragged: each cell's operator and offset as device
    # arrays, the batch's composition worked out on the device (no plan), cells shuffled
    perm = torch.from_numpy(np.random.default_rng(seed).permutation(ncells)).to(dev)
    sizes = [(km + 1) * (lm + 1) ** 2 for km, lm in shapes]
    sid = torch.from_numpy(np.repeat(np.arange(len(shapes), dtype=np.int32), counts)).to(dev)
    starts = np.concatenate([[0], np.cumsum([n * sz for n, sz in zip(counts, sizes)])[:-1]])
    off = torch.from_numpy(np.concatenate([st0 + sz * np.arange(n, dtype=np.int64)
                                           for st0, sz, n in zip(starts, sizes, counts)])).to(dev)
    sid, off = sid[perm].contiguous(), off[perm].contiguous()
    hs = [o.h for o in ops]
    gws = torch.empty(W.wef_ragged_workspace_size(hs, ncells, W.WEF_RADIAL_FP32), dtype=torch.uint8, device=dev)
    gstep = lambda: W.wef_evaluate_ragged(hs, sid.data_ptr(), off.data_ptr(), f.data_ptr(), q.data_ptr(), ncells,  # noqa: E731
                                          W.WEF_RADIAL_FP32, gws.data_ptr(), gws.numel(), st.cuda_stream)
    gms = _time_steps(gstep, args.steps, args.warmup, st, torch)
    return _line("Q(f,f) cell-evals/s, ragged (Kmax,Lmax) in {6..16}^2", ncells / (ms / 1e3), "cells/s", ms, args, world,
                 "f64+tf32",
                 f"VHS gamma=0.5, {ncells} cells, (Kmax, Lmax) drawn independently per cell, 25 shapes grouped; one "
                 f"persistent launch under a CUDA graph; autotuned granularity {g}; cores "
                 + ("from the library quadrature" if real else "random stand-ins (timing does not depend on values)"),
                 roofline={"bound": "alu", "achieved": achieved, "peak": FP64_PEAK_TFLOPS, "unit": "TFLOP/s",
                           "frac": achieved / FP64_PEAK_TFLOPS, "fp64_flops_total": flops},
                 gpu_launches=2 * args.steps,
                 ragged_call={"cells_per_s": ncells / (gms / 1e3), "ms_per_step": gms,
                              "note": "same batch, cells shuffled, through wef_evaluate_ragged (per-cell operator and "
                                      "offset on the device; set-up kernels, then each operator's persistent "
                                      "radial-first launch on streams forked from the caller's)"},
                 radial_first={"cells_per_s": ncells / (rms / 1e3), "ms_per_step": rms, "fork_streams": rg % 16,
                               "tile_group_mb": rg // 16 or 24,
                               "note": "same batch, radial-first plan: per-shape persistent launches on concurrent "
                                       "streams in one CUDA graph"})


def serving_leg(args, W, torch, dev, duration):
    """Configuration 5: a seeded Poisson stream of requests (1-4096 cells, Kmax=Lmax drawn from
    {8,10,12,16}, hard-sphere-sized operators) served by the continuous-batching loop at 0.7x
    the measured capacity for `duration` seconds of arrivals.  Requests read their cells from
    per-shape pinned pools and receive their Q in per-shape pinned result buffers (set up
    before serving); latency runs from arrival to the result in host memory."""
    import wef_inputs as wi
    from paper_2605_28475_gb300 import serve

    shapes = [(8, 8), (10, 10), (12, 12), (16, 16)]
    real = os.environ.get("WEF_BENCH_QUADRATURE_CORES") == "1"
    ops = {}
    for i, (km, lm) in enumerate(shapes):
        op = W.Operator(km, lm, 1.0)
        op.upload_core(op.build_core(device=True) if real else wi.random_core(op.n_channels, km, seed=300 + i))
        ops[(km, lm)] = op
    prec = W.PRECISIONS[args.precision]
    st = torch.cuda.current_stream(dev)
    max_cells = 4096
    # capacity: full-batch throughput per shape at the serving precision
    cap, pools = {}, {}
    for sh, op in ops.items():
        n = 2048
        f = torch.from_numpy(wi.random_cells(sh[0], sh[1], n, seed=1)).to(dev)
        q = torch.empty_like(f)
        ws = op.workspace(n, prec, dev)
        step = lambda: W.wef_evaluate(op.h, f.data_ptr(), q.data_ptr(), n, prec, ws.data_ptr(), ws.numel(), st.cuda_stream)  # noqa: E731,B023
        ms = _time_steps(step, 3, 1, st, torch)
        cap[sh] = n / (ms / 1e3)  # cells/s at this shape
        pools[sh] = (torch.from_numpy(wi.random_cells(sh[0], sh[1], max_cells, seed=2)).pin_memory(),
                     torch.empty(max_cells, sh[0] + 1, (sh[1] + 1) ** 2, dtype=torch.float64).pin_memory())
    # mean service time of a request (log-uniform size, uniform shape) at full-batch speed
    sizes = np.exp(np.linspace(0, np.log(max_cells), 2001))
    mean_cells = float(np.mean(sizes))
    mean_service = float(np.mean([mean_cells / cap[sh] for sh in shapes]))
    rate = 0.7 / mean_service
    reqs = serve.poisson_requests(rate, duration, shapes, max_cells, seed=5,
                                  make_cells=lambda sh, n, s: pools[sh][0][:n])
    for r in reqs:
        r.out = pools[r.shape][1][:r.f.shape[0]]
    cost = {sh: 1.0 / c for sh, c in cap.items()}
    # batches capped at ~50 ms of estimated GPU time so that small requests do not queue
    # behind one huge batch (a single larger request still goes alone)
    srv = serve.Server(ops, arena_bytes=24 << 30, nslots=args.serve_slots, precision=args.precision, device=str(dev),
                       cost_per_cell=cost, max_batch_s=args.serve_batch_ms / 1e3,
                       max_wait_s=args.serve_max_wait_ms / 1e3 if args.serve_max_wait_ms > 0 else None)
    with ClockSampler(dev.index or 0) as clk:
        res = serve.run(srv, reqs)
    res["clocks"] = clk.summary()
    res.update(rate_req_per_s=rate, duration_s=duration, ragged_batches=srv.ragged,
               capacity_cells_per_s={f"{k[0]}x{k[1]}": v for k, v in cap.items()},
               note=(f"Poisson arrivals at 0.7x capacity ({rate:.1f} req/s) for {duration:.0f} s; sizes log-uniform "
                     f"1-{max_cells} cells; Kmax=Lmax in {{8,10,12,16}}; {args.serve_slots} stream slots; 24 GiB admission "
                     f"arena; batches {'mixing every shape (wef_evaluate_ragged)' if srv.ragged else 'of one shape'}, "
                     f"capped at {args.serve_batch_ms:g} ms of estimated GPU time; "
                     + (f"size-aware admission (waiting > {args.serve_max_wait_ms:g} ms first, then cheapest first); "
                        if args.serve_max_wait_ms > 0 else "arrival order; ")
                     + f"latency = arrival to Q in pinned "
                     f"host memory (small: requests of <= 64 cells, large: >= 1024 cells); cores "
                     + ("from the library quadrature" if real else "random stand-ins (timing does not depend on values)")))
    for op in ops.values():
        op.close()
    return res


def bench_serve(args, W, torch, dev, world):
    """Serving alone (configuration 5), as its own JSON line."""
    res = serving_leg(args, W, torch, dev, args.duration)
    return _line("serve: p50/p99 latency and cells/s", res["cells_per_s"], "cells/s", None, args, world,
                 DTYPES[args.precision], res["note"], serving=res)


def main():
    global KMAX, LMAX, METRIC
    args = parse()
    if args.kl != KMAX:
        KMAX = LMAX = args.kl
        METRIC = f"Q(f,f) cell-evals/s at K=L={KMAX}"
    rank, world, local = dist_env()
    if args.impl == "reference":
        run_reference(args, rank, world)
        return
    import torch

    import paper_2605_28475_gb300 as W

    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)
    dist = None
    if world > 1:
        import torch.distributed as dist

        dist.init_process_group("nccl", device_id=dev)
    if args.workload != "kl12":
        fn = {"maxwell4": lambda: bench_small(args, W, torch, dev, world, "maxwell4"),
              "hs8": lambda: bench_small(args, W, torch, dev, world, "hs8"),
              "ragged": lambda: bench_ragged(args, W, torch, dev, world),
              "serve": lambda: bench_serve(args, W, torch, dev, world),
              "baselines": lambda: bench_baselines(args, W, torch, dev, world),
              "rk4": lambda: bench_rk4(args, W, torch, dev, world),
              "core": lambda: bench_core(args, W, torch, dev, world)}[args.workload]
        line = fn()
        if rank == 0:
            print(json.dumps(line), flush=True)
        if dist:
            dist.destroy_process_group()
        return
    probe = fp64_probe() if rank == 0 else None
    op = W.Operator(KMAX, LMAX, GAMMA)
    R = op.build_core(device=True)  # the library quadrature, assembled on the GPU
    op.upload_core(R)
    ncells = args.ncells
    f_host = inputs(ncells, seed=3 + rank)
    f = torch.from_numpy(f_host).to(dev)
    q = torch.empty_like(f)
    stream = torch.cuda.current_stream(dev)

    def measure(precision, with_clocks=False):
        prec = W.PRECISIONS[precision]
        ws = op.workspace(ncells, prec, dev)

        def step(ev=None):
            if ev is not None:
                W.wef_set_trace_events(op.h, ev[0].cuda_event, ev[1].cuda_event)
            W.wef_evaluate(op.h, f.data_ptr(), q.data_ptr(), ncells, prec, ws.data_ptr(), ws.numel(), stream.cuda_stream)

        for _ in range(args.warmup):
            step()
        torch.cuda.synchronize(dev)
        kev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(args.steps)]
        for a, b in kev:  # torch creates the CUDA events lazily, on first record
            a.record(stream)
            b.record(stream)
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        if dist:
            dist.barrier()
        torch.cuda.synchronize(dev)
        clk = ClockSampler(local) if with_clocks else None
        if clk:
            clk.__enter__()
        e0.record(stream)
        for i in range(args.steps):
            step(kev[i])
        e1.record(stream)
        torch.cuda.synchronize(dev)
        if clk:
            clk.__exit__()
        W.wef_set_trace_events(op.h, None, None)
        W.wef_device_status(op.h)
        ms_total = max_over_ranks(e0.elapsed_time(e1), dist, dev)
        ms_step = ms_total / args.steps
        kernel_ms = statistics.mean(a.elapsed_time(b) for a, b in kev)
        fp64_flops, radial_flops = W.wef_flops(op.h, prec)
        out = {
            "value": job_throughput(world, ncells, ms_step),
            "ms_per_step": ms_step,
            "kernel_ms": kernel_ms,
            "fp64_tflops": fp64_flops * ncells / (kernel_ms / 1e3) / 1e12,
            "fp64_flops_per_cell": fp64_flops,
            "radial_flops_per_cell": radial_flops,
            "radial_tflops": radial_flops * ncells / (kernel_ms / 1e3) / 1e12,
            "step": step,
            "clocks": clk.summary() if clk else None,
        }
        return out

    variants = {}
    # the tensor-core radial-first path (rftc) is compiled for Kmax = 8, 10 and 12
    others = [p for p in ("fp64", "bf16", "tf32", "rftc", "rf32")
              if p != args.precision and (p != "rftc" or KMAX in (8, 10, 12))]
    order = (others if args.variants == "all" else []) + [args.precision]
    nsample = min(args.cpu_sample_cells, ncells)
    q_sample, invariant_max = {}, {}
    qv = q.view(ncells, KMAX + 1, (LMAX + 1) ** 2)
    for pr in order:
        variants[pr] = measure(pr, with_clocks=(pr == args.precision))
        # the result of the last timed step: the cells the oracle checks, and the largest
        # |Q| over every cell's mass, momentum and energy outputs (exact zeros by Sec. 4.4)
        q_sample[pr] = qv[:nsample].reshape(nsample, -1).cpu().numpy()
        invariant_max[pr] = max(float(qv[:, 0, 0:4].abs().max()), float(qv[:, 1, 0].abs().max()))
    head = variants[args.precision]
    step = head["step"]
    # end to end through the C ABI with host buffers: wef_evaluate_host streams pinned f to
    # the device in chunks and Q back, the copies of one chunk overlapping the evaluation of
    # the next; every byte of f in and Q out crosses host<->device inside the timed region
    f_pin = torch.from_numpy(f_host).pin_memory()
    q_pin = torch.empty_like(f_pin).pin_memory()
    prec_h = W.PRECISIONS[args.precision]
    chunk = 4096
    hws = torch.empty(W.wef_host_workspace_size(op.h, chunk, prec_h), dtype=torch.uint8, device=dev)

    def host_step():
        W.wef_evaluate_host(op.h, f_pin.data_ptr(), q_pin.data_ptr(), ncells, chunk, prec_h, hws.data_ptr(),
                            hws.numel(), stream.cuda_stream)

    for _ in range(2):
        host_step()
    torch.cuda.synchronize(dev)
    a0, a1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    a0.record(stream)
    for _ in range(args.steps):
        host_step()
    a1.record(stream)
    torch.cuda.synchronize(dev)
    e2e_ms = a0.elapsed_time(a1) / args.steps
    # configuration 5 (serving), timed after the headline legs
    serving = None
    if world == 1 and os.environ.get("WEF_BENCH_NO_SERVE") != "1" and args.duration > 0:
        try:  # the serving figure must not cost the benchmark line
            serving = serving_leg(args, W, torch, dev, args.duration)
        except Exception as e:  # noqa: BLE001
            torch.cuda.synchronize(dev)
            serving = {"error": f"{type(e).__name__}: {e}"}
    if rank != 0:
        if dist:
            dist.destroy_process_group()
        return
    achieved = head["fp64_tflops"]
    line = {
        "metric": METRIC,
        "value": head["value"],
        "unit": "cells/s",
        "n_gpus": world,
        "steps": args.steps,
        "warmup": args.warmup,
        "ms_per_step": head["ms_per_step"],
        "higher_is_better": True,
        "scaling": "weak",
        "vs_baseline": None,
        "dtype": DTYPES[args.precision],
        "data": "synthetic",
        "config": {
            "workload": f"hard spheres (gamma=1), Kmax=Lmax={KMAX}, {ncells} cells per GPU, seeded two-Maxwellian "
                        f"mixtures, core from the library quadrature (pad 20/20)",
            "precision": args.precision,
            "l2": (f"inputs ({ncells * (KMAX + 1) * (LMAX + 1) ** 2 * 8 / 1e6:.0f} MB f + the same in Q) "
                   + ("larger than L2, no flush" if 2 * ncells * (KMAX + 1) * (LMAX + 1) ** 2 * 8 > 129e6
                      else "smaller than L2 (not a headline configuration)")),
        },
        "roofline": {
            "bound": "alu",
            "pipe": {"fp64": "FP64 FMA (angular coupling + radial contraction)",
                     "rf32": "FP64 FMA (Gaunt reduction of the radial-first products)",
                     "rftc": "FP64 FMA (Gaunt reduction of the radial-first products)"}.get(
                         args.precision, "FP64 FMA (angular coupling)"),
            "kernel": {"fp64": "fp64_kernel", "rf32": f"rf_kernel<{KMAX + 1}>",
                       "rftc": f"rft_kernel<{KMAX + 1}>"}.get(
                args.precision, f"tc_kernel<{KMAX + 1},{args.precision}>"),
            "achieved": achieved,
            "peak": FP64_PEAK_TFLOPS,
            "unit": "TFLOP/s",
            "frac": achieved / FP64_PEAK_TFLOPS,
            "traffic": TRAFFIC_BYTES.get(args.precision) if (ncells == NCELLS and KMAX == 12) else None,
            "traffic_note": "DRAM bytes per launch (one-pass ncu capture at 16384 cells); algorithmic: FP32 tiles "
                            "in + FP64 Q out = 432 MB; " + TRAFFIC_NOTE,
            "fp64_flops_per_cell": head["fp64_flops_per_cell"],
            "radial_flops_per_cell": head["radial_flops_per_cell"],
            "radial_note": "low-precision radial flops: tensor-core (bf16, tf32; rftc: stage 1 as three TF32 "
                           "products on padded tiles, stage 2 on the FP32 CUDA cores) or FP32 CUDA-core (rf32)",
            "radial_tflops": head["radial_tflops"],
            "kernel_ms": head["kernel_ms"],
            "peak_note": "peak = 152 SMs x 2 DFMA lanes/clock x 2 flop x 2070 MHz; probe = live DFMA chain",
            "peak_probe": probe,
        },
        "variants": {k: {kk: vv for kk, vv in v.items() if kk not in ("step", "clocks")} for k, v in variants.items()},
        "speedup_vs_fp64": head["value"] / variants["fp64"]["value"] if "fp64" in variants else None,
        "e2e": {
            "value": world * ncells / (e2e_ms / 1e3),
            "unit": "cells/s",
            "h2d_bytes_per_step": int(f_pin.numel() * 8),
            "d2h_bytes_per_step": int(q_pin.numel() * 8),
            "api": f"wef_evaluate_host, pinned host f and Q, chunks of {chunk} cells (copies overlap evaluations)",
        },
        "gpu_launches": 2 * args.steps,
        "clocks": head["clocks"],
    }
    if serving is not None:
        line["serving"] = {k: serving[k] for k in ("p50_ms", "p99_ms", "cells_per_s", "completed", "rejected",
                                                    "requests", "batches", "small", "large", "mean_queue_ms",
                                                    "wall_s", "clocks", "note", "error")
                           if k in serving}
    if world == 1 and os.environ.get("WEF_BENCH_NO_CPU") != "1":
        cb, (Qo, T, rows) = cpu_baseline(nsample, args.cpu_sample_rows, with_angular_first=True, R=R, f=f_host)
        line["cpu_baseline"] = cb
        line["error_vs_oracle"] = {
            "metric": f"per cell: max over its output rows of |Q - Q_oracle| / max(max |Q_oracle|, 2^-10 x max sum "
                      f"of |terms|); max and median over {nsample} cells (the oracle's sample: the batch's first "
                      f"cells, {len(rows)} output rows each, the hard-sphere core of this run); invariant_max_abs = "
                      f"largest |Q| of the mass, momentum and energy outputs over all {ncells} cells",
            **{pr: {**error_vs_oracle(q_sample[pr][:, rows], Qo, T), "invariant_max_abs": invariant_max[pr]}
               for pr in order},
        }
    else:
        line["error_vs_oracle"] = {pr: {"invariant_max_abs": invariant_max[pr]} for pr in order}
    print(json.dumps(line), flush=True)
    if dist:
        dist.destroy_process_group()


if __name__ == "__main__":
    main()
