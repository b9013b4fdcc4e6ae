"""Benchmark: batched Q(f, f) cell-evaluations per second on GB300.

Workload (one step = one pass of the whole hot path over one batch): hard spheres
(gamma = 1), Kmax = Lmax = 12, 16384 cells, each cell a seeded two-Maxwellian
mixture projected onto the basis; core from the library's own quadrature.
The batch (288 MB of f in, 288 MB of Q out) is larger than the 129 MB L2, so no
flush is needed between steps.

    python bench.py [--gpus N] [--steps K] [--warmup W] [--precision tf32|bf16|fp64] [--impl ours|reference]

The headline is the mixed path (FP64 angular coupling, radial stage on the tensor
cores; TF32 by default); the same run also times the other two precisions with the
same protocol and reports them under "variants" with the speedup over plain FP64.
Prints one JSON line (rank 0).  Under torchrun every rank evaluates its own batch
(weak scaling, no data-path collective); the barrier and the max over ranks of
the timed region are the only collectives.
"""
import argparse
import json
import os
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


def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=5)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--precision", default="tf32", choices=["fp64", "bf16", "tf32"])
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--ncells", type=int, default=NCELLS)
    ap.add_argument("--cpu-sample-rows", type=int, default=384)
    ap.add_argument("--cpu-sample-cells", type=int, default=4)
    return ap.parse_args()


def dist_env():
    rank = int(os.environ.get("RANK", "0"))
    world = int(os.environ.get("WORLD_SIZE", "1"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return rank, world, local


def inputs(ncells, seed):
    import wef_inputs as wi

    return wi.two_maxwellians(KMAX, LMAX, ncells, seed=seed, pool=min(1024, ncells))


def cpu_baseline(sample_cells, sample_rows, seed=3):
    """The oracle (dense FP64 CPU contraction) timed on a bounded sample of the workload:
    `sample_cells` cells and `sample_rows` of the N output rows, scaled to cells/s."""
    import wef_inputs as wi
    from oracle import dense, gaunt

    K, NQ = KMAX + 1, (LMAX + 1) ** 2
    N = K * NQ
    R = wi.random_core(len(gaunt.channels(LMAX)), KMAX, seed=11)  # timing does not depend on the values
    f = wi.two_maxwellians(KMAX, LMAX, sample_cells, seed=seed).reshape(sample_cells, -1)
    op = dense.DenseOperator(KMAX, LMAX, dense.conservation_zeroing(R, LMAX))
    rows = np.random.default_rng(seed).choice(N, sample_rows, replace=False)
    t0 = time.perf_counter()
    op.evaluate_rows(f, rows)
    dt = time.perf_counter() - t0
    value = sample_cells * (sample_rows / N) / dt
    return {
        "value": value,
        "unit": "cells/s",
        "cores": os.cpu_count(),
        "kind": "oracle",
        "sample": f"{sample_cells} cells x {sample_rows} of {N} output rows (dense C slices), {dt:.1f} s; "
        f"numpy BLAS threads default (all {os.cpu_count()} host cores)",
    }


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


def run_reference(args, rank, world):
    if rank != 0:
        return
    cb = cpu_baseline(args.cpu_sample_cells, args.cpu_sample_rows)
    line = {
        "impl": "reference", "metric": METRIC, "value": cb["value"], "unit": "cells/s", "n_gpus": args.gpus,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1e3 / cb["value"], "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
        "config": {"workload": f"hard spheres, Kmax=Lmax={KMAX}, two-Maxwellian cells (bounded CPU sample)"},
        "cpu_baseline": cb, "e2e": {"value": cb["value"], "unit": "cells/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }
    print(json.dumps(line), flush=True)


def main():
    args = parse()
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
    op = W.Operator(KMAX, LMAX, GAMMA)
    R = op.build_core()
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
        ms_total = e0.elapsed_time(e1)
        if dist:
            t = torch.tensor([ms_total], device=dev)
            dist.all_reduce(t, op=dist.ReduceOp.MAX)
            ms_total = float(t.item())
            dist.barrier()
        ms_step = ms_total / args.steps
        kernel_ms = statistics.mean(a.elapsed_time(b) for a, b in kev)
        fp64_flops, tc_flops = W.wef_flops(op.h, prec)
        out = {
            "value": world * ncells / (ms_step / 1e3),
            "ms_per_step": ms_step,
            "kernel_ms": kernel_ms,
            "fp64_tflops": fp64_flops * ncells / (kernel_ms / 1e3) / 1e12,
            "fp64_flops_per_cell": fp64_flops,
            "tc_flops_per_cell": tc_flops,
            "tc_tflops": tc_flops * ncells / (kernel_ms / 1e3) / 1e12,
            "step": step,
            "clocks": clk.summary() if clk else None,
        }
        return out

    variants = {}
    order = [p for p in ("fp64", "bf16", "tf32") if p != args.precision] + [args.precision]
    for pr in order:
        variants[pr] = measure(pr, with_clocks=(pr == args.precision))
    head = variants[args.precision]
    step = head["step"]
    # end to end through the public API: pinned host f -> device, evaluate, Q -> pinned host
    f_pin = torch.from_numpy(f_host).pin_memory()
    q_pin = torch.empty_like(f_pin).pin_memory()
    for _ in range(2):
        f.copy_(f_pin, non_blocking=True)
        step()
        q_pin.copy_(q, non_blocking=True)
    torch.cuda.synchronize(dev)
    a0, a1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    a0.record(stream)
    for _ in range(args.steps):
        f.copy_(f_pin, non_blocking=True)
        step()
        q_pin.copy_(q, non_blocking=True)
    a1.record(stream)
    torch.cuda.synchronize(dev)
    e2e_ms = a0.elapsed_time(a1) / args.steps
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
        "dtype": "f64" if args.precision == "fp64" else f"f64+{args.precision}",
        "data": "synthetic",
        "config": {
            "workload": f"hard spheres (gamma=1), Kmax=Lmax={KMAX}, {ncells} cells per GPU, seeded two-Maxwellian "
                        f"mixtures, core from the library quadrature (pad 20/20)",
            "precision": args.precision,
            "l2": "inputs (288 MB f + 288 MB Q) larger than L2, no flush",
        },
        "roofline": {
            "bound": "alu",
            "pipe": "FP64 FMA (angular coupling" + (" + radial contraction)" if args.precision == "fp64" else ")"),
            "kernel": "fp64_kernel" if args.precision == "fp64" else f"tc_kernel<{KMAX + 1},{args.precision}>",
            "achieved": achieved,
            "peak": FP64_PEAK_TFLOPS,
            "unit": "TFLOP/s",
            "frac": achieved / FP64_PEAK_TFLOPS,
            "traffic": None,
            "fp64_flops_per_cell": head["fp64_flops_per_cell"],
            "tc_flops_per_cell": head["tc_flops_per_cell"],
            "tc_tflops": head["tc_tflops"],
            "kernel_ms": head["kernel_ms"],
        },
        "variants": {k: {kk: vv for kk, vv in v.items() if kk not in ("step", "clocks")} for k, v in variants.items()},
        "speedup_vs_fp64": head["value"] / variants["fp64"]["value"],
        "e2e": {
            "value": world * ncells / (e2e_ms / 1e3),
            "unit": "cells/s",
            "h2d_bytes_per_step": int(f_pin.numel() * 8),
            "d2h_bytes_per_step": int(q_pin.numel() * 8),
        },
        "gpu_launches": 2 * args.steps,
        "clocks": head["clocks"],
    }
    if world == 1 and os.environ.get("WEF_BENCH_NO_CPU") != "1":
        line["cpu_baseline"] = cpu_baseline(args.cpu_sample_cells, args.cpu_sample_rows)
    print(json.dumps(line), flush=True)
    if dist:
        dist.destroy_process_group()


if __name__ == "__main__":
    main()
