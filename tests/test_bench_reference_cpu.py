"""bench.py's reference arm (the oracle on the host cores) runs without a GPU and prints one
JSON line with the fields the benchmark contract asks for."""
import json
import os
import subprocess
import sys

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def test_reference_arm_json_line():
    r = subprocess.run([sys.executable, os.path.join(ROOT, "bench.py"), "--impl", "reference", "--steps", "2",
                        "--warmup", "1", "--cpu-sample-cells", "1", "--cpu-sample-rows", "16"],
                       capture_output=True, text=True, timeout=600, cwd=ROOT)
    assert r.returncode == 0, r.stderr[-2000:]
    line = json.loads(r.stdout.strip().splitlines()[-1])
    assert line["impl"] == "reference" and line["unit"] == "cells/s" and line["value"] > 0
    assert line["steps"] == 2 and line["warmup"] == 1 and line["higher_is_better"] is True
    assert line["cpu_baseline"]["kind"] == "oracle" and line["cpu_baseline"]["cores"] >= 1
    assert line["e2e"]["h2d_bytes_per_step"] == 0 and line["e2e"]["value"] == line["value"]


def test_angular_first_all_cores_figure():
    """The all-cores CPU comparison figure (spawned processes, barrier, shared wall clock)
    runs without a GPU and reports the processes it used."""
    code = ("import json, bench; print(json.dumps(bench.cpu_angular_first_all_cores("
            "cells_per_process=2, processes=2)))")
    r = subprocess.run([sys.executable, "-c", code], capture_output=True, text=True, timeout=600, cwd=ROOT)
    assert r.returncode == 0, r.stderr[-2000:]
    d = json.loads(r.stdout.strip().splitlines()[-1])
    assert d["cores"] == 2 and d["value"] > 0 and d["unit"] == "cells/s" and d["cpu_model"]


def test_clock_summary_parsing():
    """The clocks object of the benchmark line from nvidia-smi CSV samples: median SM clock,
    maximum clock, and every throttle reason seen active in any sample."""
    sys.path.insert(0, ROOT)
    import bench

    s = bench.ClockSampler(0)
    s.lines = ["2070, 2070, 900.5, 0x0000000000000000, Not Active, Not Active, Not Active, Not Active",
               "2055, 2070, 1390.2, 0x0000000000000004, Not Active, Not Active, Not Active, Active",
               "[N/A], 2070, 1380.0, 0x0, Not Active, Not Active, Not Active, Not Active",  # unparsable: skipped
               "2040, 2070, 1395.0, 0x0000000000000008, Active, Not Active, Not Active, Not Active"]
    d = s.summary()
    assert d["sm_mhz"] == 2055.0 and d["sm_max_mhz"] == 2070.0 and d["samples"] == 3
    assert d["reasons"] == ["hw_slowdown", "sw_power_cap"]
    s.lines = []
    assert s.summary()["reasons"] == ["unsampled"]


def test_error_vs_oracle_guard():
    """The bench line's per-cell error: the infinity norm of each cell's error over its rows,
    relative to max(|Q_oracle| of the cell, 2^-10 x its largest sum of |terms|)."""
    sys.path.insert(0, ROOT)
    import numpy as np

    import bench

    Qo = np.array([[1.0, -2.0], [1e-9, 0.0]])
    T = np.array([[3.0, 4.0], [1.0, 1.0]])
    Q = Qo + np.array([[1e-6, 0.0], [0.0, 1e-9]])
    e = bench.error_vs_oracle(Q, Qo, T)
    assert abs(e["max"] - 1e-9 / 2.0 ** -10) < 1e-18  # cell 2: guarded by its terms, not by |Q| = 1e-9
    assert abs(e["median"] - (5e-7 + 1e-9 * 2.0 ** 10) / 2) < 1e-15
    assert abs(e["plain_rel_max"] - 1.0) < 1e-12
