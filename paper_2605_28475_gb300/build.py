"""Build the in-tree shared library libwef.so (sm_103a) with nvcc and g++.

Translation units are compiled in parallel; the result sits next to this file.
"""
import concurrent.futures as cf
import os
import shutil
import subprocess
import sys

HERE = os.path.dirname(os.path.abspath(__file__))
CSRC = os.path.join(HERE, "csrc")
OUT_DIR = os.path.join(HERE, "_build")
LIB = os.path.join(HERE, "libwef.so")
PROBE = os.path.join(OUT_DIR, "fp64_peak")
ARCH = ["-gencode", "arch=compute_103a,code=sm_103a"]
CUDA_HOME = os.environ.get("CUDA_HOME", "/usr/local/cuda")


def _nvcc():
    p = os.path.join(CUDA_HOME, "bin", "nvcc")
    return p if os.path.exists(p) else (shutil.which("nvcc") or "nvcc")


def _sources():
    cu = sorted(f for f in os.listdir(CSRC) if f.endswith(".cu"))
    cpp = sorted(f for f in os.listdir(CSRC) if f.endswith(".cpp"))
    return cu, cpp


def _compile(cmd):
    r = subprocess.run(cmd, capture_output=True, text=True)
    if r.returncode != 0:
        raise RuntimeError("compile failed:\n" + " ".join(cmd) + "\n" + r.stdout + r.stderr)
    return r.stdout + r.stderr


def build(verbose=False, extra_nvcc=(), defines=()):
    """Compile every translation unit and link libwef.so; returns its path.
    `defines` (e.g. ["WEF_RF_J13=4"]) go to both nvcc and g++."""
    dflags = ["-D" + d for d in defines]
    os.makedirs(OUT_DIR, exist_ok=True)
    cu, cpp = _sources()
    jobs = []
    objs = []
    for f in cu:
        o = os.path.join(OUT_DIR, f + ".o")
        objs.append(o)
        jobs.append([_nvcc(), *ARCH, "-O3", "-lineinfo", "-std=c++17", "-Xcompiler", "-fPIC", "-c",
                     os.path.join(CSRC, f), "-o", o, *dflags, *extra_nvcc])
    for f in cpp:
        o = os.path.join(OUT_DIR, f + ".o")
        objs.append(o)
        jobs.append(["g++", "-O3", "-std=c++17", "-fPIC", "-pthread", *dflags, "-c", os.path.join(CSRC, f), "-o", o])
    with cf.ThreadPoolExecutor(max_workers=max(1, min(len(jobs), os.cpu_count() or 4))) as ex:
        logs = list(ex.map(_compile, jobs))
    if verbose:
        for lg in logs:
            if lg.strip():
                print(lg)
    jobs_probe = [_nvcc(), *ARCH, "-O3", "-o", PROBE, os.path.join(CSRC, "probes", "fp64_peak.cu")]
    with cf.ThreadPoolExecutor(max_workers=2) as ex:
        fut = ex.submit(_compile, jobs_probe)
        tmp = LIB + ".tmp"
        _compile([_nvcc(), *ARCH, "-shared", "-o", tmp, *objs, "-lcudart", "-lcublas", "-lpthread"])
        os.replace(tmp, LIB)
        fut.result()
    return LIB


if __name__ == "__main__":
    print(build(verbose="-v" in sys.argv))
