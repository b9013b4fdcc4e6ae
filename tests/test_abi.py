"""The C ABI: the library loads, exports every symbol include/wef.h declares, and its
host-side parts (angular tables, core quadrature, argument checks) agree with the
oracle.  No GPU compute here."""
import os
import re

import numpy as np
import pytest

import paper_2605_28475_gb300 as W
from oracle import core as ocore
from oracle import gaunt as ogaunt

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _declared_symbols():
    names = set()
    for fn in os.listdir(os.path.join(ROOT, "include")):
        if fn.endswith(".h"):
            src = open(os.path.join(ROOT, "include", fn)).read()
            names |= set(re.findall(r"^\s*(?:wef_status|const char\*)\s+(wef_\w+)\s*\(", src, re.M))
    return names


@pytest.fixture(scope="module", autouse=True)
def built():
    if not os.path.exists(W.LIB_PATH):
        from paper_2605_28475_gb300 import build

        build.build()


def test_exports_every_declared_symbol():
    names = _declared_symbols()
    assert {"wef_create", "wef_evaluate", "wef_upload_core", "wef_destroy"} <= names
    lib = W.lib()
    for n in sorted(names):
        assert hasattr(lib, n), n


@pytest.mark.parametrize("L", [2, 4, 8, 12])
def test_gaunt_table_matches_oracle(L):
    """Exact 3-j route (library) vs sphere quadrature (oracle): same rows, same order, same weights."""
    h = W.wef_create(1, L, 0.0)
    try:
        q1, q2, q3, c, g = W.wef_gaunt_coo(h)
        o = ogaunt.coo(L)
        for a, b in zip((q1, q2, q3, c), o[:4]):
            assert np.array_equal(a, b)
        assert np.max(np.abs(g - o[4])) < 1e-13
        nq, nt, ng, rl = W.wef_sizes(h)
        assert (nq, nt, ng, rl) == (2 * (L + 1) ** 2, len(ogaunt.channels(L)), len(g), len(ogaunt.channels(L)) * 8)
    finally:
        W.wef_destroy(h)


@pytest.mark.parametrize("gamma", [0.0, 0.5, 1.0])
def test_core_builder_matches_oracle_core(gamma):
    """The library's core quadrature (Funk-Hecke sphere means, C++) against the oracle's
    (explicit scattering-sphere rule, numpy): two independent evaluations of the same integral."""
    km, lm = 2, 3
    h = W.wef_create(km, lm, gamma)
    try:
        Rp = W.wef_core_build(h).reshape(-1, km + 1, km + 1, km + 1)
    finally:
        W.wef_destroy(h)
    Ro = ocore.core(km, lm, gamma)
    assert np.max(np.abs(Rp - Ro)) < 1e-13 * np.max(np.abs(Ro))


def test_argument_errors():
    with pytest.raises(W.WefError) as e:
        W.wef_create(17, 4, 0.0)
    assert e.value.status == W.WEF_ESHAPE
    with pytest.raises(W.WefError):
        W.wef_create(4, 21, 0.0)
    with pytest.raises(W.WefError):
        W.wef_create(4, 4, -1.0)
    h = W.wef_create(2, 2, 0.0)
    try:
        with pytest.raises(W.WefError) as e:
            W.wef_upload_core(h, np.zeros(5))
        assert e.value.status == W.WEF_ESHAPE
        with pytest.raises(W.WefError):
            W.wef_workspace_size(h, -1)
        assert W.wef_workspace_size(h, 0) == 0
        assert W.wef_workspace_size(h, 33) == 64 * 3 * 9 * 8
        # an unknown precision is refused before any size is computed or any work queued
        for fn in (W.wef_workspace_size, W.wef_integrate_workspace_size, W.wef_host_workspace_size):
            with pytest.raises(W.WefError) as e:
                fn(h, 33, 7)
            assert e.value.status == W.WEF_EINVAL
        with pytest.raises(W.WefError) as e:
            W.wef_flops(h, 7)
        assert e.value.status == W.WEF_EINVAL
        with pytest.raises(W.WefError) as e:
            W.wef_evaluate(h, 0, 0, 0, 7, 0, 0, 0)
        assert e.value.status == W.WEF_EINVAL and "precision" in str(e.value)
        # the tensor-core radial-first path exists for Kmax = 8, 10, 12 only (here Kmax = 2),
        # and is a one-shape path: plans and ragged batches refuse it
        with pytest.raises(W.WefError) as e:
            W.wef_evaluate(h, 0, 0, 1, W.WEF_RADIAL_TC, 0, 0, 0)
        assert e.value.status == W.WEF_EINVAL and "Kmax" in str(e.value)
        assert W.wef_workspace_size(h, 33, W.WEF_RADIAL_TC) == W.wef_workspace_size(h, 33, W.WEF_RADIAL_FP32)
        with pytest.raises(W.WefError) as e:
            W.wef_plan_create([h], [32], W.WEF_RADIAL_TC, 0)
        assert e.value.status == W.WEF_EINVAL
        with pytest.raises(W.WefError) as e:
            W.wef_ragged_workspace_size([h], 32, W.WEF_RADIAL_TC)
        assert e.value.status == W.WEF_EINVAL
    finally:
        W.wef_destroy(h)


def test_binding_rejects_mis_shaped_tensors():
    """The Python helper refuses tensors the library would read or write past their end
    (another operator's per-cell size), wrong dtypes, non-contiguous views and tensors on
    the wrong side of the bus, before any CUDA call."""
    torch = pytest.importorskip("torch")
    op = W.Operator(2, 2, 0.0)  # 3 x 9 = 27 doubles per cell
    try:
        ok = torch.zeros(4, 3, 9, dtype=torch.float64)
        bad = [torch.zeros(4, 3, 4, dtype=torch.float64),           # another Lmax
               torch.zeros(4, 27, dtype=torch.float32),             # dtype
               torch.zeros(4, 9, 3, dtype=torch.float64).transpose(1, 2)]  # not contiguous
        for f in bad:
            with pytest.raises(ValueError):
                op.evaluate_host(f)
        with pytest.raises(ValueError):
            op.evaluate_host(ok, q=torch.zeros(3, 3, 9, dtype=torch.float64))
        with pytest.raises(ValueError):
            op.evaluate(ok)  # host tensor given to the device entry point
        with pytest.raises(ValueError):
            op.linearized_apply(ok, ok)
        with pytest.raises(ValueError):
            op.integrate(ok, 0.1, 1)
    finally:
        op.close()


@pytest.mark.parametrize("km,lm", [(4, 4), (8, 8), (12, 12), (12, 4)])
def test_flop_counts_match_the_coo_table(km, lm):
    """The per-cell work wef_flops reports (the numerator of the benchmark's roofline) against
    counts taken from the oracle's own COO table.  Radial-first: the FP64 Gaunt reduction is
    2K per symmetrised entry (q2 <= q3), the FP32 radial stages 2K^3 per distinct
    (channel, q2) and 2K^2 per distinct (channel, q2, q3).  Plain FP64 angular-first: 2K^2
    per rank-1 group (distinct channel, q1, q2), 2K per symmetrised entry and 2K^3 per
    symmetrised slice (distinct channel, q1)."""
    q1, q2, q3, c, g = ogaunt.coo(lm)
    sym = q2 <= q3
    lof = lambda q: np.floor(np.sqrt(q + 0.5)).astype(int)  # noqa: E731
    l1, l2, l3 = lof(q1[sym]), lof(q2[sym]), lof(q3[sym])
    groups = {(a, b, d, e) for a, b, d, e in zip(l1, l2, l3, q2[sym])}
    pairs = {(a, b, d, e, f) for a, b, d, e, f in zip(l1, l2, l3, q2[sym], q3[sym])}
    rank1 = {(a, b, d, e, f) for a, b, d, e, f in zip(l1, l2, l3, q1[sym], q2[sym])}
    slices = {(a, b, d, e) for a, b, d, e in zip(l1, l2, l3, q1[sym])}
    K, E = km + 1, int(sym.sum())
    h = W.wef_create(km, lm, 1.0)
    try:
        fp64, fp32 = W.wef_flops(h, W.WEF_RADIAL_FP32)
        tc64, tc = W.wef_flops(h, W.WEF_RADIAL_TC)
        plain, _ = W.wef_flops(h, W.WEF_FP64)
    finally:
        W.wef_destroy(h)
    assert fp64 == 2 * K * E
    assert fp32 == 2 * K**3 * len(groups) + 2 * K**2 * len(pairs)
    # tensor-core stage 1 as executed: per (channel, q2) group three TF32 products of the
    # 32 cells repeated over the 4 lane quadrants by 16 (padded k2) by 16 K (k1, padded k3)
    assert tc64 == fp64 and tc == len(groups) * 4 * 3 * 2 * 16 * 16 * K
    assert plain == 2 * K**2 * len(rank1) + 2 * K * E + 2 * K**3 * len(slices)


def test_plain_c_client(tmp_path):
    """include/wef.h is a C header: a C99 program (-pedantic -Werror) that includes it, links
    libwef.so and calls the host-only entry points runs and checks its results."""
    import shutil
    import subprocess

    gcc = shutil.which("gcc")
    if gcc is None:
        pytest.skip("no C compiler")
    libdir = os.path.dirname(W.LIB_PATH)
    exe = str(tmp_path / "c_abi_client")
    subprocess.run([gcc, "-std=c99", "-Wall", "-Wextra", "-pedantic", "-Werror", "-o", exe,
                    os.path.join(ROOT, "tests", "host", "c_abi_client.c"), f"-L{libdir}", "-lwef",
                    f"-Wl,-rpath,{libdir}", "-Wl,--allow-shlib-undefined"], check=True)
    r = subprocess.run([exe], capture_output=True, text=True, timeout=120)
    assert r.returncode == 0 and r.stdout.strip().endswith("ok"), r.stdout + r.stderr


def test_tensor_core_stage1_b_tiles(tmp_path):
    """The split-TF32 core tiles of the tensor-core first radial stage (WEF_RADIAL_TC), as the
    library packs them at core upload: layout, TF32 exactness, hi + lo = R to 2^-22, padding
    (tests/host/rft_pack_check.cpp, linked against libwef.so; host code only)."""
    import shutil
    import subprocess

    gxx = shutil.which("g++")
    if gxx is None:
        pytest.skip("no C++ compiler")
    libdir = os.path.dirname(W.LIB_PATH)
    exe = str(tmp_path / "rft_pack_check")
    subprocess.run([gxx, "-O2", "-std=c++17", "-o", exe, os.path.join(ROOT, "tests", "host", "rft_pack_check.cpp"),
                    f"-L{libdir}", "-lwef", f"-Wl,-rpath,{libdir}", "-Wl,--allow-shlib-undefined"], check=True)
    r = subprocess.run([exe], capture_output=True, text=True, timeout=120)
    assert r.returncode == 0 and "bad=0" in r.stdout, r.stdout + r.stderr
