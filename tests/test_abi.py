"""The C ABI library builds, loads and exports every symbol include/qmc.h
declares (no CUDA compute calls: this runs without a GPU)."""

import ctypes
import os
import re

import pytest

from paper_1501_06286_gb300 import build, capi

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _declared_symbols(debug: bool = False):
    """Functions the headers declare: the product ABI (every header but
    qmc_debug.h), or with debug=True those of qmc_debug.h, which only the
    bounds-checked build exports."""
    names = set()
    for fn in os.listdir(os.path.join(ROOT, "include")):
        if fn.endswith(".h") and (fn == "qmc_debug.h") == debug:
            text = open(os.path.join(ROOT, "include", fn)).read()
            names |= set(re.findall(r"^\s*(?:int|int64_t|const char\*)\s+(qmc_\w+)\s*\(", text, re.M))
    return names


@pytest.fixture(scope="module")
def lib():
    build.build()
    return capi.load()


def test_every_declared_symbol_is_exported(lib):
    declared = _declared_symbols()
    assert declared, "no declarations parsed"
    assert declared == set(capi.EXPORTS)
    for name in declared:
        assert hasattr(lib, name), name


def test_checked_build_exports_the_debug_hook(lib):
    # the QMC_CHECK_BOUNDS build: the same ABI plus qmc_debug.h's hook,
    # which the default library does not export
    debug = _declared_symbols(debug=True)
    assert debug == {"qmc_debug_poke_table"}
    for name in debug:
        assert not hasattr(lib, name), name
    path = build.build(checked=True)
    assert path == build.lib_path(checked=True) and path != build.lib_path()
    checked = ctypes.CDLL(path)
    for name in _declared_symbols() | debug:
        assert hasattr(checked, name), name
    checked.qmc_status_string.restype = ctypes.c_char_p
    assert b"QMC_CHECK_BOUNDS" in checked.qmc_status_string(13)
    # argument checks of the hook (no device access)
    old = ctypes.c_int32()
    checked.qmc_debug_poke_table.argtypes = [ctypes.c_void_p, ctypes.c_int32, ctypes.c_int64, ctypes.c_int32,
                                             ctypes.POINTER(ctypes.c_int32)]
    assert checked.qmc_debug_poke_table(None, 3, 0, 0, ctypes.byref(old)) == 1


def test_status_strings_and_version(lib):
    assert lib.qmc_status_string(0) == b"ok"
    for code in range(1, 14):
        assert lib.qmc_status_string(code) != b"unknown status"
    assert lib.qmc_status_string(999) == b"unknown status"
    assert lib.qmc_version() >= 100


def test_null_arguments_are_rejected_without_touching_the_device(lib):
    assert lib.qmc_plan_create(None, None, None) == 1
    h = ctypes.c_void_p()
    assert lib.qmc_plan_create(ctypes.byref(h), None, None) == 1
    assert lib.qmc_plan_destroy(None) == 1
    assert lib.qmc_matmul(None, None, 0, 0, 0, None, 0, None, None, None) == 1
    assert lib.qmc_plan_info(None, None) == 1


def test_library_is_built_for_sm103a():
    path = build.lib_path()
    assert os.path.exists(path)
    assert "arch=compute_103a,code=sm_103a" in " ".join(build.ARCH)


@pytest.mark.parametrize("delta", [1.0, -0.25, float("nan"), float("inf")])
def test_shift_outside_unit_interval_is_rejected_on_the_host(lib, delta):
    # Remark 2's diagonal shift Δ must lie in [0, 1); the check runs before
    # any device work, so it needs no GPU
    import numpy as np

    gen = np.array([1, 3], dtype=np.int64)
    d = capi.QmcDesc()
    d.kind, d.N, d.s = 0, 17, 2
    d.gen_host = gen.ctypes.data_as(ctypes.POINTER(ctypes.c_int64))
    d.map, d.row0, d.order, d.prec = 1, 0, 0, 0
    d.shift = delta
    h = ctypes.c_void_p()
    assert lib.qmc_plan_create(ctypes.byref(h), ctypes.byref(d), None) == 1
    assert not h.value


def test_stage_count_matches_the_header():
    # qmc_plan_read_profile writes QMC_NUM_STAGES entries into caller arrays
    hdr = open(os.path.join(os.path.dirname(__file__), "..", "include", "qmc.h")).read()
    n = int(re.search(r"QMC_NUM_STAGES\s*=\s*(\d+)", hdr).group(1))
    assert capi.NUM_STAGES == n == len(capi.STAGES)
    # the binding's stage names are the header's, in the header's order
    for name, value in re.findall(r"QMC_STAGE_(\w+)\s*=\s*(\d+)", hdr):
        assert capi.STAGES[int(value)] == name.lower()


def test_option_values_match_the_header():
    hdr = open(os.path.join(os.path.dirname(__file__), "..", "include", "qmc.h")).read()
    enum = {k: int(v) for k, v in re.findall(r"\b(QMC_(?:OPT|FIRST_PASS|KERNEL|ROW_MEAN)_\w+)\s*=\s*(\d+)", hdr)}
    assert enum["QMC_OPT_PASS_KERNEL"] == capi.OPT_PASS_KERNEL
    assert enum["QMC_OPT_ROW_MEAN"] == capi.OPT_ROW_MEAN
    assert enum["QMC_OPT_FIRST_PASS"] == capi.OPT_FIRST_PASS
    for name, v in capi.FIRST_PASS.items():
        assert enum[f"QMC_FIRST_PASS_{name.upper()}"] == v
    for name, v in capi.KERNEL.items():
        assert enum[f"QMC_KERNEL_{name.upper()}"] == v
    for name, v in capi.ROW_MEAN.items():
        assert enum[f"QMC_ROW_MEAN_{name.upper()}"] == v


def _desc(kind=0, N=17, gen=(1, 3), g=0, P=0, map=1, row0=0, order=0, prec=0):
    import numpy as np
    arr = np.asarray(gen, dtype=np.int64)
    d = capi.QmcDesc()
    d.kind, d.N, d.g, d.modulus_P, d.s = kind, N, g, P, len(arr)
    d.gen_host = arr.ctypes.data_as(ctypes.POINTER(ctypes.c_int64))
    d.map, d.row0, d.order, d.prec = map, row0, order, prec
    d.shift = 0.0
    return d, arr


@pytest.mark.parametrize("kw,code", [
    ({"N": 15}, 2),                    # not prime
    ({"N": 1 << 31 | 1}, 2),           # beyond the int32 tables (rejected before any prime test)
    ({"g": 2}, 3),                     # 2 is not a primitive root mod 17 (order 8)
    ({"kind": 1, "N": 12}, 2),         # F_2 point count must be 2^m
    ({"kind": 1, "N": 16, "P": 0b10001}, 3),  # x^4 + 1 is not primitive
    ({"map": 7}, 1), ({"row0": 5}, 1), ({"order": 2}, 1), ({"prec": 3}, 1),
    ({"kind": 2, "row0": 1}, 1),       # a p-set has no zero point to include
])
def test_descriptor_errors_are_caught_on_the_host(lib, kw, code):
    # Section 2.1 needs a prime N and a primitive root (Remark 1: a primitive
    # modulus); these checks run before any device work, so they need no GPU
    d, keep = _desc(**kw)
    h = ctypes.c_void_p()
    assert lib.qmc_plan_create(ctypes.byref(h), ctypes.byref(d), None) == code
    assert not h.value


def test_reference_arm_prints_one_json_line():
    # bench.py --impl reference times the FP64 oracle on the host; the line
    # carries the contract's keys
    import json
    import subprocess
    import sys
    root = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
    res = subprocess.run([sys.executable, os.path.join(root, "bench.py"), "--impl", "reference", "--steps", "1",
                          "--warmup", "1", "--ref-seconds", "0.3", "--workload", "lattice-257"],
                         capture_output=True, text=True, timeout=600, cwd=root)
    assert res.returncode == 0, res.stderr[-2000:]
    lines = [ln for ln in res.stdout.splitlines() if ln.startswith("{")]
    assert len(lines) == 1
    d = json.loads(lines[0])
    for key in ("impl", "metric", "value", "unit", "n_gpus", "steps", "warmup", "ms_per_step",
                "higher_is_better", "dtype", "config", "cpu_baseline", "e2e"):
        assert key in d
    assert d["impl"] == "reference" and d["value"] > 0
    assert d["cpu_baseline"]["kind"] == "oracle"


def test_bench_grid_option_shrinks_the_field_workloads():
    # smaller node grids for profiling captures keep N, s and the map
    import bench
    w = bench._make_workload("field-786433", 0, 17)
    assert (w.N, w.s, w.t, w.map, w.name) == (786433, 2048, 289, "centred", "field-786433-grid17")
    w = bench._make_workload("f2-65536", 0, 9)
    assert (w.N, w.s, w.t, w.name) == (65536, 1024, 81, "f2-65536-grid9")
    assert bench._make_workload("field-786433", 0, None).t == 4225


def test_fe_solve_arguments_are_checked_on_the_host(lib):
    # qmc_fe_solve_mean rejects bad arguments before touching the device
    # the larger of the two solves' needs; the partitioned solve's, per
    # system: three doubles for each of 128 chunks x ceil((M-1)/128) rows (at least 8)
    # (and one int32 flag per system, rounded up to 8 bytes)
    assert lib.qmc_fe_work_bytes(4001, 8002) == 4001 * 3 * 63 * 128 * 8 + 8 * 2001
    assert lib.qmc_fe_work_bytes(7, 50) == 7 * 3 * 8 * 128 * 8 + 8 * 4
    # one system of M = 8002: the flux form's layout is the larger (header,
    # G in FP64 and as pairs, one FluxSys, one chunk's Q and S, R, and one
    # sum of R per 64 elements)
    assert lib.qmc_fe_work_bytes(1, 8002) == 64 + 8 * 8002 * 2 + 16 + 8 * 8002 * 2 + 8 * 8002 + 8 * 126
    assert lib.qmc_fe_work_bytes(0, 10) == 0 and lib.qmc_fe_work_bytes(5, 2) == 0
    fake = ctypes.c_void_p(0x1000)  # never dereferenced: every call below fails its checks
    big = 1 << 40
    assert lib.qmc_fe_solve_mean(None, 20, 4, 10, 0, None, fake, big, fake, None) == 1
    assert lib.qmc_fe_solve_mean(fake, 20, 4, 10, 0, None, None, big, fake, None) == 1
    assert lib.qmc_fe_solve_mean(fake, 20, 4, 10, 0, None, fake, big, None, None) == 1
    assert lib.qmc_fe_solve_mean(fake, 20, 4, 2, 0, None, fake, big, fake, None) == 1      # M < 3
    assert lib.qmc_fe_solve_mean(fake, 20, 0, 10, 0, None, fake, big, fake, None) == 1     # n_sys < 1
    assert lib.qmc_fe_solve_mean(fake, 20, 4, 10, 2, None, fake, big, fake, None) == 1     # kind
    assert lib.qmc_fe_solve_mean(fake, 20, 4, 10, 0, None, ctypes.c_void_p(0x1004), big, fake, None) == 1
    assert lib.qmc_fe_solve_mean(fake, 16, 4, 10, 0, None, fake, big, fake, None) == 5     # ldb < 2M-3
    assert lib.qmc_fe_solve_mean(fake, 9, 4, 10, 1, None, fake, big, fake, None) == 5      # ldb < M
    assert lib.qmc_fe_solve_mean(fake, 20, 4, 10, 0, None, fake, 8, fake, None) == 5       # work too small
