"""The C ABI library builds, loads and exports every symbol include/qmc.h
declares (no CUDA compute calls: this runs without a GPU)."""

import ctypes
import os
import re

import pytest

from paper_1501_06286_gb300 import build, capi

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _declared_symbols():
    names = set()
    for fn in os.listdir(os.path.join(ROOT, "include")):
        if fn.endswith(".h"):
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


def test_status_strings_and_version(lib):
    assert lib.qmc_status_string(0) == b"ok"
    for code in range(1, 12):
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
