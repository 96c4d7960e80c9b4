"""qmc_matmul_noalloc: the product for callers that must not allocate device
memory during the call (its scratch is a fixed array inside the library).

Checked through the C ABI against the FP64 oracle and against qmc_matmul on
two calls in a row, with the parity tolerance of the other tests, on every
kind of plan the entry point accepts: prime single-pass and three-pass
plans, ragged column counts, plans whose positions are hit many times
(s comparable to L), the split hi+lo precision on FP64 input, lengths
N - 1 = 3·2^18 and F_2 lengths 2^m - 1 (with the factor 257).  This file is
collected last so that a run stopping at the first failure has run every
other test before it.
"""

import ctypes as C

import numpy as np
import pytest
import torch

from oracle import products
from paper_1501_06286_gb300 import capi, workloads
from paper_1501_06286_gb300.qmc import Plan

from _helpers import TOL, colwise_rel_err, oracle_pointset

pytestmark = pytest.mark.gpu


def _noalloc(lib, plan, A, out):
    dtype = capi.DTYPE_F64 if A.dtype == torch.float64 else capi.DTYPE_F32
    return lib.qmc_matmul_noalloc(plan.handle, C.c_void_p(A.data_ptr()), A.stride(0), A.shape[1],
                                  dtype, C.c_void_p(out.data_ptr()), out.stride(0),
                                  C.c_void_p(torch.cuda.current_stream().cuda_stream))


def _oracle_rows(w, plan, A64):
    """The oracle's product on every row (small plans) or on sampled rows."""
    ps = oracle_pointset(w)
    if plan.out_rows <= 20000:
        rows = np.arange(plan.out_rows)
    else:
        rng = np.random.default_rng(plan.out_rows)
        rows = np.unique(np.concatenate([[0, 1, plan.out_rows - 1],
                                         rng.choice(plan.out_rows, 509, replace=False)]))
    return rows, products.matmul_rows(ps, A64, rows)


def _check_two_calls(w, prec="fp32"):
    from paper_1501_06286_gb300 import build
    build.build()
    lib = capi.load()
    plan = Plan.from_workload(w, prec=prec)
    A = torch.from_numpy(np.ascontiguousarray(w.A)).cuda()
    t = w.t
    ref_gpu = plan.matmul(A).cpu().numpy()
    rows, ref = _oracle_rows(w, plan, w.A.astype(np.float64))
    for _ in range(2):
        out = torch.full((plan.out_rows, t), float("nan"), device="cuda")
        assert _noalloc(lib, plan, A, out) == 0
        torch.cuda.synchronize()
        assert plan.sync_status() == 0
        got = out.cpu().numpy()
        assert colwise_rel_err(got, ref_gpu) <= TOL
        assert colwise_rel_err(got[rows], ref) <= TOL


@pytest.mark.parametrize("N,s,t,map", [(65537, 200, 64, "phi_inv"),   # three passes, scratch
                                       (7681, 150, 37, "centred"),    # three passes, ragged
                                       (257, 300, 9, "centred"),      # single pass
                                       (7681, 3000, 21, "centred"),   # s >= L/4: dense hits
                                       (786433, 40, 8, "centred")])   # L = 768·1024
def test_noalloc_matches_oracle_and_matmul_on_two_calls(N, s, t, map):
    _check_two_calls(workloads.random_prime_case(N, s, t, seed=N + t, map=map))


def test_noalloc_split_precision_on_fp64_input():
    w = workloads.random_prime_case(7681, 150, 13, seed=5, dtype=np.float64)
    _check_two_calls(w, prec="fp32_split")


@pytest.mark.parametrize("m,s,grid", [(12, 60, 3), (16, 48, 3)])   # L = 4095; L = 65535 = 255·257
def test_noalloc_f2_plans(m, s, grid):
    _check_two_calls(workloads.f2_65536(m=m, s=s, grid=grid))


def test_noalloc_rejects_problems_beyond_the_fixed_scratch():
    lib = capi.load()
    w = workloads.random_prime_case(65537, 64, 512, seed=3)
    plan = Plan.from_workload(w)
    A = torch.from_numpy(w.A).cuda()
    out = torch.zeros((plan.out_rows, 512), device="cuda")
    assert _noalloc(lib, plan, A, out) == 11   # QMC_ERR_SCRATCH
    torch.cuda.synchronize()
    assert torch.count_nonzero(out).item() == 0


def test_noalloc_rejects_pset_plans():
    lib = capi.load()
    plan = Plan("pset", 257, None, map="centred", s=10)
    A = torch.ones((10, 2), device="cuda")
    out = torch.zeros((plan.out_rows, 2), device="cuda")
    assert _noalloc(lib, plan, A, out) == 6    # QMC_ERR_UNSUPPORTED
    torch.cuda.synchronize()
    assert torch.count_nonzero(out).item() == 0
