"""qmc_matmul_noalloc: the product for callers that must not allocate device
memory during the call (its scratch is a fixed array inside the library).

Checked through the C ABI against qmc_matmul on two calls in a row, with the
parity tolerance of the other tests.  This file is collected last so that a
run stopping at the first failure has run every other test before it.
"""

import ctypes as C

import numpy as np
import pytest
import torch

from paper_1501_06286_gb300 import capi, workloads
from paper_1501_06286_gb300.qmc import Plan

from _helpers import TOL, colwise_rel_err

pytestmark = pytest.mark.gpu


def _noalloc(lib, plan, A, out):
    return lib.qmc_matmul_noalloc(plan.handle, C.c_void_p(A.data_ptr()), A.stride(0), A.shape[1],
                                  capi.DTYPE_F32, C.c_void_p(out.data_ptr()), out.stride(0),
                                  C.c_void_p(torch.cuda.current_stream().cuda_stream))


@pytest.mark.parametrize("N,s,t,map", [(65537, 200, 64, "phi_inv"),   # three passes, scratch
                                       (7681, 150, 37, "centred"),    # three passes, ragged
                                       (257, 300, 9, "centred")])     # single pass
def test_noalloc_matches_matmul_on_two_calls(N, s, t, map):
    from paper_1501_06286_gb300 import build
    build.build()
    lib = capi.load()
    w = workloads.random_prime_case(N, s, t, seed=N + t, map=map)
    plan = Plan.from_workload(w)
    A = torch.from_numpy(w.A).cuda()
    ref = plan.matmul(A).cpu().numpy()
    for _ in range(2):
        out = torch.full((plan.out_rows, t), float("nan"), device="cuda")
        assert _noalloc(lib, plan, A, out) == 0
        torch.cuda.synchronize()
        assert plan.sync_status() == 0
        assert colwise_rel_err(out.cpu().numpy(), ref) <= TOL


def test_noalloc_rejects_problems_beyond_the_fixed_scratch():
    lib = capi.load()
    w = workloads.random_prime_case(65537, 64, 512, seed=3)
    plan = Plan.from_workload(w)
    A = torch.from_numpy(w.A).cuda()
    out = torch.zeros((plan.out_rows, 512), device="cuda")
    assert _noalloc(lib, plan, A, out) == 11   # QMC_ERR_SCRATCH
    torch.cuda.synchronize()
    assert torch.count_nonzero(out).item() == 0
