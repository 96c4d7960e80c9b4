"""Degenerate and boundary cases of the fast product against the FP64
oracle: the smallest point sets (N = 3, 5; F_2 with m = 2, 3), a single
coordinate, a single column, every row of A on one position (all e_j
equal), more coordinates than positions, rows whose length is not a
multiple of 8 bytes, and strided (non-contiguous) A and B."""

import ctypes

import numpy as np
import pytest
import torch

from _helpers import TOL, colwise_rel_err, oracle_pointset
from oracle import f2, products
from paper_1501_06286_gb300 import capi, workloads
from paper_1501_06286_gb300.qmc import Plan

pytestmark = pytest.mark.gpu


def _run(w, A=None, **kw):
    plan = Plan.from_workload(w, **kw)
    A = w.A if A is None else A
    B = plan.matmul(torch.from_numpy(np.ascontiguousarray(A)).cuda())
    torch.cuda.synchronize()
    return plan, B.cpu().numpy()


@pytest.mark.parametrize("N", [3, 5, 7])
@pytest.mark.parametrize("map", ["centred", "phi_inv", "identity"])
def test_smallest_prime_point_sets(N, map):
    w = workloads.random_prime_case(N, 4, 3, seed=N, map=map)
    plan, B = _run(w)
    ref = products.matmul(oracle_pointset(w), w.A.astype(np.float64))
    assert B.shape == ref.shape
    assert colwise_rel_err(B, ref) <= TOL


@pytest.mark.parametrize("m", [2, 3])
def test_smallest_f2_point_sets(m):
    P = f2.smallest_primitive(m)
    L = (1 << m) - 1
    e = np.arange(5) % L
    A = np.random.default_rng(m).standard_normal((5, 3)).astype(np.float32)
    w = workloads.Workload(f"f2-m{m}", "f2", 1 << m, 0, P, e.astype(np.int64), True, "centred", "auto", A,
                           extra={"m": m})
    plan, B = _run(w)
    ref = products.matmul(oracle_pointset(w), A.astype(np.float64))
    assert colwise_rel_err(B, ref) <= TOL


@pytest.mark.parametrize("N", [257, 65537])
def test_single_coordinate_and_single_column(N):
    w = workloads.random_prime_case(N, 1, 1, seed=3, map="centred")
    plan, B = _run(w)
    assert plan.info["n_distinct"] == 1 and plan.info["collision_adds"] == 0
    ref = products.matmul(oracle_pointset(w), w.A.astype(np.float64))
    assert colwise_rel_err(B, ref) <= TOL


@pytest.mark.parametrize("N", [257, 7681])
def test_all_rows_on_one_position(N):
    # every z_j equal: P·A has a single non-zero row, the sum of all rows of A
    s, t = 300, 6
    w = workloads.random_prime_case(N, s, t, seed=9, map="centred")
    w.gen[:] = w.gen[0]
    plan, B = _run(w)
    assert plan.info["n_distinct"] == 1 and plan.info["collision_adds"] == s - 1
    ref = products.matmul(oracle_pointset(w), w.A.astype(np.float64))
    assert colwise_rel_err(B, ref) <= TOL


def test_more_coordinates_than_positions():
    # s = 3·L: every position is hit several times
    N = 17
    w = workloads.random_prime_case(N, 48, 5, seed=4, map="tent")
    plan, B = _run(w)
    assert plan.info["n_distinct"] <= N - 1
    ref = products.matmul(oracle_pointset(w), w.A.astype(np.float64))
    assert colwise_rel_err(B, ref) <= TOL


@pytest.mark.parametrize("N,t", [(65537, 7), (786433, 3), (7681, 33)])
def test_odd_row_lengths(N, t):
    # output rows of 7, 3, 33 floats: neither 8- nor 16-byte multiples
    w = workloads.random_prime_case(N, 40, t, seed=t, map="centred")
    plan, B = _run(w)
    ps = oracle_pointset(w)
    rows = np.unique(np.random.default_rng(0).integers(0, plan.out_rows, 3000))
    ref = products.matmul_rows(ps, w.A.astype(np.float64), rows)
    full = products.matmul_rows(ps, w.A.astype(np.float64), np.arange(0, plan.out_rows, 97))
    scale = np.abs(full).max(axis=0)
    assert np.max(np.abs(B[rows] - ref) / scale[None, :]) <= TOL


def test_strided_input_and_output():
    # A and B as column blocks of wider matrices (lda, ldo > t) through the C ABI
    N, s, t = 7681, 120, 5
    w = workloads.random_prime_case(N, s, t, seed=12, map="phi_inv")
    plan = Plan.from_workload(w)
    Awide = torch.zeros((s, 16), dtype=torch.float32)
    Awide[:, 3:3 + t] = torch.from_numpy(w.A)
    Awide = Awide.cuda()
    Bwide = torch.full((plan.out_rows, 12), 7.0, device="cuda")
    lib = capi.load()
    rc = lib.qmc_matmul(plan.handle, ctypes.c_void_p(Awide.data_ptr() + 4 * 3), 16, t, 0,
                        ctypes.c_void_p(Bwide.data_ptr() + 4 * 2), 12, None, None,
                        ctypes.c_void_p(torch.cuda.current_stream().cuda_stream))
    assert rc == 0
    torch.cuda.synchronize()
    got = Bwide.cpu().numpy()
    ref = products.matmul(oracle_pointset(w), w.A.astype(np.float64))
    assert colwise_rel_err(got[:, 2:2 + t], ref) <= TOL
    # columns outside the block are untouched
    assert np.all(got[:, :2] == 7.0) and np.all(got[:, 2 + t:] == 7.0)


@pytest.mark.parametrize("N,s,t,prec", [(7681, 4000, 7, "fp32"), (12289, 5000, 4, "fp32_split"),
                                        (4001, 8002, 9, "fp32")])
def test_densely_hit_positions(N, s, t, prec):
    # s comparable to L or larger (the applications' s = 2N regime): the
    # scatter-add is streamed into the work array before the first pass
    w = workloads.random_prime_case(N, s, t, seed=s, map="centred",
                                    dtype=np.float64 if prec == "fp32_split" else np.float32)
    plan, B = _run(w, prec=prec)
    ref = products.matmul(oracle_pointset(w), w.A.astype(np.float64))
    assert colwise_rel_err(B, ref) <= TOL
