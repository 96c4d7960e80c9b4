"""Diagonal shift of Remark 2 on the GPU: every coordinate x becomes {x + Δ}
(one Δ for all coordinates), so the plan's generator sequence is
z_k = φ({x_k + Δ}) and row 0 is φ(Δ)·Σ_j a_j.  Compared with the FP64
oracle's shifted point set."""

import dataclasses

import numpy as np
import pytest
import torch

from _helpers import TOL, colwise_rel_err, oracle_pointset
from oracle import products
from paper_1501_06286_gb300 import workloads
from paper_1501_06286_gb300.qmc import Plan

pytestmark = pytest.mark.gpu

DELTA = 0.3717


def _shifted(w, delta=DELTA):
    return dataclasses.replace(w, shift=delta)


@pytest.mark.parametrize("map", ["phi_inv", "centred", "tent"])
@pytest.mark.parametrize("N", [257, 7681, 65537])
def test_shift_forward(N, map):
    w = _shifted(workloads.random_prime_case(N, 300, 9, seed=N, map=map))
    plan = Plan.from_workload(w)
    ps = oracle_pointset(w)
    assert plan.info["has_row0"] == 1          # φ(Δ) is finite for Δ in (0, 1)
    assert abs(plan.info["phi0"] - ps.phi0) <= 1e-14 * max(1.0, abs(ps.phi0))
    B = plan.matmul(torch.from_numpy(w.A).cuda())
    torch.cuda.synchronize()
    ref = products.matmul(ps, w.A.astype(np.float64))
    assert B.shape == ref.shape
    assert colwise_rel_err(B.cpu().numpy(), ref) <= TOL


def test_shift_adjoint_and_points():
    w = _shifted(workloads.random_prime_case(7681, 200, 5, seed=2, map="phi_inv"))
    plan = Plan.from_workload(w)
    ps = oracle_pointset(w)
    G = np.random.default_rng(3).standard_normal((plan.out_rows, 5)).astype(np.float32)
    dA = plan.matmul_backward(torch.from_numpy(G).cuda())
    Y = plan.generate_points()
    torch.cuda.synchronize()
    ref = products.adjoint(ps, G.astype(np.float64))
    assert colwise_rel_err(dA.cpu().numpy(), ref) <= TOL
    Yref = ps.Y()
    assert np.max(np.abs(Y.cpu().numpy() - Yref)) <= 1e-6 * np.max(np.abs(Yref))


def test_shift_f2():
    w = _shifted(workloads.f2_65536(seed=4, m=12, s=64, grid=5))
    plan = Plan.from_workload(w)
    ps = oracle_pointset(w)
    B = plan.matmul(torch.from_numpy(w.A).cuda())
    torch.cuda.synchronize()
    ref = products.matmul(ps, w.A.astype(np.float64))
    assert colwise_rel_err(B.cpu().numpy(), ref) <= TOL


def test_zero_shift_is_the_unshifted_plan():
    w = workloads.random_prime_case(7681, 100, 4, seed=5, map="centred")
    A = torch.from_numpy(w.A).cuda()
    B0 = Plan.from_workload(w).matmul(A)
    B1 = Plan.from_workload(_shifted(w, 0.0)).matmul(A)
    torch.cuda.synchronize()
    assert torch.equal(B0, B1)
