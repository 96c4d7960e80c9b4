"""GPU parity at the full workload sizes, in the launch configuration that
bench.py times (default plan options), on output rows the oracle computes
one by one, plus properties that hold at any size."""

import numpy as np
import pytest
import torch

from oracle import products
from paper_1501_06286_gb300 import workloads
from paper_1501_06286_gb300.autograd import exp_mean_loss
from paper_1501_06286_gb300.qmc import Plan

from _helpers import TOL, colwise_rel_err, oracle_pointset

pytestmark = pytest.mark.gpu


def _sample_rows(out_rows, n, seed):
    rng = np.random.default_rng(seed)
    rows = set(rng.choice(out_rows, size=n, replace=False).tolist())
    rows |= {0, 1, out_rows - 1}
    return np.array(sorted(rows))


@pytest.fixture(scope="module", autouse=True)
def _built():
    from paper_1501_06286_gb300 import build
    build.build()
    torch.cuda.set_device(0)


def test_gauss_65537_full_size():
    w = workloads.gauss_65537()
    plan = Plan.from_workload(w)
    A = torch.from_numpy(w.A).cuda()
    B = plan.matmul(A)
    torch.cuda.synchronize()
    assert B.shape == (65536, 4096)
    rows = _sample_rows(plan.out_rows, 192, 0)
    ps = oracle_pointset(w)
    ref = products.matmul_rows(ps, w.A.astype(np.float64), rows)
    assert colwise_rel_err(B[torch.from_numpy(rows).cuda()].cpu().numpy(), ref) <= TOL
    # Φ^{-1} points: every column sums to 0 over the N-1 rows (closed form)
    colsum = B.double().sum(dim=0)
    scale = B.double().abs().sum(dim=0)
    assert torch.max(colsum.abs() / scale).item() < 1e-6


@pytest.mark.parametrize("prec", ["fp32", "fp32_split"])
def test_field_786433_full_size(prec):
    dtype = np.float64 if prec == "fp32_split" else np.float32
    w = workloads.field_786433(dtype=dtype)
    plan = Plan.from_workload(w, prec=prec)
    A = torch.from_numpy(w.A).cuda()
    B, rm, _ = plan.matmul(A, row_mean=True)
    torch.cuda.synchronize()
    assert B.shape == (786433, 4225)
    rows = _sample_rows(plan.out_rows, 96, 1)
    ps = oracle_pointset(w)
    A64 = w.A.astype(np.float64)
    ref = products.matmul_rows(ps, A64, rows)
    got = B[torch.from_numpy(rows).cuda()].cpu().numpy()
    assert colwise_rel_err(got, ref) <= TOL
    # boundary nodes of the grid are exactly zero columns
    zero_cols = [k for k in range(4225) if not np.any(A64[:, k])]
    assert len(zero_cols) == 4 * 64
    assert torch.count_nonzero(B[:, zero_cols]).item() == 0
    # per-row mean: r = Y·(A·1/t)
    ref_rm = products.matmul_rows(ps, A64.mean(axis=1)[:, None], rows)[:, 0]
    assert colwise_rel_err(rm[torch.from_numpy(rows).cuda()].cpu().numpy(), ref_rm) <= TOL
    # centred points: column sums over all N rows are -1/2 sum_j A_jk
    colsum = B.double().sum(dim=0).cpu().numpy()
    target = -0.5 * A64.sum(axis=0)
    scale = B.double().abs().sum(dim=0).cpu().numpy()
    nz = scale > 0
    assert np.max(np.abs(colsum - target)[nz] / scale[nz]) < 1e-6


def test_f2_65536_full_size_loss_and_gradient():
    w = workloads.f2_65536()
    plan = Plan.from_workload(w)
    assert (plan.info["L1"], plan.info["L2"]) == (255, 257)
    A = torch.from_numpy(w.A).cuda().requires_grad_(True)
    loss = exp_mean_loss(A, plan)
    loss.backward()
    ps = oracle_pointset(w)
    ref_loss, ref_grad = products.exp_mean_loss_and_grad(ps, w.A.astype(np.float64))
    assert abs(loss.item() - ref_loss) <= 1e-5 * abs(ref_loss)
    assert colwise_rel_err(A.grad.cpu().numpy(), ref_grad) <= TOL
    B = plan.matmul(A.detach())
    rows = _sample_rows(plan.out_rows, 128, 2)
    ref = products.matmul_rows(ps, w.A.astype(np.float64), rows)
    assert colwise_rel_err(B[torch.from_numpy(rows).cuda()].cpu().numpy(), ref) <= TOL


def test_lattice_257_full():
    w = workloads.lattice_257()
    plan = Plan.from_workload(w)
    B = plan.matmul(torch.from_numpy(w.A).cuda())
    ref = products.matmul(oracle_pointset(w), w.A)
    assert colwise_rel_err(B.cpu().numpy(), ref) <= TOL
