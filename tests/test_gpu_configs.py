"""GPU parity at the full workload sizes, in the launch configuration that
bench.py times (default plan options).

Every output row of each full-size product is compared element by element
with the FP64 oracle: on all columns where the oracle's dense product fits
in host memory (the Gaussian and F_2 workloads), and on whole 8-column
panels of the work array otherwise (the field workload: the first two
panels, a middle one and the last two, the last one ragged because t is
odd), plus sampled rows across all columns.  Properties that hold at any
size (closed-form column sums, exact zero columns) cover every entry."""

import numpy as np
import pytest
import torch

from oracle import numtheory, products
from paper_1501_06286_gb300 import workloads
from paper_1501_06286_gb300.autograd import exp_mean_loss
from paper_1501_06286_gb300.qmc import Plan

from _helpers import (TOL, ColwiseErr, colwise_rel_err, conventional_output_rows,
                      oracle_pointset, oracle_row_blocks, panel_columns)

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
    # every output row, every column
    ps = oracle_pointset(w)
    acc = ColwiseErr(w.t)
    for r0, r1, ref in oracle_row_blocks(ps, w.A.astype(np.float64)):
        acc.add(B[r0:r1].cpu().numpy(), ref)
    assert acc.value() <= TOL
    # Φ^{-1} points: every column sums to 0 over the N-1 rows (closed form)
    colsum = B.double().sum(dim=0)
    scale = B.double().abs().sum(dim=0)
    assert torch.max(colsum.abs() / scale).item() < 1e-6


@pytest.fixture(scope="module")
def field_reference():
    """Oracle products of the field workload on every output row: the panel
    columns for A in FP32 (as the FP32 path reads it) and in FP64 (the split
    path), and the row means r = Y·(A·1/t) of both."""
    w32 = workloads.field_786433(dtype=np.float32)
    w64 = workloads.field_786433(dtype=np.float64)
    cols = panel_columns(w32.t, split=False)
    assert set(panel_columns(w64.t, split=True)) <= set(cols.tolist())
    A32 = w32.A.astype(np.float64)
    A64 = w64.A
    k = len(cols)
    rhs = np.concatenate([A32[:, cols], A64[:, cols], A32.mean(axis=1)[:, None],
                          A64.mean(axis=1)[:, None]], axis=1)
    ps = oracle_pointset(w32)
    ref = np.empty((ps.out_rows, rhs.shape[1]))
    for r0, r1, blk in oracle_row_blocks(ps, rhs, block=8192):
        ref[r0:r1] = blk
    return {"cols": cols, "ps": ps,
            "fp32": (ref[:, :k], ref[:, 2 * k]), "fp32_split": (ref[:, k:2 * k], ref[:, 2 * k + 1])}


@pytest.mark.parametrize("prec", ["fp32", "fp32_split"])
def test_field_786433_full_size(prec, field_reference):
    dtype = np.float64 if prec == "fp32_split" else np.float32
    w = workloads.field_786433(dtype=dtype)
    plan = Plan.from_workload(w, prec=prec)
    # integer tables of the plan itself, bit for bit
    assert plan.info["g"] == w.g == numtheory.smallest_primitive_root(w.N)
    assert np.array_equal(plan.exponents(), np.asarray(numtheory.exponents(w.gen, w.g, w.N)))
    assert np.array_equal(plan.table("out_row"), conventional_output_rows(w.N, w.g, True))
    A = torch.from_numpy(w.A).cuda()
    B, rm, _ = plan.matmul(A, row_mean=True)
    torch.cuda.synchronize()
    assert B.shape == (786433, 4225)
    cols = field_reference["cols"]
    ref_b, ref_rm = field_reference[prec]
    # every output row on whole panels, including the ragged last one
    got = B[:, torch.from_numpy(cols).cuda()].cpu().numpy()
    assert colwise_rel_err(got, ref_b) <= TOL
    # every row mean
    assert colwise_rel_err(rm.cpu().numpy(), ref_rm) <= TOL
    # sampled rows across all columns
    rows = _sample_rows(plan.out_rows, 96, 1)
    A64 = w.A.astype(np.float64)
    ref = products.matmul_rows(field_reference["ps"], A64, rows)
    assert colwise_rel_err(B[torch.from_numpy(rows).cuda()].cpu().numpy(), ref) <= TOL
    # boundary nodes of the grid are exactly zero columns
    zero_cols = [k for k in range(4225) if not np.any(A64[:, k])]
    assert len(zero_cols) == 4 * 64
    assert torch.count_nonzero(B[:, zero_cols]).item() == 0
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
    A64 = w.A.astype(np.float64)
    ref_B = products.matmul(ps, A64)
    ref_loss = products.exp_mean_loss(ref_B)
    ref_grad = products.adjoint(ps, products.exp_mean_loss_grad_B(ref_B))
    assert abs(loss.item() - ref_loss) <= 1e-5 * abs(ref_loss)
    # the gradient: every row of dA
    assert colwise_rel_err(A.grad.cpu().numpy(), ref_grad) <= TOL
    # the forward product: every output row, every column
    B = plan.matmul(A.detach())
    assert B.shape == ref_B.shape
    assert colwise_rel_err(B.cpu().numpy(), ref_B) <= TOL


def test_lattice_257_full():
    w = workloads.lattice_257()
    plan = Plan.from_workload(w)
    B = plan.matmul(torch.from_numpy(w.A).cuda())
    ref = products.matmul(oracle_pointset(w), w.A)
    assert colwise_rel_err(B.cpu().numpy(), ref) <= TOL
