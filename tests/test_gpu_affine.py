"""qmc_matmul_affine (Sections 3.2, 3.3): B = col_offset + Y·A, and
exp(col_offset + Y·A), against the FP64 oracle, on every kernel path (the
one-launch small product, pipelined and P x Q passes, row 0 kept or not,
Korobov p-set)."""

import numpy as np
import pytest
import torch

from _helpers import TOL, colwise_rel_err, oracle_pointset
from oracle import products, pset
from paper_1501_06286_gb300 import capi, workloads
from paper_1501_06286_gb300.qmc import Plan

pytestmark = pytest.mark.gpu


def _check(w, B, ref_lin):
    """ref_lin = Y·A (FP64); compares B with the workload's affine map of it.
    For exp the error of exp(θ) relative to the column's largest value is at
    most the absolute error of θ, i.e. TOL times the column's max |Y·A|."""
    off = w.extra["col_offset"].astype(np.float64)
    if w.extra["apply_exp"]:
        ref = np.exp(off[None, :] + ref_lin)
        tol = TOL * max(1.0, float(np.max(np.abs(ref_lin))))
    else:
        ref = off[None, :] + ref_lin
        tol = TOL
    assert B.shape == ref.shape
    assert colwise_rel_err(B, ref) <= tol


@pytest.mark.parametrize("kind,N,M,s", [("uniform", 257, 6, 40), ("uniform", 7681, 40, 60),
                                        ("uniform", 786433, 5, 30), ("lognormal", 257, 5, 30),
                                        ("lognormal", 65537, 33, 100), ("lognormal", 40961, 20, 64)])
def test_affine_against_oracle(kind, N, M, s):
    w = workloads.fe_workload(kind, N, M, s)
    plan = Plan.from_workload(w)
    B = plan.matmul_affine(torch.from_numpy(w.A).cuda(), torch.from_numpy(w.extra["col_offset"]).cuda(),
                           apply_exp=w.extra["apply_exp"])
    torch.cuda.synchronize()
    ps = oracle_pointset(w)
    if ps.out_rows * w.t <= 5e6:
        ref_lin = products.matmul(ps, w.A.astype(np.float64))
        _check(w, B.cpu().numpy(), ref_lin)
    else:  # sampled rows
        rows = np.unique(np.random.default_rng(2).integers(0, plan.out_rows, 4000))
        rows[0] = 0
        ref_lin = products.matmul_rows(ps, w.A.astype(np.float64), rows)
        full = B.cpu().numpy()
        off = w.extra["col_offset"].astype(np.float64)
        lin = np.log(full) - off if w.extra["apply_exp"] else full - off
        scale = np.abs(lin).max(axis=0)
        diff = np.abs(lin[rows] - ref_lin).max(axis=0)
        zero = scale == 0  # all-zero coefficient columns come out exactly zero
        assert np.all(diff[zero] == 0)
        assert np.all(diff[~zero] / scale[~zero] <= 2 * TOL)


def test_affine_without_offset_equals_plain_product():
    w = workloads.random_prime_case(7681, 80, 9, seed=3, map="centred")
    plan = Plan.from_workload(w)
    A = torch.from_numpy(w.A).cuda()
    B0 = plan.matmul(A)
    B1 = plan.matmul_affine(A)
    E = plan.matmul_affine(A, apply_exp=True)
    torch.cuda.synchronize()
    assert torch.equal(B0, B1)
    assert torch.allclose(E, torch.exp(B0), rtol=1e-6, atol=0)


def test_affine_pset():
    K, s, t = 257, 24, 5
    A = np.random.default_rng(4).standard_normal((s, t)).astype(np.float32)
    off = np.linspace(-1.0, 1.0, t).astype(np.float32)
    plan = Plan("pset", K, None, map="centred", s=s)
    B = plan.matmul_affine(torch.from_numpy(A).cuda(), torch.from_numpy(off).cuda(), apply_exp=True)
    ref_lin = pset.matmul(pset.PSet(K, s, "centred"), A.astype(np.float64))
    ref = np.exp(off.astype(np.float64)[None, :] + ref_lin)
    tol = TOL * max(1.0, float(np.max(np.abs(ref_lin))))
    assert colwise_rel_err(B.cpu().numpy(), ref) <= tol


def test_affine_rejects_bad_flag():
    w = workloads.random_prime_case(257, 10, 2, seed=1, map="centred")
    plan = Plan.from_workload(w)
    A = torch.from_numpy(w.A).cuda()
    out = torch.empty((plan.out_rows, 2), device="cuda")
    lib = capi.load()
    import ctypes
    rc = lib.qmc_matmul_affine(plan.handle, ctypes.c_void_p(A.data_ptr()), 2, 2, 0, None, 2,
                               ctypes.c_void_p(out.data_ptr()), 2, None)
    assert rc == 1
