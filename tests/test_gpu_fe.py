"""qmc_fe_solve_mean (the finite-element step of Sections 3.2 and 3.3,
Experiments 2 and 3) against the FP64 oracle: the constant-coefficient
closed form, the solver alone on the same FP32 rows, the whole pipeline
(affine product, then the solves and the mean) on small cases, and the
solver at Experiment 2's size (N = 4001, M = s = 2N)."""

import numpy as np
import pytest
import torch

from _helpers import oracle_pointset
from oracle import fe, products
from paper_1501_06286_gb300 import workloads
from paper_1501_06286_gb300.qmc import Plan, fe_solve_mean

pytestmark = pytest.mark.gpu


def _rel(a, b):
    return float(np.max(np.abs(np.asarray(a) - b)) / np.max(np.abs(b)))


@pytest.mark.parametrize("M", [3, 4, 33, 1000])
def test_constant_coefficient_closed_form(M):
    # rows of a ≡ 2 (tridiag: 4M, -2M) and a ≡ 3 (midpoint), exact in FP32
    rows = 37
    tri = torch.tensor(np.concatenate([np.full(M - 1, 4.0 * M), np.full(M - 2, -2.0 * M)]),
                       dtype=torch.float32).repeat(rows, 1).cuda()
    mid = torch.full((rows, M), 3.0, dtype=torch.float32, device="cuda")
    u_t = fe_solve_mean(tri, M, "tridiag").cpu().numpy()
    u_m = fe_solve_mean(mid, M, "midpoint").cpu().numpy()
    assert _rel(u_t, fe.constant_coefficient_solution(M, 2.0)) <= 1e-10
    assert _rel(u_m, fe.constant_coefficient_solution(M, 3.0)) <= 1e-10


@pytest.mark.parametrize("kind", ["tridiag", "midpoint"])
@pytest.mark.parametrize("n_sys,M", [(1, 57), (31, 57), (33, 57), (300, 57), (130, 777), (1, 3), (65, 4)])
def test_solver_alone_on_the_same_rows(kind, n_sys, M):
    # random diagonally dominant rows (FP32), a strided B and an explicit
    # right-hand side: both sides solve the same systems in FP64.  n_sys
    # spans whole and ragged chunks of 64 systems, M whole and ragged tiles
    # of 256 elements and the smallest systems
    rng = np.random.default_rng(n_sys + M)
    if kind == "tridiag":
        off = -rng.uniform(0.5, 1.5, size=(n_sys, M - 2))
        diag = np.abs(np.pad(off, ((0, 0), (1, 0)))) + np.abs(np.pad(off, ((0, 0), (0, 1)))) + rng.uniform(0.1, 1, (n_sys, M - 1))
        rows = np.concatenate([diag, off], axis=1).astype(np.float32)
    else:
        rows = rng.uniform(0.5, 3.0, size=(n_sys, M)).astype(np.float32)
    wide = np.zeros((n_sys, rows.shape[1] + 5), dtype=np.float32)
    wide[:, : rows.shape[1]] = rows
    g = rng.standard_normal(M - 1)
    Bw = torch.from_numpy(wide).cuda()
    u = fe_solve_mean(Bw[:, : rows.shape[1]], M, kind, torch.from_numpy(g).cuda()).cpu().numpy()
    ref = fe.mean_solution(rows.astype(np.float64), M, kind, rhs=g)
    assert _rel(u, ref) <= 1e-11


@pytest.mark.parametrize("kind,N,M,s", [("uniform", 257, 40, 30), ("uniform", 4001, 200, 150),
                                        ("lognormal", 257, 40, 30), ("lognormal", 4001, 150, 120)])
def test_pipeline_against_the_oracle(kind, N, M, s):
    # product (affine, exp for the log-normal case) then the solves: the
    # oracle does both in FP64 from the definition of the points.  The
    # product's FP32 error (1e-5 of each column's largest value; for the
    # log-normal case an absolute error of that size in the exponent, i.e. a
    # relative one in a) reaches ū about unchanged (the 1-D solution depends
    # on the coefficient like 1/a), so the bound is 10x that.
    w = workloads.fe_workload(kind, N, M, s)
    plan = Plan.from_workload(w)
    off = torch.from_numpy(w.extra["col_offset"]).cuda()
    B = plan.matmul_affine(torch.from_numpy(w.A).cuda(), off, apply_exp=w.extra["apply_exp"])
    fe_kind = "tridiag" if kind == "uniform" else "midpoint"
    u = fe_solve_mean(B, M, fe_kind).cpu().numpy()
    lin = products.matmul(oracle_pointset(w), w.A.astype(np.float64))
    Bref = w.extra["col_offset"].astype(np.float64)[None, :] + lin
    if w.extra["apply_exp"]:
        Bref = np.exp(Bref)
    ref = fe.mean_solution(Bref, M, fe_kind)
    scale = max(1.0, float(np.abs(lin).max())) if w.extra["apply_exp"] else 1.0
    assert _rel(u, ref) <= 1e-4 * scale


def test_experiment2_size_solver():
    # N = 4001, M = s = 2N (Experiment 2's largest timed case on this path):
    # the GPU product's rows, solved on the GPU and by the oracle in FP64
    N, M = 4001, 8002
    w = workloads.fe_workload("uniform", N, M, M)
    plan = Plan.from_workload(w)
    off = torch.from_numpy(w.extra["col_offset"]).cuda()
    B = plan.matmul_affine(torch.from_numpy(w.A).cuda(), off)
    u = fe_solve_mean(B, M, "tridiag").cpu().numpy()
    ref = fe.mean_solution(B.cpu().numpy().astype(np.float64), M, "tridiag")
    assert _rel(u, ref) <= 1e-9
    # the mean field is close to the y = 0 solution (a ≡ 2) in shape and size
    u0 = fe.constant_coefficient_solution(M, 2.0)
    assert 0.3 < float(u.max() / u0.max()) < 3.0


def test_experiment3_size_solver():
    # N = 4001, M = s = 2N with the log-normal coefficient exp(2 + Y·Ψ):
    # the GPU product's rows, solved on the GPU (flux form) and by the
    # oracle's elimination in FP64
    N, M = 4001, 8002
    w = workloads.fe_workload("lognormal", N, M, M)
    plan = Plan.from_workload(w)
    off = torch.from_numpy(w.extra["col_offset"]).cuda()
    B = plan.matmul_affine(torch.from_numpy(w.A).cuda(), off, apply_exp=True)
    u = fe_solve_mean(B, M, "midpoint").cpu().numpy()
    ref = fe.mean_solution(B.cpu().numpy().astype(np.float64), M, "midpoint")
    assert _rel(u, ref) <= 1e-9
    # and with a signed right-hand side
    g = np.random.default_rng(3).standard_normal(M - 1)
    u = fe_solve_mean(B, M, "midpoint", torch.from_numpy(g).cuda()).cpu().numpy()
    ref = fe.mean_solution(B.cpu().numpy().astype(np.float64), M, "midpoint", rhs=g)
    assert _rel(u, ref) <= 1e-9


def _near_element_form(rng, n_sys, M, noise, positive=False):
    # rows of the element-difference form (weights w_1..w_M) with the
    # diagonal perturbed by `noise` of itself: Experiment 2's structure
    # (positive: a one-signed perturbation, which keeps the rows diagonally
    # dominant however large it is)
    w = rng.uniform(1.0, 3.0, size=(n_sys, M)) * M
    z = rng.standard_normal((n_sys, M - 1))
    diag = (w[:, :-1] + w[:, 1:]) * (1.0 + noise * (np.abs(z) if positive else z))
    return np.concatenate([diag, -w[:, 1:-1]], axis=1).astype(np.float32)


@pytest.mark.parametrize("n_sys,M", [(40, 57), (9, 1000), (3, 8002), (2, 8192), (2, 8193)])
def test_defect_correction_rows(n_sys, M):
    # near-element-form rows take the defect correction (M up to 8192),
    # one row with a large perturbation and one random row take the
    # elimination instead: all against the oracle's elimination
    rng = np.random.default_rng(M)
    rows = _near_element_form(rng, n_sys, M, 1e-7)
    if n_sys >= 3:
        rows[1] = _near_element_form(rng, 1, M, 0.3, positive=True)[0]
        off = -rng.uniform(0.5, 1.5, size=M - 2)
        rows[2, : M - 1] = np.abs(np.pad(off, (1, 0))) + np.abs(np.pad(off, (0, 1))) + rng.uniform(0.1, 1, M - 1)
        rows[2, M - 1:] = off
    g = rng.standard_normal(M - 1)
    B = torch.from_numpy(rows).cuda()
    for rhs in (None, g):
        u = fe_solve_mean(B, M, "tridiag", None if rhs is None else torch.from_numpy(rhs).cuda()).cpu().numpy()
        ref = fe.mean_solution(rows.astype(np.float64), M, "tridiag", rhs=rhs)
        assert _rel(u, ref) <= (1e-11 if M <= 1000 else 1e-9)


@pytest.mark.parametrize("kind", ["tridiag", "midpoint"])
def test_solve_is_deterministic(kind):
    # the same rows give the same bits on every call
    rng = np.random.default_rng(11)
    M, n_sys = 300, 200
    if kind == "tridiag":
        off = -rng.uniform(0.5, 1.5, size=(n_sys, M - 2))
        diag = np.abs(np.pad(off, ((0, 0), (1, 0)))) + np.abs(np.pad(off, ((0, 0), (0, 1)))) + 0.5
        rows = np.concatenate([diag, off], axis=1).astype(np.float32)
    else:
        rows = rng.uniform(0.5, 3.0, size=(n_sys, M)).astype(np.float32)
    Bt = torch.from_numpy(rows).cuda()
    u1 = fe_solve_mean(Bt, M, kind).cpu().numpy()
    u2 = fe_solve_mean(Bt, M, kind).cpu().numpy()
    assert np.array_equal(u1, u2)


def test_pivots_outside_the_fp32_range():
    # one row scaled by 1e33 and one by 1e-33: their pivots (about M times
    # the coefficient) leave FP32's normal range, where the solve takes the
    # FP64 division instead of the FP32-seeded Newton reciprocal
    rng = np.random.default_rng(7)
    M, n_sys = 57, 40
    rows = rng.uniform(0.5, 3.0, size=(n_sys, M))
    rows[3] *= 1e33
    rows[5] *= 1e-33
    rows = rows.astype(np.float32)
    u = fe_solve_mean(torch.from_numpy(rows).cuda(), M, "midpoint").cpu().numpy()
    ref = fe.mean_solution(rows.astype(np.float64), M, "midpoint")
    assert np.all(np.isfinite(u))
    assert _rel(u, ref) <= 1e-11
    # the same with the extreme rows removed: every finite row matters
    keep = [i for i in range(n_sys) if i not in (3, 5)]
    u2 = fe_solve_mean(torch.from_numpy(rows[keep]).cuda(), M, "midpoint").cpu().numpy()
    ref2 = fe.mean_solution(rows[keep].astype(np.float64), M, "midpoint")
    assert _rel(u2, ref2) <= 1e-11
