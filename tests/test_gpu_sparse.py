"""Sparse first pass (qmc_first_pass): the spectral pass sums each of its
lines, Σ_j a_j·w_L^{-e_j·k1} over the rows j whose position e_j falls on the
line, straight from the rows of A, instead of reading the first pass's
transform from the work array (Section 2.1's scatter-add and FFT, in one
pass).  Checked against the FP64 oracle with the mode forced on and off on
the same inputs, for both pass lengths (L2 = 256, 1024), first factors L1
that are not powers of two, collisions, FP64 and split-precision A, strided
A, the affine epilogue and the fused row mean; the per-stage profile shows
which path ran."""

import ctypes as C

import numpy as np
import pytest
import torch

from _helpers import TOL, colwise_rel_err, oracle_pointset
from oracle import products
from paper_1501_06286_gb300 import capi, workloads
from paper_1501_06286_gb300.qmc import Plan

pytestmark = pytest.mark.gpu


def _profiled(plan, fn):
    """Runs fn() with per-stage events on; returns its result and the set
    of stages that launched."""
    lib = capi.load()
    lib.qmc_plan_set_profiling(plan.handle, 1)
    out = fn()
    torch.cuda.synchronize()
    ms = (C.c_double * capi.NUM_STAGES)()
    n = (C.c_int32 * capi.NUM_STAGES)()
    assert lib.qmc_plan_read_profile(plan.handle, ms, n) == 0
    lib.qmc_plan_set_profiling(plan.handle, 0)
    return out, {capi.STAGES[i] for i in range(capi.NUM_STAGES) if n[i]}


def _reference(plan, w, A64, sample=None):
    ps = oracle_pointset(w)
    if sample is None:
        return None, products.matmul(ps, A64)
    rows = np.unique(np.random.default_rng(5).integers(0, plan.out_rows, sample))
    return rows, products.matmul_rows(ps, A64, rows)


def _check(B, rows, ref):
    if rows is None:
        assert colwise_rel_err(B, ref) <= TOL
        return
    # sampled rows: error relative to each column's largest sampled value
    scale = np.abs(ref).max(axis=0)
    diff = np.abs(B[rows] - ref).max(axis=0)
    assert np.all(diff <= TOL * scale)


@pytest.mark.parametrize("N,s,t,sample", [
    (65537, 300, 20, None),      # L = 256 x 256
    (40961, 700, 16, 3000),      # L = 160 x 256: n1·k1 mod L1 off powers of two
    (786433, 2048, 19, 3000),    # L = 768 x 1024, two rows per line on average
    (7681, 90, 17, None),        # L = 80 x 96: no sparse form, the first pass runs
])
@pytest.mark.parametrize("mode", ["sparse", "transform"])
def test_forced_modes_against_oracle(N, s, t, sample, mode):
    w = workloads.random_prime_case(N, s, t, seed=N % 97, map="phi_inv")
    plan = Plan.from_workload(w)
    plan.set_first_pass(mode)
    A = torch.from_numpy(w.A).cuda()
    B, stages = _profiled(plan, lambda: plan.matmul(A))
    L2 = plan.info["L2"]
    if mode == "sparse" and L2 in (256, 1024):
        assert {"sparse_pack", "fwd_sparse"} <= stages and "fwd_scatter" not in stages
    else:
        assert "fwd_sparse" not in stages
    rows, ref = _reference(plan, w, w.A.astype(np.float64), sample)
    _check(B.cpu().numpy(), rows, ref)


def test_auto_takes_sparse_only_for_few_rows_per_line():
    # L2 = 256: s <= 256 folds the first pass, s above it keeps it
    for s, sparse in [(256, True), (257, False)]:
        w = workloads.random_prime_case(65537, s, 16, seed=s, map="centred")
        plan = Plan.from_workload(w)
        A = torch.from_numpy(w.A).cuda()
        B, stages = _profiled(plan, lambda: plan.matmul(A))
        assert ("fwd_sparse" in stages) == sparse
        rows, ref = _reference(plan, w, w.A.astype(np.float64), 2000)
        _check(B.cpu().numpy(), rows, ref)


def test_narrow_products_fall_back_to_the_transform():
    # fewer than 8 complex columns: no 8-column panels, the first pass runs
    w = workloads.random_prime_case(65537, 100, 5, seed=8, map="centred")
    plan = Plan.from_workload(w)
    plan.set_first_pass("sparse")
    B, stages = _profiled(plan, lambda: plan.matmul(torch.from_numpy(w.A).cuda()))
    assert "fwd_sparse" not in stages and "fwd_scatter" in stages
    _, ref = _reference(plan, w, w.A.astype(np.float64))
    _check(B.cpu().numpy(), None, ref)


@pytest.mark.parametrize("N", [65537, 40961])
def test_collisions_and_many_rows_per_line(N):
    # every row on one of three positions, and s far above the AUTO bound
    s, t = 3000, 18
    w = workloads.random_prime_case(N, s, t, seed=21, map="centred")
    w.gen[:] = w.gen[np.arange(s) % 3]
    plan = Plan.from_workload(w)
    plan.set_first_pass("sparse")
    B, stages = _profiled(plan, lambda: plan.matmul(torch.from_numpy(w.A).cuda()))
    assert "fwd_sparse" in stages
    rows, ref = _reference(plan, w, w.A.astype(np.float64), 3000)
    _check(B.cpu().numpy(), rows, ref)


@pytest.mark.parametrize("prec", ["fp32", "fp32_split"])
def test_fp64_input(prec):
    w = workloads.random_prime_case(65537, 400, 21, seed=30, map="phi_inv", dtype=np.float64)
    plan = Plan.from_workload(w, prec=prec)
    plan.set_first_pass("sparse")
    B, stages = _profiled(plan, lambda: plan.matmul(torch.from_numpy(w.A).cuda()))
    assert "fwd_sparse" in stages
    _, ref = _reference(plan, w, w.A)
    _check(B.cpu().numpy(), None, ref)


def test_strided_input():
    # A as a column block of a wider FP32 matrix (lda > t, odd offset)
    N, s, t = 40961, 200, 19
    w = workloads.random_prime_case(N, s, t, seed=14, map="tent")
    plan = Plan.from_workload(w)
    plan.set_first_pass("sparse")
    wide = torch.zeros((s, 27), dtype=torch.float32)
    wide[:, 5:5 + t] = torch.from_numpy(w.A)
    wide = wide.cuda()
    B = torch.empty((plan.out_rows, t), device="cuda")
    lib = capi.load()

    def run():
        rc = lib.qmc_matmul(plan.handle, C.c_void_p(wide.data_ptr() + 4 * 5), 27, t, 0,
                            C.c_void_p(B.data_ptr()), t, None, None,
                            C.c_void_p(torch.cuda.current_stream().cuda_stream))
        assert rc == 0
        return B

    B, stages = _profiled(plan, run)
    assert "fwd_sparse" in stages
    _, ref = _reference(plan, w, w.A.astype(np.float64))
    _check(B.cpu().numpy(), None, ref)


def test_affine_and_row_mean_on_the_sparse_path():
    w = workloads.random_prime_case(65537, 250, 24, seed=40, map="centred")
    A64 = w.A.astype(np.float64)
    off = np.linspace(-0.5, 0.5, w.t).astype(np.float32)
    plan = Plan.from_workload(w)
    plan.set_first_pass("sparse")
    A = torch.from_numpy(w.A).cuda()
    E, stages = _profiled(plan, lambda: plan.matmul_affine(A, torch.from_numpy(off).cuda(), apply_exp=True))
    assert "fwd_sparse" in stages
    _, lin = _reference(plan, w, A64)
    ref = np.exp(off.astype(np.float64)[None, :] + lin)
    assert colwise_rel_err(E.cpu().numpy(), ref) <= TOL * max(1.0, float(np.abs(lin).max()))
    B, r = plan.matmul(A, row_mean=True)[:2]
    torch.cuda.synchronize()
    assert colwise_rel_err(B.cpu().numpy(), lin) <= TOL
    mean_ref = lin.mean(axis=1)
    assert np.max(np.abs(r.cpu().numpy() - mean_ref)) <= TOL * np.abs(lin).max()


def test_modes_agree_closely():
    # the two forms sum the same terms in different orders: FP32 rounding apart
    w = workloads.random_prime_case(786433, 1500, 40, seed=3, map="centred")
    A = torch.from_numpy(w.A).cuda()
    out = {}
    for mode in ("sparse", "transform"):
        plan = Plan.from_workload(w)
        plan.set_first_pass(mode)
        out[mode] = plan.matmul(A).cpu().numpy()
    scale = np.abs(out["transform"]).max(axis=0)
    assert np.all(np.abs(out["sparse"] - out["transform"]).max(axis=0) <= 2 * TOL * scale)


def _case_with_lines(N, lines, t, seed, extra_rows=0):
    """Rows of A placed on chosen first-pass lines of the N = 786433 plan
    (L = 768 x 1024, position e = n1·1024 + n2 on line n2): lines maps a
    line n2 to the list of its n1 values (repeats collide), plus
    extra_rows rows at random positions."""
    rng = np.random.default_rng(seed)
    e = [n1 * 1024 + n2 for n2, n1s in lines.items() for n1 in n1s]
    e += list(rng.integers(0, N - 1, size=extra_rows))
    e = np.array(e, dtype=np.int64)
    g = workloads.PRIMITIVE_ROOT[N]
    z = np.array([pow(g, int(v), N) for v in e], dtype=np.int64)
    A = rng.standard_normal((len(e), t)).astype(np.float32)
    return workloads.Workload(f"lines-{N}", "prime", N, g, 0, z, False, "centred", "auto", A, exponents=e)


@pytest.mark.parametrize("t", [17, 32])
def test_first_pass_lines_summed_term_by_term(t):
    # lines of 4 entries take the term-by-term DFT, lines of 5 the transform;
    # a point hit three times, a line whose points include n1 = 0 and
    # n1 = 767, and odd rows (t = 17: 64-byte output runs by shuffles)
    N = 786433
    lines = {7: [0, 5, 100, 767], 9: [1, 2, 3, 4, 5], 11: [300, 300, 300, 12], 13: [767], 1023: [0]}
    w = _case_with_lines(N, lines, t, seed=t, extra_rows=40)
    plan = Plan.from_workload(w)
    plan.set_first_pass("transform")
    A = torch.from_numpy(w.A).cuda()
    B = plan.matmul(A)
    torch.cuda.synchronize()
    ps = oracle_pointset(w)
    rows = np.unique(np.concatenate([np.random.default_rng(1).integers(0, plan.out_rows, 3000),
                                     [0, 1, plan.out_rows - 1]]))
    ref = products.matmul_rows(ps, w.A.astype(np.float64), rows)
    _check(B.cpu().numpy(), rows, ref)
    # exp-sum epilogue on the same path: Σ exp(B) against the oracle's B
    B2, _, es = plan.matmul(A, exp_sum=True)
    torch.cuda.synchronize()
    assert torch.allclose(B2, B, rtol=1e-6, atol=0)
    full = B.double()
    assert abs(float(es.item()) - float(torch.exp(full).sum())) <= 1e-5 * float(torch.exp(full).sum())
