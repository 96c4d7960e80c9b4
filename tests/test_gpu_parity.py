"""GPU parity: the CUDA path (through the C ABI) against the FP64 oracle.

Integer tables are compared bit for bit; values within the per-column
∞-norm relative tolerance TOL (1e-5).
"""

import numpy as np
import pytest
import torch

from oracle import circulant, f2, numtheory, points, products
from paper_1501_06286_gb300 import capi, workloads
from paper_1501_06286_gb300.qmc import Plan

from _helpers import TOL, colwise_rel_err, conventional_output_rows, internal_order, oracle_pointset

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _built():
    from paper_1501_06286_gb300 import build
    build.build()
    torch.cuda.set_device(0)


def _run(w, prec="fp32", order="conventional", A=None, **kw):
    plan = Plan.from_workload(w, prec=prec, order=order)
    A = w.A if A is None else A
    At = torch.from_numpy(np.ascontiguousarray(A)).cuda()
    out = plan.matmul(At, **kw)
    torch.cuda.synchronize()
    return plan, out


# --------------------------------------------------------------------------
# Plan tables: bit-exact integer indexing
# --------------------------------------------------------------------------

@pytest.mark.parametrize("N", [7, 17, 257, 7681, 12289, 40961, 65537, 786433])
def test_prime_tables_bit_exact(N):
    w = workloads.random_prime_case(N, 97, 3, seed=N)
    plan = Plan.from_workload(w)
    assert plan.info["g"] == numtheory.smallest_primitive_root(N) == w.g
    pw = plan.table("pow")
    assert np.array_equal(pw, np.array(numtheory.power_table(w.g, N)))
    lg = plan.table("log")
    ref_lg = np.array(numtheory.log_table(w.g, N))
    assert np.array_equal(lg, ref_lg)
    e = plan.exponents()
    assert np.array_equal(e, np.array(numtheory.exponents(w.gen, w.g, N)))
    assert np.array_equal(e, plan.table("exponents"))
    assert np.array_equal(plan.table("out_row"), conventional_output_rows(N, w.g, True))
    # scatter lists: positions and j lists equal to the selector P's rows
    rp, jl = plan.table("row_ptr"), plan.table("jlist")
    for u in np.unique(e):
        assert list(jl[rp[u]:rp[u + 1]]) == [j for j in range(len(e)) if e[j] == u]
    assert plan.info["collision_adds"] == circulant.collision_adds(e)
    assert plan.info["n_distinct"] == len(set(e.tolist()))
    assert plan.info["row0_adds"] == w.s - 1


@pytest.mark.parametrize("m", [4, 8, 12, 16])
def test_f2_tables_bit_exact(m):
    w = workloads.f2_65536(m=m, s=50, grid=3)
    plan = Plan.from_workload(w)
    P = f2.smallest_primitive(m)
    assert plan.info["modulus_P"] == P
    L = (1 << m) - 1
    pw = plan.table("pow")
    v, ref = 1, []
    for _ in range(L):
        ref.append(v)
        v = f2.mod(v << 1, P)
    assert np.array_equal(pw, np.array(ref))
    assert np.array_equal(plan.exponents(), np.asarray(w.gen))
    # out rows: circulant row r is the point n(x) = x^{-r} mod P (row 0 dropped)
    n_of_r = np.array([ref[(L - r) % L] for r in range(L)])
    assert np.array_equal(plan.table("out_row"), n_of_r - 1)
    zeta = plan.table("zeta")
    zref = circulant.generator_sequence_f2(P, "phi_inv")
    assert np.max(np.abs(zeta - zref) / np.maximum(1.0, np.abs(zref))) < 1e-14


@pytest.mark.parametrize("N,map", [(7, "identity"), (17, "centred"), (257, "phi_inv"),
                                   (257, "tent"), (65537, "phi_inv"), (786433, "centred")])
def test_generator_sequence(N, map):
    w = workloads.random_prime_case(N, 8, 1, seed=1, map=map)
    plan = Plan.from_workload(w)
    zeta = plan.table("zeta")
    zref = circulant.generator_sequence_prime(N, w.g, map)
    if map == "phi_inv":
        # CUDA normcdfinv vs the oracle's AS241, both FP64
        assert np.max(np.abs(zeta - zref) / np.maximum(1.0, np.abs(zref))) < 1e-14
    else:
        assert np.array_equal(zeta, zref)


@pytest.mark.parametrize("N", [7, 17, 257, 7681, 65537])
def test_spectrum_fp64(N):
    w = workloads.random_prime_case(N, 8, 1, seed=2, map="phi_inv")
    plan = Plan.from_workload(w)
    zref = circulant.generator_sequence_prime(N, w.g, "phi_inv")
    Href = circulant.spectrum(zref) if N <= 257 else circulant.spectrum_fft(zref)
    H = plan.table("spectrum64")
    Hn = np.empty_like(H)
    Hn[internal_order(plan.info["L1"], plan.info["L2"])] = H
    assert np.max(np.abs(Hn - Href)) <= 1e-13 * np.max(np.abs(Href)) + 1e-15


# --------------------------------------------------------------------------
# Forward product
# --------------------------------------------------------------------------

@pytest.mark.parametrize("N", [7, 17, 257])
@pytest.mark.parametrize("map", ["identity", "centred", "phi_inv", "tent"])
@pytest.mark.parametrize("t", [1, 2, 5, 17])
def test_forward_small(N, map, t):
    w = workloads.random_prime_case(N, 3 * N // 2 + 1, t, seed=N * t, map=map)
    plan, B = _run(w)
    ps = oracle_pointset(w)
    ref = products.matmul(ps, w.A.astype(np.float64))
    assert B.shape == ref.shape
    assert colwise_rel_err(B.cpu().numpy(), ref) <= TOL


@pytest.mark.parametrize("N,s,t", [(7681, 300, 21), (12289, 200, 16), (40961, 64, 9),
                                   (65537, 300, 37), (257, 1000, 64)])
def test_forward_multipass(N, s, t):
    w = workloads.random_prime_case(N, s, t, seed=s + t, map="centred")
    plan, B = _run(w)
    ps = oracle_pointset(w)
    ref = products.matmul(ps, w.A.astype(np.float64))
    assert colwise_rel_err(B.cpu().numpy(), ref) <= TOL


@pytest.mark.parametrize("row0", ["include", "exclude"])
@pytest.mark.parametrize("order", ["conventional", "circulant"])
def test_row0_policy_and_order(row0, order):
    w = workloads.random_prime_case(7681, 120, 6, seed=4, map="centred", row0=row0)
    plan, B = _run(w, order=order)
    ps = oracle_pointset(w)
    ref = products.matmul(ps, w.A.astype(np.float64))
    if order == "circulant":
        rows = conventional_output_rows(w.N, w.g, row0 == "include")
        if row0 == "include":
            ref = np.vstack([ref[:1], ref[rows]])
        else:
            ref = ref[rows]
    assert colwise_rel_err(B.cpu().numpy(), ref) <= TOL


def test_lattice_257_config():
    w = workloads.lattice_257()
    plan, B = _run(w)
    ps = oracle_pointset(w)
    ref = products.matmul(ps, w.A)
    assert B.shape == (257, 1)
    assert colwise_rel_err(B.cpu().numpy(), ref) <= TOL
    assert plan.info["collision_adds"] == circulant.collision_adds(w.exponents)


def test_split_precision_fp64_input():
    w = workloads.random_prime_case(7681, 150, 7, seed=8, map="centred", dtype=np.float64)
    plan, B = _run(w, prec="fp32_split")
    ref = products.matmul(oracle_pointset(w), w.A)
    assert colwise_rel_err(B.cpu().numpy(), ref) <= TOL


@pytest.mark.parametrize("t", [1, 2, 7, 17, 40])
def test_split_precision_pipelined_768(t):
    # N = 786433 (L = 768 x 1024): the split loader and store of the
    # pipelined first pass (term-by-term pairs and singles, transformed
    # lines) and of the two-panel un-permute pass, with a ragged last panel
    # and a lone last panel; s = 5000 puts about five rows on a line
    w = workloads.random_prime_case(786433, 5000, t, seed=t, map="centred", dtype=np.float64)
    plan, B = _run(w, prec="fp32_split")
    rows = np.unique(np.concatenate([[0, 1, plan.out_rows - 1],
                                     np.random.default_rng(t).integers(0, plan.out_rows, 250)]))
    ref = products.matmul_rows(oracle_pointset(w), w.A, rows)
    assert colwise_rel_err(B[torch.from_numpy(rows).cuda()].cpu().numpy(), ref) <= TOL
    # every row: the centred points' column sums are -1/2 Σ_j A_jk, to
    # within 1e-6 of the sum of |B| (the rounding of the rows adds up)
    colsum = B.double().sum(dim=0).cpu().numpy()
    scale = B.double().abs().sum(dim=0).cpu().numpy()
    assert np.max(np.abs(colsum + 0.5 * w.A.sum(axis=0)) / scale) < 1e-6


def test_row_mean_and_exp_sum():
    w = workloads.random_prime_case(7681, 100, 13, seed=9, map="centred")
    A = (w.A * 0.1).astype(np.float32)
    plan, (B, rm, es) = _run(w, A=A, row_mean=True, exp_sum=True)
    ref = products.matmul(oracle_pointset(w), A.astype(np.float64))
    assert colwise_rel_err(rm.cpu().numpy(), products.row_mean(ref)) <= TOL
    assert abs(es.item() - np.exp(ref).sum()) <= 1e-5 * np.exp(ref).sum()


def test_zero_columns_give_exact_zeros():
    w = workloads.random_prime_case(7681, 64, 6, seed=10)
    A = w.A.copy()
    A[:, 2] = 0.0
    plan, B = _run(w, A=A)
    assert torch.all(B[:, 2] == 0)


def test_generate_points_matches_definition():
    w = workloads.random_prime_case(257, 40, 1, seed=12, map="phi_inv")
    plan = Plan.from_workload(w)
    Y = plan.generate_points().cpu().numpy()
    Yref = oracle_pointset(w).Y()
    assert np.max(np.abs(Y - Yref) / np.maximum(1, np.abs(Yref))) < 1e-6


def test_plan_round_trip_from_exponents():
    w = workloads.random_prime_case(65537, 200, 8, seed=13)
    p1, B1 = _run(w)
    e = p1.exponents()
    p2 = Plan("prime", w.N, e, map=w.map, g=p1.info["g"], gen_is_exponent=True)
    B2 = p2.matmul(torch.from_numpy(w.A).cuda())
    assert torch.equal(B1, B2)


# --------------------------------------------------------------------------
# Adjoint
# --------------------------------------------------------------------------

@pytest.mark.parametrize("N,s,t,map", [(17, 30, 3, "centred"), (257, 300, 8, "phi_inv"),
                                       (7681, 200, 11, "centred"), (65537, 100, 6, "phi_inv"),
                                       (786433, 60, 5, "centred")])
def test_adjoint_against_oracle(N, s, t, map):
    w = workloads.random_prime_case(N, s, t, seed=N + s, map=map)
    plan = Plan.from_workload(w)
    rng = np.random.default_rng(0)
    G = rng.standard_normal((plan.out_rows, t)).astype(np.float32)
    dA = plan.matmul_backward(torch.from_numpy(G).cuda()).cpu().numpy()
    ref = products.adjoint(oracle_pointset(w), G.astype(np.float64))
    assert colwise_rel_err(dA, ref) <= TOL


def test_adjoint_dot_product_on_gpu():
    w = workloads.random_prime_case(7681, 150, 10, seed=21, map="centred")
    plan = Plan.from_workload(w)
    A = torch.from_numpy(w.A).cuda()
    G = torch.randn(plan.out_rows, 10, device="cuda")
    lhs = (plan.matmul(A).double() * G.double()).sum().item()
    rhs = (A.double() * plan.matmul_backward(G).double()).sum().item()
    assert abs(lhs - rhs) <= 1e-5 * (abs(lhs) + abs(rhs))


# --------------------------------------------------------------------------
# Errors are status codes, never faults
# --------------------------------------------------------------------------

def _status_of(fn):
    try:
        fn()
    except capi.QmcError as e:
        return e.code
    return 0


def test_error_statuses():
    assert _status_of(lambda: Plan("prime", 15, [1, 2])) == 2            # not prime
    assert _status_of(lambda: Plan("prime", 7, [1, 2], g=2)) == 3        # 2 not primitive mod 7
    assert _status_of(lambda: Plan("prime", 7, [1, 7])) == 4             # z = 7 ≡ 0
    assert _status_of(lambda: Plan("prime", 7, [1, 6], gen_is_exponent=True)) == 4
    assert _status_of(lambda: Plan("f2", 16, [1, 2], P=0b11111)) == 3    # not primitive
    assert _status_of(lambda: Plan("prime", 7, [1], map="phi_inv", row0="include")) == 1
    p = Plan("prime", 7, [1, 5, 3])
    A = torch.zeros(3, 2, device="cuda")
    out = torch.zeros(7, 2, device="cuda")
    lib = capi.load()
    assert lib.qmc_matmul(p.handle, A.data_ptr(), 2, 0, 0, out.data_ptr(), 2, None, None, None) == 5
    assert lib.qmc_matmul(p.handle, A.data_ptr(), 1, 2, 0, out.data_ptr(), 2, None, None, None) == 5
    assert lib.qmc_matmul(p.handle, A.data_ptr(), 2, 2, 7, out.data_ptr(), 2, None, None, None) == 1
    assert p.sync_status() == 0


# --------------------------------------------------------------------------
# Polynomial lattice rules over F_2 (Remark 1), Rader-257 inside L = 65535
# --------------------------------------------------------------------------

@pytest.mark.parametrize("m,s,grid", [(6, 20, 3), (8, 40, 5), (12, 64, 5), (16, 48, 3)])
def test_f2_forward(m, s, grid):
    w = workloads.f2_65536(m=m, s=s, grid=grid)
    plan, B = _run(w)
    ps = oracle_pointset(w)
    ref = products.matmul(ps, w.A.astype(np.float64))
    assert B.shape == ref.shape == (w.N - 1, w.t)
    assert colwise_rel_err(B.cpu().numpy(), ref) <= TOL
    if m == 16:
        assert (plan.info["L1"], plan.info["L2"]) == (255, 257)


@pytest.mark.parametrize("m", [8, 16])
def test_f2_adjoint(m):
    w = workloads.f2_65536(m=m, s=40, grid=3)
    plan = Plan.from_workload(w)
    rng = np.random.default_rng(m)
    G = rng.standard_normal((plan.out_rows, w.t)).astype(np.float32)
    dA = plan.matmul_backward(torch.from_numpy(G).cuda()).cpu().numpy()
    ref = products.adjoint(oracle_pointset(w), G.astype(np.float64))
    assert colwise_rel_err(dA, ref) <= TOL


def test_f2_exp_loss_and_gradient():
    from paper_1501_06286_gb300.autograd import exp_mean_loss
    w = workloads.f2_65536(m=12, s=32, grid=5)
    plan = Plan.from_workload(w)
    A = torch.from_numpy(w.A).cuda().requires_grad_(True)
    loss = exp_mean_loss(A, plan)
    loss.backward()
    ps = oracle_pointset(w)
    ref_loss, ref_grad = products.exp_mean_loss_and_grad(ps, w.A.astype(np.float64))
    assert abs(loss.item() - ref_loss) <= 1e-5 * abs(ref_loss)
    assert colwise_rel_err(A.grad.cpu().numpy(), ref_grad) <= TOL


def test_autograd_matmul_matches_adjoint():
    from paper_1501_06286_gb300.autograd import qmc_matmul
    w = workloads.random_prime_case(7681, 90, 6, seed=31, map="phi_inv")
    plan = Plan.from_workload(w)
    A = torch.from_numpy(w.A).cuda().requires_grad_(True)
    B = qmc_matmul(A, plan)
    G = torch.randn_like(B)
    (B * G).sum().backward()
    ref = products.adjoint(oracle_pointset(w), G.cpu().numpy().astype(np.float64))
    assert colwise_rel_err(A.grad.cpu().numpy(), ref) <= TOL


def test_paired_columns_of_very_different_scale():
    # column pairs sharing one complex FFT column: each keeps its own
    # relative accuracy thanks to the power-of-two column scaling
    w = workloads.random_prime_case(65537, 100, 8, seed=41, map="phi_inv")
    A = w.A.copy()
    A[:, 0::2] *= 1e-4
    A[:, 5] = 0.0
    plan, B = _run(w, A=A)
    ref = products.matmul(oracle_pointset(w), A.astype(np.float64))
    assert colwise_rel_err(B.cpu().numpy(), ref) <= TOL


# --------------------------------------------------------------------------
# Register-resident pass kernels (LP = 256, 1024) against the oracle and
# against the generic kernel
# --------------------------------------------------------------------------

@pytest.mark.parametrize("N,s,t", [(257, 300, 19), (65537, 200, 21), (40961, 100, 8),
                                   (786433, 16, 6), (786433, 40, 7), (12289, 64, 3), (7681, 120, 40),
                                   (25601, 90, 7), (4001, 50, 5)])
@pytest.mark.parametrize("direction", ["forward", "adjoint"])
def test_pass_kernels_agree(N, s, t, direction):
    w = workloads.random_prime_case(N, s, t, seed=N % 1000 + s, map="phi_inv")
    ps = oracle_pointset(w)
    outs = {}
    for kind in ("generic", "register", "pipelined"):
        plan = Plan.from_workload(w)
        plan.set_pass_kernel(kind)
        if direction == "forward":
            outs[kind] = plan.matmul(torch.from_numpy(w.A).cuda()).cpu().numpy()
        else:
            G = np.random.default_rng(5).standard_normal((plan.out_rows, t)).astype(np.float32)
            outs[kind] = plan.matmul_backward(torch.from_numpy(G).cuda()).cpu().numpy()
    if direction == "forward":
        ref = products.matmul(ps, w.A.astype(np.float64))
    else:
        ref = products.adjoint(ps, G.astype(np.float64))
    for kind, got in outs.items():
        assert colwise_rel_err(got, ref) <= TOL, kind


@pytest.mark.parametrize("direction", ["forward", "adjoint"])
def test_pass_kernels_agree_f2(direction):
    w = workloads.f2_65536(m=16, s=48, grid=5)
    ps = oracle_pointset(w)
    G = np.random.default_rng(9).standard_normal((w.N - 1, w.t)).astype(np.float32)
    ref = (products.matmul(ps, w.A.astype(np.float64)) if direction == "forward"
           else products.adjoint(ps, G.astype(np.float64)))
    for kind in ("generic", "register", "pipelined"):
        plan = Plan.from_workload(w)
        plan.set_pass_kernel(kind)
        if direction == "forward":
            got = plan.matmul(torch.from_numpy(w.A).cuda()).cpu().numpy()
        else:
            got = plan.matmul_backward(torch.from_numpy(G).cuda()).cpu().numpy()
        assert colwise_rel_err(got, ref) <= TOL, kind


@pytest.mark.parametrize("mode", ["linear", "fused"])
def test_row_mean_modes(mode):
    w = workloads.field_786433(s=64, grid=9)
    plan = Plan.from_workload(w)
    plan.set_row_mean_mode(mode)
    B, rm, _ = plan.matmul(torch.from_numpy(w.A).cuda(), row_mean=True)
    ps = oracle_pointset(w)
    rows = np.arange(0, w.N, 1013)
    ref = products.matmul_rows(ps, w.A.astype(np.float64).mean(axis=1)[:, None], rows)[:, 0]
    assert colwise_rel_err(rm[torch.from_numpy(rows).cuda()].cpu().numpy(), ref) <= TOL


def test_f2_adjoint_with_row0():
    # F_2 plan with row 0 (centred map), L = 255 x 257: the adjoint's last
    # pass adds φ(0)·G_0 to every row of dA
    import dataclasses
    w = dataclasses.replace(workloads.f2_65536(m=16, s=40, grid=3), map="centred", row0="auto")
    plan = Plan.from_workload(w)
    assert plan.info["has_row0"] == 1
    G = np.random.default_rng(21).standard_normal((plan.out_rows, w.t)).astype(np.float32)
    dA = plan.matmul_backward(torch.from_numpy(G).cuda()).cpu().numpy()
    ref = products.adjoint(oracle_pointset(w), G.astype(np.float64))
    assert colwise_rel_err(dA, ref) <= TOL


def test_nonfinite_input_column_is_reported():
    # a NaN and an infinity in columns 2 and 6 of A: those columns and their
    # complex partners (3 and 7) come out non-finite, the other columns are
    # the product, and the plan reports QMC_ERR_NONFINITE
    w = workloads.random_prime_case(7681, 60, 9, seed=11)
    plan = Plan.from_workload(w)
    A = w.A.copy()
    A[5, 2] = np.nan
    A[17, 6] = np.inf
    B = plan.matmul(torch.from_numpy(A).cuda())
    torch.cuda.synchronize()
    assert plan.sync_status() == 12   # QMC_ERR_NONFINITE
    assert plan.sync_status() == 0    # read and cleared
    got = B.cpu().numpy()
    assert not np.any(np.isfinite(got[1:, [2, 3, 6, 7]]))
    keep = [0, 1, 4, 5, 8]
    ref = products.matmul(oracle_pointset(w), w.A.astype(np.float64))
    assert colwise_rel_err(got[:, keep], ref[:, keep]) <= TOL
