"""Polynomial lattice rules over F_b (b prime; Remark 1) on the GPU against
the FP64 oracle (oracle.fb, oracle.points): the plan's integer tables bit
for bit, the generator sequence, forward products and the adjoint on single-
and two-pass lengths L = b^m - 1, the F_b kind at b = 2 against the F_2
kind, and the statuses of unsupported or invalid descriptors."""

import numpy as np
import pytest
import torch

from oracle import circulant, f2, fb, products
from paper_1501_06286_gb300 import capi, workloads
from paper_1501_06286_gb300.qmc import Plan

from _helpers import TOL, colwise_rel_err, oracle_pointset

pytestmark = pytest.mark.gpu

# (b, m): L = b^m - 1 = 8, 80, 242 = 2·11², 728, 624, 168, 2400 (two passes)
CASES = [(3, 2), (3, 4), (3, 5), (3, 6), (5, 4), (13, 2), (7, 4)]


@pytest.fixture(scope="module", autouse=True)
def _built():
    from paper_1501_06286_gb300 import build
    build.build()
    torch.cuda.set_device(0)


@pytest.mark.parametrize("b,m", CASES)
def test_fb_tables_bit_exact(b, m):
    w = workloads.fb_case(b, m, 40, 3, seed=b * 10 + m, map="centred")
    plan = Plan.from_workload(w)
    Pc = fb.smallest_primitive(m, b)
    assert plan.info["modulus_P"] == fb.encode(Pc, b)
    assert plan.info["base"] == b
    L = b ** m - 1
    assert plan.L == L
    # pow[k] = x^k mod P (base-b encoding), stepping by x in the oracle
    ref = []
    v = [1]
    for _ in range(L):
        ref.append(fb.encode(v, b))
        v = fb.divmod_poly([0] + v, Pc, b)[1]
    assert np.array_equal(plan.table("pow"), np.array(ref))
    lg = fb.log_table(Pc, b)
    assert np.array_equal(plan.table("log"), np.array(lg))
    assert np.array_equal(plan.exponents(), np.array([lg[int(q)] for q in w.gen]))
    # output rows: circulant row r is the point n(x) = x^{-r} (row 0 kept: centred)
    assert np.array_equal(plan.table("out_row"), np.array(circulant.reordered_conventional_index_fb(Pc, b)))
    # generator sequence: exact for the centred map
    assert np.array_equal(plan.table("zeta"), circulant.generator_sequence_fb(Pc, b, "centred"))


@pytest.mark.parametrize("map", ["phi_inv", "tent"])
def test_fb_generator_sequence_maps(map):
    b, m = 3, 5
    w = workloads.fb_case(b, m, 20, 2, seed=1, map=map)
    plan = Plan.from_workload(w)
    ref = circulant.generator_sequence_fb(fb.smallest_primitive(m, b), b, map)
    got = plan.table("zeta")
    if map == "phi_inv":
        assert np.max(np.abs(got - ref) / np.maximum(1.0, np.abs(ref))) <= 1e-14
        assert plan.out_rows == b ** m - 1
    else:
        assert np.array_equal(got, ref)


@pytest.mark.parametrize("b,m", CASES)
@pytest.mark.parametrize("map", ["centred", "phi_inv"])
def test_fb_forward_against_oracle(b, m, map):
    N = b ** m
    s = 2 * N if N < 200 else 150          # collisions on the short lengths
    w = workloads.fb_case(b, m, s, 9, seed=N + s, map=map)
    plan = Plan.from_workload(w)
    B = plan.matmul(torch.from_numpy(w.A).cuda())
    torch.cuda.synchronize()
    assert plan.sync_status() == 0
    ref = products.matmul(oracle_pointset(w), w.A.astype(np.float64))
    assert B.shape == ref.shape
    assert colwise_rel_err(B.cpu().numpy(), ref) <= TOL


@pytest.mark.parametrize("b,m", [(3, 6), (7, 4)])
def test_fb_adjoint_against_oracle(b, m):
    w = workloads.fb_case(b, m, 90, 7, seed=7, map="centred")
    plan = Plan.from_workload(w)
    rng = np.random.default_rng(3)
    G = rng.standard_normal((plan.out_rows, 7)).astype(np.float32)
    dA = plan.matmul_backward(torch.from_numpy(G).cuda())
    ref = products.adjoint(oracle_pointset(w), G.astype(np.float64))
    assert colwise_rel_err(dA.cpu().numpy(), ref) <= TOL


def test_fb_base2_equals_f2_kind():
    m, s, t = 12, 60, 5
    rng = np.random.default_rng(5)
    q = rng.integers(1, 1 << m, size=s)
    A = torch.from_numpy(rng.standard_normal((s, t)).astype(np.float32)).cuda()
    pf2 = Plan("f2", 1 << m, q, map="phi_inv")
    pfb = Plan("fb", 1 << m, q, map="phi_inv", base=2)
    assert pfb.info["modulus_P"] == pf2.info["modulus_P"] == f2.smallest_primitive(m)
    for name in ("pow", "log", "exponents", "out_row", "zeta"):
        assert np.array_equal(pfb.table(name), pf2.table(name))
    assert torch.equal(pfb.matmul(A), pf2.matmul(A))


def test_fb_generate_points_matches_definition():
    w = workloads.fb_case(5, 4, 30, 1, seed=2, map="centred")
    plan = Plan.from_workload(w)
    Y = plan.generate_points().cpu().numpy()
    ref = oracle_pointset(w).Y()
    assert np.array_equal(Y, ref.astype(np.float32))


def test_fb_statuses():
    q = np.array([1, 2, 3], dtype=np.int64)
    with pytest.raises(capi.QmcError) as e:
        Plan("fb", 81, q, base=4)                 # base not prime
    assert e.value.code == 2
    with pytest.raises(capi.QmcError) as e:
        Plan("fb", 80, q, base=3)                 # N not a power of b
    assert e.value.code == 2
    with pytest.raises(capi.QmcError) as e:
        Plan("fb", 3 ** 8, q, base=3)             # L = 6560 = 2^5·5·41: no FFT factorisation
    assert e.value.code == 6
    with pytest.raises(capi.QmcError) as e:
        Plan("fb", 9, q, base=3, P=9 + 1)         # x^2 + 1: not primitive over F_3
    assert e.value.code == 3
    with pytest.raises(capi.QmcError) as e:
        Plan("fb", 81, np.array([0, 5]), base=3)  # q_j = 0
    assert e.value.code == 4
    with pytest.raises(capi.QmcError) as e:
        Plan("fb", 81, np.array([81, 5]), base=3)  # q_j >= N: degree >= m
    assert e.value.code == 4
