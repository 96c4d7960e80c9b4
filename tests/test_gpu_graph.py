"""The library's calls can be captured in a CUDA graph (the steady state the
throughput is quoted in): after qmc_plan_reserve nothing in a product
allocates or synchronises, so a capture of the forward product (with its
row-mean and exp-sum epilogues), the adjoint, the affine product and the
finite-element step replays to the same bits as the eager calls, for new
inputs copied into the captured buffers too."""

import numpy as np
import pytest
import torch

from _helpers import TOL, colwise_rel_err, oracle_pointset
from oracle import products
from paper_1501_06286_gb300 import workloads
from paper_1501_06286_gb300.qmc import Plan, fe_solve_mean

pytestmark = pytest.mark.gpu


def _capture(fn):
    side = torch.cuda.Stream()
    side.wait_stream(torch.cuda.current_stream())
    with torch.cuda.stream(side):
        fn()
    torch.cuda.current_stream().wait_stream(side)
    torch.cuda.synchronize()
    g = torch.cuda.CUDAGraph()
    with torch.cuda.graph(g):
        res = fn()
    torch.cuda.synchronize()
    return g, res


CASES = {
    "prime-65537": lambda: workloads.random_prime_case(65537, 300, 24, seed=1, map="centred"),
    "prime-786433": lambda: workloads.random_prime_case(786433, 64, 33, seed=2, map="centred"),
    "prime-7681-dense": lambda: workloads.random_prime_case(7681, 3000, 8, seed=3, map="centred"),
    "f2-65536": lambda: workloads.f2_65536(s=64, grid=4),
}


@pytest.mark.parametrize("case", sorted(CASES))
def test_forward_and_adjoint_replay_bit_exact(case):
    w = CASES[case]()
    t = w.t
    plan = Plan.from_workload(w)
    plan.reserve(t)
    A = torch.from_numpy(w.A.astype(np.float32)).cuda()
    out = torch.empty((plan.out_rows, t), device="cuda")
    G = torch.randn(plan.out_rows, t, device="cuda")
    dA = torch.empty((w.s, t), device="cuda")

    def step():
        _, rm, _ = plan.matmul(A, out=out, row_mean=True)
        plan.matmul_backward(G, dA=dA)
        return rm

    g, rm_g = _capture(step)
    rm_e = step().clone()
    out_e, dA_e = out.clone(), dA.clone()
    out.zero_()
    dA.zero_()
    g.replay()
    torch.cuda.synchronize()
    assert torch.equal(out, out_e) and torch.equal(dA, dA_e) and torch.equal(rm_g, rm_e)
    assert plan.sync_status() == 0
    # new inputs copied into the captured buffers: the replay computes them
    A2 = np.random.default_rng(1).standard_normal((w.s, t)).astype(np.float32)
    A.copy_(torch.from_numpy(A2))
    g.replay()
    torch.cuda.synchronize()
    rows = np.unique(np.random.default_rng(2).integers(0, plan.out_rows, 64))
    ref = products.matmul_rows(oracle_pointset(w), A2.astype(np.float64), rows)
    assert colwise_rel_err(out[torch.from_numpy(rows).cuda()].cpu().numpy(), ref) <= TOL


def test_affine_and_fe_step_replay_bit_exact():
    # Experiment 3's pipeline (exp(c + Y·Ψ), then the midpoint solves and
    # the mean) at a small size, captured whole
    w = workloads.fe_workload("lognormal", 257, 64, 40)
    plan = Plan.from_workload(w)
    plan.reserve(w.t)
    A = torch.from_numpy(w.A).cuda()
    off = torch.from_numpy(w.extra["col_offset"]).cuda()
    out = torch.empty((plan.out_rows, w.t), device="cuda")

    def step():
        plan.matmul_affine(A, off, apply_exp=True, out=out)
        return fe_solve_mean(out, 64, "midpoint")

    g, u_g = _capture(step)
    u_e = step().clone()
    u_g.zero_()
    g.replay()
    torch.cuda.synchronize()
    assert torch.equal(u_g, u_e)
