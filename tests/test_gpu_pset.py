"""Korobov p-set (Section 2.2) on the GPU against the FP64 oracle
(oracle.pset).  Every block of the reordered set is Z·P_b with one shared
circulant, so the library runs the (K-1) blocks as one product with
(K-1)·t right-hand sides; the output is (K-1)^2 x t."""

import ctypes

import numpy as np
import pytest
import torch

from _helpers import TOL, colwise_rel_err
from oracle import pset
from paper_1501_06286_gb300 import capi
from paper_1501_06286_gb300.qmc import Plan

pytestmark = pytest.mark.gpu


def _A(s, t, seed, dtype=np.float32):
    rng = np.random.default_rng(seed)
    return (rng.standard_normal((s, t)) * np.arange(1, s + 1)[:, None] ** -1.0).astype(dtype)


@pytest.mark.parametrize("K,s,t,map", [(257, 40, 5, "centred"), (257, 300, 4, "phi_inv"),
                                       (17, 6, 3, "tent"), (7681, 25, 3, "centred")])
def test_pset_forward(K, s, t, map):
    A = _A(s, t, K + s)
    plan = Plan("pset", K, None, map=map, s=s)
    assert plan.out_rows == (K - 1) ** 2
    B = plan.matmul(torch.from_numpy(A).cuda())
    torch.cuda.synchronize()
    ps = pset.PSet(K, s, map)
    if ps.out_rows <= 70000:
        ref = pset.matmul(ps, A.astype(np.float64))
        assert colwise_rel_err(B.cpu().numpy(), ref) <= TOL
    else:
        # sampled rows against the oracle, scaled by the full column maxima
        # of the GPU result (the oracle's full product is too large here)
        rows = np.sort(np.random.default_rng(1).choice(ps.out_rows, 20000, replace=False))
        ref = ps.Y_rows(rows) @ A.astype(np.float64)
        got = B[torch.from_numpy(rows).cuda()].cpu().numpy().astype(np.float64)
        scale = B.abs().amax(dim=0).cpu().numpy().astype(np.float64)
        assert np.max(np.abs(got - ref) / scale[None, :]) <= TOL


def test_pset_fp64_input_shift_and_circulant_order():
    K, s, t = 257, 50, 3
    A = _A(s, t, 7, np.float64)
    plan = Plan("pset", K, None, map="phi_inv", s=s, shift=0.125)
    B = plan.matmul(torch.from_numpy(A).cuda())
    ps = pset.PSet(K, s, "phi_inv", shift=0.125)
    ref = pset.matmul(ps, A)
    assert colwise_rel_err(B.cpu().numpy(), ref) <= TOL
    # circulant order: block b, row r holds the point n = g^{-r}, γ = g^b
    cplan = Plan("pset", K, None, map="phi_inv", s=s, shift=0.125, order="circulant")
    Bc = cplan.matmul(torch.from_numpy(A).cuda()).cpu().numpy()
    g = int(plan.info["g"])
    ginv = pow(g, K - 2, K)
    L = K - 1
    conv_rows = np.array([(pow(g, b, K) - 1) * L + pow(ginv, r, K) - 1
                          for b in range(L) for r in range(L)])
    assert colwise_rel_err(Bc, ref[conv_rows]) <= TOL


def test_pset_generate_points():
    K, s = 257, 33
    plan = Plan("pset", K, None, map="centred", s=s)
    Y = plan.generate_points()
    torch.cuda.synchronize()
    Yref = pset.PSet(K, s, "centred").Y()
    assert np.max(np.abs(Y.cpu().numpy() - Yref)) <= 1e-7


def test_pset_rejects_what_it_does_not_offer():
    K, s, t = 257, 10, 2
    plan = Plan("pset", K, None, map="centred", s=s)
    A = torch.from_numpy(_A(s, t, 3)).cuda()
    with pytest.raises(capi.QmcError):
        plan.matmul(A, row_mean=True)
    with pytest.raises(capi.QmcError):
        plan.matmul_backward(torch.zeros(plan.out_rows, t, device="cuda"))
    out = torch.empty(plan.out_rows, t, device="cuda")
    lib = capi.load()
    rc = lib.qmc_matmul_noalloc(plan.handle, ctypes.c_void_p(A.data_ptr()), t, t, 0,
                                ctypes.c_void_p(out.data_ptr()), t, None)
    assert rc == 6  # QMC_ERR_UNSUPPORTED
    with pytest.raises(ValueError):
        Plan("pset", K, [1, 2], s=2)
