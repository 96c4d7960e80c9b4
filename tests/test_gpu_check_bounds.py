"""The bounds-checked build (-DQMC_CHECK_BOUNDS, libqmcfft_checked.so):
its products equal the oracle's like the default build's, and an index
planted out of range in a plan table (qmc_debug_poke_table) is caught by
the kernels' checks, which latch QMC_ERR_BOUNDS instead of reading or
writing outside a buffer; with the entry restored the plan works again.

Each planted index is read only by kernels that check it: the out-row table
by the un-permute stores (every pass kernel of the forward product), the
adjoint's loads of G and the point generator; the j list by the dense first
pass and the adjoint's stores of dA (the pipelined first passes read the
gather table built from it at plan time, which is not touched).  The
product runs in a child process that loads the checked library through
QMC_LIBRARY."""

import json
import os
import subprocess
import sys
import textwrap

import pytest

pytestmark = pytest.mark.gpu

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))

CHILD = textwrap.dedent(r"""
    import ctypes as C, json, sys
    import numpy as np, torch
    sys.path.insert(0, "tests")
    from _helpers import colwise_rel_err, oracle_pointset
    from oracle import products
    from paper_1501_06286_gb300 import capi, workloads
    from paper_1501_06286_gb300.qmc import Plan

    lib = capi.load()
    assert hasattr(lib, "qmc_debug_poke_table"), "not the checked build"
    OUT_ROW, JLIST = 3, 7
    res = {}

    def poke(plan, which, idx, val):
        torch.cuda.synchronize()
        old = C.c_int32()
        rc = lib.qmc_debug_poke_table(plan.handle, which, idx, val, C.byref(old))
        assert rc == 0, rc
        return old.value

    def fwd_case(name, w, which, idx, bad):
        plan = Plan.from_workload(w)
        A = torch.from_numpy(w.A).cuda()
        clean = plan.matmul(A).cpu().numpy()
        st0 = plan.sync_status()
        ref = products.matmul(oracle_pointset(w), w.A.astype(np.float64))
        old = poke(plan, which, idx, bad(plan))
        plan.matmul(A)
        st_bad = plan.sync_status()
        poke(plan, which, idx, old)
        again = plan.matmul(A).cpu().numpy()
        st1 = plan.sync_status()
        res[name] = {"clean": st0, "planted": st_bad, "restored": st1,
                     "err": colwise_rel_err(clean, ref), "same": bool(np.array_equal(clean, again))}

    # 256 x 256 transform (pipelined passes, two-panel un-permute)
    w = workloads.random_prime_case(65537, 100, 16, seed=3)
    fwd_case("prime65537_orow", w, OUT_ROW, 5, lambda p: p.out_rows + 1000)
    # s >= L/4: the dense first pass reads the j list
    w = workloads.random_prime_case(7681, 3000, 8, seed=4)
    fwd_case("prime7681_dense_jlist", w, JLIST, 10, lambda p: -5)
    # 768 x 1024 (P x Q first pass and two-panel un-permute)
    w = workloads.random_prime_case(786433, 40, 12, seed=5)
    fwd_case("prime786433_orow", w, OUT_ROW, 123457, lambda p: -2)
    # F_2, L = 255 x 257 (Rader-257 spectral pass, P x Q un-permute)
    w = workloads.f2_65536(s=64, grid=4)
    fwd_case("f2_65536_orow", w, OUT_ROW, 777, lambda p: 1 << 30)

    # adjoint: loads of G by the out-row table, stores of dA by the j list
    w = workloads.random_prime_case(65537, 100, 16, seed=6)
    plan = Plan.from_workload(w)
    G = torch.randn(plan.out_rows, 16, device="cuda")
    d_clean = plan.matmul_backward(G).cpu().numpy()
    st0 = plan.sync_status()
    sts = []
    for which, idx, bad in ((JLIST, 3, plan.s + 7), (OUT_ROW, 9, -1)):
        old = poke(plan, which, idx, bad)
        plan.matmul_backward(G)
        sts.append(plan.sync_status())
        poke(plan, which, idx, old)
    d_again = plan.matmul_backward(G).cpu().numpy()
    res["adjoint"] = {"clean": st0, "planted": sts, "restored": plan.sync_status(),
                      "same": bool(np.array_equal(d_clean, d_again))}

    # the point generator reads the out-row table
    old = poke(plan, OUT_ROW, 0, plan.out_rows)
    plan.generate_points()
    st_bad = plan.sync_status()
    poke(plan, OUT_ROW, 0, old)
    plan.generate_points()
    res["points"] = {"planted": st_bad, "restored": plan.sync_status()}
    print("RESULT " + json.dumps(res), flush=True)
""")


@pytest.fixture(scope="module")
def checked_lib():
    from paper_1501_06286_gb300 import build
    build.build()
    return build.build(checked=True)


def test_checked_build_catches_planted_indices(checked_lib):
    env = dict(os.environ, QMC_LIBRARY=checked_lib)
    r = subprocess.run([sys.executable, "-c", CHILD], cwd=ROOT, env=env, capture_output=True, text=True,
                       timeout=900)
    assert r.returncode == 0, r.stderr[-3000:]
    line = [ln for ln in r.stdout.splitlines() if ln.startswith("RESULT ")]
    assert line, r.stdout[-2000:]
    res = json.loads(line[0][len("RESULT "):])
    BOUNDS = 13
    for name in ("prime65537_orow", "prime7681_dense_jlist", "prime786433_orow", "f2_65536_orow"):
        c = res[name]
        assert c["clean"] == 0 and c["restored"] == 0, (name, c)
        assert c["planted"] == BOUNDS, (name, c)
        assert c["same"], name                 # restored: the same bits as before
        assert c["err"] <= 1e-5, (name, c)     # the checked build's product against the oracle
    adj = res["adjoint"]
    assert adj["clean"] == 0 and adj["restored"] == 0 and adj["same"], adj
    assert adj["planted"] == [BOUNDS, BOUNDS], adj
    assert res["points"] == {"planted": BOUNDS, "restored": 0}
