"""The transform's factorisation as a plan option (QMC_OPT_FFT_SPLIT) and
the batch autotuner that searches it: every split gives the oracle's
product; invalid splits are rejected and leave the plan as it was; the
tuner's choices are cached per problem shape and, with QMC_AUTOTUNE_CACHE,
written to and read back from a file by a later process."""

import os
import subprocess
import sys
import textwrap

import numpy as np
import pytest
import torch

from oracle import products
from paper_1501_06286_gb300 import capi, workloads
from paper_1501_06286_gb300.qmc import Plan

from _helpers import TOL, colwise_rel_err, oracle_pointset

pytestmark = pytest.mark.gpu

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module", autouse=True)
def _built():
    from paper_1501_06286_gb300 import build
    build.build()
    torch.cuda.set_device(0)


@pytest.mark.parametrize("N,splits", [(65537, [256, 128, 64]), (7681, [80, 64, 60, 48]),
                                      (12289, [96, 64, 48]), (40961, [160, 128, 80])])
def test_every_split_gives_the_product(N, splits):
    w = workloads.random_prime_case(N, 150, 19, seed=N, map="centred")
    plan = Plan.from_workload(w)
    assert plan.info["L1"] == splits[0]          # the default split comes first
    A = torch.from_numpy(w.A).cuda()
    ref = products.matmul(oracle_pointset(w), w.A.astype(np.float64))
    for L1 in splits + [0]:
        plan.set_fft_split(L1)
        want = splits[0] if L1 == 0 else L1
        assert (plan.info["L1"], plan.info["L2"]) == (want, plan.L // want)
        B = plan.matmul(A)
        torch.cuda.synchronize()
        assert plan.sync_status() == 0
        assert colwise_rel_err(B.cpu().numpy(), ref) <= TOL, L1


def test_invalid_splits_keep_the_plan():
    w = workloads.random_prime_case(65537, 40, 6, seed=1)
    plan = Plan.from_workload(w)
    A = torch.from_numpy(w.A).cuda()
    B0 = plan.matmul(A).clone()
    for L1, code in [(3, 1), (32, 1), (65536, 1), (1, 1)]:   # no divisor / a factor above 1024
        with pytest.raises(capi.QmcError) as e:
            plan.set_fft_split(L1)
        assert e.value.code == code
    assert (plan.info["L1"], plan.info["L2"]) == (256, 256)
    assert torch.equal(plan.matmul(A), B0)
    ps = Plan("pset", 257, None, map="centred", s=5)
    with pytest.raises(capi.QmcError) as e:
        ps.set_fft_split(16)
    assert e.value.code == 6


_CHILD = textwrap.dedent("""
    import ctypes as C, sys, torch
    sys.path.insert(0, {root!r})
    from paper_1501_06286_gb300 import capi, workloads
    from paper_1501_06286_gb300.qmc import Batch, Plan
    ws = workloads.batch_64(seed=11, count=6, primes=(7681, 12289, 65537), s_max=300, t_max=24)
    plans = [Plan.from_workload(w) for w in ws]
    As = [torch.from_numpy(w.A).cuda() for w in ws]
    outs = [torch.empty((p.out_rows, w.t), device="cuda") for p, w in zip(plans, ws)]
    Batch(plans, [w.t for w in ws]).matmul(As, outs)
    torch.cuda.synchronize()
    out = []
    for p in plans:
        info = capi.QmcInfo()
        capi.load().qmc_plan_info(p.handle, C.byref(info))
        out.append(f"{{info.L}}:{{info.L1}}")
    print("SPLITS", " ".join(out))
""")


def test_autotune_cache_file_round_trip(tmp_path):
    cache = tmp_path / "tune.txt"
    env = dict(os.environ, QMC_AUTOTUNE_CACHE=str(cache))
    code = _CHILD.format(root=ROOT)
    r1 = subprocess.run([sys.executable, "-c", code], env=env, capture_output=True, text=True, timeout=600)
    assert r1.returncode == 0, r1.stderr
    lines = cache.read_text().splitlines()
    assert lines, "no cache entries written"
    chosen = {}
    for ln in lines:
        f = ln.split()
        assert len(f) == 9
        kind, L, sb, tb, arch, L1, kern, first = (int(v) for v in f[:8])
        assert kind == 0 and L % L1 == 0 and arch >= 100 and float(f[8]) > 0
        chosen.setdefault(L, set()).add(L1)
    # a second process reads the file: the same splits, nothing appended
    r2 = subprocess.run([sys.executable, "-c", code], env=env, capture_output=True, text=True, timeout=600)
    assert r2.returncode == 0, r2.stderr
    assert len(cache.read_text().splitlines()) == len(lines)
    s1 = [l for l in r1.stdout.splitlines() if l.startswith("SPLITS")]
    s2 = [l for l in r2.stdout.splitlines() if l.startswith("SPLITS")]
    assert s1 and s1 == s2
    for item in s1[0].split()[1:]:
        L, L1 = (int(v) for v in item.split(":"))
        assert L1 in chosen[L]
