"""Batched products (graph and persistent modes) against the FP64 oracle,
and the bounded wait of the persistent mode (a dependency that never
completes ends in QMC_ERR_TIMEOUT, with the context still usable)."""

import numpy as np
import pytest
import torch

from oracle import products
from paper_1501_06286_gb300 import workloads
from paper_1501_06286_gb300.qmc import Batch, Plan

from _helpers import TOL, colwise_rel_err, oracle_pointset

pytestmark = pytest.mark.gpu

SMALL_PRIMES = (257, 7681, 12289, 40961, 65537)


@pytest.fixture(scope="module", autouse=True)
def _built():
    from paper_1501_06286_gb300 import build
    build.build()
    torch.cuda.set_device(0)


def _problems(count=12, seed=3):
    ws = workloads.batch_64(seed=seed, count=count, primes=SMALL_PRIMES, s_max=600, t_max=40)
    plans = [Plan.from_workload(w) for w in ws]
    As = [torch.from_numpy(w.A).cuda() for w in ws]
    outs = [torch.full((p.out_rows, w.t), float("nan"), device="cuda") for p, w in zip(plans, ws)]
    return ws, plans, As, outs


@pytest.mark.parametrize("mode", ["graph", "persistent"])
def test_batch_matches_oracle(mode):
    ws, plans, As, outs = _problems()
    batch = Batch(plans, [w.t for w in ws])
    batch.set_option("mode", mode)
    for _ in range(2):   # second call replays (graph) / relaunches (persistent)
        for o in outs:
            o.fill_(float("nan"))
        batch.matmul(As, outs)
        torch.cuda.synchronize()
        assert batch.sync_status() == 0
        for w, o in zip(ws, outs):
            ref = products.matmul(oracle_pointset(w), w.A.astype(np.float64))
            assert colwise_rel_err(o.cpu().numpy(), ref) <= TOL, w.name


def test_batch_graph_recaptures_on_new_pointers():
    ws, plans, As, outs = _problems(count=5, seed=7)
    batch = Batch(plans, [w.t for w in ws])
    batch.matmul(As, outs)
    outs2 = [torch.empty_like(o) for o in outs]
    batch.matmul(As, outs2)
    torch.cuda.synchronize()
    for o, o2 in zip(outs, outs2):
        assert torch.equal(o, o2)


def test_persistent_wait_times_out_and_context_survives():
    ws, plans, As, outs = _problems(count=6, seed=11)
    batch = Batch(plans, [w.t for w in ws])
    batch.set_option("mode", "persistent")
    batch.set_option("wait_limit_us", 200000)   # 0.2 s
    # pass-major items: the first len(multi-pass problems) items are first
    # passes; item index n_first is a second pass, which waits on a first pass
    n_first = len(ws)
    batch.set_option("test_block_item", n_first)
    batch.matmul(As, outs)
    torch.cuda.synchronize()
    assert batch.sync_status() == 9           # QMC_ERR_TIMEOUT
    batch.set_option("test_block_item", -1)
    batch.matmul(As, outs)
    torch.cuda.synchronize()
    assert batch.sync_status() == 0
    for w, o in zip(ws, outs):
        ref = products.matmul(oracle_pointset(w), w.A.astype(np.float64))
        assert colwise_rel_err(o.cpu().numpy(), ref) <= TOL
