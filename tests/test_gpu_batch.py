"""Batched products (graph and persistent modes) against the FP64 oracle,
and the bounded wait of the persistent mode (a dependency that never
completes ends in QMC_ERR_TIMEOUT, with the context still usable).  The
persistent queue runs specialised tile loops for some pass shapes (every
pass of the 768 x 1024 transform, the sparse first pass, the register tile
of length 256) and the generic tile for the rest; the mixed-shape test
reaches each of them."""

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


def _sampled_rows(n_out, seed, k=48):
    rows = np.random.default_rng(seed).integers(0, n_out, k)
    return np.unique(np.concatenate([rows, [0, n_out - 1]]))


def test_persistent_queue_mixed_shapes_match_oracle():
    ws = [
        # N = 786433 (L = 768 x 1024), s <= 1024 and 8+ complex columns: the
        # sparse first pass (row packing, spectral pass from the packed rows)
        workloads.random_prime_case(786433, 600, 40, seed=21),
        # s > 1024, odd t: term-by-term lines (pairs and singles) and
        # gathered lines, spectral pass, un-permute pass; two panels, ragged
        workloads.random_prime_case(786433, 3000, 17, seed=22),
        # five complex columns: one 8-column panel, mostly empty
        workloads.random_prime_case(786433, 200, 9, seed=23),
        # two complex columns: narrower panels, the generic tile
        workloads.random_prime_case(786433, 300, 3, seed=24),
        # L = 256 x 256 and L = 160 x 256: register tiles of length 256 next
        # to generic tiles of length 160
        workloads.random_prime_case(65537, 500, 33, seed=25),
        workloads.random_prime_case(40961, 150, 12, seed=26),
        # L = 256 in one pass
        workloads.random_prime_case(257, 100, 20, seed=27),
        workloads.random_prime_case(257, 40, 1, seed=28),
    ]
    plans = [Plan.from_workload(w) for w in ws]
    As = [torch.from_numpy(w.A).cuda() for w in ws]
    outs = [torch.full((p.out_rows, w.t), float("nan"), device="cuda") for p, w in zip(plans, ws)]
    batch = Batch(plans, [w.t for w in ws])
    batch.set_option("mode", "persistent")
    for _ in range(2):   # the second call reuses the uploaded queue description
        for o in outs:
            o.fill_(float("nan"))
        batch.matmul(As, outs)
        torch.cuda.synchronize()
        assert batch.sync_status() == 0
        for i, (w, p, o) in enumerate(zip(ws, plans, outs)):
            if p.out_rows > 70000:
                rows = _sampled_rows(p.out_rows, seed=100 + i)
                ref = products.matmul_rows(oracle_pointset(w), w.A.astype(np.float64), rows)
                got = o[torch.from_numpy(rows).cuda()].cpu().numpy()
            else:
                ref = products.matmul(oracle_pointset(w), w.A.astype(np.float64))
                got = o.cpu().numpy()
            assert np.isfinite(got).all(), w.name
            assert colwise_rel_err(got, ref) <= TOL, w.name
