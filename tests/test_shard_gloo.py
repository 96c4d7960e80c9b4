"""Column sharding over ranks, on CPU with the gloo backend (world size 2):
each rank computes its column block with the FP64 oracle, and the gathered
blocks, the combined row mean and the combined exp-sum equal the unsharded
oracle results."""

import os
import socket

import numpy as np
import pytest
import torch
import torch.distributed as dist
import torch.multiprocessing as mp

from oracle import points, products
from paper_1501_06286_gb300 import workloads
from paper_1501_06286_gb300.shard import column_shard, combine_exp_sums, combine_row_means


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _worker(rank, world, port, result_dir):
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    w = workloads.random_prime_case(257, 40, 11, seed=5, dtype=np.float64)
    ps = points.PointSet("prime", w.N, w.gen, w.map, w.row0)
    c0, c1 = column_shard(w.t, world, rank)
    B_local = products.matmul(ps, w.A[:, c0:c1])
    # gather the column blocks
    blocks = [None] * world
    dist.all_gather_object(blocks, (c0, c1, B_local))
    # row mean and exp-sum combined over ranks
    rm = torch.from_numpy(products.row_mean(B_local) if c1 > c0 else np.zeros(ps.out_rows))
    combine_row_means(rm, c1 - c0, w.t)
    es = torch.tensor([np.exp(B_local).sum()])
    combine_exp_sums(es)
    if rank == 0:
        B = np.zeros((ps.out_rows, w.t))
        for a, b, blk in blocks:
            B[:, a:b] = blk
        np.save(os.path.join(result_dir, "B.npy"), B)
        np.save(os.path.join(result_dir, "rm.npy"), rm.numpy())
        np.save(os.path.join(result_dir, "es.npy"), es.numpy())
    dist.barrier()
    dist.destroy_process_group()


def test_column_shard_covers_columns():
    for t in (1, 2, 7, 4225, 4096):
        for world in (1, 2, 3, 8):
            spans = [column_shard(t, world, r) for r in range(world)]
            assert spans[0][0] == 0 and spans[-1][1] == t
            for (a0, b0), (a1, b1) in zip(spans, spans[1:]):
                assert b0 == a1
            assert all(a % 2 == 0 for a, b in spans if b > a)


def test_sharded_product_matches_unsharded(tmp_path):
    port = _free_port()
    mp.spawn(_worker, args=(2, port, str(tmp_path)), nprocs=2, join=True)
    w = workloads.random_prime_case(257, 40, 11, seed=5, dtype=np.float64)
    ps = points.PointSet("prime", w.N, w.gen, w.map, w.row0)
    B = products.matmul(ps, w.A)
    assert np.allclose(np.load(tmp_path / "B.npy"), B, rtol=0, atol=1e-13)
    assert np.allclose(np.load(tmp_path / "rm.npy"), products.row_mean(B), rtol=0, atol=1e-13)
    assert abs(np.load(tmp_path / "es.npy")[0] - np.exp(B).sum()) <= 1e-10 * np.exp(B).sum()
