"""Column sharding of B = Y·A over ranks (one process per GPU).

Every column of A is an independent matvec Y·a (Section 1), so ranks own
contiguous column blocks of A and B and the product needs no exchange.
Only the epilogues that reduce across columns combine over ranks:
  * per-row mean r_n = (1/t) Σ_k B_nk: each rank contributes
    (t_r / t) · (its block's row mean) — one sum-reduce of N floats;
  * exp-mean loss: each rank contributes its Σ exp(B_nk) — one scalar.
"""

from __future__ import annotations


def column_shard(t_total: int, world: int, rank: int) -> tuple[int, int]:
    """[start, stop) of rank's columns: contiguous, sizes differ by at most
    one, an even start for every rank when possible (columns pair into
    complex FFT columns)."""
    if world < 1 or not (0 <= rank < world):
        raise ValueError("bad rank/world")
    pairs = (t_total + 1) // 2
    base, extra = divmod(pairs, world)
    start_pair = rank * base + min(rank, extra)
    stop_pair = start_pair + base + (1 if rank < extra else 0)
    return min(2 * start_pair, t_total), min(2 * stop_pair, t_total)


def combine_row_means(local_mean, t_local: int, t_total: int, group=None):
    """Row mean over all columns from each rank's row mean of its block
    (in place on `local_mean`, a torch tensor)."""
    import torch.distributed as dist
    local_mean.mul_(t_local / t_total)
    dist.all_reduce(local_mean, op=dist.ReduceOp.SUM, group=group)
    return local_mean


def combine_exp_sums(local_sum, group=None):
    """Σ exp(B) over all ranks' columns (in place on a 1-element tensor)."""
    import torch.distributed as dist
    dist.all_reduce(local_sum, op=dist.ReduceOp.SUM, group=group)
    return local_sum
