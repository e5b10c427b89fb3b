"""Query-sharded data parallelism of the fit over several GPUs (one process
per GPU, torch.distributed for the one exchange step).

The cull and the evaluation work per tile of queries (Section 3.2: a
candidate list per tile; Eq. 8: a sum per query), so a step's query set
splits into contiguous tile ranges, one per rank: every rank culls,
evaluates and back-propagates its own tiles with the unchanged kernels.
What couples the ranks is the gradient: each Gaussian's gradient is a sum
over all tiles, so the ranks' partial gradients are summed once per step,
and every rank then applies the same Adam update to its full copy of the
mixture.  The loss of a shard is normalised by the whole set's query count
(ndg_loss_l2_shard), so that the shards' losses and gradients add up to the
whole set's.

The sum is deterministic: every rank gathers all ranks' gradient buffers
and adds them in rank order, so the ranks stay bit-identical and a run is
reproducible (an all-reduce may associate the sum differently per rank).
The paper fits on one GPU; this partitioning is this library's.
"""
from __future__ import annotations

import torch


def tile_range(T: int, rank: int, world: int) -> tuple[int, int]:
    """Contiguous tiles [t0, t1) of `rank`: the T tiles in `world` runs whose
    lengths differ by at most one (the first T % world runs one longer)."""
    if not (0 <= rank < world):
        raise ValueError(f"rank {rank} outside a world of {world}")
    base, extra = divmod(T, world)
    t0 = rank * base + min(rank, extra)
    return t0, t0 + base + (1 if rank < extra else 0)


def query_range(Q: int, tile: int, rank: int, world: int) -> tuple[int, int]:
    """Queries [q0, q1) of `rank`: whole tiles of `tile` queries (the last
    tile of the set may be short)."""
    T = (Q + tile - 1) // tile
    t0, t1 = tile_range(T, rank, world)
    return min(Q, t0 * tile), min(Q, t1 * tile)


def sum_over_ranks_(tensors, group=None) -> None:
    """In place: every tensor becomes the sum over all ranks of that tensor,
    added in rank order (all_gather, then rank 0 + rank 1 + ...), so that the
    result is bit-identical on every rank and from run to run."""
    import torch.distributed as dist
    world = dist.get_world_size(group)
    if world == 1:
        return
    for t in tensors:
        if t is None:
            continue
        parts = [torch.empty_like(t) for _ in range(world)]
        dist.all_gather(parts, t.contiguous(), group=group)
        acc = parts[0].clone()
        for p in parts[1:]:
            acc.add_(p)
        t.copy_(acc)


def shard_trainer(mix, x_all: torch.Tensor, target_all: torch.Tensor, tile: int, cp, rank: int,
                  world: int, group=None, **trainer_kw):
    """A Trainer on this rank's tile range of the query set (x_all [Q][N],
    target_all [Q][3]): the shard's loss is normalised by the whole Q and its
    gradients are summed over the ranks before Adam."""
    from .train import Trainer
    Q = int(x_all.shape[0])
    q0, q1 = query_range(Q, tile, rank, world)
    tr = Trainer(mix, x_all[q0:q1].contiguous(), target_all[q0:q1].contiguous(), tile, cp,
                 loss_norm_queries=Q, **trainer_kw)
    # rows >= G are not gradients of anything: only the G rows in use travel
    tr.grad_hook = lambda tensors: sum_over_ranks_(
        [t[:tr.mix.G] for t in tensors if t is not None], group)
    return tr
