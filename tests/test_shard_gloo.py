"""Query-sharded data parallelism (shard.py) on CPU: two gloo ranks on
127.0.0.1, no GPU.  Each rank takes its tile range of the query set; the
per-rank gradient is the oracle's gradient of that shard's loss normalised
by the whole set's query count (what ndg_loss_l2_shard gives the CUDA path);
the ordered sum over the ranks must equal the oracle's gradient of the whole
set (FP64, up to the summation order), be bit-identical on both ranks and
reproducible, and the shards' losses must add up to the whole set's."""
import os
import socket

import numpy as np
import pytest

from paper_2405_20067_gb300 import shard


def _free_port() -> int:
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def test_tile_ranges_partition_the_tiles():
    for T in (0, 1, 5, 64, 4097):
        for world in (1, 2, 3, 8):
            r = [shard.tile_range(T, k, world) for k in range(world)]
            assert r[0][0] == 0 and r[-1][1] == T
            assert all(a[1] == b[0] for a, b in zip(r, r[1:]))
            lens = [b - a for a, b in r]
            assert max(lens) - min(lens) <= 1
    # query ranges are whole tiles; the last tile of the set may be short
    Q, tile = 1000, 64
    qs = [shard.query_range(Q, tile, k, 3) for k in range(3)]
    assert qs[0][0] == 0 and qs[-1][1] == Q and all(a[1] == b[0] for a, b in zip(qs, qs[1:]))
    assert all(a % tile == 0 for a, _ in qs)
    with pytest.raises(ValueError):
        shard.tile_range(10, 2, 2)


N, G, Q, TILE, K, CUTOFF, B = 4, 60, 3000, 64, 8, 1.0 / 255.0, 32
NAMES = ["mean", "theta", "alpha_raw", "color_raw", "u_theta", "m_u", "c_alpha_raw",
         "c_color_raw"]


def _problem():
    from paper_2405_20067_gb300 import synth
    mix = synth.mixture(N, G, 1201)
    ch = synth.children(N, G, 1202, spread=0.2)
    x = synth.queries_box(N, Q, 1203).astype(np.float64)
    target = synth.targets_uniform(Q, 1204).astype(np.float64)
    proj = synth.projections(N, K, 1205)
    return mix, ch, x, target, proj


def _shard_grad(oracle, rank, world):
    """(loss share, gradient arrays) of this rank's shard, the loss
    normalised by the whole set's Q."""
    mix, ch, x, target, proj = _problem()
    raw = oracle.Raw.from_arrays([mix[n] for n in NAMES[:4]] + [ch[n] for n in NAMES[4:]], True)
    L, m, w = oracle.activate(raw)
    T = (Q + TILE - 1) // TILE
    t0, t1 = shard.tile_range(T, rank, world)
    q0, q1 = shard.query_range(Q, TILE, rank, world)
    # the shard's lists: the contract of the whole set restricted to its tiles
    offs, ids = oracle.cull_contract(L, m, w, x, TILE, proj, CUTOFF, 3.0, B,
                                     tiles=np.arange(t0, t1))
    y = oracle.eval(L, m, w, x[q0:q1], TILE, offs, ids)
    loss_r, gbar = oracle.loss_l2(y, target[q0:q1])
    scale = (q1 - q0) / Q  # the oracle normalises by the shard's own count
    g = oracle.grad(raw, x[q0:q1], TILE, offs, ids, gbar * scale)
    return loss_r * scale, {n: np.array(getattr(g, n)) for n in NAMES}


def _rank_main(rank, world, port, q):
    import torch
    import torch.distributed as dist
    import oracle
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank),
                      WORLD_SIZE=str(world))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    loss_r, g = _shard_grad(oracle, rank, world)
    tensors = [torch.as_tensor(g[n]) for n in NAMES] + [torch.tensor([loss_r], dtype=torch.float64)]
    again = [t.clone() for t in tensors]
    shard.sum_over_ranks_(tensors)
    shard.sum_over_ranks_(again)
    assert all(torch.equal(a, b) for a, b in zip(tensors, again)), "not reproducible"
    dist.barrier()
    dist.destroy_process_group()
    q.put((rank, [t.numpy() for t in tensors]))


def test_sharded_gradient_equals_whole_set_gradient(oracle):
    import torch.multiprocessing as mp
    world = 2
    ctx = mp.get_context("spawn")
    qu = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_rank_main, args=(r, world, port, qu)) for r in range(world)]
    for p in procs:
        p.start()
    out = dict(qu.get(timeout=300) for _ in procs)
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    # bit-identical on both ranks
    for a, b in zip(out[0], out[1]):
        assert np.array_equal(a, b)
    # the whole set on one rank
    loss_all, g_all = _shard_grad(oracle, 0, 1)
    summed = dict(zip(NAMES, out[0][:-1]))
    for n in NAMES:
        want = g_all[n]
        err = np.linalg.norm(summed[n] - want) / np.linalg.norm(want)
        assert err <= 1e-12, (n, err)
    assert abs(out[0][-1][0] - loss_all) <= 1e-12 * loss_all
