"""Parity at the full workload sizes, in the launch configuration bench.py
times (tiles of 256 queries, 16 projections, cutoff 1/255, k_sigma 3, 64
buckets; the lifted tensor-core form with the plain FP32 form beside it).

The oracle cannot evaluate these workloads whole in seconds, so each check
samples what the oracle can compute one by one:

* config 1 (N = 6 fit step: 100,000 parents + 100,000 children at brightness
  t/10, below the cutoff but evaluated within 3 sigma, 2^20 Morton-tiled
  queries): the candidate lists of all 4,096 tiles
  bit-exact; the outputs of 48 sampled tiles; the gradients of 64 sampled
  parents.  With dy fixed, a Gaussian's gradient involves only its own
  pairs, so the oracle differentiates the mixture restricted to the sampled
  Gaussians (their own candidate entries, renumbered), exactly their rows
  of the full gradient.  Central differences (h = 1e-3) of the oracle's
  restricted functional sum(dy * y) pin 12 of those parameters as well.
* config 2 (N = 10, 500,000 Gaussians, 2^22 queries on 256 planes): the
  lists of 6 sampled tiles bit-exact (the oracle runs the contract for those
  tiles only) and their outputs.
* config 3 (N = 10 fit: 50,000 parents with children evaluated within 3
  sigma, 2^18-query minibatch, targets from a 2M-Gaussian ground truth):
  gradients of 48 sampled parents (FP32 and tensor-core backward), graph
  replays equal eager steps, the loss decreases.
* config 4 (batched render specs): three of the 64 frames (the largest, the
  smallest, one N = 8), outputs of sampled tiles including the ragged edges.
"""
import numpy as np
import pytest

from helpers import NAMES, assert_grads_close, assert_outputs_close, oracle_raw
from paper_2405_20067_gb300 import synth

pytestmark = pytest.mark.gpu

TILE, K, CUTOFF, KS, B = 256, 16, 1.0 / 255.0, 3.0, 64
KMIN = 3.0  # children's radius floor (Section 3.3, reading R7), as bench.py


@pytest.fixture(scope="module")
def ndg():
    import torch
    from paper_2405_20067_gb300 import build, ndg as _ndg
    build.build()
    assert torch.cuda.is_available(), "GPU tests need a GPU"
    return _ndg


# ---------------------------------------------------------------- helpers

def gpu_lists_ascending(ev, E):
    """(offsets, ids) of the device lists with ids ascending inside each tile
    (the fill pass emits a tile's list in bucket-run order), on the device."""
    import torch
    offs = ev.cull.offsets[:ev.T + 1]
    ids = ev.cull.ids[:E].to(torch.int64)
    tile = torch.repeat_interleave(torch.arange(ev.T, device=ids.device), offs[1:] - offs[:-1])
    key, _ = torch.sort((tile << 32) | ids)
    return offs, (key & 0xFFFFFFFF).to(torch.int32)


def gpu_tile_lists(ev, tiles):
    """Ascending device lists of the given tiles only (for lists too large to
    sort whole)."""
    offs = ev.cull.offsets.cpu().numpy()
    return [np.sort(ev.cull.ids[int(offs[t]):int(offs[t + 1])].cpu().numpy()) for t in tiles]


def tile_subset(offs, ids, tiles):
    """Lists of the given tiles, concatenated (offsets renumbered)."""
    lens = offs[tiles + 1] - offs[tiles]
    o = np.concatenate([[0], np.cumsum(lens)]).astype(np.int64)
    i = np.concatenate([ids[offs[t]:offs[t + 1]] for t in tiles]).astype(np.int32)
    return o, i


def queries_of(x, tiles, Q):
    rows = np.concatenate([np.arange(t * TILE, min((t + 1) * TILE, Q)) for t in tiles])
    return rows, x[rows]


def restrict(offs, ids, sel_e, Ge):
    """Lists restricted to the evaluated Gaussians sel_e (ascending),
    renumbered 0 .. len(sel_e) - 1; ascending order is kept."""
    mp = np.full(Ge, -1, dtype=np.int64)
    mp[sel_e] = np.arange(sel_e.size)
    sub = mp[ids]
    keep = sub >= 0
    c = np.concatenate([[0], np.cumsum(keep)]).astype(np.int64)
    return c[offs], sub[keep].astype(np.int32)


def raw_rows(mix, ch, S):
    par = {k: np.asarray(mix[k])[S] for k in NAMES[:4]}
    chd = None if ch is None else {k: np.asarray(ch[k])[S] for k in NAMES[4:]}
    return par, chd


def sampled_tiles(rng, T, n, extra=()):
    t = np.sort(rng.choice(T, size=min(n, T), replace=False))
    return np.unique(np.concatenate([t, np.asarray(extra, dtype=np.int64)])).astype(np.int64)


# ---------------------------------------------------------------- config 1

@pytest.fixture(scope="module")
def cfg1(ndg, oracle):
    """The bench's fit workload (same recipe and seeds as bench.py)."""
    import torch
    N, G, Q = 6, 100_000, 1 << 20
    c = synth.config1(G=G, Q=Q)
    ch = synth.children(N, G, 11, spread=0.05, brightness=(0.0009, 0.0011))
    gm = ndg.Mixture.from_arrays(N, c["mix"], ch, G_cap=G + G // 10)
    x = torch.as_tensor(c["x"]).cuda()
    cp = ndg.CullParams(K, torch.as_tensor(c["proj"]).cuda(), CUTOFF, KS, B, child_k_min=KMIN)
    ev = ndg.Evaluator(gm, x, TILE, cp)
    E = ev.build(gm)
    raw = oracle_raw(oracle, c["mix"], ch)
    L, m, w = oracle.activate(raw)
    xd = c["x"].astype(np.float64)
    o_offs, o_ids = oracle.cull_contract(L, m, w, xd, TILE, c["proj"], CUTOFF, KS, B,
                                         n_parents=G, child_k_min=KMIN)
    return dict(N=N, G=G, Q=Q, c=c, ch=ch, gm=gm, x=x, xd=xd, ev=ev, E=E, L=L, m=m, w=w,
                o_offs=o_offs, o_ids=o_ids)


def test_config1_lists_bit_exact_full(cfg1):
    import torch
    E, ev = cfg1["E"], cfg1["ev"]
    assert E == int(cfg1["o_offs"][-1])
    offs, ids = gpu_lists_ascending(ev, E)
    assert np.array_equal(offs.cpu().numpy(), cfg1["o_offs"])
    assert torch.equal(ids, torch.as_tensor(cfg1["o_ids"]).cuda())
    print(f"config 1: E = {E} entries in {ev.T} tiles, identical")


@pytest.mark.parametrize("mode", ["tc", "fp32"])
def test_config1_outputs_sampled_tiles(ndg, oracle, cfg1, mode):
    d = cfg1
    ev = d["ev"]
    md = ndg.NDG_MODE_TC if mode == "tc" else ndg.NDG_MODE_FP32
    y = ev.forward(d["gm"], mode=md).cpu().numpy()
    tiles = sampled_tiles(synth.rng(71), ev.T, 48, extra=[0, ev.T - 1])
    so, si = tile_subset(d["o_offs"], d["o_ids"], tiles)
    rows, xs = queries_of(d["xd"], tiles, d["Q"])
    want = oracle.eval(d["L"], d["m"], d["w"], xs, TILE, so, si)
    kw = dict(rtol=1e-3, floor=1e-3) if mode == "tc" else {}
    worst = assert_outputs_close(y[rows], want, what=f"config 1 {mode} forward", **kw)
    print(f"config 1 {mode}: {tiles.size} tiles, worst relative error {worst:.2e}")


@pytest.mark.parametrize("mode", ["tc", "fp32"])
def test_config1_gradients_sampled_gaussians(ndg, oracle, cfg1, mode):
    import torch
    d = cfg1
    N, G, Q, ev = d["N"], d["G"], d["Q"], d["ev"]
    dy = (synth.rng(73).standard_normal((Q, 3)) / (3 * Q)).astype(np.float32)
    md = ndg.NDG_MODE_TC if mode == "tc" else ndg.NDG_MODE_FP32
    grad = ev.backward(d["gm"], torch.as_tensor(dy).cuda(), mode=md)
    S = np.sort(synth.rng(74).choice(G, size=64, replace=False))
    par, chd = raw_rows(d["c"]["mix"], d["ch"], S)
    raw_s = oracle_raw(oracle, par, chd)
    sel_e = np.concatenate([S, G + S])
    so, si = restrict(d["o_offs"], d["o_ids"], sel_e, 2 * G)
    assert si.size > 0
    want = oracle.grad(raw_s, d["xd"], TILE, so, si, dy.astype(np.float64))
    got = {n: getattr(grad, n)[torch.as_tensor(S).cuda()].cpu().numpy() for n in NAMES}
    rep = assert_grads_close(got, want, NAMES, rtol=1e-3 if mode == "tc" else 1e-4)
    print(f"config 1 {mode} gradients, 64 parents ({si.size} entries): "
          + " ".join(f"{n}={v:.1e}" for n, v in rep.items()))
    if mode != "fp32":
        return
    # central differences of the oracle's restricted functional sum(dy * y)
    dyd = dy.astype(np.float64)

    def f(r):
        Lr, mr, wr = oracle.activate(r)
        return float(np.sum(dyd * oracle.eval(Lr, mr, wr, d["xd"], TILE, so, si)))

    pick = synth.rng(75)
    h = 1e-3
    for name in ("mean", "theta", "alpha_raw", "color_raw"):
        for _ in range(3):
            arr = getattr(raw_s, name)
            idx = tuple(int(pick.integers(0, s)) for s in arr.shape)
            plus, minus = [oracle_raw(oracle, par, chd) for _ in range(2)]
            getattr(plus, name)[idx] += h
            getattr(minus, name)[idx] -= h
            fd = (f(plus) - f(minus)) / (2 * h)
            an = float(getattr(want, name)[idx])
            gg = float(got[name][idx])
            scale = max(abs(fd), 1e-3 * float(np.abs(getattr(want, name)).max()), 1e-30)
            assert abs(an - fd) <= 1e-3 * scale, (name, idx, an, fd)
            assert abs(gg - fd) <= 2e-3 * scale, (name, idx, gg, fd)


# ---------------------------------------------------------------- config 2

def test_config2_sampled_tiles(ndg, oracle):
    """N = 10 surface workload at full size: candidate lists of sampled tiles
    bit-exact, tensor-core and FP32 outputs of those tiles."""
    import torch
    c = synth.config2()
    N, Q = c["N"], c["x"].shape[0]
    gm = ndg.Mixture.from_arrays(N, c["mix"])
    x = torch.as_tensor(c["x"]).cuda()
    cp = ndg.CullParams(K, torch.as_tensor(c["proj"]).cuda(), CUTOFF, KS, B)
    T = (Q + TILE - 1) // TILE
    ev = ndg.Evaluator(gm, x, TILE, cp, E_cap=T * gm.Ge + 1024, backward=False)
    E = ev.build(gm)
    tiles = sampled_tiles(synth.rng(81), T, 5, extra=[T - 1])
    raw = oracle_raw(oracle, c["mix"])
    L, m, w = oracle.activate(raw)
    xd = c["x"].astype(np.float64)
    so, si = oracle.cull_contract(L, m, w, xd, TILE, c["proj"], CUTOFF, KS, B, tiles=tiles)
    for i, (t, got) in enumerate(zip(tiles, gpu_tile_lists(ev, tiles))):
        assert np.array_equal(got, si[so[i]:so[i + 1]]), f"tile {t}"
    rows, xs = queries_of(xd, tiles, Q)
    want = oracle.eval(L, m, w, xs, TILE, so, si)
    for mode, md, kw in (("tc", ndg.NDG_MODE_TC, dict(rtol=1e-3, floor=1e-3)),
                         ("fp32", ndg.NDG_MODE_FP32, {})):
        y = ev.forward(gm, mode=md).cpu().numpy()
        worst = assert_outputs_close(y[rows], want, what=f"config 2 {mode} forward", **kw)
        print(f"config 2 {mode}: E = {E}, {tiles.size} tiles ({int(so[-1])} entries), "
              f"worst relative error {worst:.2e}")
    assert ndg.read_status(ev.ws) == 0


# ---------------------------------------------------------------- config 3

def test_config3_fit_full_size(ndg, oracle):
    """N = 10 fit at full size: targets from the 2M-Gaussian ground truth
    (tensor-core forward); gradients of sampled parents against the oracle
    (FP32 backward at 1e-4, the tensor-core beta form at 1e-3); CUDA-graph
    replays equal eager steps (tensor-core forward and backward); the loss
    decreases."""
    import torch
    from paper_2405_20067_gb300.train import Trainer
    c = synth.config3()
    N, G = c["N"], c["mix"]["mean"].shape[0]
    x = torch.as_tensor(c["x"]).cuda()
    Q = x.shape[0]
    cp = ndg.CullParams(K, torch.as_tensor(c["proj"]).cuda(), CUTOFF, KS, B, child_k_min=KMIN)
    gt = ndg.Mixture.from_arrays(N, c["gt"])
    ev_gt = ndg.Evaluator(gt, x, TILE, cp, backward=False)
    ev_gt.build(gt)
    target = ev_gt.forward(gt, mode=ndg.NDG_MODE_TC).clone()
    assert ndg.read_status(ev_gt.ws) == 0
    del ev_gt, gt
    torch.cuda.empty_cache()

    # gradients of 48 sampled parents for a fixed dy
    gm = ndg.Mixture.from_arrays(N, c["mix"], c["children"], G_cap=c["G_max"])
    ev = ndg.Evaluator(gm, x, TILE, cp)
    E = ev.build(gm)
    dy = (synth.rng(91).standard_normal((Q, 3)) / (3 * Q)).astype(np.float32)
    grad = ev.backward(gm, torch.as_tensor(dy).cuda(), mode=ndg.NDG_MODE_FP32)
    grad_tc = ev.backward(gm, torch.as_tensor(dy).cuda(), mode=ndg.NDG_MODE_TC)
    assert ndg.read_status(ev.ws) == 0
    offs, ids = gpu_lists_ascending(ev, E)
    S = np.sort(synth.rng(92).choice(G, size=48, replace=False))
    raw = oracle_raw(oracle, c["mix"], c["children"])
    L, m, w = oracle.activate(raw)
    xd = c["x"].astype(np.float64)
    T = ev.T
    o_offs, o_ids = oracle.cull_contract(L, m, w, xd, TILE, c["proj"], CUTOFF, KS, B,
                                         n_parents=G, child_k_min=KMIN)
    assert np.array_equal(offs.cpu().numpy(), o_offs)
    assert torch.equal(ids, torch.as_tensor(o_ids).cuda())
    par, chd = raw_rows(c["mix"], c["children"], S)
    so, si = restrict(o_offs, o_ids, np.concatenate([S, G + S]), 2 * G)
    want = oracle.grad(oracle_raw(oracle, par, chd), xd, TILE, so, si, dy.astype(np.float64))
    got = {n: getattr(grad, n)[torch.as_tensor(S).cuda()].cpu().numpy() for n in NAMES}
    rep = assert_grads_close(got, want, NAMES, rtol=1e-4)
    got_tc = {n: getattr(grad_tc, n)[torch.as_tensor(S).cuda()].cpu().numpy() for n in NAMES}
    rep_tc = assert_grads_close(got_tc, want, NAMES, rtol=1e-3)
    print(f"config 3: E = {E} in {T} tiles; 48 parents: fp32 "
          + " ".join(f"{n}={v:.1e}" for n, v in rep.items()) + " | tc "
          + " ".join(f"{n}={v:.1e}" for n, v in rep_tc.items()))
    del ev, grad, grad_tc
    torch.cuda.empty_cache()

    # graph replays against eager steps, then the loss over 30 replays
    def trainer():
        mix = ndg.Mixture.from_arrays(N, c["mix"], c["children"], G_cap=c["G_max"])
        return Trainer(mix, x, target, TILE, cp, lr=1e-3, t=c["t"], phase=300,
                       mode=ndg.NDG_MODE_TC, bwd_mode=ndg.NDG_MODE_TC)

    eager, graphed = trainer(), trainer()
    # the capture's two warm-up steps are steps too: match them eagerly
    for _ in range(2):
        eager.step(refine=False)
        eager.refine(sync=False)
    graphed.capture(refine_each_step=True)
    for _ in range(3):
        eager.step(refine=False)
        eager.refine(sync=False)
        graphed.replay()
    torch.cuda.synchronize()
    assert eager.check() == ndg.NDG_OK and graphed.check() == ndg.NDG_OK
    assert torch.equal(eager.loss, graphed.loss)
    for f in NAMES:
        pa, pb = getattr(eager.mix, f), getattr(graphed.mix, f)
        assert torch.equal(pa.detach(), pb.detach()), f
    first = float(graphed.loss.item())
    for _ in range(30):
        graphed.replay()
    torch.cuda.synchronize()
    last = float(graphed.loss.item())
    assert graphed.check() == ndg.NDG_OK
    assert last < first, (first, last)
    print(f"config 3: loss {first:.4e} -> {last:.4e} over 30 replays")


# ---------------------------------------------------------------- config 4

@pytest.mark.parametrize("which", ["largest", "smallest", "n8"])
def test_config4_frames_sampled_tiles(ndg, oracle, which):
    import torch
    frames = synth.config4_frames()
    if which == "largest":
        f = max(frames, key=lambda s: s["W"] * s["H"] * s["G"])
    elif which == "smallest":
        f = min(frames, key=lambda s: s["W"] * s["H"] * s["G"])
    else:
        f = next(s for s in frames if s["N"] == 8)
    N, G, W, H, sd = f["N"], f["G"], f["W"], f["H"], f["seed"]
    mix = synth.mixture(N, G, sd)
    xn = synth.queries_frame(N, W, H, sd + 1)
    proj = synth.projections(N, K, sd + 2)
    Q = xn.shape[0]
    T = (Q + TILE - 1) // TILE
    gm = ndg.Mixture.from_arrays(N, mix)
    cp = ndg.CullParams(K, torch.as_tensor(proj).cuda(), CUTOFF, KS, B)
    ev = ndg.Evaluator(gm, torch.as_tensor(xn).cuda(), TILE, cp, backward=False)
    E = ev.build(gm)
    y = ev.forward(gm, mode=ndg.NDG_MODE_TC).cpu().numpy()
    # tiles are runs of 256 consecutive queries in 16 x 16 pixel-tile order;
    # the last one is ragged when W H is not a multiple of 256
    tiles = sampled_tiles(synth.rng(sd + 7), T, 6, extra=[0, T - 1])
    raw = oracle_raw(oracle, mix)
    L, m, w = oracle.activate(raw)
    xd = xn.astype(np.float64)
    so, si = oracle.cull_contract(L, m, w, xd, TILE, proj, CUTOFF, KS, B, tiles=tiles)
    for i, (t, got) in enumerate(zip(tiles, gpu_tile_lists(ev, tiles))):
        assert np.array_equal(got, si[so[i]:so[i + 1]]), f"tile {t}"
    rows, xs = queries_of(xd, tiles, Q)
    want = oracle.eval(L, m, w, xs, TILE, so, si)
    worst = assert_outputs_close(y[rows], want, rtol=1e-3, floor=1e-3,
                                 what=f"frame {W}x{H} N={N} G={G}")
    print(f"config 4 {which}: N={N} G={G} {W}x{H}, E = {E}, worst relative error {worst:.2e}")
