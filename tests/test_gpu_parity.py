"""Parity of the CUDA path (through the C ABI) with the FP64 oracle on the
same seeded inputs: candidate lists bit-exact, outputs within 1e-5 relative,
gradients within 1e-4 (tolerances in helpers.py)."""
import math

import numpy as np
import pytest

from helpers import (NAMES, assert_grads_close, assert_outputs_close, csr_sets, oracle_raw)
from paper_2405_20067_gb300 import synth

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def ndg():
    import torch
    from paper_2405_20067_gb300 import build, ndg as _ndg
    build.build()
    assert torch.cuda.is_available(), "GPU tests need a GPU"
    return _ndg


def make_case(N, G, Q, seed, children=False, queries="box"):
    mix = synth.mixture(N, G, seed)
    ch = synth.children(N, G, seed + 1, spread=0.2) if children else None
    if queries == "box":
        x = synth.queries_box(N, Q, seed + 2)
    else:
        x = queries
    return mix, ch, x


def gpu_setup(ndg, N, mix, ch, x, tile, k, cutoff, k_sigma, B, seed, E_cap=None, G_cap=None):
    import torch
    gm = ndg.Mixture.from_arrays(N, mix, ch, G_cap=G_cap)
    xt = torch.as_tensor(x).cuda()
    proj = synth.projections(N, k, seed + 3) if k > 0 else np.zeros((0, N), np.float32)
    cp = ndg.CullParams(k, torch.as_tensor(proj).cuda() if k > 0 else None, cutoff, k_sigma, B)
    ev = ndg.Evaluator(gm, xt, tile, cp, E_cap=E_cap)
    E = ev.build(gm)
    return gm, xt, proj, cp, ev, E


CULL_CASES = [
    # N, G, Q, tile, k, cutoff, k_sigma, B, children
    (6, 2000, 20000, 256, 16, 1 / 255, 3.0, 64, False),
    (6, 1500, 9000, 100, 8, 0.0, 3.0, 200, True),
    (10, 1200, 12288, 256, 16, 1 / 255, 3.0, 128, False),
    (3, 500, 5000, 64, 1, 0.0, 2.0, 32, False),
    (2, 300, 3000, 17, 32, 1 / 255, 3.0, 255, True),
    (6, 800, 4096, 256, 4, 0.0, 3.0, 1, False),
    (12, 400, 2000, 256, 24, 1 / 255, 3.0, 16, False),
]


@pytest.mark.parametrize("N,G,Q,tile,k,cutoff,k_sigma,B,children", CULL_CASES)
def test_cull_lists_bit_exact_and_forward(ndg, oracle, N, G, Q, tile, k, cutoff, k_sigma, B,
                                          children):
    seed = 100 + N + k
    mix, ch, x = make_case(N, G, Q, seed, children)
    gm, xt, proj, cp, ev, E = gpu_setup(ndg, N, mix, ch, x, tile, k, cutoff, k_sigma, B, seed)
    raw = oracle_raw(oracle, mix, ch)
    L, m, w = oracle.activate(raw)
    offs, ids = oracle.cull_contract(L, m, w, x.astype(np.float64), tile, proj, cutoff, k_sigma, B)
    assert E == offs[-1], (E, offs[-1])
    g_off = ev.cull.offsets.cpu().numpy()
    g_ids = ev.cull.ids[:E].cpu().numpy()
    assert np.array_equal(g_off, offs)
    for t, (a, b) in enumerate(zip(csr_sets(g_off, g_ids), csr_sets(offs, ids))):
        assert np.array_equal(a, b), f"tile {t}: {len(a)} vs {len(b)} candidates"
    assert 0 < E
    if k > 0 and B > 1:
        assert E < len(offs[:-1]) * L.shape[0], "nothing culled"
    y = ev.forward(gm).cpu().numpy()
    yo = oracle.eval(L, m, w, x.astype(np.float64), tile, offs, ids)
    assert_outputs_close(y, yo)
    assert ndg.read_status(ev.ws) == 0


TC_CASES = [
    # N, G, Q, tile, k, cutoff, B, children
    (6, 2000, 20000, 256, 16, 1 / 255, 64, False),
    (6, 900, 7000, 100, 8, 0.0, 64, True),
    (10, 1200, 12288, 256, 16, 1 / 255, 128, False),
    (10, 300, 3000, 17, 4, 0.0, 32, True),
    (3, 500, 5000, 64, 2, 0.0, 32, False),
    (1, 200, 2000, 256, 1, 1 / 255, 64, False),
    (12, 400, 2000, 256, 24, 1 / 255, 16, False),
    (8, 800, 6000, 256, 16, 1 / 255, 64, True),
    (5, 500, 4000, 200, 8, 0.0, 32, False),
]


@pytest.mark.parametrize("N,G,Q,tile,k,cutoff,B,children", TC_CASES)
def test_tc_forward_matches_oracle(ndg, oracle, N, G, Q, tile, k, cutoff, B, children):
    """Lifted tensor-core form: within 1e-3 relative of the FP64 oracle on
    outputs above 1e-3 (|a - b| / max(|b|, 1e-3) <= 1e-3)."""
    seed = 500 + N + k
    mix, ch, x = make_case(N, G, Q, seed, children)
    gm, xt, proj, cp, ev, E = gpu_setup(ndg, N, mix, ch, x, tile, k, cutoff, 3.0, B, seed)
    y = ev.forward(gm, mode=ndg.NDG_MODE_TC).cpu().numpy()
    raw = oracle_raw(oracle, mix, ch)
    L, m, w = oracle.activate(raw)
    offs, ids = oracle.cull_contract(L, m, w, x.astype(np.float64), tile, proj, cutoff, 3.0, B)
    assert E == offs[-1]
    yo = oracle.eval(L, m, w, x.astype(np.float64), tile, offs, ids)
    worst = assert_outputs_close(y, yo, rtol=1e-3, floor=1e-3, what="tensor-core forward")
    print(f"tc forward N={N} tile={tile}: worst relative error {worst:.2e}")
    print(f"N={N} tile={tile}: worst relative error {worst:.2e}")
    assert ndg.read_status(ev.ws) == 0


def test_dense_forward_config0(ndg, oracle):
    """N = 6, 1000 Gaussians, 16384 queries, no culling (k = 0)."""
    c = synth.config0()
    N = c["N"]
    gm, xt, proj, cp, ev, E = gpu_setup(ndg, N, c["mix"], None, c["x"], 256, 0, 0.0, 3.0, 1, 0)
    assert E == 64 * 1000
    y = ev.forward(gm).cpu().numpy()
    raw = oracle_raw(oracle, c["mix"])
    L, m, w = oracle.activate(raw)
    yo = oracle.eval(L, m, w, c["x"].astype(np.float64))
    assert_outputs_close(y, yo)


GRAD_CASES = [
    # N, G, Q, tile, k, cutoff, children, mode
    (6, 1000, 16384, 256, 0, 0.0, False, "fp32"),
    (6, 600, 8192, 256, 16, 1 / 255, True, "fp32"),
    (10, 400, 6000, 128, 16, 1 / 255, True, "fp32"),
    (3, 200, 3000, 33, 8, 0.0, True, "fp32"),
    (6, 1000, 16384, 256, 0, 0.0, False, "tc"),
    (6, 600, 8192, 256, 16, 1 / 255, True, "tc"),
    (5, 400, 6000, 200, 16, 1 / 255, True, "tc"),
    (3, 200, 3000, 33, 8, 0.0, True, "tc"),
    (1, 100, 1000, 256, 1, 0.0, False, "tc"),
    # the beta form of the tensor-core backward (N > 6)
    (7, 300, 4000, 100, 8, 0.0, True, "tc"),
    (8, 500, 6000, 256, 16, 1 / 255, True, "tc"),
    (9, 300, 4000, 200, 8, 1 / 255, False, "tc"),
    (10, 400, 6000, 128, 16, 1 / 255, True, "tc"),
    (11, 200, 3000, 64, 8, 0.0, True, "tc"),
    (12, 200, 3000, 256, 16, 1 / 255, False, "tc"),
]


@pytest.mark.parametrize("N,G,Q,tile,k,cutoff,children,mode", GRAD_CASES)
def test_backward_matches_oracle(ndg, oracle, N, G, Q, tile, k, cutoff, children, mode):
    """FP32 form: 1e-4 relative per tensor; lifted tensor-core form: 1e-3."""
    import torch
    seed = 300 + N + k
    mix, ch, x = make_case(N, G, Q, seed, children)
    gm, xt, proj, cp, ev, E = gpu_setup(ndg, N, mix, ch, x, tile, k, cutoff, 3.0, 64, seed)
    dy = (synth.rng(seed + 9).standard_normal((Q, 3)) / (3 * Q)).astype(np.float32)
    md = ndg.NDG_MODE_TC if mode == "tc" else ndg.NDG_MODE_FP32
    grad = ev.backward(gm, torch.as_tensor(dy).cuda(), mode=md)
    raw = oracle_raw(oracle, mix, ch)
    offs = ev.cull.offsets.cpu().numpy()
    ids_sorted = np.concatenate(csr_sets(offs, ev.cull.ids[:E].cpu().numpy())).astype(np.int32)
    # the oracle's own lists, identical as sets (checked above)
    L, m, w = oracle.activate(raw)
    o_offs, o_ids = (oracle.cull_contract(L, m, w, x.astype(np.float64), tile, proj, cutoff, 3.0, 64)
                     if k > 0 else (None, None))
    if k > 0:
        assert np.array_equal(o_ids, ids_sorted)
    want = oracle.grad(raw, x.astype(np.float64), tile, o_offs, o_ids, dy.astype(np.float64))
    names = NAMES if children else NAMES[:4]
    got = {n: getattr(grad, n)[:G].cpu().numpy() for n in names}
    rep = assert_grads_close(got, want, names, rtol=1e-3 if mode == "tc" else 1e-4)
    print(f"{mode} N={N}: " + " ".join(f"{n}={v:.1e}" for n, v in rep.items()))
    # determinism: a second backward is bit-identical
    grad2 = ev.backward(gm, torch.as_tensor(dy).cuda(), mode=md)
    for n in names:
        assert torch.equal(getattr(grad, n), getattr(grad2, n)), n


def test_loss_matches_oracle(ndg, oracle):
    import torch
    r = synth.rng(5)
    Q = 70001
    y = r.uniform(0, 2, (Q, 3)).astype(np.float32)
    t = r.uniform(0, 2, (Q, 3)).astype(np.float32)
    yt, tt = torch.as_tensor(y).cuda(), torch.as_tensor(t).cuda()
    dy = torch.empty_like(yt)
    loss = torch.zeros(1, dtype=torch.float64, device="cuda")
    ws = ndg.workspace(1 << 16)
    ndg.loss_l2(yt, tt, dy, loss, ws)
    lo, go = oracle.loss_l2(y.astype(np.float64), t.astype(np.float64))
    assert abs(loss.item() - lo) <= 1e-12 * lo
    assert_outputs_close(dy.cpu().numpy(), go, rtol=1e-6, floor=1e-12)


def test_shard_loss_matches_oracle(ndg, oracle):
    """ndg_loss_l2_shard: a shard of Q outputs normalised by the whole set's
    Q_total: its loss is the oracle's loss of the shard times Q / Q_total, dy
    likewise; two shards add up to the whole set's loss."""
    import torch
    r = synth.rng(8)
    Q_total, Q = 90001, 40000
    y = r.uniform(0, 2, (Q_total, 3)).astype(np.float32)
    t = r.uniform(0, 2, (Q_total, 3)).astype(np.float32)
    ws = ndg.workspace(1 << 16)
    parts = []
    for q0, q1 in ((0, Q), (Q, Q_total)):
        yt, tt = torch.as_tensor(y[q0:q1]).cuda(), torch.as_tensor(t[q0:q1]).cuda()
        dy = torch.empty_like(yt)
        loss = torch.zeros(1, dtype=torch.float64, device="cuda")
        ndg.loss_l2_shard(yt, tt, dy, loss, ws, Q_total)
        lo, go = oracle.loss_l2(y[q0:q1].astype(np.float64), t[q0:q1].astype(np.float64))
        f = (q1 - q0) / Q_total
        assert abs(loss.item() - lo * f) <= 1e-12 * lo * f
        assert_outputs_close(dy.cpu().numpy(), go * f, rtol=1e-6, floor=1e-12)
        parts.append(loss.item())
    whole, _ = oracle.loss_l2(y.astype(np.float64), t.astype(np.float64))
    assert abs(sum(parts) - whole) <= 1e-12 * whole
    with pytest.raises(ndg.NDGError):  # Q_total below the shard's Q
        ndg.loss_l2_shard(torch.zeros(10, 3, device="cuda"), torch.zeros(10, 3, device="cuda"),
                          torch.zeros(10, 3, device="cuda"),
                          torch.zeros(1, dtype=torch.float64, device="cuda"), ws, 9)


def test_relative_loss_matches_oracle(ndg, oracle):
    """Relative L2 (Section 4.1 reading): loss to 1e-12, dy to 1e-6, with
    outputs near zero (where the eps term dominates) included."""
    import torch
    r = synth.rng(6)
    Q = 50003
    y = r.uniform(0, 2, (Q, 3)).astype(np.float32)
    y[:100] *= 1e-3
    t = r.uniform(0, 2, (Q, 3)).astype(np.float32)
    yt, tt = torch.as_tensor(y).cuda(), torch.as_tensor(t).cuda()
    dy = torch.empty_like(yt)
    loss = torch.zeros(1, dtype=torch.float64, device="cuda")
    ws = ndg.workspace(1 << 16)
    for eps in (1e-2, 0.5):
        ndg.loss_rel_l2(yt, tt, dy, loss, ws, eps=eps)
        lo, go = oracle.loss_rel_l2(y.astype(np.float64), t.astype(np.float64),
                                    eps=float(np.float32(eps)))
        assert abs(loss.item() - lo) <= 1e-12 * lo
        assert_outputs_close(dy.cpu().numpy(), go, rtol=1e-6, floor=1e-12)


def test_fit_with_relative_loss_reduces_it(ndg):
    """The trainer's relative-L2 option drives the same graph-capturable step."""
    import torch
    from paper_2405_20067_gb300.train import Trainer
    N, G, Q = 6, 400, 8192
    mix = synth.mixture(N, G, 90)
    gm = ndg.Mixture.from_arrays(N, mix, G_cap=2 * G)
    x = torch.as_tensor(synth.queries_box(N, Q, 91)).cuda()
    target = torch.as_tensor(synth.targets_uniform(Q, 92)).cuda()
    cp = ndg.CullParams(8, torch.as_tensor(synth.projections(N, 8, 93)).cuda(), 1 / 255, 3.0, 64)
    tr = Trainer(gm, x, target, 256, cp, lr=1e-2, t=0.01, phase=0, loss="rel_l2")
    first = float(tr.step(refine=False).item())
    for _ in range(40):
        tr.step(refine=False)
    last = float(tr.loss.item())
    assert tr.check() == ndg.NDG_OK
    assert last < 0.9 * first, (first, last)


def test_adam_matches_oracle(ndg, oracle):
    import torch
    N, G = 6, 500
    mix = synth.mixture(N, G, 7)
    ch = synth.children(N, G, 8)
    p = ndg.Mixture.from_arrays(N, mix, ch, G_cap=G + 10)
    r = synth.rng(9)
    grads = {n: r.standard_normal(getattr(p, n).shape).astype(np.float32) for n in NAMES}
    g = p.zeros_like()
    for n in NAMES:
        getattr(g, n).copy_(torch.as_tensor(grads[n]))
    m1, m2 = p.zeros_like(), p.zeros_like()
    step = torch.zeros(1, dtype=torch.int32, device="cuda")
    before = {n: getattr(p, n).cpu().numpy().astype(np.float64) for n in NAMES}
    for it in range(3):
        ndg.adam(p, g, m1, m2, step, 1e-2)
    assert step.item() == 3
    for n in NAMES:
        pw = before[n][:G].ravel()
        om1 = np.zeros_like(pw)
        om2 = np.zeros_like(pw)
        for it in range(3):
            pw, om1, om2 = oracle.adam(pw, grads[n][:G].ravel().astype(np.float64), om1, om2,
                                       it + 1, 1e-2)
        got = getattr(p, n)[:G].cpu().numpy().ravel()
        np.testing.assert_allclose(got, pw, rtol=1e-5, atol=1e-6, err_msg=n)
        # rows beyond G untouched
        assert np.array_equal(getattr(p, n)[G:].cpu().numpy(), before[n][G:].astype(np.float32))


@pytest.mark.parametrize("first", [True, False])
def test_densify_matches_oracle(ndg, oracle, first):
    import torch
    N, G, cap = 6, 300, 340
    mix = synth.mixture(N, G, 21)
    ch = None if first else synth.children(N, G, 22, spread=0.1, brightness=(0.001, 0.03))
    gm = ndg.Mixture.from_arrays(N, mix, ch, G_cap=cap)
    m1, m2 = gm.zeros_like(), gm.zeros_like()
    for mm in (m1, m2):
        for n in NAMES:
            getattr(mm, n).fill_(7.0)
    noise = synth.noise(cap, N, 23)
    ws = ndg.workspace(ndg.workspace_size(gm, None, 1, None, 0))
    G_new = torch.zeros(1, dtype=torch.int32, device="cuda")
    t = 0.01
    ndg.densify(gm, t, torch.as_tensor(noise).cuda(), m1, m2, G_new, ws)
    raw = oracle_raw(oracle, mix, ch)
    a_thr = float(np.float32(math.log(t)))
    new, Gn, flag = oracle.densify(raw, cap, a_thr, math.log(t / 10), noise.astype(np.float64))
    assert gm.G == Gn
    if first:
        assert Gn == G
    else:
        assert Gn == cap, "capacity-limited case expected"
    for n in NAMES:
        got = getattr(gm, n)[:Gn].cpu().numpy().astype(np.float64)
        want = getattr(new, n)[:Gn]
        np.testing.assert_allclose(got, want, rtol=2e-6, atol=2e-6, err_msg=n)
    # moments of touched rows zeroed, others kept
    fresh = np.zeros(cap, bool)
    fresh[:Gn] = True if first else False
    if not first:
        fresh[np.nonzero(flag)[0]] = True
        fresh[G:Gn] = True
    c1 = m1.u_theta.cpu().numpy()
    assert np.all(c1[fresh] == 0) and np.all(c1[~fresh] == 7.0)
    p1 = m1.mean.cpu().numpy()
    assert np.all(p1[G:Gn] == 0) and np.all(p1[:G] == 7.0)


def test_capacity_overflow_reports_and_truncates(ndg, oracle):
    import torch
    N, G, Q, tile = 6, 500, 4096, 256
    mix, ch, x = make_case(N, G, Q, 41)
    gm = ndg.Mixture.from_arrays(N, mix)
    xt = torch.as_tensor(x).cuda()
    proj = torch.as_tensor(synth.projections(N, 8, 42)).cuda()
    cp = ndg.CullParams(8, proj, 1 / 255, 3.0, 64)
    cull = ndg.Cull(16, 100)
    ws = ndg.workspace(ndg.workspace_size(gm, xt, tile, cp, 100))
    ndg.build_cull(gm, xt, tile, cp, cull, ws)
    E = cull.E()
    assert E > 100
    assert ndg.read_status(ws) == ndg.NDG_ERR_CAPACITY
    assert ndg.read_status(ws) == 0  # reading clears
    offs = cull.offsets.cpu().numpy()
    assert offs.max() <= 100 and np.all(np.diff(offs) >= 0)


def test_empty_inputs(ndg):
    import torch
    N = 6
    mix = synth.mixture(N, 10, 3)
    gm = ndg.Mixture.from_arrays(N, mix)
    proj = torch.as_tensor(synth.projections(N, 4, 1)).cuda()
    cp = ndg.CullParams(4, proj, 1 / 255, 3.0, 64)
    # no queries
    x0 = torch.zeros(0, N, device="cuda")
    ev = ndg.Evaluator(gm, x0, 256, cp, E_cap=16)
    assert ev.build(gm) == 0
    assert ev.forward(gm).shape == (0, 3)
    # no Gaussians
    g0 = ndg.Mixture.from_arrays(N, {k: v[:0] for k, v in mix.items()}, G_cap=4)
    x = torch.as_tensor(synth.queries_box(N, 300, 2)).cuda()
    ev = ndg.Evaluator(g0, x, 256, cp, E_cap=16)
    assert ev.build(g0) == 0
    y = ev.forward(g0)
    assert torch.count_nonzero(y) == 0
    grad = ev.backward(g0, torch.ones(300, 3, device="cuda"))
    assert ndg.read_status(ev.ws) == 0


def test_value_at_mean_exact(ndg):
    """Eq. 1: a query at a Gaussian's mean with nothing else nearby returns w
    to FP32 rounding (s = 0 exactly, exp2(0) = 1)."""
    import torch
    N = 6
    mix = synth.mixture(N, 1, 4)
    gm = ndg.Mixture.from_arrays(N, mix)
    x = torch.as_tensor(mix["mean"]).cuda()
    cp = ndg.CullParams(0, None, 0.0, 3.0, 1)
    ev = ndg.Evaluator(gm, x, 1, cp, E_cap=4)
    ev.build(gm)
    y = ev.forward(gm).cpu().numpy()[0]
    a = np.float64(mix["alpha_raw"][0])
    c = 1.0 / (1.0 + np.exp(-mix["color_raw"][0].astype(np.float64)))
    np.testing.assert_allclose(y, np.exp(a) * c, rtol=1e-6)


def test_auto_forward_picks_form_per_tile(ndg, oracle):
    """NDG_MODE_AUTO: tiles with at least NDG_AUTO_MIN_CANDIDATES(N) candidates
    get the tensor-core form, the others the FP32 form; each tile's outputs
    equal that form's bit for bit, and all are within the tensor-core
    tolerance of the oracle.  The Gaussians crowd one corner of the box so
    that the tiles' candidate counts span both sides of the threshold."""
    N, G, Q, tile, k = 6, 4000, 30000, 256, 16
    seed = 640
    mix, _, x = make_case(N, G, Q, seed)
    mix = dict(mix)
    mix["mean"] = (0.2 * (mix["mean"] + 1.0) - 1.0).astype(np.float32)  # means in [-1, -0.6]^6
    gm, xt, proj, cp, ev, E = gpu_setup(ndg, N, mix, None, x, tile, k, 1 / 255, 3.0, 64, seed)
    counts = np.diff(ev.cull.offsets.cpu().numpy())
    dense = counts >= ndg.auto_min_candidates(N)
    assert dense.any() and (~dense).any(), (counts.min(), counts.max())
    y_tc = ev.forward(gm, mode=ndg.NDG_MODE_TC).cpu().numpy()
    y_fp = ev.forward(gm, mode=ndg.NDG_MODE_FP32).cpu().numpy()
    y_au = ev.forward(gm, mode=ndg.NDG_MODE_AUTO).cpu().numpy()
    rows_dense = np.repeat(dense, tile)[:Q]
    assert np.array_equal(y_au[rows_dense], y_tc[rows_dense])
    assert np.array_equal(y_au[~rows_dense], y_fp[~rows_dense])
    raw = oracle_raw(oracle, mix)
    L, m, w = oracle.activate(raw)
    offs, ids = oracle.cull_contract(L, m, w, x.astype(np.float64), tile, proj, 1 / 255, 3.0, 64)
    yo = oracle.eval(L, m, w, x.astype(np.float64), tile, offs, ids)
    worst = assert_outputs_close(y_au, yo, rtol=1e-3, floor=1e-3, what="auto forward")
    print(f"auto: {int(dense.sum())} of {dense.size} tiles on the tensor cores, worst {worst:.2e}")
    assert ndg.read_status(ev.ws) == 0


@pytest.mark.parametrize("N,G,Q,tile,k,children", [(6, 3000, 20000, 256, 16, False),
                                                   (10, 2000, 9000, 128, 8, True),
                                                   (4, 500, 3000, 64, 4, False)])
def test_conditioned_cull_bit_exact_and_forward(ndg, oracle, N, G, Q, tile, k, children):
    """Section 3.2 with the inputs beyond position constant: the lists of
    ndg_build_cull_conditioned equal the oracle's conditioned contract (same
    sets per tile, bit-exact), are shorter than the unconditioned ones, and
    the forward over them matches the oracle in both forms."""
    import torch
    seed = 700 + N
    mix, ch, _ = make_case(N, G, 16, seed, children)
    r = synth.rng(seed + 5)
    xc = r.uniform(-0.5, 0.5, size=N - 3).astype(np.float32)
    xp = synth.queries_box(3, Q, seed + 6)
    x = np.concatenate([xp, np.repeat(xc[None, :], Q, axis=0)], axis=1).astype(np.float32)
    gm, xt, proj, cp, ev, E_full = gpu_setup(ndg, N, mix, ch, x, tile, k, 1 / 255, 3.0, 64, seed)
    E = ev.build(gm, xc=torch.as_tensor(xc).cuda())
    assert E < E_full
    raw = oracle_raw(oracle, mix, ch)
    L, m, w = oracle.activate(raw)
    xd = x.astype(np.float64)
    offs, ids = oracle.cull_contract(L, m, w, xd, tile, proj, 1 / 255, 3.0, 64,
                                     xc=xc.astype(np.float64))
    assert E == offs[-1]
    got = csr_sets(ev.cull.offsets.cpu().numpy(), ev.cull.ids[:E].cpu().numpy())
    want = csr_sets(offs, ids)
    assert all(np.array_equal(a, b) for a, b in zip(got, want))
    yo = oracle.eval(L, m, w, xd, tile, offs, ids)
    assert_outputs_close(ev.forward(gm, mode=ndg.NDG_MODE_FP32).cpu().numpy(), yo)
    assert_outputs_close(ev.forward(gm, mode=ndg.NDG_MODE_TC).cpu().numpy(), yo, rtol=1e-3,
                         floor=1e-3)
    print(f"conditioned N={N}: E = {E} (unconditioned {E_full})")
    assert ndg.read_status(ev.ws) == 0


def test_config0_l2_loss_and_gradient(ndg, oracle):
    """Config 0 as specified: N = 6, 1000 Gaussians, 16384 queries, no
    culling, the plain L2 loss against a 200-Gaussian ground truth (its
    values from the oracle), seed 0: loss and every raw-parameter gradient
    of the FP32 path against the oracle."""
    import torch
    c = synth.config0()
    N = c["N"]
    x = c["x"].astype(np.float64)
    Lg, mg, wg = oracle.activate(oracle_raw(oracle, c["gt"]))
    target = oracle.eval(Lg, mg, wg, x).astype(np.float32)
    gm, xt, proj, cp, ev, E = gpu_setup(ndg, N, c["mix"], None, c["x"], 256, 0, 0.0, 3.0, 1, 0)
    y = ev.forward(gm)
    dy = torch.empty_like(y)
    loss = torch.zeros(1, dtype=torch.float64, device="cuda")
    ndg.loss_l2(y, torch.as_tensor(target).cuda(), dy, loss, ev.ws)
    grad = ev.backward(gm, dy)
    raw = oracle_raw(oracle, c["mix"])
    L, m, w = oracle.activate(raw)
    yo = oracle.eval(L, m, w, x)
    lo, go = oracle.loss_l2(yo, target.astype(np.float64))
    assert abs(loss.item() - lo) <= 1e-5 * lo
    want = oracle.grad(raw, x, 256, None, None, go)
    got = {n: getattr(grad, n)[:1000].cpu().numpy() for n in NAMES[:4]}
    rep = assert_grads_close(got, want, NAMES[:4])
    print("config 0: loss %.6e; " % loss.item() + " ".join(f"{n}={v:.1e}" for n, v in rep.items()))


@pytest.mark.parametrize("mode", ["fp32", "tc"])
def test_backward_above_32768_tiles_matches_oracle(ndg, oracle, mode):
    """More than 32768 tiles: the backward orders the entries Gaussian-major by
    a radix sort of the ids (the counting sort covers up to 32768 tiles).
    Tiles of 16 queries over 540,000 queries (33,750 tiles); gradients
    against the oracle (FP32 form 1e-4, tensor-core form 1e-3 per tensor) and
    a second backward bit-identical."""
    import torch
    N, G, Q, tile, k = 6, 1000, 540_000, 16, 16
    seed = 910
    mix, ch, x = make_case(N, G, Q, seed, children=True)
    gm, xt, proj, cp, ev, E = gpu_setup(ndg, N, mix, ch, x, tile, k, 1 / 255, 3.0, 64, seed)
    assert ev.T > 32768
    dy = (synth.rng(seed + 9).standard_normal((Q, 3)) / (3 * Q)).astype(np.float32)
    md = ndg.NDG_MODE_TC if mode == "tc" else ndg.NDG_MODE_FP32
    dyt = torch.as_tensor(dy).cuda()
    grad = ev.backward(gm, dyt, mode=md)
    assert ndg.read_status(ev.ws) == 0
    raw = oracle_raw(oracle, mix, ch)
    L, m, w = oracle.activate(raw)
    o_offs, o_ids = oracle.cull_contract(L, m, w, x.astype(np.float64), tile, proj, 1 / 255, 3.0, 64)
    assert E == o_offs[-1]
    want = oracle.grad(raw, x.astype(np.float64), tile, o_offs, o_ids, dy.astype(np.float64))
    got = {n: getattr(grad, n)[:G].cpu().numpy() for n in NAMES}
    rep = assert_grads_close(got, want, NAMES, rtol=1e-3 if mode == "tc" else 1e-4)
    print(f"{mode} T={ev.T} E={E}: " + " ".join(f"{n}={v:.1e}" for n, v in rep.items()))
    grad2 = ev.backward(gm, dyt, mode=md)
    for n in NAMES:
        assert torch.equal(getattr(grad, n), getattr(grad2, n)), n
    # the radix-sorted order computed ahead (ndg_backward_order), then used
    ndg.backward_order(gm, xt, tile, ev.cull, ev.ws)
    grad3 = ev.backward(gm, dyt, mode=md | ndg.NDG_BWD_ORDER_READY)
    assert ndg.read_status(ev.ws) == 0
    for n in NAMES:
        assert torch.equal(getattr(grad, n), getattr(grad3, n)), n


@pytest.mark.parametrize("N,mode", [(6, "tc"), (6, "fp32"), (10, "tc")])
def test_backward_order_ahead_on_a_side_stream(ndg, N, mode):
    """ndg_backward_order on a second stream while the forward runs, then
    ndg_backward with NDG_BWD_ORDER_READY: gradients bit-identical to the
    backward that orders the entries itself."""
    import torch
    G, Q, tile, k = 800, 8192, 256, 16
    seed = 930 + N
    mix, ch, x = make_case(N, G, Q, seed, children=True)
    gm, xt, proj, cp, ev, E = gpu_setup(ndg, N, mix, ch, x, tile, k, 1 / 255, 3.0, 64, seed)
    md = ndg.NDG_MODE_TC if mode == "tc" else ndg.NDG_MODE_FP32
    dyt = torch.as_tensor((synth.rng(seed + 1).standard_normal((Q, 3)) / (3 * Q))
                          .astype(np.float32)).cuda()
    want = ev.backward(gm, dyt, mode=md)
    torch.cuda.synchronize()
    side = torch.cuda.Stream()
    side.wait_stream(torch.cuda.current_stream())
    ndg.backward_order(gm, xt, tile, ev.cull, ev.ws, stream=side)
    ev.forward(gm, mode=md)  # on the current stream, beside the order
    torch.cuda.current_stream().wait_stream(side)
    got = ev.backward(gm, dyt, mode=md | ndg.NDG_BWD_ORDER_READY)
    torch.cuda.synchronize()
    assert ndg.read_status(ev.ws) == 0
    for n in NAMES:
        assert torch.equal(getattr(want, n), getattr(got, n)), n


@pytest.mark.parametrize("N", [6, 10])
def test_records_prepared_by_the_cull_are_reused_exactly(ndg, N):
    """NDG_RECORDS_READY: after ndg_build_cull the evaluation (every form)
    and the tensor-core backward skip their own preparation and give the
    same outputs and gradients, bit for bit."""
    import torch
    G, Q, tile, k = 900, 8192, 256, 16
    seed = 950 + N
    mix, ch, x = make_case(N, G, Q, seed, children=True)
    gm, xt, proj, cp, ev, E = gpu_setup(ndg, N, mix, ch, x, tile, k, 1 / 255, 3.0, 64, seed)
    dyt = torch.as_tensor((synth.rng(seed + 1).standard_normal((Q, 3)) / (3 * Q))
                          .astype(np.float32)).cuda()
    for md in (ndg.NDG_MODE_TC, ndg.NDG_MODE_FP32, ndg.NDG_MODE_AUTO):
        want = ev.forward(gm, mode=md).clone()
        ev.build(gm)  # leaves the records
        got = ev.forward(gm, mode=md | ndg.NDG_RECORDS_READY)
        assert torch.equal(want, got), md
    want = ev.backward(gm, dyt, mode=ndg.NDG_MODE_TC)
    ev.build(gm)
    tr = ndg.Trace()
    got = ndg.Mixture.zeros_like(gm)
    ndg.backward(gm, xt, tile, ev.cull, dyt, got, ev.ws,
                 mode=ndg.NDG_MODE_TC | ndg.NDG_RECORDS_READY, trace=tr)
    torch.cuda.synchronize()
    assert ndg.read_status(ev.ws) == ndg.NDG_OK
    for n in NAMES:
        assert torch.equal(getattr(want, n), getattr(got, n)), n


def test_backward_with_a_stale_order_stays_inside_its_buffers(ndg):
    """NDG_BWD_ORDER_READY with an order left from other lists (a caller
    error): the segmented sum clamps segment bounds and checks entry indices
    against the capacity, so the call completes, reads nothing outside the
    workspace and may report NDG_ERR_INVALID_ARG; the next backward that
    orders the entries itself is correct again."""
    import torch
    N, G, Q, tile, k = 6, 800, 8192, 256, 16
    seed = 940
    mix, ch, x = make_case(N, G, Q, seed, children=True)
    gm, xt, proj, cp, ev, E = gpu_setup(ndg, N, mix, ch, x, tile, k, 1 / 255, 3.0, 64, seed)
    dyt = torch.as_tensor((synth.rng(seed + 1).standard_normal((Q, 3)) / (3 * Q))
                          .astype(np.float32)).cuda()
    want = ev.backward(gm, dyt, mode=ndg.NDG_MODE_TC)
    ndg.backward_order(gm, xt, tile, ev.cull, ev.ws)
    # other lists in the same buffers: queries shifted, so the tiles' candidates change
    x0 = xt.clone()
    xt.add_(0.25)
    E2 = ev.build(gm)
    assert E2 <= ev.E_cap
    ev.backward(gm, dyt, mode=ndg.NDG_MODE_TC | ndg.NDG_BWD_ORDER_READY)
    torch.cuda.synchronize()
    assert ndg.read_status(ev.ws) in (ndg.NDG_OK, ndg.NDG_ERR_INVALID_ARG)
    xt.copy_(x0)
    assert ev.build(gm) == E
    again = ev.backward(gm, dyt, mode=ndg.NDG_MODE_TC)
    torch.cuda.synchronize()
    assert ndg.read_status(ev.ws) == ndg.NDG_OK
    for n in NAMES:
        assert torch.equal(getattr(want, n), getattr(again, n)), n


def test_non_finite_parameter_sets_numeric_status(ndg):
    """A raw parameter whose activation is not finite (NaN, or +inf
    brightness; planted on the host) makes the preparation report
    NDG_ERR_NUMERIC in the workspace status word; nothing faults, and the
    next call with finite parameters reports NDG_OK."""
    import torch
    N, G, Q, tile, k = 6, 500, 4096, 256, 8
    seed = 920
    mix, ch, x = make_case(N, G, Q, seed, children=True)
    gm, xt, proj, cp, ev, E = gpu_setup(ndg, N, mix, ch, x, tile, k, 1 / 255, 3.0, 64, seed)
    assert ndg.read_status(ev.ws) == 0
    for field, value in (("theta", float("nan")), ("alpha_raw", float("inf")),
                         ("m_u", float("nan")), ("c_color_raw", float("nan"))):
        t = getattr(gm, field)
        keep = t.clone()
        t.view(-1)[7] = value
        ev.forward(gm, mode=ndg.NDG_MODE_TC)
        assert ndg.read_status(ev.ws) == ndg.NDG_ERR_NUMERIC, field
        assert ndg.read_status(ev.ws) == 0  # reading clears the word
        ndg.build_cull(gm, xt, tile, cp, ev.cull, ev.ws)
        assert ndg.read_status(ev.ws) == ndg.NDG_ERR_NUMERIC, field
        t.copy_(keep)
        ev.build(gm)
        ev.forward(gm, mode=ndg.NDG_MODE_TC)
        ev.backward(gm, torch.ones(Q, 3, device="cuda") / Q, mode=ndg.NDG_MODE_TC)
        assert ndg.read_status(ev.ws) == 0, field
    # a raw colour of -inf activates to the finite colour 0: not an error
    gm.c_color_raw.view(-1)[7] = float("-inf")
    ev.forward(gm, mode=ndg.NDG_MODE_TC)
    assert ndg.read_status(ev.ws) == 0


@pytest.mark.parametrize("N,tile,conditioned", [(6, 256, False), (10, 128, False), (6, 256, True)])
def test_children_below_cutoff_keep_radius_floor(ndg, oracle, N, tile, conditioned):
    """Section 3.3 with a contribution cutoff (reading R7): children start at
    brightness t/10 = 1e-3, below the 1/255 cutoff, and keep a radius of 3
    sigma (child_k_min) so that they are evaluated where they span their
    parents.  Lists bit-exact against the oracle's contract with the same
    floor, children present in them (absent without the floor), forward
    within tolerance in both forms."""
    import torch
    G, Q, k = 800, 12000, 16
    seed = 950 + N + int(conditioned)
    mix = synth.mixture(N, G, seed)
    ch = synth.children(N, G, seed + 1, spread=0.05, brightness=(0.0009, 0.0011))
    xc = None
    if conditioned:
        xc_np = synth.rng(seed + 4).uniform(-0.5, 0.5, size=N - 3).astype(np.float32)
        xp = synth.queries_box(3, Q, seed + 2)
        x = np.concatenate([xp, np.repeat(xc_np[None, :], Q, axis=0)], axis=1).astype(np.float32)
        xc = torch.as_tensor(xc_np).cuda()
    else:
        x = synth.queries_box(N, Q, seed + 2)
    gm = ndg.Mixture.from_arrays(N, mix, ch)
    xt = torch.as_tensor(x).cuda()
    proj = synth.projections(N, k, seed + 3)
    raw = oracle_raw(oracle, mix, ch)
    L, m, w = oracle.activate(raw)
    xd = x.astype(np.float64)
    sets = {}
    for floor in (0.0, 3.0):
        cp = ndg.CullParams(k, torch.as_tensor(proj).cuda(), 1 / 255, 3.0, 64, child_k_min=floor)
        ev = ndg.Evaluator(gm, xt, tile, cp)
        E = ev.build(gm, xc=xc)
        offs, ids = oracle.cull_contract(L, m, w, xd, tile, proj, 1 / 255, 3.0, 64,
                                         xc=None if xc is None else xc.cpu().numpy(),
                                         n_parents=G, child_k_min=floor)
        assert E == offs[-1], (floor, E, offs[-1])
        g_off = ev.cull.offsets.cpu().numpy()
        g_ids = ev.cull.ids[:E].cpu().numpy()
        assert np.array_equal(g_off, offs)
        for t, (a, b) in enumerate(zip(csr_sets(g_off, g_ids), csr_sets(offs, ids))):
            assert np.array_equal(a, b), f"floor {floor} tile {t}"
        sets[floor] = (E, int((g_ids >= G).sum()))
        for mode, tol in ((ndg.NDG_MODE_FP32, 1e-5), (ndg.NDG_MODE_TC, 1e-3)):
            y = ev.forward(gm, mode=mode).cpu().numpy()
            yo = oracle.eval(L, m, w, xd, tile, offs, ids)
            assert_outputs_close(y, yo, rtol=tol, floor=1e-3)
        assert ndg.read_status(ev.ws) == 0
    assert sets[0.0][1] == 0, "children below the cutoff must be culled without the floor"
    assert sets[3.0][1] > 0, "with the floor the children must be evaluated"
    print(f"N={N} conditioned={conditioned}: entries {sets[0.0][0]} -> {sets[3.0][0]} "
          f"({sets[3.0][1]} child entries)")
