"""Many frames in one persistent launch (ndg_forward_batch): mixtures and
query sets of uneven size (N = 3..12, ragged last tiles, tile sizes 128,
200 and 256, a frame without queries, a frame without Gaussians).  Each
frame's output equals its own tensor-core ndg_forward bit for bit, sampled
frames match the FP64 oracle at the tensor-core tolerance, the device
completion stamps are consistent, and a repeated batch gives the same
outputs."""
import numpy as np
import pytest

from helpers import assert_outputs_close, oracle_raw
from paper_2405_20067_gb300 import synth

pytestmark = pytest.mark.gpu

K, CUTOFF, B = 16, 1 / 255, 64

# N, G, W, H (pixels; W = 0: no queries), tile, children, checked against the oracle
FRAMES = [
    (6, 2000, 96, 80, 256, False, True),
    (10, 1200, 64, 48, 256, True, False),
    (3, 500, 50, 37, 200, False, True),
    (12, 400, 40, 40, 128, False, False),
    (8, 800, 128, 72, 256, True, True),
    (6, 300, 0, 0, 256, False, False),
    (6, 0, 32, 32, 256, False, False),
]


@pytest.fixture(scope="module")
def ndg():
    import torch
    from paper_2405_20067_gb300 import build, ndg as _ndg
    build.build()
    assert torch.cuda.is_available(), "GPU tests need a GPU"
    return _ndg


def make_frames(ndg):
    import torch
    out = []
    for i, (N, G, W, H, tile, children, _) in enumerate(FRAMES):
        seed = 700 + 10 * i
        mix = synth.mixture(N, max(G, 1), seed)
        if G == 0:
            mix = {k: v[:0] for k, v in mix.items()}
        ch = synth.children(N, G, seed + 1, spread=0.2) if children else None
        x = synth.queries_frame(N, W, H, seed + 2) if W > 0 else np.zeros((0, N), np.float32)
        proj = synth.projections(N, K, seed + 3)
        gm = ndg.Mixture.from_arrays(N, mix, ch, G_cap=max(G, 4))
        xt = torch.as_tensor(x).cuda()
        cp = ndg.CullParams(K, torch.as_tensor(proj).cuda(), CUTOFF, 3.0, B)
        ev = ndg.Evaluator(gm, xt, tile, cp, backward=False)
        ev.build(gm)
        y_ref = ev.forward(gm, mode=ndg.NDG_MODE_TC).clone()
        y = torch.full_like(y_ref, float("nan"))
        out.append(dict(N=N, mix=mix, ch=ch, x=x, proj=proj, tile=tile, gm=gm, xt=xt, ev=ev,
                        y_ref=y_ref, y=y))
    return out


def test_batch_equals_per_frame_forward_and_oracle(ndg, oracle):
    import torch
    fr = make_frames(ndg)
    bws = ndg.batch_workspace(len(fr))
    stamps = torch.zeros(1 + len(fr), dtype=torch.int64, device="cuda")
    items = [(f["gm"], f["xt"], f["tile"], f["ev"].cull, f["y"], f["ev"].ws) for f in fr]
    tr = ndg.Trace()
    ndg.forward_batch(items, bws, stamps, trace=tr)
    torch.cuda.synchronize()
    # one prep per frame with Gaussians, and the one persistent launch
    assert tr.launches == sum(1 for f in FRAMES if f[1] > 0) + 1
    for i, f in enumerate(fr):
        assert ndg.read_status(f["ev"].ws) == ndg.NDG_OK
        assert torch.equal(f["y"], f["y_ref"]), f"frame {i}: batch differs from ndg_forward"
    st = stamps.cpu().numpy()
    assert st[0] > 0
    for i, (N, G, W, H, tile, _, _) in enumerate(FRAMES):
        if W * H > 0:
            assert st[1 + i] >= st[0], i
        else:
            assert st[1 + i] == 0, i  # no work, no stamp
    assert torch.count_nonzero(fr[6]["y"]) == 0  # no Gaussians
    # sampled frames against the FP64 oracle
    for i, f in enumerate(fr):
        if not FRAMES[i][6]:
            continue
        raw = oracle_raw(oracle, f["mix"], f["ch"])
        L, m, w = oracle.activate(raw)
        xd = f["x"].astype(np.float64)
        offs, ids = oracle.cull_contract(L, m, w, xd, f["tile"], f["proj"], CUTOFF, 3.0, B,
                                         n_parents=f["mix"]["mean"].shape[0])
        yo = oracle.eval(L, m, w, xd, f["tile"], offs, ids)
        worst = assert_outputs_close(f["y"].cpu().numpy(), yo, rtol=1e-3, floor=1e-3,
                                     what=f"batched frame {i}")
        print(f"batched frame {i} (N={f['N']}, tile {f['tile']}): worst relative error {worst:.2e}")
    # the same batch again (the work list is rebuilt per call)
    for f in fr:
        f["y"].fill_(float("nan"))
    ndg.forward_batch(items, bws, None)
    torch.cuda.synchronize()
    for i, f in enumerate(fr):
        assert torch.equal(f["y"], f["y_ref"]), f"frame {i}: second batch differs"
    # after fresh culls, reusing the records they prepared (NDG_RECORDS_READY)
    for f in fr:
        f["ev"].build(f["gm"])
        f["y"].fill_(float("nan"))
    tr2 = ndg.Trace()
    ndg.forward_batch(items, bws, None, trace=tr2, records_ready=True)
    torch.cuda.synchronize()
    assert tr2.launches == 1  # no preparation, the one persistent launch
    for i, f in enumerate(fr):
        assert torch.equal(f["y"], f["y_ref"]), f"frame {i}: batch on the cull's records differs"


def test_batch_of_one_frame_fills_every_sm(ndg):
    """A single large frame through the batch entry point: more tiles than
    SMs, so each persistent CTA renders several tiles in turn."""
    import torch
    N, G, W, H = 6, 3000, 320, 256  # 320 tiles
    mix = synth.mixture(N, G, 91)
    x = synth.queries_frame(N, W, H, 92)
    gm = ndg.Mixture.from_arrays(N, mix)
    xt = torch.as_tensor(x).cuda()
    cp = ndg.CullParams(K, torch.as_tensor(synth.projections(N, K, 93)).cuda(), CUTOFF, 3.0, B)
    ev = ndg.Evaluator(gm, xt, 256, cp, backward=False)
    ev.build(gm)
    y_ref = ev.forward(gm, mode=ndg.NDG_MODE_TC).clone()
    y = torch.zeros_like(y_ref)
    stamps = torch.zeros(2, dtype=torch.int64, device="cuda")
    ndg.forward_batch([(gm, xt, 256, ev.cull, y, ev.ws)], ndg.batch_workspace(1), stamps)
    torch.cuda.synchronize()
    assert torch.equal(y, y_ref)
    st = stamps.cpu().numpy()
    assert st[1] > st[0] > 0
