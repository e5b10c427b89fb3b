"""ndg_forward_noalloc: the evaluation for callers that cannot allocate device
memory (a plugin whose host application owns all device memory, a frame
callback that cannot afford an allocation's device synchronisation).  Its
scratch is a fixed static device array shared by every call, so these checks
call it through the C ABI several times in a row -- a larger mixture, then a
smaller one of the same dimension (leftover records of the first call must
not leak into the second), then another dimension -- and compare each result
with the FP64 oracle at the FP32 tolerance and with the workspace-based
ndg_forward (the same kernels: identical bits); an input larger than the
fixed scratch is refused."""
import numpy as np
import pytest

from helpers import assert_outputs_close, oracle_raw
from paper_2405_20067_gb300 import synth

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def ndg():
    import torch
    from paper_2405_20067_gb300 import build, ndg as _ndg
    build.build()
    assert torch.cuda.is_available()
    return _ndg


def _case(ndg, N, G, Q, tile, k, children, seed):
    import torch
    mix = synth.mixture(N, G, seed)
    ch = synth.children(N, G, seed + 1, spread=0.2) if children else None
    gm = ndg.Mixture.from_arrays(N, mix, ch)
    x = synth.queries_box(N, Q, seed + 2)
    proj = synth.projections(N, k, seed + 3)
    cp = ndg.CullParams(k, torch.as_tensor(proj).cuda(), 1 / 255, 3.0, 64)
    xt = torch.as_tensor(x).cuda()
    ev = ndg.Evaluator(gm, xt, tile, cp)
    ev.build(gm)
    return mix, ch, x, proj, gm, xt, ev


def test_noalloc_forward_matches_oracle_and_workspace_forward(ndg, oracle):
    import torch
    cases = [(6, 3000, 8192, 256, 8, True, 10),    # 6000 evaluated Gaussians
             (6, 1000, 5000, 256, 8, False, 15),   # same N, fewer records than the last call
             (10, 2000, 6000, 100, 16, False, 20)]
    for N, G, Q, tile, k, children, seed in cases:
        mix, ch, x, proj, gm, xt, ev = _case(ndg, N, G, Q, tile, k, children, seed)
        got = torch.full((Q, 3), float("nan"), device="cuda")
        ndg.forward_noalloc(gm, xt, tile, ev.cull, got)
        torch.cuda.synchronize()
        ref = ev.forward(gm)  # ndg_forward, FP32 form
        L, m, w = oracle.activate(oracle_raw(oracle, mix, ch))
        offs, ids = oracle.cull_contract(L, m, w, x.astype(np.float64), tile, proj, 1 / 255,
                                         3.0, 64)
        yo = oracle.eval(L, m, w, x.astype(np.float64), tile, offs, ids)
        g = got.cpu().numpy()
        worst = assert_outputs_close(g, yo, what=f"noalloc N={N} G={G}")
        assert np.array_equal(g, ref.cpu().numpy()), f"noalloc N={N} G={G}: differs from ndg_forward"
        print(f"noalloc N={N} G={G}: worst relative error {worst:.2e} against the oracle")


def test_noalloc_forward_refuses_inputs_beyond_its_scratch(ndg):
    import torch
    N, G = 6, 70_000  # 140,000 evaluated Gaussians x 128 B > 16 MiB
    gm = ndg.Mixture.from_arrays(N, synth.mixture(N, G, 5), synth.children(N, G, 6))
    x = torch.zeros(256, N, device="cuda")
    cull = ndg.Cull(1, 16)
    y = torch.zeros(256, 3, device="cuda")
    with pytest.raises(ndg.NDGError) as err:
        ndg.forward_noalloc(gm, x, 256, cull, y)
    assert err.value.status == ndg.NDG_ERR_SCRATCH_LIMIT
    assert "scratch" in str(err.value)
