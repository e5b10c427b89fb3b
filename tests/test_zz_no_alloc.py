"""ndg_forward_noalloc: the evaluation for callers that cannot allocate device
memory (a plugin whose host application owns all device memory, a frame
callback that cannot afford an allocation's device synchronisation).  Its
scratch is a fixed static device array, so these checks call it through the
C ABI and compare it with the workspace-based ndg_forward on two different
inputs in a row (the second call must not see the first call's leftovers),
and check that an input larger than the fixed scratch is refused."""
import numpy as np
import pytest

from helpers import assert_outputs_close
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
    x = torch.as_tensor(synth.queries_box(N, Q, seed + 2)).cuda()
    cp = ndg.CullParams(k, torch.as_tensor(synth.projections(N, k, seed + 3)).cuda(), 1 / 255, 3.0, 64)
    ev = ndg.Evaluator(gm, x, tile, cp)
    ev.build(gm)
    return gm, x, ev


def test_noalloc_forward_matches_workspace_forward_twice(ndg):
    import torch
    cases = [(6, 3000, 8192, 256, 8, True, 10), (10, 2000, 6000, 100, 16, False, 20)]
    for N, G, Q, tile, k, children, seed in cases:
        gm, x, ev = _case(ndg, N, G, Q, tile, k, children, seed)
        ref = ev.forward(gm)
        got = torch.full_like(ref, float("nan"))
        ndg.forward_noalloc(gm, x, tile, ev.cull, got)
        torch.cuda.synchronize()
        assert_outputs_close(got.cpu().numpy(), ref.cpu().numpy().astype(np.float64),
                             what=f"noalloc N={N}")


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
