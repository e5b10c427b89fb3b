"""Failure detection without a GPU fault: the bounded device waits end, the
status word reports NDG_ERR_TIMEOUT, and the context stays usable."""
import time

import numpy as np
import pytest

from helpers import assert_outputs_close, oracle_raw
from paper_2405_20067_gb300 import synth

pytestmark = pytest.mark.gpu
NDG_ERR_TIMEOUT = 5


@pytest.fixture(scope="module")
def ndg():
    import torch
    from paper_2405_20067_gb300 import build, ndg as _ndg
    build.build()
    assert torch.cuda.is_available(), "GPU tests need a GPU"
    return _ndg


@pytest.mark.parametrize("which", [0, 1])
def test_wait_on_a_barrier_nothing_completes_times_out(ndg, oracle, which):
    import torch
    ws = ndg.workspace(1 << 16)
    t0 = time.time()
    ndg.selftest_timeout(which, ws)
    st = ndg.read_status(ws)
    dt = time.time() - t0
    assert st == NDG_ERR_TIMEOUT, st
    assert ndg.read_status(ws) == 0  # read_status clears the word
    assert dt < 60.0
    print(f"wait {which}: timed out after {dt:.2f} s")
    # the context still works: a small culled forward against the oracle
    N, G, Q, tile = 3, 200, 2000, 64
    mix = synth.mixture(N, G, 31)
    x = synth.queries_box(N, Q, 32)
    gm = ndg.Mixture.from_arrays(N, mix)
    proj = synth.projections(N, 4, 33)
    cp = ndg.CullParams(4, torch.as_tensor(proj).cuda(), 1 / 255, 3.0, 32)
    ev = ndg.Evaluator(gm, torch.as_tensor(x).cuda(), tile, cp)
    ev.build(gm)
    y = ev.forward(gm, mode=ndg.NDG_MODE_TC).cpu().numpy()
    L, m, w = oracle.activate(oracle_raw(oracle, mix))
    offs, ids = oracle.cull_contract(L, m, w, x.astype(np.float64), tile, proj, 1 / 255, 3.0, 32)
    yo = oracle.eval(L, m, w, x.astype(np.float64), tile, offs, ids)
    assert_outputs_close(y, yo, rtol=1e-3, floor=1e-3)
    assert ndg.read_status(ev.ws) == 0
