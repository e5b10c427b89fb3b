"""Shared test helpers: the same seeded inputs fed to the CUDA path and to the
oracle, and the comparison rules used by every parity test.

Tolerances (FP32 path against the FP64 oracle):
  outputs   |a - b| / max(|b|, 1e-3) <= 1e-5
  gradients per tensor ||a - b||_2 / ||b||_2 <= 1e-4, and elementwise
            |a - b| <= 1e-4 |b| + 1e-3 max|b| (relative floor for entries
            that are sums of cancelling contributions)
  candidate lists: identical sets per tile (bit-exact integer contract).
"""
from __future__ import annotations

import numpy as np

FWD_RTOL = 1e-5
FWD_FLOOR = 1e-3
GRAD_RTOL = 1e-4
GRAD_FLOOR = 1e-3

NAMES = ["mean", "theta", "alpha_raw", "color_raw", "u_theta", "m_u", "c_alpha_raw", "c_color_raw"]


def oracle_raw(oracle, parents: dict, children: dict | None = None):
    arrs = [parents[k] for k in NAMES[:4]]
    arrs += [None] * 4 if children is None else [children[k] for k in NAMES[4:]]
    return oracle.Raw.from_arrays(arrs, has_children=children is not None)


def assert_outputs_close(got, want, rtol=FWD_RTOL, floor=FWD_FLOOR, what="output"):
    got = np.asarray(got, dtype=np.float64)
    want = np.asarray(want, dtype=np.float64)
    assert got.shape == want.shape
    err = np.abs(got - want) / np.maximum(np.abs(want), floor)
    worst = float(err.max()) if err.size else 0.0
    assert worst <= rtol, f"{what}: worst relative error {worst:.3e} > {rtol:.1e}"
    return worst


def assert_grads_close(got: dict, want, names, rtol=GRAD_RTOL, floor=GRAD_FLOOR):
    report = {}
    for n in names:
        g = np.asarray(got[n], dtype=np.float64)
        w = np.asarray(getattr(want, n), dtype=np.float64).reshape(g.shape)
        nw = np.linalg.norm(w)
        rel = np.linalg.norm(g - w) / nw if nw > 0 else np.linalg.norm(g)
        scale = np.abs(w).max() if w.size else 0.0
        elem = np.abs(g - w) <= rtol * np.abs(w) + floor * scale + 1e-30
        report[n] = rel
        assert rel <= rtol, f"grad {n}: relative L2 error {rel:.3e} > {rtol:.1e}"
        assert elem.all(), (f"grad {n}: {int((~elem).sum())} entries off; worst "
                            f"{np.abs(g - w)[~elem].max():.3e}")
    return report


def csr_sets(offsets, ids):
    offsets = np.asarray(offsets)
    ids = np.asarray(ids)
    return [np.sort(ids[offsets[t]:offsets[t + 1]]) for t in range(len(offsets) - 1)]


def sorted_csr(offsets, ids):
    """Same lists with ascending ids inside each tile."""
    sets = csr_sets(offsets, ids)
    return np.asarray(offsets, dtype=np.int64), (np.concatenate(sets).astype(np.int32)
                                                 if sets else np.zeros(0, np.int32))
