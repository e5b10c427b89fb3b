"""Seeded synthetic inputs shaped like the paper's 6-D and 10-D workloads.

This module only draws numbers (numpy PCG64) and arranges them; it evaluates,
culls and differentiates nothing.  Both the CUDA path and the FP64 oracle are
fed from it, so it imports neither.

Recipes (the paper's datasets are Mitsuba G-buffers and captured scenes that
are not available; these stand in with the same dimensionality and layout):

* Gaussians: means uniform in [-1, 1]^N.  Shape: the published recipe gives a
  lower-triangular factor with diagonal log-uniform in [2, 20] and
  off-diagonals N(0, 0.5^2); those numbers describe the inverse (precision)
  factor M = L^-1, so that widths are 0.05 .. 0.5 in a box of width 2.  The
  covariance factor the paper optimises is L = M^-1 and the raw parameters
  are theta_ii = ln L_ii and theta_ij = ln((1 + L_ij) / (1 - L_ij)); draws
  with |L_ij| >= 0.999 are redrawn.  Weights: w ~ U[0, 1]^3 split into
  brightness alpha = max_c w (raw ln alpha) and colour c = w / alpha clamped
  to [1e-4, 1 - 1e-4] (raw logit c).
* Unstructured queries (6-D): uniform in [-1, 1]^N, ordered along a Morton
  curve of 60 / N bits per dimension so that consecutive runs of 256 form
  compact tiles.
* Surface queries (10-D): 256 random planes through [-1, 1]^3, a 128 x 128
  grid on each (position = 3 dims), the other 7 dims i.i.d. uniform in
  [-1, 1] per query; 16 x 16 pixel tiles, row-major inside a tile.
* Frame queries (10-D, 1920 x 1080): one plane seen head-on, one query per
  pixel, the other dims uniform per query; 16 x 16 tiles, the last tile row
  half full.
* Projections: k unit vectors, normalised N(0, I) draws.
"""
from __future__ import annotations

import numpy as np


def rng(seed: int) -> np.random.Generator:
    return np.random.Generator(np.random.PCG64(seed))


def tri_size(N: int) -> int:
    return N * (N + 1) // 2


def _tril_pack(A: np.ndarray) -> np.ndarray:
    """[..., N, N] lower triangle -> [..., P] packed row by row."""
    N = A.shape[-1]
    rows, cols = np.tril_indices(N)
    return A[..., rows, cols]


def mixture(N: int, G: int, seed: int, literal_shape: bool = False) -> dict:
    """Raw parent parameters (float32) of G Gaussians."""
    r = rng(seed)
    mean = r.uniform(-1.0, 1.0, size=(G, N))
    rows, cols = np.tril_indices(N, -1)
    L = np.zeros((G, N, N))
    todo = np.arange(G)
    while todo.size:
        n = todo.size
        M = np.zeros((n, N, N))
        M[:, np.arange(N), np.arange(N)] = np.exp(r.uniform(np.log(2.0), np.log(20.0), size=(n, N)))
        M[:, rows, cols] = r.normal(0.0, 0.5, size=(n, rows.size))
        Lb = M if literal_shape else np.linalg.inv(M)
        Lb = np.tril(Lb)
        bad = np.any(np.abs(Lb[:, rows, cols]) >= 0.999, axis=1) if rows.size else np.zeros(n, bool)
        L[todo[~bad]] = Lb[~bad]
        todo = todo[bad]
    theta = np.zeros((G, N, N))
    d = np.arange(N)
    theta[:, d, d] = np.log(L[:, d, d])
    off = L[:, rows, cols]
    theta[:, rows, cols] = np.log((1.0 + off) / (1.0 - off))
    w = r.uniform(0.0, 1.0, size=(G, 3))
    alpha = np.maximum(w.max(axis=1), 1e-6)
    c = np.clip(w / alpha[:, None], 1e-4, 1.0 - 1e-4)
    return {
        "mean": mean.astype(np.float32),
        "theta": _tril_pack(theta).astype(np.float32),
        "alpha_raw": np.log(alpha).astype(np.float32),
        "color_raw": np.log(c / (1.0 - c)).astype(np.float32),
    }


def children(N: int, G: int, seed: int, spread: float = 0.3,
             brightness=(0.05, 0.5)) -> dict:
    """Raw child parameters with visible contributions (for tests)."""
    r = rng(seed)
    P = tri_size(N)
    return {
        "u_theta": r.normal(0.0, spread, size=(G, P)).astype(np.float32),
        "m_u": r.normal(0.0, spread, size=(G, N)).astype(np.float32),
        "c_alpha_raw": np.log(r.uniform(*brightness, size=G)).astype(np.float32),
        "c_color_raw": r.normal(0.0, 1.0, size=(G, 3)).astype(np.float32),
    }


def morton_order(x: np.ndarray) -> np.ndarray:
    """Stable permutation sorting points in [-1, 1]^N along a Morton curve."""
    Q, N = x.shape
    bits = max(1, 60 // N)
    q = np.clip(((x + 1.0) * 0.5 * (1 << bits)).astype(np.int64), 0, (1 << bits) - 1)
    code = np.zeros(Q, dtype=np.uint64)
    for b in range(bits):
        for dd in range(N):
            code |= (((q[:, dd] >> b) & 1).astype(np.uint64)) << np.uint64(b * N + dd)
    return np.argsort(code, kind="stable")


def queries_box(N: int, Q: int, seed: int, morton: bool = True) -> np.ndarray:
    r = rng(seed)
    x = r.uniform(-1.0, 1.0, size=(Q, N))
    if morton:
        x = x[morton_order(x)]
    return np.ascontiguousarray(x, dtype=np.float32)


def _plane_basis(r, n):
    normal = r.normal(size=(n, 3))
    normal /= np.linalg.norm(normal, axis=1, keepdims=True)
    a = np.where(np.abs(normal[:, :1]) < 0.9, np.array([[1.0, 0, 0]]), np.array([[0, 1.0, 0]]))
    u = np.cross(normal, a)
    u /= np.linalg.norm(u, axis=1, keepdims=True)
    v = np.cross(normal, u)
    return u, v


def _tiled_grid(W: int, H: int, tile_w: int = 16):
    """(row, col) of each pixel in tile order: tiles row-major over the image,
    pixels row-major inside a tile; edge tiles are ragged."""
    tr = (H + tile_w - 1) // tile_w
    tc = (W + tile_w - 1) // tile_w
    out_r, out_c = [], []
    for ty in range(tr):
        for tx in range(tc):
            rr = np.arange(ty * tile_w, min(H, (ty + 1) * tile_w))
            cc = np.arange(tx * tile_w, min(W, (tx + 1) * tile_w))
            R, C = np.meshgrid(rr, cc, indexing="ij")
            out_r.append(R.ravel())
            out_c.append(C.ravel())
    return np.concatenate(out_r), np.concatenate(out_c)


def tile_sizes(W: int, H: int, tile_w: int = 16) -> np.ndarray:
    """Number of pixels in each tile of _tiled_grid order."""
    tr = (H + tile_w - 1) // tile_w
    tc = (W + tile_w - 1) // tile_w
    hs = np.minimum(tile_w, H - np.arange(tr) * tile_w)
    ws = np.minimum(tile_w, W - np.arange(tc) * tile_w)
    return (hs[:, None] * ws[None, :]).ravel()


def queries_planes(N: int, n_planes: int, res: int, seed: int, extent: float = 1.0) -> np.ndarray:
    """Surface queries: n_planes planes with a res x res grid each, 16 x 16
    tiles (res must be a multiple of 16); dims beyond position uniform."""
    r = rng(seed)
    centre = r.uniform(-1.0, 1.0, size=(n_planes, 3))
    u, v = _plane_basis(r, n_planes)
    pr, pc = _tiled_grid(res, res)
    s = (pc + 0.5) / res - 0.5
    t = (pr + 0.5) / res - 0.5
    pos = centre[:, None, :] + extent * (s[None, :, None] * u[:, None, :] + t[None, :, None] * v[:, None, :])
    x = np.empty((n_planes, res * res, N))
    x[..., :3] = pos
    x[..., 3:] = r.uniform(-1.0, 1.0, size=(n_planes, res * res, N - 3))
    return np.ascontiguousarray(x.reshape(-1, N), dtype=np.float32)


def queries_frame(N: int, W: int, H: int, seed: int) -> np.ndarray:
    """One W x H frame of surface queries (plane z = 0 spanning [-1, 1] in x),
    16 x 16 tiles; dims beyond position uniform per query."""
    r = rng(seed)
    pr, pc = _tiled_grid(W, H)
    x = np.empty((pr.size, N))
    x[:, 0] = (pc + 0.5) / W * 2.0 - 1.0
    x[:, 1] = ((pr + 0.5) / H * 2.0 - 1.0) * (H / W)
    x[:, 2] = 0.0
    x[:, 3:] = r.uniform(-1.0, 1.0, size=(pr.size, N - 3))
    return np.ascontiguousarray(x, dtype=np.float32)


def projections(N: int, k: int, seed: int) -> np.ndarray:
    r = rng(seed)
    p = r.normal(size=(k, N))
    p /= np.linalg.norm(p, axis=1, keepdims=True)
    return np.ascontiguousarray(p, dtype=np.float32)


def targets_uniform(Q: int, seed: int) -> np.ndarray:
    return rng(seed).uniform(0.0, 1.0, size=(Q, 3)).astype(np.float32)


def noise(rows: int, N: int, seed: int) -> np.ndarray:
    """Standard normals for re-initialising children: one row of
    P + N + 4 values per slot."""
    return rng(seed).standard_normal(size=(rows, tri_size(N) + N + 4)).astype(np.float32)


# Workload recipes ----------------------------------------------------------

def config0(seed: int = 0) -> dict:
    """N=6, 1000 Gaussians, 16384 queries, ground truth mixture of 200; dense."""
    N = 6
    return {
        "N": N, "mix": mixture(N, 1000, seed), "gt": mixture(N, 200, seed + 100),
        "x": queries_box(N, 16384, seed + 1), "tile": 256,
    }


def config1(seed: int = 1, G: int = 100_000, Q: int = 1 << 20, k: int = 16) -> dict:
    """N=6 culled fwd+bwd: 100k Gaussians, 2^20 Morton-tiled queries, 16
    projections, contribution cutoff 1/255."""
    N = 6
    return {
        "N": N, "mix": mixture(N, G, seed), "x": queries_box(N, Q, seed + 1),
        "proj": projections(N, k, seed + 2), "target": targets_uniform(Q, seed + 3),
        "tile": 256, "cutoff": 1.0 / 255.0, "k_sigma": 3.0, "buckets": 64,
    }


def config2(seed: int = 2, G: int = 500_000, n_planes: int = 256, res: int = 128,
            k: int = 16) -> dict:
    """N=10 surface queries: 500k Gaussians, 256 random planes with a 128 x 128
    grid each (2^22 queries, 16 x 16 tiles), 16 projections, cutoff 1/255."""
    N = 10
    return {
        "N": N, "mix": mixture(N, G, seed), "x": queries_planes(N, n_planes, res, seed + 1),
        "proj": projections(N, k, seed + 2), "tile": 256, "cutoff": 1.0 / 255.0,
        "k_sigma": 3.0, "buckets": 64,
    }


def config3(seed: int = 3, G: int = 50_000, G_gt: int = 2_000_000, G_max: int = 1_000_000,
            n_planes: int = 16, res: int = 128, k: int = 16) -> dict:
    """N=10 fit: a ground-truth mixture of 2M Gaussians drawn as in config 2,
    a fitted mixture of 50k parents whose children start at brightness t/10
    (t = 0.01) and may grow it to 1M, minibatches of 2^18 surface queries
    (16 planes x 128^2), 16 projections, cutoff 1/255."""
    N = 10
    return {
        "N": N, "mix": mixture(N, G, seed), "gt": mixture(N, G_gt, seed + 100),
        "children": children(N, G, seed + 1, spread=0.05, brightness=(0.0009, 0.0011)),
        "x": queries_planes(N, n_planes, res, seed + 2), "proj": projections(N, k, seed + 3),
        "G_max": G_max, "t": 0.01, "tile": 256, "cutoff": 1.0 / 255.0, "k_sigma": 3.0,
        "buckets": 64,
    }


def config4_frames(seed: int = 4, n: int = 64) -> list:
    """Batched render specs: n independent frames, G log-uniform in
    [1e4, 5e5], N in {6, 8, 10}, resolution log-uniform between 256 x 256 and
    1920 x 1080 (one exponent for both sides), one query per pixel.  Each
    spec carries the seeds of its mixture, queries and projections."""
    r = rng(seed)
    out = []
    for i in range(n):
        t = r.uniform()
        out.append({
            "N": int(r.choice([6, 8, 10])),
            "G": int(round(np.exp(r.uniform(np.log(1e4), np.log(5e5))))),
            "W": int(round(256 * (1920 / 256) ** t)), "H": int(round(256 * (1080 / 256) ** t)),
            "seed": seed * 1000 + 3 * i,
        })
    return out
