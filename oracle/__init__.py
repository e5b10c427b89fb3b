"""FP64 CPU oracle for the N-dimensional Gaussian mixture (test infrastructure).

Only the tests, ``__graft_entry__.smoke()`` and the CPU-baseline leg of
``bench.py`` may import this package.  The product path never does, and this
package imports nothing from the product package: the two share no code.

The arithmetic lives in ``ndg_oracle.c`` (plain loops in FP64, compiled with
``-ffp-contract=off``); this module only marshals numpy arrays.  Every raw
parameter array is widened to float64 exactly before the call.

Functions and the passages they follow (paper sections / equations):
  activate        Section 3.1 Eq. 1-2, Section 3.3 Eq. 6-7, Section 4.1 Eq. 8
  eval            Eq. 1 and Eq. 8 (dense or restricted to candidate lists)
  cull_exact      Section 3.2 Eq. 3-5, real-valued test in FP64
  cull_contract   the FP32 bucket contract that makes candidate lists
                  reproducible bit for bit (conservative w.r.t. cull_exact);
                  optionally on position for Gaussians restricted to xc
  condition       Section 3.2: a Gaussian restricted to constant inputs
                  beyond position (completing the square in the precision)
  loss_l2, grad   plain L2 loss and the analytic gradient (Section 4.1)
  loss_rel_l2     the relative L2 loss (Section 4.1; reading: (y - t)^2 / (y^2 + eps))
  adam            Adam update (the paper does not name its optimiser)
  densify         Section 3.3 materialisation of child Gaussians
  threads, set_threads   host threads of the parallel loops (for timing)
"""
from __future__ import annotations

import ctypes
import os
import subprocess
from dataclasses import dataclass

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "ndg_oracle.c")
_OUT = os.path.join(_HERE, "_build", "liboracle.so")
_lib = None

_D = ctypes.POINTER(ctypes.c_double)
_I = ctypes.POINTER(ctypes.c_int)
_LL = ctypes.POINTER(ctypes.c_longlong)
_U8 = ctypes.POINTER(ctypes.c_ubyte)


def compile_source(src: str, out: str) -> str:
    """gcc (OpenMP, no FP contraction) of one oracle source into a shared library."""
    os.makedirs(os.path.dirname(out), exist_ok=True)
    tmp = out + f".{os.getpid()}.tmp"
    cmd = ["gcc", "-O2", "-std=c11", "-ffp-contract=off", "-fno-fast-math", "-fopenmp",
           "-fPIC", "-shared", "-o", tmp, src, "-lm"]
    subprocess.run(cmd, check=True)
    os.replace(tmp, out)
    return out


def build(force: bool = False) -> str:
    """Compile the oracle (skipped while the library is newer than the source)."""
    if not force and os.path.exists(_OUT) and os.path.getmtime(_OUT) >= os.path.getmtime(_SRC):
        return _OUT
    return compile_source(_SRC, _OUT)


def _load():
    """The oracle library; NDG_ORACLE_LIB names another build of it (the
    pin-sensitivity test loads copies with planted mistakes that way)."""
    global _lib
    if _lib is None:
        lib = ctypes.CDLL(os.environ.get("NDG_ORACLE_LIB") or build())
        lib.oracle_activate.restype = None
        lib.oracle_eval.restype = None
        lib.oracle_cull_exact.restype = None
        lib.oracle_cull_contract.restype = ctypes.c_longlong
        lib.oracle_condition.restype = None
        lib.oracle_loss_l2.restype = ctypes.c_double
        lib.oracle_loss_rel_l2.restype = ctypes.c_double
        lib.oracle_grad.restype = None
        lib.oracle_adam.restype = None
        lib.oracle_densify.restype = ctypes.c_int
        lib.oracle_max_threads.restype = ctypes.c_int
        lib.oracle_set_threads.restype = None
        _lib = lib
    return _lib


def _d(a):
    """float64 C-contiguous copy (or None) and its pointer."""
    if a is None:
        return None, None
    a = np.ascontiguousarray(a, dtype=np.float64)
    return a, a.ctypes.data_as(_D)


@dataclass
class Raw:
    """Raw (pre-activation) mixture parameters, float64, row per parent."""
    mean: np.ndarray
    theta: np.ndarray
    alpha_raw: np.ndarray
    color_raw: np.ndarray
    u_theta: np.ndarray | None = None
    m_u: np.ndarray | None = None
    c_alpha_raw: np.ndarray | None = None
    c_color_raw: np.ndarray | None = None

    @property
    def N(self) -> int:
        return int(self.mean.shape[1])

    @property
    def G(self) -> int:
        return int(self.mean.shape[0])

    @property
    def has_children(self) -> bool:
        return self.u_theta is not None

    def arrays(self):
        return [self.mean, self.theta, self.alpha_raw, self.color_raw,
                self.u_theta, self.m_u, self.c_alpha_raw, self.c_color_raw]

    @staticmethod
    def from_arrays(arrs, has_children=True):
        a = [None if x is None else np.array(x, dtype=np.float64) for x in arrs]
        if not has_children:
            a[4:] = [None] * 4
        return Raw(*a)


def _raw_ptrs(raw: Raw):
    keep, ptrs = [], []
    for a in raw.arrays():
        if a is None:
            keep.append(None)
            ptrs.append(None)
        else:
            c, p = _d(a)
            keep.append(c)
            ptrs.append(p)
    return keep, ptrs


def activate(raw: Raw):
    """Evaluated Gaussians (L [Ge,N,N], m [Ge,N], w [Ge,3]) in FP64."""
    lib = _load()
    N, G = raw.N, raw.G
    Ge = 2 * G if raw.has_children else G
    L = np.zeros((Ge, N, N))
    m = np.zeros((Ge, N))
    w = np.zeros((Ge, 3))
    keep, p = _raw_ptrs(raw)
    lib.oracle_activate(N, G, int(raw.has_children), *p,
                        L.ctypes.data_as(_D), m.ctypes.data_as(_D), w.ctypes.data_as(_D))
    return L, m, w


def eval(L, m, w, x, tile=256, offsets=None, ids=None):
    """y [Q,3] = culled (or dense when offsets is None) mixture sum, FP64."""
    lib = _load()
    L, pL = _d(L)
    m, pm = _d(m)
    w, pw = _d(w)
    x, px = _d(x)
    Ge, N = m.shape
    Q = x.shape[0]
    y = np.zeros((Q, 3))
    if offsets is not None:
        offsets = np.ascontiguousarray(offsets, dtype=np.int64)
        ids = np.ascontiguousarray(ids, dtype=np.int32)
        po, pi = offsets.ctypes.data_as(_LL), ids.ctypes.data_as(_I)
    else:
        po = pi = None
    lib.oracle_eval(N, Ge, pL, pm, pw, ctypes.c_longlong(Q), px, tile, po, pi,
                    y.ctypes.data_as(_D))
    return y


def cull_exact(L, m, w, x, tile, proj, cutoff, k_sigma, n_parents=None, child_k_min=0.0):
    """keep [T, Ge] uint8 from the real-valued FP64 test (Eq. 3-5).
    n_parents: evaluated Gaussians at or above this index are children, whose
    radius is at least child_k_min (> 0; reading R7, Section 3.3); None: no
    children."""
    lib = _load()
    L, pL = _d(L)
    m, pm = _d(m)
    w, pw = _d(w)
    x, px = _d(x)
    proj, pp = _d(np.asarray(proj).reshape(-1, m.shape[1]))
    Ge, N = m.shape
    Q = x.shape[0]
    T = (Q + tile - 1) // tile
    keep = np.zeros((T, Ge), dtype=np.uint8)
    lib.oracle_cull_exact(N, Ge, pL, pm, pw, ctypes.c_longlong(Q), px, tile,
                          proj.shape[0], pp, ctypes.c_double(cutoff),
                          ctypes.c_double(k_sigma), Ge if n_parents is None else int(n_parents),
                          ctypes.c_double(child_k_min), keep.ctypes.data_as(_U8))
    return keep


def cull_contract(L, m, w, x, tile, proj, cutoff, k_sigma, buckets, tiles=None, xc=None,
                  n_parents=None, child_k_min=0.0):
    """(offsets, ids [E] int32) from the FP32 bucket contract.

    tiles=None: every tile, offsets [T+1] int64.  Otherwise the lists of the
    given tile indices only (in that order), offsets [len(tiles)+1]; each list
    equals that tile's list in the full run (the ranges and keys still come
    from the whole query set).  xc (N - 3 values): the contract on position
    for the Gaussians restricted to the constant inputs xc (condition()).
    n_parents, child_k_min: children's radius floor, as in cull_exact."""
    lib = _load()
    L, pL = _d(L)
    m, pm = _d(m)
    w, pw = _d(w)
    x, px = _d(x)
    Ge, N = m.shape
    proj, pp = _d(np.asarray(proj, dtype=np.float64).reshape(-1, N))
    k = proj.shape[0]
    Q = x.shape[0]
    T = (Q + tile - 1) // tile
    if tiles is None:
        n_sel, psel, nt = 0, None, T
    else:
        sel = np.ascontiguousarray(tiles, dtype=np.int64)
        assert sel.size == 0 or (sel.min() >= 0 and sel.max() < T)
        n_sel, psel, nt = sel.size, sel.ctypes.data_as(_LL), sel.size
    offsets = np.zeros(nt + 1, dtype=np.int64)
    if xc is not None:
        xc, pxc = _d(np.asarray(xc, dtype=np.float64).reshape(N - 3))
    else:
        pxc = None
    args = (N, Ge, pL, pm, pw, ctypes.c_longlong(Q), px, tile, k, pp,
            ctypes.c_double(cutoff), ctypes.c_double(k_sigma), buckets,
            Ge if n_parents is None else int(n_parents), ctypes.c_double(child_k_min),
            ctypes.c_longlong(n_sel), psel, pxc)
    E = lib.oracle_cull_contract(*args, offsets.ctypes.data_as(_LL), None)
    ids = np.zeros(max(E, 1), dtype=np.int32)
    E2 = lib.oracle_cull_contract(*args, offsets.ctypes.data_as(_LL), ids.ctypes.data_as(_I))
    assert E2 == E
    return offsets, ids[:E]


def condition(L, m, w, xc):
    """Gaussians restricted to the constant inputs xc = (x_4 .. x_N):
    (mu [Ge, 3], T [Ge, 3, 3] lower with covariance T^T T, wc [Ge, 3])."""
    lib = _load()
    L, pL = _d(L)
    m, pm = _d(m)
    w, pw = _d(w)
    Ge, N = m.shape
    xc, pxc = _d(np.asarray(xc, dtype=np.float64).reshape(N - 3))
    mu, T, wc = np.zeros((Ge, 3)), np.zeros((Ge, 3, 3)), np.zeros((Ge, 3))
    lib.oracle_condition(N, Ge, pL, pm, pw, pxc, mu.ctypes.data_as(_D), T.ctypes.data_as(_D),
                         wc.ctypes.data_as(_D))
    return mu, T, wc


def loss_l2(y, target):
    """(loss, gbar [Q,3]) for the plain L2 loss over Q x 3 outputs."""
    lib = _load()
    y, py = _d(y)
    t, pt = _d(target)
    gbar = np.zeros_like(y)
    loss = lib.oracle_loss_l2(ctypes.c_longlong(y.shape[0]), py, pt, gbar.ctypes.data_as(_D))
    return loss, gbar


def loss_rel_l2(y, target, eps=1e-2):
    """(loss, gbar [Q,3]) for the relative L2 loss: squared errors divided by
    y^2 + eps (the denominator held constant for the gradient)."""
    lib = _load()
    y, py = _d(y)
    t, pt = _d(target)
    gbar = np.zeros_like(y)
    loss = lib.oracle_loss_rel_l2(ctypes.c_longlong(y.shape[0]), py, pt, ctypes.c_double(eps),
                                  gbar.ctypes.data_as(_D))
    return loss, gbar


def grad(raw: Raw, x, tile, offsets, ids, gbar) -> Raw:
    """Gradient of the loss w.r.t. every raw parameter given gbar = dl/dy."""
    lib = _load()
    keep, p = _raw_ptrs(raw)
    x, px = _d(x)
    gbar, pg = _d(gbar)
    out = Raw(*[None if a is None else np.zeros_like(np.asarray(a, dtype=np.float64))
                for a in raw.arrays()])
    okeep, op = _raw_ptrs(out)
    if offsets is not None:
        offsets = np.ascontiguousarray(offsets, dtype=np.int64)
        ids = np.ascontiguousarray(ids, dtype=np.int32)
        po, pi = offsets.ctypes.data_as(_LL), ids.ctypes.data_as(_I)
    else:
        po = pi = None
    lib.oracle_grad(raw.N, raw.G, int(raw.has_children), *p, ctypes.c_longlong(x.shape[0]),
                    px, tile, po, pi, pg, *op)
    return Raw(*okeep)


def loss_of_raw(raw: Raw, x, target, tile=256, offsets=None, ids=None):
    """Loss as a function of the raw parameters (activate -> eval -> L2)."""
    L, m, w = activate(raw)
    y = eval(L, m, w, x, tile, offsets, ids)
    return loss_l2(y, target)[0]


def adam(p, g, m1, m2, t, lr, b1=0.9, b2=0.999, eps=1e-8):
    """One Adam step in FP64 on flat arrays (updated copies are returned)."""
    lib = _load()
    p, pp = _d(np.array(p, dtype=np.float64).ravel())
    g, pg = _d(np.asarray(g).ravel())
    m1, pm1 = _d(np.array(m1, dtype=np.float64).ravel())
    m2, pm2 = _d(np.array(m2, dtype=np.float64).ravel())
    lib.oracle_adam(ctypes.c_longlong(p.size), pp, pg, pm1, pm2, t, ctypes.c_double(lr),
                    ctypes.c_double(b1), ctypes.c_double(b2), ctypes.c_double(eps))
    return p, m1, m2


def densify(raw: Raw, G_cap: int, a_thr: float, a_child0: float, noise):
    """Materialise children (Section 3.3).  Returns (raw' with G_cap rows and
    G' valid, G', mat_flag[G])."""
    lib = _load()
    N, G = raw.N, raw.G
    P = N * (N + 1) // 2
    has = raw.has_children

    def grow(a, cols):
        out = np.zeros((G_cap,) + cols, dtype=np.float64)
        if a is not None:
            out[:G] = np.asarray(a, dtype=np.float64).reshape((G,) + cols)
        return out

    arrs = [grow(raw.mean, (N,)), grow(raw.theta, (P,)), grow(raw.alpha_raw, ()),
            grow(raw.color_raw, (3,)), grow(raw.u_theta, (P,)), grow(raw.m_u, (N,)),
            grow(raw.c_alpha_raw, ()), grow(raw.c_color_raw, (3,))]
    noise, pn = _d(noise)
    assert noise.size >= G_cap * (P + N + 4)
    flag = np.zeros(max(G, 1), dtype=np.uint8)
    Gn = lib.oracle_densify(N, G, G_cap, int(has), ctypes.c_double(a_thr),
                            ctypes.c_double(a_child0),
                            *[a.ctypes.data_as(_D) for a in arrs], pn,
                            flag.ctypes.data_as(_U8))
    return Raw(*arrs), Gn, flag[:G]


def threads() -> int:
    """Host threads the oracle's parallel loops use."""
    return int(_load().oracle_max_threads())


def set_threads(n: int) -> None:
    """Sets the host threads of the oracle's parallel loops (n >= 1)."""
    _load().oracle_set_threads(ctypes.c_int(int(n)))
