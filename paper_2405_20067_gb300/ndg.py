"""Thin Python binding of libndg (include/ndg.h).

Every function here only marshals arguments (torch tensors -> device
pointers, the current CUDA stream) and calls the C ABI of the same name; all
arithmetic runs in the library's CUDA kernels.  There is no CPU fallback:
loading fails loudly when the library is missing.

Layouts follow the C header: a mixture is a set of FP32 device tensors with
G_cap rows, G of them in use (theta packed lower-triangular row by row).
"""
from __future__ import annotations

import ctypes
import math
import os
from dataclasses import dataclass, field

import torch

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "_build", "libndg.so")
_lib = None

NDG_OK = 0
NDG_ERR_INVALID_ARG = 1
NDG_ERR_CAPACITY = 2
NDG_ERR_CUDA = 3
NDG_ERR_NUMERIC = 4
NDG_ERR_TIMEOUT = 5
NDG_ERR_WORKSPACE = 6
NDG_MODE_FP32 = 0
NDG_MODE_TC = 1
NDG_MODE_AUTO = 2  # forward: tensor cores on tiles with >= auto_min_candidates(N) candidates


def auto_min_candidates(N: int) -> int:
    """NDG_AUTO_MIN_CANDIDATES(N) of the header."""
    return 192 if N <= 6 else 128

MAX_N, MAX_K, MAX_BUCKETS, MAX_TILE = 12, 32, 255, 256
_P = ctypes.c_void_p


class NDGError(RuntimeError):
    def __init__(self, status: int, where: str):
        self.status = status
        super().__init__(f"{where}: {status_string(status)} (status {status})")


class MixtureC(ctypes.Structure):
    _fields_ = [("N", ctypes.c_int), ("G", ctypes.c_int), ("G_cap", ctypes.c_int),
                ("has_children", ctypes.c_int),
                ("mean", _P), ("theta", _P), ("alpha_raw", _P), ("color_raw", _P),
                ("u_theta", _P), ("m_u", _P), ("c_alpha_raw", _P), ("c_color_raw", _P)]


class QueriesC(ctypes.Structure):
    _fields_ = [("Q", ctypes.c_longlong), ("tile_size", ctypes.c_int), ("x", _P)]


class CullParamsC(ctypes.Structure):
    _fields_ = [("k", ctypes.c_int), ("proj", _P), ("cutoff", ctypes.c_float),
                ("k_sigma", ctypes.c_float), ("buckets", ctypes.c_int),
                ("child_k_min", ctypes.c_float)]


class CullC(ctypes.Structure):
    _fields_ = [("offsets", _P), ("ids", _P), ("E_cap", ctypes.c_longlong), ("E_dev", _P)]


class FrameC(ctypes.Structure):
    _fields_ = [("mix", ctypes.POINTER(MixtureC)), ("q", ctypes.POINTER(QueriesC)),
                ("cull", ctypes.POINTER(CullC)), ("y", _P), ("ws", _P), ("ws_bytes", ctypes.c_size_t),
                ("flags", ctypes.c_int)]


class TraceC(ctypes.Structure):
    _fields_ = [("main_begin", _P), ("main_end", _P), ("launches", ctypes.c_longlong)]


class Trace:
    """Events around a call's main kernel and a running launch count.
    The events are torch.cuda.Events (created on first use)."""

    def __init__(self, timing: bool = True):
        self.timing = timing
        self.c = TraceC(None, None, 0)
        if timing:
            self.begin = torch.cuda.Event(enable_timing=True)
            self.end = torch.cuda.Event(enable_timing=True)
            self.begin.record()  # materialise the underlying cudaEvent_t
            self.end.record()
            self.c.main_begin = ctypes.c_void_p(self.begin.cuda_event)
            self.c.main_end = ctypes.c_void_p(self.end.cuda_event)

    @property
    def launches(self) -> int:
        return int(self.c.launches)

    def ms(self) -> float:
        return self.begin.elapsed_time(self.end)


def _tr(trace):
    return ctypes.byref(trace.c) if trace is not None else None


EXPORTS = ["ndg_workspace_size", "ndg_build_cull", "ndg_build_cull_conditioned", "ndg_forward",
           "ndg_loss_l2", "ndg_loss_rel_l2", "ndg_backward", "ndg_adam", "ndg_densify",
           "ndg_read_status", "ndg_status_string", "ndg_version", "ndg_forward_noalloc",
           "ndg_selftest_timeout", "ndg_probe_pipe", "ndg_loss_l2_shard",
           "ndg_batch_workspace_size", "ndg_forward_batch", "ndg_backward_order"]
NDG_ERR_SCRATCH_LIMIT = 7


def lib():
    """The loaded libndg (raises if it has not been built)."""
    global _lib
    if _lib is None:
        if not os.path.exists(LIB_PATH):
            raise RuntimeError(f"{LIB_PATH} is missing: build it with "
                               "`python -m paper_2405_20067_gb300.build` (there is no CPU path)")
        L = ctypes.CDLL(LIB_PATH)
        M, Qp, CP, C, TR = (ctypes.POINTER(MixtureC), ctypes.POINTER(QueriesC),
                            ctypes.POINTER(CullParamsC), ctypes.POINTER(CullC),
                            ctypes.POINTER(TraceC))
        sz = ctypes.c_size_t
        L.ndg_workspace_size.argtypes = [M, Qp, CP, ctypes.c_longlong]
        L.ndg_workspace_size.restype = sz
        L.ndg_build_cull.argtypes = [M, Qp, CP, C, _P, sz, _P, TR]
        L.ndg_build_cull_conditioned.argtypes = [M, Qp, CP, _P, C, _P, sz, _P, TR]
        L.ndg_forward.argtypes = [M, Qp, C, ctypes.c_int, _P, _P, sz, _P, TR]
        L.ndg_loss_l2.argtypes = [ctypes.c_longlong, _P, _P, _P, _P, _P, sz, _P, TR]
        L.ndg_loss_l2_shard.argtypes = [ctypes.c_longlong, ctypes.c_longlong, _P, _P, _P, _P, _P,
                                        sz, _P, TR]
        L.ndg_loss_rel_l2.argtypes = [ctypes.c_longlong, _P, _P, ctypes.c_float, _P, _P, _P, sz,
                                      _P, TR]
        L.ndg_backward.argtypes = [M, Qp, C, ctypes.c_int, _P, M, _P, sz, _P, TR]
        L.ndg_adam.argtypes = [M, M, M, M, _P, ctypes.c_float, ctypes.c_float, ctypes.c_float,
                               ctypes.c_float, _P, TR]
        L.ndg_densify.argtypes = [M, ctypes.c_float, ctypes.c_float, _P, M, M, _P, _P, sz, _P, TR]
        L.ndg_forward_noalloc.argtypes = [M, Qp, C, _P, _P]
        L.ndg_backward_order.argtypes = [M, Qp, C, _P, sz, _P, TR]
        L.ndg_batch_workspace_size.argtypes = [ctypes.c_int]
        L.ndg_batch_workspace_size.restype = sz
        L.ndg_forward_batch.argtypes = [ctypes.POINTER(FrameC), ctypes.c_int, _P, sz, _P, _P, TR]
        L.ndg_selftest_timeout.argtypes = [ctypes.c_int, _P, sz, _P]
        L.ndg_probe_pipe.argtypes = [ctypes.c_int, ctypes.c_int, ctypes.c_int, ctypes.c_int, _P,
                                     _P, _P]
        L.ndg_read_status.argtypes = [_P, _P, ctypes.POINTER(ctypes.c_int)]
        L.ndg_status_string.argtypes = [ctypes.c_int]
        L.ndg_status_string.restype = ctypes.c_char_p
        L.ndg_version.restype = ctypes.c_int
        for name in ["ndg_build_cull", "ndg_build_cull_conditioned", "ndg_forward", "ndg_loss_l2",
                     "ndg_loss_rel_l2", "ndg_backward", "ndg_adam", "ndg_densify",
                     "ndg_read_status", "ndg_forward_noalloc", "ndg_selftest_timeout",
                     "ndg_probe_pipe", "ndg_loss_l2_shard", "ndg_forward_batch",
                     "ndg_backward_order"]:
            getattr(L, name).restype = ctypes.c_int
        _lib = L
    return _lib


def status_string(status: int) -> str:
    return lib().ndg_status_string(int(status)).decode()


def _check(status: int, where: str):
    if status != NDG_OK:
        raise NDGError(status, where)


def _ptr(t):
    return None if t is None else ctypes.c_void_p(t.data_ptr())


def _stream(stream=None):
    s = stream if stream is not None else torch.cuda.current_stream()
    return ctypes.c_void_p(s.cuda_stream)


def tri(N: int) -> int:
    return N * (N + 1) // 2


# ---- data holders ----------------------------------------------------------------

_FIELDS = ["mean", "theta", "alpha_raw", "color_raw", "u_theta", "m_u", "c_alpha_raw",
           "c_color_raw"]


@dataclass
class Mixture:
    """Raw parameters on the device: G_cap rows each, G in use."""
    N: int
    G: int
    mean: torch.Tensor
    theta: torch.Tensor
    alpha_raw: torch.Tensor
    color_raw: torch.Tensor
    u_theta: torch.Tensor | None = None
    m_u: torch.Tensor | None = None
    c_alpha_raw: torch.Tensor | None = None
    c_color_raw: torch.Tensor | None = None
    has_children: bool = False

    @property
    def G_cap(self) -> int:
        return int(self.mean.shape[0])

    @property
    def Ge(self) -> int:
        return self.G * (2 if self.has_children else 1)

    @staticmethod
    def empty(N: int, G_cap: int, device="cuda", with_children=True) -> "Mixture":
        P = tri(N)
        z = lambda *s: torch.zeros(*s, dtype=torch.float32, device=device)
        m = Mixture(N, 0, z(G_cap, N), z(G_cap, P), z(G_cap), z(G_cap, 3))
        if with_children:
            m.u_theta, m.m_u, m.c_alpha_raw, m.c_color_raw = (z(G_cap, P), z(G_cap, N), z(G_cap),
                                                              z(G_cap, 3))
        return m

    @staticmethod
    def from_arrays(N: int, parents: dict, children: dict | None = None, G_cap: int | None = None,
                    device="cuda") -> "Mixture":
        G = int(parents["mean"].shape[0])
        cap = G_cap or G
        m = Mixture.empty(N, cap, device, with_children=True)
        for k in ["mean", "theta", "alpha_raw", "color_raw"]:
            getattr(m, k)[:G] = torch.as_tensor(parents[k], dtype=torch.float32).to(device)
        if children is not None:
            for k in ["u_theta", "m_u", "c_alpha_raw", "c_color_raw"]:
                getattr(m, k)[:G] = torch.as_tensor(children[k], dtype=torch.float32).to(device)
            m.has_children = True
        m.G = G
        return m

    def zeros_like(self) -> "Mixture":
        m = Mixture(self.N, self.G, *[None if getattr(self, f) is None
                                      else torch.zeros_like(getattr(self, f)) for f in _FIELDS],
                    has_children=self.has_children)
        return m

    def tensors(self):
        return [getattr(self, f) for f in _FIELDS]

    def c(self) -> MixtureC:
        return MixtureC(self.N, self.G, self.G_cap, int(self.has_children),
                        *[_ptr(getattr(self, f)) for f in _FIELDS])


@dataclass
class Cull:
    """Candidate lists (CSR over tiles) on the device."""
    T: int
    E_cap: int
    device: str = "cuda"
    offsets: torch.Tensor = field(init=False)
    ids: torch.Tensor = field(init=False)
    E_dev: torch.Tensor = field(init=False)

    def __post_init__(self):
        self.offsets = torch.zeros(self.T + 1, dtype=torch.int64, device=self.device)
        self.ids = torch.zeros(max(self.E_cap, 1), dtype=torch.int32, device=self.device)
        self.E_dev = torch.zeros(1, dtype=torch.int64, device=self.device)

    def c(self) -> CullC:
        return CullC(_ptr(self.offsets), _ptr(self.ids), self.E_cap, _ptr(self.E_dev))

    def E(self) -> int:
        return int(self.E_dev.item())


@dataclass
class CullParams:
    k: int
    proj: torch.Tensor | None
    cutoff: float
    k_sigma: float = 3.0
    buckets: int = 64
    child_k_min: float = 0.0  # children's radius floor (Section 3.3); 0: none

    def c(self) -> CullParamsC:
        return CullParamsC(self.k, _ptr(self.proj), self.cutoff, self.k_sigma, self.buckets,
                           self.child_k_min)


def queries_c(x: torch.Tensor, tile: int) -> QueriesC:
    return QueriesC(int(x.shape[0]), tile, _ptr(x))


# ---- the C ABI, one wrapper per entry point -----------------------------------------

def workspace_size(mix: Mixture, x: torch.Tensor | None, tile: int, cp: CullParams | None,
                   E_cap: int) -> int:
    q = queries_c(x, tile) if x is not None else None
    return int(lib().ndg_workspace_size(ctypes.byref(mix.c()), ctypes.byref(q) if q else None,
                                        ctypes.byref(cp.c()) if cp else None, E_cap))


def workspace(nbytes: int, device="cuda") -> torch.Tensor:
    # torch's caching allocator returns blocks aligned to at least 512 bytes
    return torch.zeros(max(int(nbytes), 256), dtype=torch.uint8, device=device)


def build_cull(mix: Mixture, x: torch.Tensor, tile: int, cp: CullParams, cull: Cull,
               ws: torch.Tensor, stream=None, trace: Trace | None = None):
    _check(lib().ndg_build_cull(ctypes.byref(mix.c()), ctypes.byref(queries_c(x, tile)),
                                ctypes.byref(cp.c()), ctypes.byref(cull.c()), _ptr(ws), ws.numel(),
                                _stream(stream), _tr(trace)), "ndg_build_cull")


def build_cull_conditioned(mix: Mixture, x: torch.Tensor, tile: int, cp: CullParams,
                           xc: torch.Tensor, cull: Cull, ws: torch.Tensor, stream=None,
                           trace: Trace | None = None):
    """The cull on position for the Gaussians restricted to the constant
    inputs xc [N - 3] (device FP32), which the queries carry beyond position."""
    assert xc.is_cuda and xc.dtype == torch.float32 and xc.numel() == mix.N - 3
    _check(lib().ndg_build_cull_conditioned(ctypes.byref(mix.c()),
                                            ctypes.byref(queries_c(x, tile)),
                                            ctypes.byref(cp.c()), _ptr(xc),
                                            ctypes.byref(cull.c()), _ptr(ws), ws.numel(),
                                            _stream(stream), _tr(trace)),
           "ndg_build_cull_conditioned")


def forward(mix: Mixture, x: torch.Tensor, tile: int, cull: Cull, y: torch.Tensor,
            ws: torch.Tensor, mode: int = NDG_MODE_FP32, stream=None, trace: Trace | None = None):
    _check(lib().ndg_forward(ctypes.byref(mix.c()), ctypes.byref(queries_c(x, tile)),
                             ctypes.byref(cull.c()), mode, _ptr(y), _ptr(ws), ws.numel(),
                             _stream(stream), _tr(trace)), "ndg_forward")


def forward_noalloc(mix: Mixture, x: torch.Tensor, tile: int, cull: Cull, y: torch.Tensor,
                    stream=None):
    """ndg_forward_noalloc: the evaluation without a workspace, for callers
    that cannot allocate device memory (see include/ndg.h)."""
    _check(lib().ndg_forward_noalloc(ctypes.byref(mix.c()), ctypes.byref(queries_c(x, tile)),
                                     ctypes.byref(cull.c()), _ptr(y), _stream(stream)),
           "ndg_forward_noalloc")


def batch_workspace(n_frames: int, device="cuda") -> torch.Tensor:
    """The descriptor workspace of forward_batch for n_frames frames."""
    return workspace(int(lib().ndg_batch_workspace_size(int(n_frames))), device)


def forward_batch(frames, batch_ws: torch.Tensor, stamps: torch.Tensor | None = None,
                  stream=None, trace: Trace | None = None, records_ready: bool = False):
    """ndg_forward_batch: the tensor-core forward of many frames in one
    persistent launch.  frames: sequence of (mix, x, tile, cull, y, ws), each
    as for forward(); stamps: int64 [1 + len(frames)] on the device or None
    (%globaltimer ns: [0] launch start, [1 + f] frame f complete);
    records_ready: every frame's cull has just prepared its records
    (NDG_RECORDS_READY)."""
    keep = []
    arr = (FrameC * len(frames))()
    fl = NDG_RECORDS_READY if records_ready else 0
    for i, (mix, x, tile, cull, y, ws) in enumerate(frames):
        mc, qc, cc = mix.c(), queries_c(x, tile), cull.c()
        keep += [mc, qc, cc]
        arr[i] = FrameC(ctypes.pointer(mc), ctypes.pointer(qc), ctypes.pointer(cc),
                        y.data_ptr(), ws.data_ptr(), ws.numel(), fl)
    _check(lib().ndg_forward_batch(arr, len(frames), _ptr(batch_ws), batch_ws.numel(),
                                   _ptr(stamps) if stamps is not None else None,
                                   _stream(stream), _tr(trace)), "ndg_forward_batch")


def loss_l2(y: torch.Tensor, target: torch.Tensor, dy: torch.Tensor, loss: torch.Tensor,
            ws: torch.Tensor, stream=None, trace: Trace | None = None):
    _check(lib().ndg_loss_l2(int(y.shape[0]), _ptr(y), _ptr(target), _ptr(dy), _ptr(loss),
                             _ptr(ws), ws.numel(), _stream(stream), _tr(trace)), "ndg_loss_l2")


def loss_l2_shard(y: torch.Tensor, target: torch.Tensor, dy: torch.Tensor, loss: torch.Tensor,
                  ws: torch.Tensor, Q_total: int, stream=None, trace: Trace | None = None):
    """Plain L2 of this shard's outputs normalised by the whole query set's
    Q_total (the shards' losses and gradients add up to the whole set's)."""
    _check(lib().ndg_loss_l2_shard(int(y.shape[0]), int(Q_total), _ptr(y), _ptr(target), _ptr(dy),
                                   _ptr(loss), _ptr(ws), ws.numel(), _stream(stream), _tr(trace)),
           "ndg_loss_l2_shard")


def selftest_timeout(which: int, ws: torch.Tensor, stream=None):
    """Bounded-wait self-test: a CTA waits on a barrier nothing completes and
    records NDG_ERR_TIMEOUT in the workspace status word (read_status)."""
    _check(lib().ndg_selftest_timeout(int(which), _ptr(ws), ws.numel(), _stream(stream)),
           "ndg_selftest_timeout")


def probe_pipe(which: int, reps: int = 5, iters: int = 2048, threads: int = 1024) -> dict:
    """Throughput of one arithmetic pipe (0: MUFU ex2, 1: FP32 FMA) through
    ndg_probe_pipe: the best of `reps` launches of one block per SM.  Returns
    the rate per SM per clock (from the blocks' clock64 cycles) and per
    second (from CUDA events around the launch)."""
    dev = torch.cuda.current_device()
    sms = torch.cuda.get_device_properties(dev).multi_processor_count
    blocks = sms
    cycles = torch.zeros(blocks, dtype=torch.int64, device="cuda")
    sink = torch.zeros(blocks * threads, dtype=torch.float32, device="cuda")
    ops = blocks * threads * 8 * iters
    best = None
    for _ in range(reps + 1):  # the first launch warms up
        b, e = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        b.record()
        _check(lib().ndg_probe_pipe(int(which), blocks, threads, iters, _ptr(cycles), _ptr(sink),
                                    _stream()), "ndg_probe_pipe")
        e.record()
        torch.cuda.synchronize()
        ms = b.elapsed_time(e)
        cyc = float(cycles.float().median().item())
        r = {"per_clk_per_sm": threads * 8 * iters / cyc, "per_s": ops / (ms * 1e-3),
             "ms": ms, "cycles": cyc, "sms": sms}
        if best is None or r["per_s"] > best["per_s"]:
            best = r
    return best


def loss_rel_l2(y: torch.Tensor, target: torch.Tensor, dy: torch.Tensor, loss: torch.Tensor,
                ws: torch.Tensor, eps: float = 1e-2, stream=None, trace: Trace | None = None):
    """Relative L2: sum (y - t)^2 / (y^2 + eps) / (3Q), dy with the
    denominator held constant."""
    _check(lib().ndg_loss_rel_l2(int(y.shape[0]), _ptr(y), _ptr(target), float(eps), _ptr(dy),
                                 _ptr(loss), _ptr(ws), ws.numel(), _stream(stream), _tr(trace)),
           "ndg_loss_rel_l2")


def backward(mix: Mixture, x: torch.Tensor, tile: int, cull: Cull, dy: torch.Tensor,
             grad: Mixture, ws: torch.Tensor, mode: int = NDG_MODE_FP32, stream=None,
             trace: Trace | None = None):
    _check(lib().ndg_backward(ctypes.byref(mix.c()), ctypes.byref(queries_c(x, tile)),
                              ctypes.byref(cull.c()), mode, _ptr(dy), ctypes.byref(grad.c()),
                              _ptr(ws), ws.numel(), _stream(stream), _tr(trace)), "ndg_backward")


NDG_BWD_ORDER_READY = 0x100
NDG_RECORDS_READY = 0x200  # the records ndg_build_cull left in ws are current


def backward_order(mix: Mixture, x: torch.Tensor, tile: int, cull: Cull, ws: torch.Tensor,
                   stream=None, trace: Trace | None = None):
    """ndg_backward_order: the Gaussian-major order of the entries, computed
    ahead of backward(..., mode | NDG_BWD_ORDER_READY) (e.g. on a side
    stream while the forward runs)."""
    _check(lib().ndg_backward_order(ctypes.byref(mix.c()), ctypes.byref(queries_c(x, tile)),
                                    ctypes.byref(cull.c()), _ptr(ws), ws.numel(), _stream(stream),
                                    _tr(trace)), "ndg_backward_order")


def adam(params: Mixture, grad: Mixture, m1: Mixture, m2: Mixture, step: torch.Tensor, lr: float,
         beta1: float = 0.9, beta2: float = 0.999, eps: float = 1e-8, stream=None,
         trace: Trace | None = None):
    _check(lib().ndg_adam(ctypes.byref(params.c()), ctypes.byref(grad.c()), ctypes.byref(m1.c()),
                          ctypes.byref(m2.c()), _ptr(step), lr, beta1, beta2, eps,
                          _stream(stream), _tr(trace)), "ndg_adam")


def densify_async(mix: Mixture, t: float, noise: torch.Tensor, m1: Mixture, m2: Mixture,
                  G_new: torch.Tensor, ws: torch.Tensor, stream=None, trace: Trace | None = None):
    """Section 3.3 refinement with threshold t (a_thr = ln t rounded to FP32,
    fresh children at brightness ln(t / 10)); the new row count stays on
    the device in G_new."""
    a_thr = float(torch.tensor(math.log(t), dtype=torch.float32))
    _check(lib().ndg_densify(ctypes.byref(mix.c()), a_thr, math.log(t / 10.0), _ptr(noise),
                             ctypes.byref(m1.c()), ctypes.byref(m2.c()), _ptr(G_new), _ptr(ws),
                             ws.numel(), _stream(stream), _tr(trace)), "ndg_densify")


def densify(mix: Mixture, t: float, noise: torch.Tensor, m1: Mixture, m2: Mixture,
            G_new: torch.Tensor, ws: torch.Tensor, stream=None, trace: Trace | None = None):
    """densify_async, then reads the new count (one synchronisation) and
    updates G / has_children of the mixture and its moments."""
    densify_async(mix, t, noise, m1, m2, G_new, ws, stream, trace)
    mix.G = int(G_new.item())
    mix.has_children = True
    for m in (m1, m2):
        m.G, m.has_children = mix.G, True


def read_status(ws: torch.Tensor, stream=None) -> int:
    v = ctypes.c_int(0)
    _check(lib().ndg_read_status(_ptr(ws), _stream(stream), ctypes.byref(v)), "ndg_read_status")
    return int(v.value)


# ---- conveniences built from the calls above -----------------------------------------

class Evaluator:
    """Owns the cull buffers and the workspace for one query set and grows
    them on NDG_ERR_CAPACITY.  Used by NDGEval, the fit driver and bench."""

    def __init__(self, mix: Mixture, x: torch.Tensor, tile: int, cp: CullParams,
                 E_cap: int | None = None, backward: bool = True):
        self.x, self.tile, self.cp = x, tile, cp
        self.T = (int(x.shape[0]) + tile - 1) // tile
        self.want_bwd = backward
        self.E_cap = int(E_cap) if E_cap else max(self.T * 64, 1024)
        self.cull = Cull(self.T, self.E_cap, str(x.device))
        self._alloc_ws(mix)

    def _alloc_ws(self, mix):
        n = workspace_size(mix, self.x, self.tile, self.cp, self.E_cap if self.want_bwd else 0)
        self.ws = workspace(n, self.x.device)

    def build(self, mix: Mixture, exact_capacity: bool = True,
              xc: torch.Tensor | None = None) -> int:
        """Builds the candidate lists (conditioned on the constant inputs xc
        when given); returns E (synchronises once)."""
        def run():
            if xc is None:
                build_cull(mix, self.x, self.tile, self.cp, self.cull, self.ws)
            else:
                build_cull_conditioned(mix, self.x, self.tile, self.cp, xc, self.cull, self.ws)
        run()
        E = self.cull.E()
        if E > self.E_cap:
            st = read_status(self.ws)
            assert st in (NDG_OK, NDG_ERR_CAPACITY), status_string(st)
            self.E_cap = int(E * 1.25) + 1024
            self.cull = Cull(self.T, self.E_cap, str(self.x.device))
            self._alloc_ws(mix)
            run()
            E = self.cull.E()
        return E

    def forward(self, mix: Mixture, y: torch.Tensor | None = None,
                mode: int = NDG_MODE_FP32) -> torch.Tensor:
        if y is None:
            y = torch.empty(self.x.shape[0], 3, dtype=torch.float32, device=self.x.device)
        forward(mix, self.x, self.tile, self.cull, y, self.ws, mode=mode)
        return y

    def backward(self, mix: Mixture, dy: torch.Tensor, grad: Mixture | None = None,
                 mode: int = NDG_MODE_FP32) -> Mixture:
        if grad is None:
            grad = mix.zeros_like()
        backward(mix, self.x, self.tile, self.cull, dy, grad, self.ws, mode=mode)
        return grad
