"""Differentiable evaluation and the fit loop (Sections 3.3 and 4.1).

NDGEval is a torch.autograd.Function whose forward is ndg_forward and whose
backward is ndg_backward; Trainer drives the fit: per step the cull
(ndg_build_cull), the evaluation, the plain L2 loss (ndg_loss_l2), the
analytic backward, Adam (ndg_adam) and, at phase boundaries, the refinement
(ndg_densify).  Every step of that path runs in libndg's kernels; torch
provides device memory, streams and the autograd plumbing only.
"""
from __future__ import annotations

import torch

from . import ndg

_PARAMS = ["mean", "theta", "alpha_raw", "color_raw", "u_theta", "m_u", "c_alpha_raw",
           "c_color_raw"]


class NDGEval(torch.autograd.Function):
    """y = culled mixture value at the evaluator's queries (Eq. 1, Eq. 8).
    Gradients flow to the eight raw parameter tensors of the mixture."""

    @staticmethod
    def forward(ctx, ev: ndg.Evaluator, mix: ndg.Mixture, *params):
        y = torch.empty(ev.x.shape[0], 3, dtype=torch.float32, device=ev.x.device)
        ndg.forward(mix, ev.x, ev.tile, ev.cull, y, ev.ws, mode=getattr(ev, "mode", ndg.NDG_MODE_FP32),
                    trace=getattr(ev, "trace_fwd", None))
        ctx.ev, ctx.mix = ev, mix
        return y

    @staticmethod
    def backward(ctx, dy):
        ev, mix = ctx.ev, ctx.mix
        # fresh (uninitialised) gradient tensors: autograd adopts them as
        # .grad without a copy; rows >= G are never read
        grad = ndg.Mixture(mix.N, mix.G, *[None if getattr(mix, f) is None
                                           else torch.empty_like(getattr(mix, f))
                                           for f in _PARAMS], has_children=mix.has_children)
        mode = getattr(ev, "bwd_mode", ndg.NDG_MODE_FP32)
        order_stream = getattr(ev, "order_stream", None)
        if order_stream is not None and getattr(ev, "order_pending", False):
            # the Gaussian-major order of this cull ran beside the forward
            torch.cuda.current_stream().wait_stream(order_stream)
            mode |= ndg.NDG_BWD_ORDER_READY
            ev.order_pending = False
        ndg.backward(mix, ev.x, ev.tile, ev.cull, dy.contiguous(), grad, ev.ws, mode=mode,
                     trace=getattr(ev, "trace_bwd", None))
        outs = [getattr(grad, f) if (mix.has_children or i < 4) else None
                for i, f in enumerate(_PARAMS)]
        return (None, None, *outs)


def evaluate(ev: ndg.Evaluator, mix: ndg.Mixture) -> torch.Tensor:
    """Differentiable evaluation; mix tensors must require grad for a backward."""
    return NDGEval.apply(ev, mix, *[getattr(mix, f) for f in _PARAMS])


class Trainer:
    """Adam fit of a mixture to targets at a fixed query set.

    step() does one whole iteration on the device without host
    synchronisation; the candidate capacity is checked by check()."""

    def __init__(self, mix: ndg.Mixture, x: torch.Tensor, target: torch.Tensor, tile: int,
                 cp: ndg.CullParams, lr: float = 1e-3, t: float = 0.01, phase: int = 300,
                 E_cap: int | None = None, seed: int = 0, mode: int = ndg.NDG_MODE_FP32,
                 bwd_mode: int | None = None, loss: str = "l2", rel_eps: float = 1e-2,
                 loss_norm_queries: int | None = None, overlap_order: bool = True):
        """mode / bwd_mode: NDG_MODE_FP32 or NDG_MODE_TC for the forward and
        the backward; bwd_mode
        defaults to mode.  loss: "l2" (plain) or "rel_l2" (the relative L2 of
        Section 4.1, squared errors over y^2 + rel_eps).  loss_norm_queries:
        these queries are a shard of a set of that many (plain L2 only; see
        shard.py); grad_hook, when set, is called with the gradient tensors
        before Adam (the shards' sum).  overlap_order: the backward's
        Gaussian-major order of each step's lists (ndg_backward_order) runs on
        a side stream while the forward and the loss run."""
        if loss not in ("l2", "rel_l2"):
            raise ValueError(f"unknown loss {loss!r}")
        self.loss_kind, self.rel_eps = loss, rel_eps
        if loss_norm_queries is not None and loss != "l2":
            raise ValueError("a sharded loss is the plain L2")
        self.loss_norm_queries = loss_norm_queries
        self.grad_hook = None
        self.mix, self.tile, self.cp, self.mode = mix, tile, cp, mode
        self.bwd_mode = mode if bwd_mode is None else bwd_mode
        self.lr, self.t, self.phase = lr, t, phase
        for f in _PARAMS:
            p = getattr(mix, f)
            if p is not None:
                p.requires_grad_(True)
        self.m1, self.m2 = mix.zeros_like(), mix.zeros_like()
        for m in (self.m1, self.m2):
            for f in _PARAMS:
                if getattr(m, f) is not None:
                    getattr(m, f).requires_grad_(False)
        self.x = x.contiguous()
        self.target = target.contiguous()
        self.ev = ndg.Evaluator(mix, self.x, tile, cp, E_cap=E_cap)
        if E_cap is None:  # size the candidate buffers once from the initial state
            E = self.ev.build(mix)
            self.ev = ndg.Evaluator(mix, self.x, tile, cp, E_cap=int(E * 1.5) + 4096)
        dev = self.x.device
        self.dy = torch.empty_like(self.target)
        self.loss = torch.zeros(1, dtype=torch.float64, device=dev)
        self.step_dev = torch.zeros(1, dtype=torch.int32, device=dev)
        self.G_new = torch.zeros(1, dtype=torch.int32, device=dev)
        gen = torch.Generator(device=dev)
        gen.manual_seed(seed)
        P = mix.N * (mix.N + 1) // 2
        self.noise = torch.randn(mix.G_cap, P + mix.N + 4, device=dev, generator=gen)
        self.iteration = 0
        self.traces = None
        self.graph = None
        self.overlap_order = overlap_order
        # high priority: the order's blocks are placed first and finish early
        # (the forward's one CTA per SM waits for their room), so that the
        # loss after the forward is not held up by them; the two share the
        # SMs, so the overlap saves ~1 ms of the order's ~6.5 ms (measured
        # on the 2^20-query N = 6 step)
        self.order_stream = (torch.cuda.Stream(device=dev, priority=-1) if overlap_order
                             else None)

    def set_traces(self, traces: dict | None):
        """traces: dict name -> ndg.Trace for build_cull / forward / loss /
        backward / adam / densify, or None."""
        self.traces = traces
        self.ev.mode, self.ev.bwd_mode = self.mode, self.bwd_mode
        self.ev.trace_fwd = traces.get("forward") if traces else None
        self.ev.trace_bwd = traces.get("backward") if traces else None

    def _tr(self, name):
        return self.traces.get(name) if self.traces else None

    def step(self, x: torch.Tensor | None = None, target: torch.Tensor | None = None,
             refine: bool | None = None) -> torch.Tensor:
        """One iteration; x / target (host or device) replace the query set's
        contents when given.  Returns the loss as a device tensor."""
        if x is not None:
            self.x.copy_(x, non_blocking=True)
        if target is not None:
            self.target.copy_(target, non_blocking=True)
        mix = self.mix
        # the cull prepares the records the evaluation and the backward read
        # (the parameters do not change in between)
        self.ev.mode = self.mode | ndg.NDG_RECORDS_READY
        self.ev.bwd_mode = self.bwd_mode | ndg.NDG_RECORDS_READY
        ndg.build_cull(mix, self.x, self.tile, self.cp, self.ev.cull, self.ev.ws,
                       trace=self._tr("build_cull"))
        if self.overlap_order:
            # fork: the order depends on the lists only; the backward joins it
            self.order_stream.wait_stream(torch.cuda.current_stream())
            ndg.backward_order(mix, self.x, self.tile, self.ev.cull, self.ev.ws,
                               stream=self.order_stream)
            self.ev.order_stream, self.ev.order_pending = self.order_stream, True
        with torch.enable_grad():
            y = evaluate(self.ev, mix)
            if self.loss_kind == "rel_l2":
                ndg.loss_rel_l2(y.detach(), self.target, self.dy, self.loss, self.ev.ws,
                                eps=self.rel_eps, trace=self._tr("loss"))
            elif self.loss_norm_queries is not None:
                ndg.loss_l2_shard(y.detach(), self.target, self.dy, self.loss, self.ev.ws,
                                  self.loss_norm_queries, trace=self._tr("loss"))
            else:
                ndg.loss_l2(y.detach(), self.target, self.dy, self.loss, self.ev.ws,
                            trace=self._tr("loss"))
            y.backward(self.dy)
        grad = ndg.Mixture(mix.N, mix.G, *[getattr(mix, f).grad if getattr(mix, f) is not None
                                           else None for f in _PARAMS],
                           has_children=mix.has_children)
        if not mix.has_children:
            grad.u_theta = grad.m_u = grad.c_alpha_raw = grad.c_color_raw = None
        if self.grad_hook is not None:
            self.grad_hook(grad.tensors())
        with torch.no_grad():
            pm = self._detached(mix)
            ndg.adam(pm, grad, self._sync_meta(self.m1), self._sync_meta(self.m2), self.step_dev,
                     self.lr, trace=self._tr("adam"))
        for f in _PARAMS:
            if getattr(mix, f) is not None:
                getattr(mix, f).grad = None
        self.iteration += 1
        if refine is None:
            refine = self.phase > 0 and self.iteration % self.phase == 0
        if refine:
            self.refine(sync=False)
        return self.loss

    def capture(self, refine_each_step: bool = True):
        """Captures one whole step (cull, forward, loss, backward, Adam and,
        with refine_each_step, the refinement launches) as a CUDA graph;
        replay() runs it.  The graph reads the query and target buffers in
        place (refill them with copy_ between replays); a change of the row
        count G (check() after a materialising refinement) or of the
        candidate capacity needs a new capture.  Two warm-up steps run on a
        side stream first, as CUDA-graph capture of autograd requires."""
        self.set_traces(None)
        side = torch.cuda.Stream()
        side.wait_stream(torch.cuda.current_stream())
        with torch.cuda.stream(side):
            for _ in range(2):
                self._step_body(refine_each_step)
        torch.cuda.current_stream().wait_stream(side)
        g = torch.cuda.CUDAGraph()
        with torch.cuda.graph(g):
            self._step_body(refine_each_step)
        self.graph = g
        return g

    def _step_body(self, refine: bool):
        self.step(refine=False)
        if refine:
            self.refine(sync=False)

    def replay(self) -> torch.Tensor:
        """One captured step; returns the (device) loss buffer."""
        if self.graph is None:
            raise RuntimeError("capture() first")
        self.graph.replay()
        self.iteration += 1
        return self.loss

    def _detached(self, mix):
        return ndg.Mixture(mix.N, mix.G, *[None if getattr(mix, f) is None
                                           else getattr(mix, f).detach() for f in _PARAMS],
                           has_children=mix.has_children)

    def _sync_meta(self, m):
        m.G, m.has_children = self.mix.G, self.mix.has_children
        return m

    def refine(self, sync: bool = True):
        """Section 3.3 refinement.  With sync the new row count is read back
        and the mixture grows; without it the count stays on the device and
        check() applies it."""
        pm = self._detached(self.mix)
        ndg.densify_async(pm, self.t, self.noise, self._sync_meta(self.m1),
                          self._sync_meta(self.m2), self.G_new, self.ev.ws,
                          trace=self._tr("densify"))
        self.mix.has_children = True
        if sync:
            self.check()

    def check(self):
        """Synchronises: applies a pending row count, verifies the device
        status word and the candidate capacity (rebuilding larger buffers
        when it overflowed).  Steps taken since the overflow used truncated
        candidate lists: their outputs and gradients miss the dropped pairs
        (Adam has applied them); a captured graph has to be captured again."""
        st = ndg.read_status(self.ev.ws)
        Gn = int(self.G_new.item())
        if self.mix.has_children and Gn >= self.mix.G:
            self.mix.G = Gn
        self._sync_meta(self.m1)
        self._sync_meta(self.m2)
        if st == ndg.NDG_ERR_CAPACITY or self.ev.cull.E() > self.ev.E_cap:
            E = self.ev.cull.E()
            self.ev = ndg.Evaluator(self.mix, self.x, self.tile, self.cp, E_cap=int(E * 1.5) + 4096)
            self.set_traces(self.traces)
        elif st != ndg.NDG_OK:
            raise ndg.NDGError(st, "device status")
        return st
