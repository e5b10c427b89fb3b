"""Frame rendering with an autotuned launch configuration.

A frame is one query per pixel against one mixture: the cull (Section 3.2)
and the forward (Eq. 1, Eq. 8) through the C ABI, nothing else.  The
launch configuration of a frame -- the evaluation form (tensor cores, the
per-tile automatic choice, or FP32) and the query-tile size (256 or 128
queries: 16 x 16 or 16 x 8 pixels) -- is picked by `Autotuner`: the first
frame of each class (N, G rounded to a power of two, pixel count rounded to
a power of two) is rendered `reps` times with every candidate configuration,
the configuration with the lowest median time is kept for the class, and
later frames of the class reuse it.

`render_batch` renders many frames with one persistent launch of the
tensor-core forward (ndg_forward_batch) after their culls, and returns the
device's per-frame completion stamps.
"""
from __future__ import annotations

import math
from dataclasses import dataclass, field

import torch

from . import ndg

#: candidate launch configurations: (form, queries per tile)
CANDIDATES = (("tc", 256), ("auto", 256), ("tc", 128), ("fp32", 256))
_MODES = {"tc": ndg.NDG_MODE_TC, "auto": ndg.NDG_MODE_AUTO, "fp32": ndg.NDG_MODE_FP32}


def frame_class(N: int, G: int, Q: int) -> tuple:
    """Frames of one class share a tuned configuration."""
    return (N, int(round(math.log2(max(G, 1)))), int(round(math.log2(max(Q, 1)))))


@dataclass
class Autotuner:
    candidates: tuple = CANDIDATES
    reps: int = 5
    cache: dict = field(default_factory=dict)
    trials: dict = field(default_factory=dict)

    def choose(self, key: tuple, time_config) -> tuple:
        """time_config(cfg) -> ms of one frame; each candidate is timed
        `reps` times (interleaved, so that drifts hit every candidate alike)
        on the first frame of a class, and the lowest median wins."""
        if key not in self.cache:
            samples = {cfg: [] for cfg in self.candidates}
            for _ in range(self.reps):
                for cfg in self.candidates:
                    samples[cfg].append(time_config(cfg))
            med = {cfg: sorted(v)[len(v) // 2] for cfg, v in samples.items()}
            self.trials[key] = samples
            self.cache[key] = min(med, key=med.get)
        return self.cache[key]


class Frame:
    """One frame's device state: mixture, queries, cull buffers and
    workspace per tile size (built lazily), output."""

    def __init__(self, mix: ndg.Mixture, x: torch.Tensor, cp: ndg.CullParams):
        self.mix, self.x, self.cp = mix, x, cp
        self.Q = int(x.shape[0])
        self.y = torch.empty(self.Q, 3, dtype=torch.float32, device=x.device)
        self._ev = {}

    def evaluator(self, tile: int) -> ndg.Evaluator:
        if tile not in self._ev:
            ev = ndg.Evaluator(self.mix, self.x, tile, self.cp, backward=False)
            ev.build(self.mix)  # sizes the candidate buffers (synchronises once)
            self._ev[tile] = ev
        return self._ev[tile]

    def render(self, cfg: tuple) -> torch.Tensor:
        """Cull + forward on the current stream, no synchronisation."""
        form, tile = cfg
        ev = self.evaluator(tile)
        ndg.build_cull(self.mix, self.x, tile, self.cp, ev.cull, ev.ws)
        # the cull has just prepared the records from the same parameters
        ndg.forward(self.mix, self.x, tile, ev.cull, self.y, ev.ws,
                    mode=_MODES[form] | ndg.NDG_RECORDS_READY)
        return self.y

    def time(self, cfg: tuple, reps: int = 1) -> float:
        """ms of one frame (CUDA events on the current stream, after one
        untimed frame)."""
        self.render(cfg)
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record()
        for _ in range(reps):
            self.render(cfg)
        e1.record()
        torch.cuda.synchronize()
        return e0.elapsed_time(e1) / reps

    def release(self):
        self._ev.clear()


def render_batch(frames, batch_ws: torch.Tensor, stamps: torch.Tensor | None = None,
                 tile: int = 256, trace: ndg.Trace | None = None):
    """Culls every frame (its own launches, in order), then evaluates all of
    them with one persistent tensor-core launch (ndg_forward_batch, work list
    in frame order).  stamps: int64 [1 + len(frames)] on the device or None
    (%globaltimer ns: launch start, then each frame's completion).  No
    synchronisation; each frame's output is frame.y."""
    items = []
    for fr in frames:
        ev = fr.evaluator(tile)
        ndg.build_cull(fr.mix, fr.x, tile, fr.cp, ev.cull, ev.ws)
        items.append((fr.mix, fr.x, tile, ev.cull, fr.y, ev.ws))
    ndg.forward_batch(items, batch_ws, stamps, trace=trace, records_ready=True)
