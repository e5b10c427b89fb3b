#!/usr/bin/env python
"""Throughput of the culled forward + backward of an N-dimensional Gaussian
mixture (the fit step of "N-Dimensional Gaussians for Fitting of High
Dimensional Functions"), in Gaussian-query pairs per second.

Workload (synthetic, seeded): N = 6, 100,000 Gaussians (each with a child
of negligible brightness, the state after the first refinement), 2^20
queries uniform in [-1, 1]^6 in Morton-ordered tiles of 256, 16 random
projections, contribution cutoff 1/255.  One step = cull + forward + L2 loss
+ backward + Adam + refinement check, all in libndg's kernels.  Pairs per
step = sum over tiles of (queries in tile x candidates in tile).

    python bench.py [--gpus N] [--steps K] [--warmup W] [--impl reference]

Prints one JSON line (rank 0).  With --gpus N > 1 (under torchrun) every rank
fits its own independent replica (no collective): weak scaling.
"""
from __future__ import annotations

import argparse
import json
import math
import os
import statistics
import subprocess
import sys
import threading
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "culled fwd+bwd Gaussian-query pairs/s and N=10 1080p render ms, vs plain FP32"
UNIT = "pairs/s"
N_DIM, K_PROJ, TILE, BUCKETS = 6, 16, 256, 64
CUTOFF = 1.0 / 255.0
# the headline workload and a small case of the same density for profiling
WORKLOADS = {"fit_n6": (100_000, 1 << 20), "small_n6": (12_500, 1 << 17)}
G, Q = WORKLOADS["fit_n6"]


def workload_name(g, q):
    return (f"N={N_DIM} culled fit step: {g} Gaussians (+{g} children at brightness t/10, "
            "evaluated within 3 sigma), "
            f"Q=2^{q.bit_length() - 1} Morton-tiled queries, tile {TILE}, k={K_PROJ} projections, "
            f"cutoff 1/255, {BUCKETS} buckets, Adam lr 1e-3")


# DRAM bytes per candidate entry of one bwd_h_kernel<6> launch:
# dram__bytes_read.sum + dram__bytes_write.sum = 36.69 MB + 621.08 MB from one
# ncu capture of the 1/8 workload (5,196,498 entries in that run's step),
# i.e. 126.6 B per entry; a full launch's traffic is this times its entries
# (the kernel streams one gradient record per entry, so traffic grows in
# proportion).  To be re-taken whenever the kernel changes.
BWD_BYTES_PER_ENTRY = (36.689408e6 + 621.075456e6) / 5196498


def flops_per_pair(N: int):
    """Algorithmic FP32 flops per Gaussian-query pair (FMA = 2):
    forward  d = x - m (N), z = M d (N(N+1)), s = |z|^2 (2N), scale (1),
             w e (6)                                 -> N^2 + 4N + 7
    backward the forward's N^2 + 4N + 1 again, sum dy e (6), beta (6),
             beta z (N), sum beta z (N), sum beta z d^T (N(N+1))
                                                     -> 2N^2 + 7N + 13."""
    return N * N + 4 * N + 7, 2 * N * N + 7 * N + 13


def tc_flops_per_pair(N: int):
    """Tensor-core flops per pair.  Algorithmic (the lifted contraction
    counted once): forward 2F (s = phi . coef), backward 4F (s recomputed and
    the gradient contraction sum_q beta phi), F = N(N+1)/2 + N + 1.
    Executed by the kernels (FP16 hi/lo split, K padded to KP = 16 ceil(F /
    16)): forward 6 KP (three products); backward 6 KP for S (three
    products) plus 12 KP for D2 = E Psi (E single FP16, Psi hi/lo: two
    products; Psi has 3 KP columns, one block per colour)."""
    P = N * (N + 1) // 2
    F = P + N + 1
    KP = (F + 15) // 16 * 16
    return 2 * F, 4 * F, 6 * KP, 6 * KP + 12 * KP


def fp32_peak_tflops(sm_mhz: float, sms: int = 152) -> float:
    """FP32 FMA pipe: 128 lanes x 2 flops per SM per clock."""
    return sms * 128 * 2 * sm_mhz * 1e6 / 1e12


def load_peaks():
    p = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(p):
        with open(p) as f:
            return json.load(f), "measured"
    return {"hbm_gbs": 6800.0, "bf16_tflops": 1900.0, "sm_max_mhz": 2070.0}, "fallback"


class ClockSampler:
    """nvidia-smi samples (SM clock, reasons) while the timed region runs."""
    Q = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
         "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
         "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, index: int):
        self.index = index
        self.proc = None
        self.lines = []

    def __enter__(self):
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", f"--id={self.index}", f"--query-gpu={self.Q}",
                 "--format=csv,noheader,nounits", "-lms", "200"],
                stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
            self.thread = threading.Thread(target=self._read, daemon=True)
            self.thread.start()
        except (OSError, FileNotFoundError):
            self.proc = None
        return self

    def _read(self):
        for line in self.proc.stdout:
            self.lines.append(line.strip())

    def __exit__(self, *a):
        if self.proc is not None:
            self.proc.terminate()
            try:
                self.proc.wait(timeout=5)
            except subprocess.TimeoutExpired:
                self.proc.kill()

    def summary(self):
        mhz, mx, reasons = [], 0.0, set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for ln in self.lines:
            parts = [p.strip() for p in ln.split(",")]
            if len(parts) < 9:
                continue
            try:
                mhz.append(float(parts[1]))
                mx = max(mx, float(parts[2]))
            except ValueError:
                continue
            for n, v in zip(names, parts[5:9]):
                if v.lower() == "active":
                    reasons.add(n)
        return {"sm_mhz": statistics.median(mhz) if mhz else None, "sm_max_mhz": mx or None,
                "samples": len(mhz), "reasons": sorted(reasons)}


def build_workload(device):
    import torch
    from paper_2405_20067_gb300 import ndg, synth
    c = synth.config1(G=G, Q=Q)
    mix = c["mix"]
    ch = synth.children(N_DIM, G, 11, spread=0.05, brightness=(0.0009, 0.0011))
    gm = ndg.Mixture.from_arrays(N_DIM, mix, ch, G_cap=G + G // 10, device=device)
    x = torch.as_tensor(c["x"]).to(device)
    target = torch.as_tensor(c["target"]).to(device)
    proj = torch.as_tensor(c["proj"]).to(device)
    # children below the cutoff keep a 3-sigma radius (Section 3.3): they are
    # evaluated, and optimised, where they span their parents
    cp = ndg.CullParams(K_PROJ, proj, CUTOFF, 3.0, BUCKETS, child_k_min=3.0)
    return c, ch, gm, x, target, cp


RENDER = {"N": 10, "G": 500_000, "W": 1920, "H": 1080, "k": 16, "buckets": 64}


def render_n10_1080p(device, steps: int, warmup: int, flush, res: tuple | None = None):
    """Second metric: one 1920 x 1080 frame (16 x 16 pixel tiles, 8160 tiles,
    the last tile row half full) of 10-D surface queries against 500,000
    10-D Gaussians: cull + forward (S1-S4), ms per frame, for the lifted
    tensor-core form (the value) and the plain FP32 form."""
    import torch
    from paper_2405_20067_gb300 import ndg, synth
    r = dict(RENDER) if res is None else dict(RENDER, W=res[0], H=res[1])
    mix = synth.mixture(r["N"], r["G"], 2)
    gm = ndg.Mixture.from_arrays(r["N"], mix, device=device)
    x = torch.as_tensor(synth.queries_frame(r["N"], r["W"], r["H"], 3)).to(device)
    proj = torch.as_tensor(synth.projections(r["N"], r["k"], 4)).to(device)
    cp = ndg.CullParams(r["k"], proj, CUTOFF, 3.0, r["buckets"])
    ev = ndg.Evaluator(gm, x, TILE, cp, E_cap=1 << 24, backward=False)
    E = ev.build(gm)
    y = torch.empty(x.shape[0], 3, dtype=torch.float32, device=device)
    tc, tf = ndg.Trace(), ndg.Trace()
    out = {}
    for form, mode in (("tc", ndg.NDG_MODE_TC), ("fp32", ndg.NDG_MODE_FP32)):
        def frame(trace_c=None, trace_f=None):
            ndg.build_cull(gm, x, TILE, cp, ev.cull, ev.ws, trace=trace_c)
            # the cull has just prepared the records from the same parameters
            ndg.forward(gm, x, TILE, ev.cull, y, ev.ws, mode=mode | ndg.NDG_RECORDS_READY,
                        trace=trace_f)

        for _ in range(warmup):
            frame()
        ms, cull_ms, fwd_ms, launches = [], [], [], 0
        n = steps if form == "tc" else max(2, steps // 2)
        for _ in range(n):
            flush.zero_()
            a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            tc.c.launches = tf.c.launches = 0
            a.record()
            frame(tc, tf)
            b.record()
            torch.cuda.synchronize()
            ms.append(a.elapsed_time(b))
            cull_ms.append(tc.ms())
            fwd_ms.append(tf.ms())
            launches += tc.launches + tf.launches
        out[form] = {"ms": statistics.median(ms), "fwd_kernel_ms": statistics.median(fwd_ms),
                     "cull_fill_kernel_ms": statistics.median(cull_ms), "gpu_launches": launches}
    assert ndg.read_status(ev.ws) == ndg.NDG_OK
    pairs = pairs_of(ev.cull, x.shape[0], TILE)
    fwd_f, _ = flops_per_pair(r["N"])
    return {"metric": "N=10 1080p render ms", "value": out["tc"]["ms"], "unit": "ms",
            "higher_is_better": False, "form": "lifted tensor-core forward",
            "fp32_form_ms": out["fp32"]["ms"],
            "workload": f"{r['W']}x{r['H']} frame, 16x16 tiles, N=10, {r['G']} Gaussians, "
                        f"k={r['k']}, cutoff 1/255 (non-position dims uniform per pixel)",
            "candidates": E, "pairs": pairs, "tc": out["tc"], "fp32": out["fp32"],
            "fp32_fwd_tflops": round(pairs * fwd_f / (out["fp32"]["fwd_kernel_ms"] / 1e3) / 1e12, 3),
            "tc_pairs_per_s": pairs / (out["tc"]["fwd_kernel_ms"] / 1e3)}


def pairs_of(cull, Qn, tile):
    import torch
    offs = cull.offsets
    cnt = offs[1:] - offs[:-1]
    T = cnt.shape[0]
    qt = torch.full((T,), tile, dtype=torch.int64, device=offs.device)
    if T:
        qt[-1] = Qn - tile * (T - 1)
    return int((cnt * qt).sum().item())


def cpu_baseline(c, ch, seconds: float = 15.0, single_seconds: float = 0.0):
    """The FP64 oracle on a bounded sample of the same workload: culled
    forward + L2 loss + gradient on a subset of tiles, on all host cores
    (its OpenMP loops) and, when single_seconds > 0, on one core with a
    sample sized to take about that long."""
    import oracle
    from paper_2405_20067_gb300 import synth  # noqa: F401  (inputs only)
    oracle.build()
    names = ["mean", "theta", "alpha_raw", "color_raw", "u_theta", "m_u", "c_alpha_raw",
             "c_color_raw"]
    raw = oracle.Raw.from_arrays([c["mix"][n] for n in names[:4]] + [ch[n] for n in names[4:]], True)
    x = c["x"].astype(np.float64)
    L, m, w = oracle.activate(raw)
    offs, ids = oracle.cull_contract(L, m, w, x, TILE, c["proj"], CUTOFF, 3.0, BUCKETS,
                                     n_parents=int(c["mix"]["mean"].shape[0]), child_k_min=3.0)
    T = len(offs) - 1
    rng = np.random.default_rng(0)
    order = rng.permutation(T)

    def run(ntiles):
        sel = np.sort(order[:ntiles])
        xs = np.concatenate([x[t * TILE:(t + 1) * TILE] for t in sel])
        ts = np.concatenate([c["target"][t * TILE:(t + 1) * TILE] for t in sel]).astype(np.float64)
        so = np.zeros(ntiles + 1, np.int64)
        lists = [ids[offs[t]:offs[t + 1]] for t in sel]
        so[1:] = np.cumsum([len(l) for l in lists])
        si = np.concatenate(lists).astype(np.int32) if lists else np.zeros(0, np.int32)
        pairs = int(sum(len(l) for l in lists) * TILE)
        t0 = time.perf_counter()
        La, ma, wa = oracle.activate(raw)
        y = oracle.eval(La, ma, wa, xs, TILE, so, si)
        _, gbar = oracle.loss_l2(y, ts)
        oracle.grad(raw, xs, TILE, so, si, gbar)
        return pairs, time.perf_counter() - t0

    cores = oracle.threads()
    p1, t1 = run(4)
    n = int(min(T, max(4, 4 * seconds / max(t1, 1e-3))))
    p, t = run(n)
    out = {"value": p / t, "unit": UNIT, "cores": cores, "kind": "oracle",
           "sample": f"{n} of {T} tiles ({p:.3g} pairs), FP64 culled forward + loss + gradient",
           "seconds": round(t, 2)}
    if single_seconds > 0:
        n1 = int(min(T, max(1, single_seconds * n / max(t * cores, 1e-3))))
        oracle.set_threads(1)
        try:
            q1, s1 = run(n1)
        finally:
            oracle.set_threads(cores)
        out["single_thread"] = {"value": q1 / s1, "unit": UNIT, "cores": 1,
                                "sample": f"{n1} of {T} tiles ({q1:.3g} pairs)",
                                "seconds": round(s1, 2)}
    return out


def max_over_ranks(v: float, world: int, device="cpu") -> float:
    """The largest of the ranks' values (the job's time is its slowest rank's)."""
    if world <= 1:
        return v
    import torch
    import torch.distributed as dist
    t = torch.tensor([v], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def job_throughput(pairs_per_rank: float, world: int, total_ms: float) -> float:
    """Whole-job pairs/s of `world` independent replicas (weak scaling: every
    rank evaluates the same workload), timed by the slowest rank."""
    return pairs_per_rank * world / (total_ms / 1e3)


def run_reference(args):
    """The oracle as it stands, timed on the host cores (rank 0 only)."""
    rank = int(os.environ.get("RANK", "0"))
    if rank != 0:
        return
    from paper_2405_20067_gb300 import synth
    c = synth.config1(G=G, Q=Q)
    ch = synth.children(N_DIM, G, 11, spread=0.05, brightness=(0.0009, 0.0011))
    vals = []
    for i in range(args.warmup + args.steps):
        cb = cpu_baseline(c, ch, seconds=5.0)
        if i >= args.warmup:
            vals.append(cb)
    v = statistics.median([cb["value"] for cb in vals])
    cb = dict(vals[-1])
    cb["value"] = v
    out = {"impl": "reference", "metric": METRIC, "value": v, "unit": UNIT,
           "n_gpus": args.gpus, "steps": args.steps, "warmup": args.warmup,
           "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
           "data": "synthetic", "config": {"workload": workload_name(G, Q), "l2": "n/a (host)"},
           "cpu_baseline": cb,
           "e2e": {"value": v, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(out), flush=True)


def run_fit(form: str, steps: int, warmup: int, device: str, flush, world: int, e2e_steps: int,
            bwd_form: str | None = None, graph: bool = False):
    """Times `steps` fit steps of the workload in one form ("tc": lifted
    tensor-core forward; "fp32": plain FP32 forward); backward, cull, loss,
    Adam and the refinement check are shared."""
    import torch
    from paper_2405_20067_gb300 import ndg
    from paper_2405_20067_gb300.train import Trainer
    import torch.distributed as dist
    c, ch, gm, x, target, cp = build_workload(device)
    mode = ndg.NDG_MODE_TC if form == "tc" else ndg.NDG_MODE_FP32
    bmode = ndg.NDG_MODE_TC if (bwd_form or form) == "tc" else ndg.NDG_MODE_FP32
    tr = Trainer(gm, x, target, TILE, cp, lr=1e-3, t=0.01, phase=0, mode=mode, bwd_mode=bmode)
    names = ["build_cull", "forward", "loss", "backward", "adam", "densify"]

    def one_step(traces):
        tr.set_traces(traces)
        tr.step(refine=False)
        tr.refine(sync=False)

    for _ in range(warmup):
        one_step(None)
    torch.cuda.synchronize()
    tr.check()
    # per-kernel times and launch counts: traced eager steps (CUDA events
    # around each call's main kernel on the launching stream), with the
    # backward's order computed inside the backward (not beside the forward),
    # so that each kernel's time is its own and every launch is counted
    ntr = max(3, steps // 4)
    traces = [{n: ndg.Trace() for n in names} for _ in range(ntr)]
    overlap = tr.overlap_order
    tr.overlap_order = False
    for i in range(ntr):
        flush.zero_()
        one_step(traces[i])
    torch.cuda.synchronize()
    tr.overlap_order = overlap
    kern = {n: statistics.mean(tr_[n].ms() for tr_ in traces) for n in names}
    launches_per_step = sum(tr_[n].launches for tr_ in traces for n in names) / ntr
    # the timed steps: the whole step captured once as a CUDA graph and replayed
    if graph:
        tr.capture(refine_each_step=True)
    starts = [torch.cuda.Event(enable_timing=True) for _ in range(steps)]
    ends = [torch.cuda.Event(enable_timing=True) for _ in range(steps)]
    pairs = []
    if world > 1:
        dist.barrier()
    torch.cuda.synchronize()
    eager_ms = []
    with ClockSampler(torch.cuda.current_device()) as clk:
        for i in range(steps):
            flush.zero_()
            starts[i].record()
            if graph:
                tr.replay()
            else:
                one_step(None)
            ends[i].record()
            torch.cuda.synchronize()
            pairs.append(pairs_of(tr.ev.cull, Q, TILE))  # counted outside the timed region
            if graph:
                # the same step launched eagerly, timed the same way right
                # after each replay (untimed for the metric): graph against eager
                flush.zero_()
                e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
                e0.record()
                one_step(None)
                e1.record()
                torch.cuda.synchronize()
                eager_ms.append(e0.elapsed_time(e1))
    torch.cuda.synchronize()
    if world > 1:
        dist.barrier()
    st = tr.check()
    assert st == ndg.NDG_OK, ndg.status_string(st)
    total_ms = max_over_ranks(sum(s.elapsed_time(e) for s, e in zip(starts, ends)), world, device)
    res = {"value": job_throughput(sum(pairs), world, total_ms), "ms_per_step": total_ms / steps,
           "pairs_per_step": statistics.mean(pairs), "candidates_per_step": int(tr.ev.cull.E()),
           "kernels_ms": kern, "gpu_launches": int(round(launches_per_step * steps)),
           "graph": graph, "clocks": clk.summary()}
    if eager_ms:
        res["eager_ms_per_step"] = statistics.mean(eager_ms)
    if e2e_steps:
        xh = x.cpu().pin_memory()
        th = target.cpu().pin_memory()
        e2e_ms = []
        for i in range(e2e_steps + 1):
            flush.zero_()  # the same L2 flush as between the device-timed steps (untimed)
            torch.cuda.synchronize()
            t0 = time.perf_counter()
            loss = tr.step(xh, th, refine=False)
            tr.refine(sync=False)
            float(loss.item())
            e2e_ms.append((time.perf_counter() - t0) * 1e3)
        res["e2e"] = {"value": res["pairs_per_step"] / (statistics.mean(e2e_ms[1:]) / 1e3) * world,
                      "unit": UNIT, "h2d_bytes_per_step": int(xh.numel() * 4 + th.numel() * 4),
                      "d2h_bytes_per_step": 8}
    res["_c"], res["_ch"] = c, ch
    del tr, gm, x, target
    torch.cuda.empty_cache()
    return res


def run_ablation(device) -> dict:
    """The paper's culling ablations in shape (Section 3.2 and its
    evaluation): for an N = 6 fit workload (20,000 Gaussians, 2^18
    Morton-tiled queries) the fixed-k_sigma sweep (average candidates per
    tile, FP32 forward time, largest dropped contribution against the unculled
    evaluation), the contribution-cutoff mode, and culling on / off for
    inference (tensor-core forward) and for training (50 Adam steps)."""
    import torch
    from paper_2405_20067_gb300 import ndg, synth
    from paper_2405_20067_gb300.train import Trainer
    N, Gs, Qs, k = 6, 20_000, 1 << 18, 16
    c = synth.config1(G=Gs, Q=Qs)
    gm = ndg.Mixture.from_arrays(N, c["mix"], G_cap=Gs, device=device)
    x = torch.as_tensor(c["x"]).to(device)
    target = torch.as_tensor(c["target"]).to(device)
    proj = torch.as_tensor(c["proj"]).to(device)
    T = (Qs + TILE - 1) // TILE

    def timed(fn, reps=5):
        for _ in range(2):
            fn()
        torch.cuda.synchronize()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record()
        for _ in range(reps):
            fn()
        e1.record()
        torch.cuda.synchronize()
        return e0.elapsed_time(e1) / reps

    def evaluator(cp):
        ev = ndg.Evaluator(gm, x, TILE, cp, backward=False)
        E = ev.build(gm)
        return ev, E

    dense_cp = ndg.CullParams(0, None, 0.0, 3.0, 1)
    ev_d, E_d = evaluator(dense_cp)
    y_dense = ev_d.forward(gm, mode=ndg.NDG_MODE_FP32).clone()
    ymax = float(y_dense.abs().max())
    rows = []
    settings = [("k_sigma", ks, 0.0) for ks in (1.0, 1.5, 2.0, 2.5, 3.0, 4.0, 5.0)]
    settings.append(("cutoff 1/255", 3.0, CUTOFF))
    for name, ks, cut in settings:
        cp = ndg.CullParams(k, proj, cut, ks, BUCKETS)
        ev, E = evaluator(cp)
        y = ev.forward(gm, mode=ndg.NDG_MODE_FP32)
        drop = float((y_dense - y).abs().max())
        ms = timed(lambda: ev.forward(gm, mode=ndg.NDG_MODE_FP32))
        rows.append({"mode": name, "k_sigma": ks, "cutoff": cut, "avg_candidates": E / T,
                     "fraction_of_dense": E / E_d, "max_dropped": drop,
                     "max_dropped_rel": drop / ymax, "fp32_forward_ms": round(ms, 4)})
    cull_cp = ndg.CullParams(k, proj, CUTOFF, 3.0, BUCKETS)
    ev_c, E_c = evaluator(cull_cp)
    inf = {"tc_forward_ms_culled": round(timed(lambda: ev_c.forward(gm, mode=ndg.NDG_MODE_TC)), 4),
           "tc_forward_ms_dense": round(timed(lambda: ev_d.forward(gm, mode=ndg.NDG_MODE_TC)), 4),
           "cull_build_ms": round(timed(lambda: ev_c.build(gm)), 4)}
    train = {}
    for name, cp in (("culled", cull_cp), ("dense", dense_cp)):
        mix = ndg.Mixture.from_arrays(N, c["mix"], G_cap=Gs, device=device)
        tr = Trainer(mix, x, target, TILE, cp, lr=1e-3, t=0.01, phase=0,
                     mode=ndg.NDG_MODE_TC, bwd_mode=ndg.NDG_MODE_TC)
        first = float(tr.step(refine=False).item())
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        for _ in range(50):
            tr.step(refine=False)
        torch.cuda.synchronize()
        dt = (time.perf_counter() - t0) / 50 * 1e3
        assert tr.check() == ndg.NDG_OK
        train[name] = {"ms_per_step": round(dt, 3), "loss_first": first,
                       "loss_after_50": float(tr.loss.item())}
    # Section 3.2's easy case: the inputs beyond position constant for a frame
    # (N = 10, 500,000 Gaussians, one 1920 x 1080 frame): the cull on all
    # inputs against the cull on position for the Gaussians restricted to
    # the constants
    del ev_d, ev_c
    torch.cuda.empty_cache()
    Nr = RENDER["N"]
    mixr = synth.mixture(Nr, RENDER["G"], 2)
    gr = ndg.Mixture.from_arrays(Nr, mixr, device=device)
    xf = synth.queries_frame(Nr, RENDER["W"], RENDER["H"], 3)
    xcn = synth.rng(5).uniform(-1.0, 1.0, size=Nr - 3).astype(xf.dtype)
    xf[:, 3:] = xcn
    xr = torch.as_tensor(xf).to(device)
    xc = torch.as_tensor(xcn).to(device)
    cpr = ndg.CullParams(RENDER["k"], torch.as_tensor(synth.projections(Nr, RENDER["k"], 4)).to(device),
                         CUTOFF, 3.0, RENDER["buckets"])
    cond = {}
    for name, xcv in (("all inputs", None), ("conditioned on position", xc)):
        ev = ndg.Evaluator(gr, xr, TILE, cpr, E_cap=1 << 24, backward=False)
        E = ev.build(gr, xc=xcv)

        def frame():
            if xcv is None:
                ndg.build_cull(gr, xr, TILE, cpr, ev.cull, ev.ws)
            else:
                ndg.build_cull_conditioned(gr, xr, TILE, cpr, xcv, ev.cull, ev.ws)
            ev.forward(gr, mode=ndg.NDG_MODE_TC)

        cond[name] = {"entries": E, "frame_ms": round(timed(frame, reps=3), 3)}
        del ev
        torch.cuda.empty_cache()
    return {"workload": f"N=6, {Gs} Gaussians, 2^18 Morton-tiled queries, tile {TILE}, k={k}",
            "dense_entries": E_d, "sweep": rows, "inference": inf, "training": train,
            "constant_inputs_frame": {"workload": "N=10, 500,000 Gaussians, 1920 x 1080, "
                                                  "inputs beyond position constant", **cond}}


def run_render_batch(device, n_frames: int = 64) -> dict:
    """Batched render (64 frame specs: G log-uniform in [1e4, 5e5], N in
    {6, 8, 10}, 256^2 .. 1920 x 1080 pixels, one query per pixel, dims beyond
    position uniform), two ways:
    - one frame at a time: per-frame latency of cull + forward (CUDA events,
      one untimed frame first) with the autotuned configuration (median of 5
      timings per candidate on a class's first frame), p50 / p99 over the
      frames, next to the fixed configuration (tensor cores, 256-query
      tiles);
    - all frames at once: every frame's cull, then one persistent launch of
      the tensor-core forward over the (frame, tile) work list
      (ndg_forward_batch).  The device stamps each frame's completion with
      %globaltimer; p50 / p99 of completion since the launch started, the
      makespan, and the whole batch (culls + launch) against the sum of the
      one-at-a-time tensor-core frames.  Every frame's batched output is
      compared with its own ndg_forward output (bit for bit)."""
    import numpy as np
    import torch
    from paper_2405_20067_gb300 import ndg, synth
    from paper_2405_20067_gb300.render import Autotuner, Frame, frame_class, render_batch
    specs = synth.config4_frames(n=n_frames)
    tuner = Autotuner()
    rows, frames = [], []
    for f in specs:
        N, G, W, H, sd = f["N"], f["G"], f["W"], f["H"], f["seed"]
        gm = ndg.Mixture.from_arrays(N, synth.mixture(N, G, sd), device=device)
        x = torch.as_tensor(synth.queries_frame(N, W, H, sd + 1)).to(device)
        proj = torch.as_tensor(synth.projections(N, K_PROJ, sd + 2)).to(device)
        fr = Frame(gm, x, ndg.CullParams(K_PROJ, proj, CUTOFF, 3.0, BUCKETS))
        key = frame_class(N, G, W * H)
        tuned_now = key not in tuner.cache
        cfg = tuner.choose(key, fr.time)
        ms = fr.time(cfg)
        ms_fixed = fr.time(("tc", 256))  # leaves the tensor-core output in fr.y
        fr._ev.pop(128, None)  # keep the 256-query tile state for the batch
        rows.append({"N": N, "G": G, "W": W, "H": H, "config": f"{cfg[0]}/{cfg[1]}",
                     "tuned_here": tuned_now, "ms": round(ms, 4), "ms_tc256": round(ms_fixed, 4),
                     "E": int(fr.evaluator(256).cull.E())})
        frames.append((fr, fr.y.clone()))
    torch.cuda.synchronize()
    ms = np.array([r["ms"] for r in rows])
    fx = np.array([r["ms_tc256"] for r in rows])
    out = {"frames": len(rows), "classes_tuned": len(tuner.cache), "tuner_reps": tuner.reps,
           "candidates": [f"{a}/{b}" for a, b in tuner.candidates],
           "p50_ms": round(float(np.percentile(ms, 50)), 4),
           "p99_ms": round(float(np.percentile(ms, 99)), 4),
           "mean_ms": round(float(ms.mean()), 4),
           "fixed_tc256_p50_ms": round(float(np.percentile(fx, 50)), 4),
           "fixed_tc256_p99_ms": round(float(np.percentile(fx, 99)), 4),
           "pixels": int(sum(r["W"] * r["H"] for r in rows))}
    # ---- all frames in one persistent launch (after their culls)
    frs = [fr for fr, _ in frames]
    bws = ndg.batch_workspace(len(frs), device)
    stamps = torch.zeros(1 + len(frs), dtype=torch.int64, device=device)
    render_batch(frs, bws, stamps)  # untimed
    torch.cuda.synchronize()
    tr = ndg.Trace()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record()
    render_batch(frs, bws, stamps, trace=tr)
    e1.record()
    torch.cuda.synchronize()
    st = stamps.cpu().numpy().astype(np.int64)
    done_ms = (st[1:] - st[0]) / 1e6
    same = all(torch.equal(fr.y, ref) for fr, ref in frames)
    status = [ndg.read_status(fr.evaluator(256).ws) for fr in frs]
    out["batch"] = {
        "launches_forward": 1, "culls": len(frs),
        "total_ms": round(e0.elapsed_time(e1), 3),
        "forward_launch_ms": round(tr.ms(), 3),
        "sum_one_at_a_time_tc256_ms": round(float(fx.sum()), 3),
        "makespan_ms_device": round(float(done_ms.max()), 3),
        "completion_p50_ms_device": round(float(np.percentile(done_ms, 50)), 3),
        "completion_p99_ms_device": round(float(np.percentile(done_ms, 99)), 3),
        "outputs_equal_one_at_a_time": bool(same),
        "status_ok": all(v == ndg.NDG_OK for v in status),
        "entries": int(sum(r["E"] for r in rows))}
    for r, d in zip(rows, done_ms):
        r["batch_done_ms"] = round(float(d), 3)
    out["per_frame"] = rows
    return out


def run_frame_fwd_bwd(device, N: int, G: int, W: int, H: int, steps: int) -> dict:
    """One frame (W x H surface queries, 16 x 16 pixel tiles) against G
    N-dimensional Gaussians: cull once, then `steps` tensor-core forwards and
    backwards (dy fixed), each timed with CUDA events; a small, seeded case
    for profiling the evaluation kernels (S4, S5, S7)."""
    import torch
    from paper_2405_20067_gb300 import ndg, synth
    gm = ndg.Mixture.from_arrays(N, synth.mixture(N, G, 21), device=device)
    x = torch.as_tensor(synth.queries_frame(N, W, H, 22)).to(device)
    cp = ndg.CullParams(K_PROJ, torch.as_tensor(synth.projections(N, K_PROJ, 23)).to(device),
                        CUTOFF, 3.0, BUCKETS)
    ev = ndg.Evaluator(gm, x, TILE, cp)
    E = ev.build(gm)
    dy = torch.as_tensor((synth.rng(24).standard_normal((x.shape[0], 3)) / x.shape[0])
                         .astype("float32")).to(device)
    fwd, bwd = [], []
    for _ in range(steps):
        e0, e1, e2 = (torch.cuda.Event(enable_timing=True) for _ in range(3))
        e0.record()
        ev.forward(gm, mode=ndg.NDG_MODE_TC)
        e1.record()
        ev.backward(gm, dy, mode=ndg.NDG_MODE_TC)
        e2.record()
        torch.cuda.synchronize()
        fwd.append(e0.elapsed_time(e1))
        bwd.append(e1.elapsed_time(e2))
    assert ndg.read_status(ev.ws) == ndg.NDG_OK
    return {"workload": f"N={N} {W}x{H} frame, {G} Gaussians, tile {TILE}, k={K_PROJ}, "
                        "cutoff 1/255", "entries": int(E), "pairs": int(E) * TILE,
            "forward_ms": [round(v, 4) for v in fwd], "backward_call_ms": [round(v, 4) for v in bwd]}


def run_fit_n10(device, steps: int = 5000, pool: int = 8, time_cap_s: float = 540.0) -> dict:
    """The N = 10 fit (config 3 shape): a synthetic ground truth of 2M
    Gaussians drawn as the 10-D recipe, a fitted mixture of 50k parents
    (children at brightness t/10, t = 0.01) that may grow to 1M under the
    Section 3.3 refinement every 300 steps, Adam lr 1e-3, minibatches of 2^18
    surface queries (16 planes x 128^2) cycled from a pool of pre-evaluated
    batches, the whole step captured as a CUDA graph (tensor-core forward and
    backward).  Reports the loss curve, G(t), ms per step and
    the wall time (stopped at time_cap_s)."""
    import torch
    from paper_2405_20067_gb300 import ndg, synth
    from paper_2405_20067_gb300.train import Trainer
    c = synth.config3()
    N = c["N"]
    # contribution cutoff 1/255 with the children's 3-sigma radius floor
    # (Section 3.3): children start at brightness t/10, below the cutoff, and
    # are still evaluated and optimised where they span their parents
    cp = ndg.CullParams(K_PROJ, torch.as_tensor(c["proj"]).to(device), CUTOFF, 3.0, BUCKETS,
                        child_k_min=3.0)
    # pre-evaluated pool: queries on planes, targets from the ground truth
    gt = ndg.Mixture.from_arrays(N, c["gt"], device=device)
    xs, ts = [], []
    for b in range(pool):
        xb = torch.as_tensor(c["x"] if b == 0 else synth.queries_planes(N, 16, 128, 1000 + b)).to(device)
        ev = ndg.Evaluator(gt, xb, TILE, cp, backward=False)
        ev.build(gt)
        ts.append(ev.forward(gt, mode=ndg.NDG_MODE_TC).clone())
        xs.append(xb)
        del ev
    del gt
    torch.cuda.empty_cache()
    mix = ndg.Mixture.from_arrays(N, c["mix"], c["children"], G_cap=c["G_max"], device=device)
    tr = Trainer(mix, xs[0].clone(), ts[0].clone(), TILE, cp, lr=1e-3, t=c["t"], phase=0,
                 mode=ndg.NDG_MODE_TC, bwd_mode=ndg.NDG_MODE_TC)
    tr.capture(refine_each_step=False)
    curve, growth = [], [(0, int(mix.G))]
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    done = 0
    for it in range(1, steps + 1):
        b = it % pool
        tr.x.copy_(xs[b])
        tr.target.copy_(ts[b])
        tr.replay()
        if it % 300 == 0:  # Section 3.3 refinement, then re-capture for the new size
            tr.refine(sync=True)
            growth.append((it, int(tr.mix.G)))
            tr.capture(refine_each_step=False)
        if it % 50 == 0:
            curve.append((it, float(tr.loss.item())))
        done = it
        if time.perf_counter() - t0 > time_cap_s:
            break
    torch.cuda.synchronize()
    wall = time.perf_counter() - t0
    assert tr.check() == ndg.NDG_OK
    return {"workload": "N=10 fit: 2M-Gaussian ground truth, 50k parents -> <= 1M, 2^18-query "
                        f"minibatches from a pool of {pool}, Adam lr 1e-3, refinement every 300 "
                        "steps, cutoff 1/255 with a 3-sigma radius floor for children, "
                        "graph-captured step (tensor-core forward and backward); each "
                        "capture runs two extra warm-up steps",
            "steps": done, "wall_s": round(wall, 2), "ms_per_step": round(wall / done * 1e3, 2),
            "loss_curve": curve, "G": growth}


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=20)
    ap.add_argument("--warmup", type=int, default=5)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-render", action="store_true", help="skip the N=10 1080p render metric")
    ap.add_argument("--no-fp32-form", action="store_true",
                    help="skip timing the plain FP32 form next to the chosen form")
    ap.add_argument("--bwd-form", default="tc", choices=["fp32", "tc"],
                    help="backward of the chosen form (its forward is the tensor-core one)")
    ap.add_argument("--no-graph", action="store_true",
                    help="time eager steps instead of replays of the CUDA-graph-captured step")
    ap.add_argument("--workload", default="fit_n6", choices=sorted(WORKLOADS),
                    help="fit_n6: the headline workload; small_n6: 1/8 of it for profiling")
    ap.add_argument("--render-batch", action="store_true",
                    help="only the batched render of 64 frame specs (autotuned launch "
                         "configuration, p50 / p99 frame latency); one JSON line")
    ap.add_argument("--render-only", metavar="WxH", default=None,
                    help="only the N = 10 render metric at this resolution (e.g. 480x272, a "
                         "small frame for profiling); one JSON line")
    ap.add_argument("--fit-n10", action="store_true",
                    help="only the N = 10 fit with refinement (loss curve, G(t), wall time); "
                         "one JSON line")
    ap.add_argument("--frame-fwd-bwd", metavar="N,G,WxH", default=None,
                    help="only tensor-core forwards and backwards of one seeded frame (e.g. "
                         "10,5000,960x544: a small case for profiling); one JSON line")
    ap.add_argument("--ablation", action="store_true",
                    help="only the culling ablations (k_sigma sweep, culling on / off); one "
                         "JSON line")
    args = ap.parse_args()
    global G, Q
    G, Q = WORKLOADS[args.workload]
    if args.impl == "reference":
        run_reference(args)
        return
    import torch
    import torch.distributed as dist
    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    torch.cuda.set_device(local)
    device = f"cuda:{local}"
    if world > 1:
        dist.init_process_group("nccl", device_id=torch.device(device))
    from paper_2405_20067_gb300 import build
    build.build()
    if args.ablation:
        if rank == 0:
            print(json.dumps({"ablation": run_ablation(device)}))
        return
    if args.render_only:
        w_, h_ = (int(v) for v in args.render_only.lower().split("x"))
        flush = torch.empty(256 << 20, dtype=torch.uint8, device=device)
        if rank == 0:
            print(json.dumps({"render": render_n10_1080p(device, max(3, args.steps // 4), args.warmup,
                                                         flush, res=(w_, h_))}))
        return
    if args.frame_fwd_bwd:
        n_, g_, wh = args.frame_fwd_bwd.split(",")
        w_, h_ = (int(v) for v in wh.lower().split("x"))
        if rank == 0:
            print(json.dumps({"frame_fwd_bwd": run_frame_fwd_bwd(device, int(n_), int(g_), w_, h_,
                                                                 args.steps)}))
        return
    if args.fit_n10:
        if rank == 0:
            print(json.dumps({"fit_n10": run_fit_n10(device, steps=args.steps if args.steps != 20 else 5000)}))
        return
    if args.render_batch:
        if rank == 0:
            print(json.dumps({"render_batch": run_render_batch(device)}))
        return
    peaks, peak_kind = load_peaks()
    from paper_2405_20067_gb300 import ndg as _ndg
    # measured pipe rates of this GPU (ndg_probe_pipe): the MUFU exponential
    # (one per pair in every evaluation kernel) and the FP32 FMA
    probe = {"ex2": _ndg.probe_pipe(0), "ffma": _ndg.probe_pipe(1)}
    flush = torch.empty(256 << 20, dtype=torch.uint8, device=device)  # > 129 MB L2
    chosen = run_fit("tc", args.steps, args.warmup, device, flush, world,
                     max(3, args.steps // 2), bwd_form=args.bwd_form, graph=not args.no_graph)
    plain = None
    if not args.no_fp32_form:
        plain = run_fit("fp32", max(3, args.steps // 2), 3, device, flush, world, 0)
    fwd_f, bwd_f = flops_per_pair(N_DIM)
    alg_fwd, alg_bwd, exe_fwd, exe_bwd = tc_flops_per_pair(N_DIM)
    mean_pairs = chosen["pairs_per_step"]
    kern = chosen["kernels_ms"]
    peak_mhz = float(peaks.get("sm_max_mhz", 2070.0))
    fp32_peak = fp32_peak_tflops(peak_mhz)
    tc_peak = float(peaks.get("bf16_tflops_sustained", peaks.get("bf16_tflops", 1900.0)))
    t_bwd = kern["backward"] / 1e3
    t_fwd = kern["forward"] / 1e3
    kernels = {n: {"ms": round(v, 4)} for n, v in kern.items()}
    if args.bwd_form == "tc":
        achieved = mean_pairs * alg_bwd / t_bwd / 1e12
        executed = mean_pairs * exe_bwd / t_bwd / 1e12
        roofline = {"bound": "tensor", "kernel": f"bwd_h_kernel<{N_DIM}> (tcgen05 kind::f16)",
                    "achieved": round(achieved, 3), "peak": round(tc_peak, 1), "unit": "TFLOP/s",
                    "frac": round(achieved / tc_peak, 4),
                    "traffic": round(BWD_BYTES_PER_ENTRY * chosen["candidates_per_step"]),
                    "peak_source": f"bf16 dense sustained, {peak_kind} (FP16 operands run at "
                                   "the bf16 rate)",
                    "algorithmic": f"{alg_bwd} flop/pair (4F: recompute s, gradient contraction)",
                    "executed_tflops": round(executed, 2),
                    "executed_frac": round(executed / tc_peak, 4),
                    "executed_note": f"{exe_bwd} MMA flop/pair issued: S from FP16 hi/lo (3 "
                                     "products), E Psi from single-FP16 E and hi/lo Psi (2 "
                                     "products) with the colour-blocked Psi operand",
                    "tensor_frac": round(achieved / tc_peak, 4)}
        mufu_frac = mean_pairs / t_bwd / probe["ex2"]["per_s"]
        roofline["mufu"] = {"achieved": mean_pairs / t_bwd, "peak": probe["ex2"]["per_s"],
                            "unit": "ex2/s", "frac": round(mufu_frac, 4),
                            "per_clk_per_sm": round(probe["ex2"]["per_clk_per_sm"], 2),
                            "algorithmic": "1 ex2 per pair",
                            "peak_source": "ndg_probe_pipe(0) in this run (MUFU ex2.approx, "
                                           "all SMs, best of 5)"}
        roofline["binding"] = "mufu" if mufu_frac > roofline["tensor_frac"] else "tensor"
        roofline["binding_frac"] = round(max(mufu_frac, roofline["tensor_frac"]), 4)
    else:
        achieved = mean_pairs * bwd_f / t_bwd / 1e12
        roofline = {"bound": "alu", "kernel": f"bwd_kernel<{N_DIM}> (per-pair partials, FP32 pipe)",
                    "achieved": round(achieved, 3), "peak": round(fp32_peak, 2), "unit": "TFLOP/s",
                    "frac": round(achieved / fp32_peak, 4), "traffic": None,
                    "peak_source": f"152 SMs x 128 FP32 lanes x 2 x {peak_mhz:.0f} MHz "
                                   f"(clock from {peak_kind} peaks file)"}
    kernels["backward"]["form"] = ("tensor-core (tcgen05; S FP16x3, E Psi FP16x2)"
                                   if args.bwd_form == "tc" else "FP32 per-pair partials")
    kernels["backward"]["fp32_equiv_tflops"] = round(mean_pairs * bwd_f / t_bwd / 1e12, 3)
    kernels["forward"]["form"] = "lifted tensor-core (tcgen05 FP16x3)"
    kernels["forward"]["tc_alg_tflops"] = round(mean_pairs * alg_fwd / t_fwd / 1e12, 3)
    kernels["forward"]["tc_executed_tflops"] = round(mean_pairs * exe_fwd / t_fwd / 1e12, 2)
    kernels["forward"]["fp32_equiv_tflops"] = round(mean_pairs * fwd_f / t_fwd / 1e12, 3)
    kernels["forward"]["tensor_frac"] = round(mean_pairs * alg_fwd / t_fwd / 1e12 / tc_peak, 4)
    kernels["forward"]["mufu_frac"] = round(mean_pairs / t_fwd / probe["ex2"]["per_s"], 4)
    if rank != 0:
        return
    out = {"metric": METRIC, "value": chosen["value"], "unit": UNIT, "n_gpus": world,
           "steps": args.steps, "warmup": args.warmup, "ms_per_step": chosen["ms_per_step"],
           "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f32",
           "data": "synthetic",
           "config": {"workload": workload_name(G, Q),
                      "form": f"tensor-core forward + {args.bwd_form} backward",
                      "step": ("one CUDA graph replay (cull, forward, loss, backward, Adam, "
                               "refinement launches)" if chosen["graph"] else "eager launches"),
                      "pairs_per_step": mean_pairs,
                      "candidates_per_step": chosen["candidates_per_step"],
                      "l2": "256 MB buffer written between timed steps (untimed)",
                      "parallelism": f"{world} independent replicas" if world > 1 else "1 GPU"},
           "roofline": roofline, "kernels_ms": kernels, "gpu_launches": chosen["gpu_launches"],
           "e2e": chosen["e2e"], "clocks": chosen["clocks"],
           "eager_ms_per_step": chosen.get("eager_ms_per_step"),
           "pipe_probe": {k: {"per_clk_per_sm": round(v["per_clk_per_sm"], 2),
                              "per_s": v["per_s"]} for k, v in probe.items()}}
    if plain is not None:
        out["fp32_form"] = {"value": plain["value"], "ms_per_step": plain["ms_per_step"],
                            "forward_ms": round(plain["kernels_ms"]["forward"], 4),
                            "speedup_of_chosen": round(chosen["value"] / plain["value"], 3)}
    if not args.no_render and args.workload == "fit_n6":
        out["render"] = render_n10_1080p(device, max(3, args.steps // 4), 2, flush)
    if world == 1 and not args.no_cpu_baseline:
        out["cpu_baseline"] = cpu_baseline(chosen["_c"], chosen["_ch"], single_seconds=5.0)
    print(json.dumps(out), flush=True)
    if world > 1:
        dist.destroy_process_group()


if __name__ == "__main__":
    main()
