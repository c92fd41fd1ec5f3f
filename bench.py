#!/usr/bin/env python
"""Throughput of the object-centric 2DGS training step on GB300.

One step is one pass of the whole hot path over one batch of views:
surfel projection, depth sort, tile binning, tile sort, front-to-back
compositing with the per-Gaussian contribution record, the masked L1 of
Eq. 2 and the background loss of Eq. 1 with their adjoints, the backward
compositing, the chain rule to the parameters and the pruning keep-set with
compaction.  The workload is 500k surfels (SH degree 3) seen by 16 views of
uneven resolution (640x480 / 800x800 / 1024x768 / 1600x1200), synthetic and
seeded.  The metric is pixels per second of the step (Mpix/s), batched (all
16 views in one pass) and per view (16 passes of one view).

    python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference] [--workload c4|c5]

--workload c5 times the full training iteration instead: 1M surfels seen by
64 views of 1600x1200, the same losses and backward, a fused Adam update of
every parameter array and the pruning of the parameters and of both Adam
moments with the same keep-set.

prints one JSON line (rank 0).  With --impl reference the FP64 CPU oracle is
timed instead, on a bounded pixel sample of the same workload.
"""
from __future__ import annotations

import argparse
import json
import math
import os
import re
import statistics
import subprocess
import sys
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

import numpy as np  # noqa: E402

METRIC = "fwd+bwd Mpix/s at 500k surfels, batched vs per-view; % of HBM roofline"
METRIC_C5 = "training-iteration Mpix/s at 1M surfels x 64 views (fwd+bwd, Eq. 3 loss, pruning, Adam)"
UNIT = "Mpix/s"
# Adam learning rates of the c5 iteration: the 3DGS defaults per array scaled by
# 1e-3, so that the timed scene stays stationary over the timed steps (the
# update does the same work at any rate; the parameters here are the activated
# values, which the default rates would push out of range within a few steps)
ADAM_LR = dict(xyz=1.6e-7, quat=1e-6, scale=5e-6, opacity=5e-5, sh=2.5e-6)
GAMMA = 0.5      # background-loss weight (Sec. 5.1)
LAMBDA_DSSIM = 0.2  # D-SSIM share of the 3DGS photometric loss that Eq. 2 masks (training iteration)
ALPHA_DIST = 1000.0  # 2DGS depth-distortion weight of Eq. 3 (bounded scenes)
BETA_NORMAL = 0.05   # 2DGS normal-consistency weight of Eq. 3
TAU = 0.01       # pruning threshold of the sweep configuration
# Algorithmic FP32 operations per evaluated (pixel, Gaussian) pair of the method (an FMA
# counts 2): about 35 in the forward (intersection, rho, alpha, blending) and about 100 in
# the backward (the same evaluation plus the adjoint), the per-unit figures of the roofline
# model; they are fixed, so a kernel that needs fewer instructions shows as a higher rate.
FLOPS_FWD = 35
FLOPS_BWD = 100


def parse_args():
    p = argparse.ArgumentParser(description=__doc__, formatter_class=argparse.RawDescriptionHelpFormatter)
    p.add_argument("--gpus", type=int, default=1)
    p.add_argument("--steps", type=int, default=30)
    p.add_argument("--warmup", type=int, default=3)
    p.add_argument("--impl", choices=("ours", "reference"), default="ours")
    p.add_argument("--workload", choices=("c4", "c5", "ewa"), default="c4",
                   help="c4: 500k surfels x 16 uneven views (the metric's workload); "
                        "c5: training iteration, 1M surfels x 64 views 1600x1200 with Adam; "
                        "ewa: the 3DGS pruning sweep (Appendix B) over the c4 views")
    p.add_argument("--n", type=int, default=None, help="surfels (default 500k for c4, 1M for c5)")
    p.add_argument("--views", type=int, default=None, help="views (default 16 for c4, 64 for c5)")
    p.add_argument("--tile", default="16x16")
    p.add_argument("--persistent", type=int, default=1)
    p.add_argument("--ppt", type=int, default=4, help="pixels per thread")
    p.add_argument("--front", type=float, default=None,
                   help="share of the depth order binned in the first of two passes (0 = one pass; "
                        "default: the library's)")
    p.add_argument("--no-tune", action="store_true",
                   help="time the options given by --tile/--persistent/--ppt/--front/--batch instead of the "
                        "autotuner's choice")
    p.add_argument("--batch", type=int, default=32, help="Gaussians per batch (16, 32 or 64)")
    p.add_argument("--no-cpu-baseline", action="store_true")
    p.add_argument("--no-e2e", action="store_true")
    p.add_argument("--no-per-view", action="store_true")
    p.add_argument("--cpu-sample", type=int, default=1536, help="pixels of the oracle's timed sample")
    p.add_argument("--prune-record", choices=("fused", "graph"), default="fused",
                   help="fused: the contribution record rides on the step's forward; graph: the step renders "
                        "without it and the pruning sweep over the same views runs as the captured CUDA graph")
    a = p.parse_args()
    if a.n is None:
        a.n = 1_000_000 if a.workload == "c5" else 500_000
    if a.views is None:
        a.views = 64 if a.workload == "c5" else 16
    return a


def workload_name(a) -> str:
    if a.workload == "c5":
        return (f"object-centric 2DGS training iteration: {a.n} surfels SH3 (60% object ball r=0.8, 40% shell "
                f"r=2-4), {a.views} hemisphere views 1600x1200 with object masks, masked 0.8 L1 + 0.2 D-SSIM + 1000 L_d + 0.05 L_n + 0.5 L_b, fwd+bwd, "
                f"Adam on all parameters, prune of parameters and moments at tau={TAU}")
    return (f"object-centric 2DGS training step: {a.n} surfels SH3 (70% object ball r=0.8, 30% shell r=2-4), "
            f"{a.views} hemisphere views of uneven resolution, masked L1 + 0.5 L_b, fwd+bwd, prune tau={TAU}")


def metric_name(a) -> str:
    return METRIC if a.workload == "c4" else METRIC_C5


# ----------------------------------------------------------------------------- clocks
class ClockSampler:
    """nvidia-smi samples during the timed region (every 50 ms)."""
    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_index: int, path: str):
        self.path = path
        self.proc = None
        try:
            self.fh = open(path, "w")
            self.proc = subprocess.Popen(["nvidia-smi", f"--query-gpu={self.FIELDS}", "--format=csv,noheader,nounits",
                                          "-lms", "50", "-i", str(gpu_index)], stdout=self.fh,
                                         stderr=subprocess.DEVNULL)
        except (OSError, FileNotFoundError):
            self.proc = None

    def stop(self) -> dict:
        if self.proc is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except subprocess.TimeoutExpired:
            self.proc.kill()
        self.fh.close()
        sm, smax, power, reasons = [], [], [], set()
        names = ("hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap")
        for line in open(self.path):
            f = [x.strip() for x in line.split(",")]
            if len(f) < 9:
                continue
            try:
                sm.append(float(f[1]))
                smax.append(float(f[2]))
                power.append(float(f[3]))
            except ValueError:
                continue
            for name, val in zip(names, f[5:9]):
                if val.lower().startswith("active"):
                    reasons.add(name)
        if not sm:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["no samples"]}
        return {"sm_mhz": statistics.median(sm), "sm_max_mhz": max(smax), "reasons": sorted(reasons),
                "samples": len(sm), "power_w_max": max(power)}


# ----------------------------------------------------------------------------- distributed
def dist_info():
    rank = int(os.environ.get("RANK", "0"))
    world = int(os.environ.get("WORLD_SIZE", "1"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return rank, world, local


def _all_reduce(x: float, world: int, op: str, device=None) -> float:
    if world <= 1:
        return x
    import torch
    import torch.distributed as dist
    t = torch.tensor([x], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX if op == "max" else dist.ReduceOp.SUM)
    return float(t.item())


def max_over_ranks(x: float, world: int, device=None) -> float:
    """The largest x over the ranks: a replicated step is as slow as its slowest rank."""
    return _all_reduce(x, world, "max", device)


def sum_over_ranks(x: float, world: int, device=None) -> float:
    """x summed over the ranks (work units of independent replicas)."""
    return _all_reduce(x, world, "sum", device)


def samples_dir() -> str:
    """Where the raw nvidia-smi clock samples of the timed region go (the JSON line
    carries their summary): $OCGS_BENCH_OUT, else the system temporary directory."""
    import tempfile
    d = os.environ.get("OCGS_BENCH_OUT") or tempfile.gettempdir()
    os.makedirs(d, exist_ok=True)
    return d


def workload_args(a, opts: dict) -> str:
    """The bench arguments that reproduce this workload with launch options ``opts``."""
    tw, th = opts["tile"]
    return (f"--n {a.n} --views {a.views} --tile {tw}x{th} --persistent {int(opts['persistent'])} "
            f"--ppt {opts['pixels_per_thread']} --front {opts['front_fraction']:g} --batch {opts['batch']} --no-tune")


def load_peaks() -> dict:
    path = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(path):
        with open(path) as f:
            d = json.load(f)
        return {"hbm_gbs": d["hbm_gbs"], "sm_max_mhz": d.get("sm_max_mhz", 2070.0), "source": "measured"}
    return {"hbm_gbs": 6800.0, "sm_max_mhz": 2070.0, "source": "fallback"}


# ----------------------------------------------------------------------------- measured DRAM traffic
TRAFFIC_FILE = os.path.join(ROOT, "profiles", "dram_traffic_500k_16views.md")


def sources_digest() -> str:
    """sha256 (first 16 hex digits) over the kernel sources and their build flags."""
    import hashlib
    pkg = os.path.join(ROOT, "paper_2501_08174_gb300")
    csrc = os.path.join(pkg, "csrc")
    files = sorted(os.path.join(csrc, f) for f in os.listdir(csrc) if f.endswith((".cu", ".cuh")))
    files.append(os.path.join(pkg, "build.py"))
    h = hashlib.sha256()
    for path in files:
        h.update(os.path.relpath(path, ROOT).encode())
        with open(path, "rb") as f:
            h.update(f.read())
    return h.hexdigest()[:16]


def measured_traffic(kernel: str, workload_args: str):
    """DRAM bytes (read + write) per launch of `kernel` from the ncu summary in profiles/.

    The summary records the source digest and the bench arguments it was captured
    with; a capture of other sources or another workload gives None."""
    if not os.path.exists(TRAFFIC_FILE):
        return None
    text = open(TRAFFIC_FILE).read()
    dig = re.search(r"^sources-sha256: *(\w+)", text, re.M)
    wl = re.search(r"^workload-args: *(.+?) *$", text, re.M)
    if not dig or not wl or dig.group(1) != sources_digest() or wl.group(1) != workload_args:
        return None
    row = re.search(r"^\| *" + re.escape(kernel) + r" *\|([^\n]*)$", text, re.M)
    if not row:
        return None
    cells = [c.strip() for c in row.group(1).split("|") if c.strip()]
    return int(cells[2])  # columns: read, write, read + write, ...


# ----------------------------------------------------------------------------- roofline model
def algorithmic(stage: str, N: int, V: int, P: int, K: int, T: int, E: int, tile_passes: int, kept: int,
                prune_calls: int = 1, M: int = 0) -> dict:
    """Minimum HBM bytes (and FP32 flops) of each stage for one step (M: records binned in the
    first of two passes, 0 for one pass)."""
    VN = V * N
    if M:
        # front: counts (order, 48 B record, count, ntiles), scan, duplication; behind the front:
        # the open-tile test (order, 16 B box, flag), its scan and compaction, the counts and their
        # scan (the candidates' coverage reads are left out: a lower bound); pairs and tile
        # ranges of both passes, the open flags and their prefix
        binning = (M * (64 + 16 + 60) + (VN - M) * (24 + 12 + 24) + K * 12 + T * 32)
    else:
        # counts (48 B record in, 8 B out), count gather + scan (28 B), duplication (60 B in per
        # record, 8 B out per pair), tile ranges (4 B per pair, 8 B per tile)
        binning = VN * (56 + 28 + 60) + K * 12 + T * 8
    ssim_px = 24 + 1 + 36 + 36 + 24 + 24  # images + mask, adjoint maps out and back, images again, d_rgb
    b = {
        "preprocess": N * 232 + VN * (72 + 4 + 48 + 4),   # record, ntiles, binning record, depth key
        "depth_sort": VN * 4 + 4 * VN * 20,
        "binning": binning,
        "tile_sort": tile_passes * K * 20,
        "raster_fwd": VN * 72 + K * 4 + P * 40,
        "loss": P * (4 + 1 + 8) + P * (12 + 12 + 1 + 24) + (ssim_px * P if prune_calls > 1 else 0),
        "raster_bwd": VN * (72 + 80) + K * 4 + P * 40,
        "preprocess_bwd": N * 232 * 3 + VN * 84,
        "prune": prune_calls * (N * 24 + kept * 232 * 2),
        "adam": N * 232 * 7,  # parameters, gradients, m, v read; parameters, m, v written
    }[stage]
    f = {"raster_fwd": E * FLOPS_FWD, "raster_bwd": E * FLOPS_BWD}.get(stage, 0)
    return {"bytes": b, "flops": f}


# ----------------------------------------------------------------------------- CPU oracle leg
def oracle_sample(g_np, cam, n_pix: int, seed: int = 0):
    rng = np.random.default_rng(seed)
    P = cam["width"] * cam["height"]
    pix = np.sort(rng.choice(P, size=min(n_pix, P), replace=False))
    d_out = dict(rgb=rng.normal(size=(len(pix), 3)), alpha=rng.normal(size=len(pix)),
                 depth=np.zeros(len(pix)), normal=np.zeros((len(pix), 3)))
    return pix, d_out


def time_oracle(sc, n_pix: int) -> dict:
    import torch
    import oracle
    cam = sc["cameras"][0]
    pix, d_out = oracle_sample(sc["gaussians"], cam, n_pix)
    t0 = time.perf_counter()
    oracle.render(sc["gaussians"], cam, pixels=pix, d_out=d_out)
    dt = time.perf_counter() - t0
    return {"value": len(pix) / dt / 1e6, "unit": UNIT, "cores": torch.get_num_threads(), "kind": "oracle",
            "sample": f"fwd+bwd (FP64 autograd) of {len(pix)} seeded pixels of view 0 ({cam['width']}x{cam['height']}) "
                      f"over all {len(sc['gaussians']['opacity'])} surfels; {dt:.1f} s"}


def run_reference(a, rank: int, world: int):
    if rank != 0:
        return
    import synthetic
    import torch
    sc = synthetic.config5(n=a.n, n_views=a.views) if a.workload == "c5" else synthetic.config4(n=a.n, n_views=a.views)
    n_pix = max(16, a.cpu_sample // 6)
    times = []
    for i in range(a.warmup + a.steps):
        cam = sc["cameras"][i % len(sc["cameras"])]
        pix, d_out = oracle_sample(sc["gaussians"], cam, n_pix, seed=i)
        t0 = time.perf_counter()
        import oracle
        oracle.render(sc["gaussians"], cam, pixels=pix, d_out=d_out)
        if i >= a.warmup:
            times.append(time.perf_counter() - t0)
    ms = 1e3 * sum(times) / len(times)
    value = n_pix / (ms / 1e3) / 1e6
    cores = torch.get_num_threads()
    line = {"impl": "reference", "metric": metric_name(a), "value": value, "unit": UNIT, "n_gpus": a.gpus,
            "steps": a.steps, "warmup": a.warmup, "ms_per_step": ms, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
            "config": {"workload": workload_name(a), "sample": f"{n_pix} pixels of one view per step"},
            "cpu_baseline": {"value": value, "unit": UNIT, "cores": cores, "kind": "oracle",
                             "sample": f"FP64 oracle fwd+bwd of {n_pix} seeded pixels of one view per step"},
            "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)


# ----------------------------------------------------------------------------- GPU step
class TrainingStep:
    """One training step through the library (all arithmetic in libocgs kernels)."""

    def __init__(self, rast, g, cams, target, mask, per_view: bool, adam: bool = False, graph=None):
        import torch
        from paper_2501_08174_gb300 import pixel_offsets
        self.rast, self.g, self.cams, self.target, self.mask = rast, g, cams, target, mask
        self.per_view = per_view
        self.adam = adam
        self.graph = graph  # the pruning sweep as a captured graph (the forward then keeps no record)
        self.t = 0
        if adam:
            self.m = {k: torch.zeros_like(v) for k, v in g.items()}
            self.v = {k: torch.zeros_like(v) for k, v in g.items()}
        self.off = pixel_offsets(cams)
        P = self.off[-1]
        dev = g["xyz"].device
        self.d_rgb = torch.zeros(P, 3, device=dev)
        self.d_alpha = torch.zeros(P, device=dev)
        if adam:  # cotangents of the planes the Eq. 3 regularisers read
            self.d_depth = torch.zeros(P, device=dev)
            self.d_depth2 = torch.zeros(P, device=dev)
            self.d_normal = torch.zeros(P, 3, device=dev)
        self.grads = {k: torch.zeros_like(v) for k, v in g.items()}
        self.score = graph.score if graph is not None else torch.zeros(g["opacity"].shape[0], device=dev)
        self.loss = torch.zeros(2, len(cams), dtype=torch.float64, device=dev)
        self.kept = 0

    def _views(self, cams, lo, hi):
        r = self.rast
        out, st = r.render(self.g, cams, score=None if self.graph is not None else self.score, depth2=self.adam)
        tgt = self.target[lo:hi]
        msk = self.mask[lo:hi]
        d_rgb, d_alpha = self.d_rgb[lo:hi], self.d_alpha[lo:hi]
        cot = {"rgb": d_rgb, "alpha": d_alpha}
        if self.adam:  # Eq. 3 in full: L_c^M ((1 - lambda) L1 + lambda D-SSIM) + alpha L_d + beta L_n + gamma L_b
            l1 = r.masked_l1(out["rgb"], tgt, msk, cams, weight=1.0 - LAMBDA_DSSIM, d_rgb=d_rgb)
            r.ssim(out["rgb"], tgt, msk, cams, weight=LAMBDA_DSSIM, d_rgb=d_rgb)
            cot.update(depth=self.d_depth[lo:hi], depth2=self.d_depth2[lo:hi], normal=self.d_normal[lo:hi])
            r.depth_distortion(out["alpha"], out["depth"], out["depth2"], cams, weight=ALPHA_DIST,
                               grads={"alpha": d_alpha, "depth": cot["depth"], "depth2": cot["depth2"]})
            r.normal_consistency(out["alpha"], out["depth"], out["normal"], cams, weight=BETA_NORMAL,
                                 grads={"alpha": d_alpha, "depth": cot["depth"], "normal": cot["normal"]})
        else:
            l1 = r.masked_l1(out["rgb"], tgt, msk, cams, weight=1.0, d_rgb=d_rgb)
        lb = r.background_loss(out["alpha"], msk, cams, gamma=GAMMA, d_alpha=d_alpha)
        r.render_backward(st, self.g, cot, grads=self.grads)
        st.release()
        return l1, lb

    def __call__(self):
        if self.graph is None:
            self.score.zero_()
        self.d_rgb.zero_()
        self.d_alpha.zero_()
        if self.adam:
            self.d_depth.zero_()
            self.d_depth2.zero_()
            self.d_normal.zero_()
        for v in self.grads.values():
            v.zero_()
        if self.per_view:
            for i, cam in enumerate(self.cams):
                l1, lb = self._views([cam], self.off[i], self.off[i + 1])
                self.loss[0, i:i + 1].copy_(l1)
                self.loss[1, i:i + 1].copy_(lb)
        else:
            l1, lb = self._views(self.cams, 0, self.off[-1])
            self.loss[0].copy_(l1)
            self.loss[1].copy_(lb)
        if self.graph is not None:
            self.graph.launch()  # zeroes the score and sweeps every view
        if self.adam:
            self.t += 1
            self.rast.adam_step(self.g, self.grads, self.m, self.v, ADAM_LR, step=self.t)
        kept, _, _ = self.rast.prune(self.g, self.score, TAU)
        if self.adam:  # the moments follow the parameters through the keep-set
            self.rast.prune(self.m, self.score, TAU)
            self.rast.prune(self.v, self.score, TAU)
        self.kept = kept["xyz"].shape[0]


class E2EPipeline:
    """Training steps through the public API with host buffers, double-buffered as a data
    loader would run them: while step i computes on one set of device inputs, a copy stream
    uploads step i+1's parameters, target image and mask from pinned host memory into the
    other set and downloads step i's gradients and losses once step i is done.  Every step
    does its full upload and download; the caller's final device synchronisation (and its
    wall clock) covers the last download."""

    def __init__(self, rast, cams, pin, tgt_h, msk_h, adam: bool, dev):
        import torch
        self.pin, self.tgt_h, self.msk_h = pin, tgt_h, msk_h
        self.sets = []
        for _ in range(2):
            g = {k: torch.empty(v.shape, dtype=v.dtype, device=dev) for k, v in pin.items()}
            target = torch.empty(tgt_h.shape, dtype=tgt_h.dtype, device=dev)
            mask = torch.empty(msk_h.shape, dtype=msk_h.dtype, device=dev)
            self.sets.append((g, target, mask, TrainingStep(rast, g, cams, target, mask, per_view=False, adam=adam)))
        self.grads_h = [{k: torch.empty_like(v).pin_memory() for k, v in pin.items()} for _ in range(2)]
        self.loss_h = [torch.empty(2, len(cams), dtype=torch.float64).pin_memory() for _ in range(2)]
        self.cs = torch.cuda.Stream(dev)
        self.copied = [torch.cuda.Event() for _ in range(2)]
        self.computed = [torch.cuda.Event() for _ in range(2)]
        self.consumed = [torch.cuda.Event() for _ in range(2)]  # inputs used and results downloaded
        self.i = 0

    def _upload(self, b):
        import torch
        g, target, mask, _ = self.sets[b]
        with torch.cuda.stream(self.cs):
            self.cs.wait_event(self.consumed[b])
            for k in g:
                g[k].copy_(self.pin[k], non_blocking=True)
            target.copy_(self.tgt_h, non_blocking=True)
            mask.copy_(self.msk_h, non_blocking=True)
            self.copied[b].record(self.cs)

    def _download(self, b):
        import torch
        st = self.sets[b][3]
        with torch.cuda.stream(self.cs):
            self.cs.wait_event(self.computed[b])
            for k in st.grads:
                self.grads_h[b][k].copy_(st.grads[k], non_blocking=True)
            self.loss_h[b].copy_(st.loss, non_blocking=True)
            self.consumed[b].record(self.cs)

    def __call__(self):
        import torch
        b = self.i % 2
        if self.i == 0:
            self._upload(0)
        self._upload(1 - b)  # the next step's inputs, once the previous user of that set is done
        main = torch.cuda.current_stream()
        main.wait_event(self.copied[b])
        self.sets[b][3]()
        self.computed[b].record(main)
        self._download(b)
        self.i += 1


def timed(step, k: int, warmup: int, world: int, dev, sampler_path=None, gpu_index=0):
    import torch
    import torch.distributed as dist
    for _ in range(warmup):
        step()
    torch.cuda.synchronize(dev)
    if world > 1:
        dist.barrier()
    sampler = ClockSampler(gpu_index, sampler_path) if sampler_path else None
    s = torch.cuda.current_stream(dev)
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    t0 = time.perf_counter()
    e0.record(s)
    for _ in range(k):
        step()
    e1.record(s)
    torch.cuda.synchronize(dev)
    wall = time.perf_counter() - t0
    if world > 1:
        dist.barrier()
    clocks = sampler.stop() if sampler else None
    ms = max_over_ranks(e0.elapsed_time(e1) / k, world, dev)
    return ms, max_over_ranks(wall / k * 1e3, world, dev), clocks


def run_ours(a, rank: int, world: int, local: int):
    import torch
    import torch.distributed as dist

    import synthetic
    from paper_2501_08174_gb300 import FRONT_FRACTION, Rasterizer, n_pixels

    dev = torch.device("cuda", local)
    torch.cuda.set_device(dev)
    if world > 1:
        dist.init_process_group("nccl", device_id=dev)
    out_dir = samples_dir()

    if a.workload == "c5":
        sc = synthetic.config5(seed=5 + rank, n=a.n, n_views=a.views)
    else:
        sc = synthetic.config4(seed=4 + rank, n=a.n, n_views=a.views)
    cams = sc["cameras"]
    P = n_pixels(cams)
    P_job = int(sum_over_ranks(P, world, dev))  # pixels of one step over all replicas
    g_np = sc["gaussians"]
    N = len(g_np["opacity"])
    rng = np.random.default_rng(40 + rank)
    target_np = rng.uniform(0.0, 1.0, size=(P, 3)).astype(np.float32)
    mask_np = np.concatenate([m.reshape(-1) for m in sc["masks"]]).astype(np.uint8)
    g = {k: torch.tensor(np.asarray(g_np[k], np.float32), device=dev) for k in ("xyz", "quat", "scale", "opacity", "sh")}
    target = torch.tensor(target_np, device=dev)
    mask = torch.tensor(mask_np, device=dev)
    tw, th = (int(x) for x in a.tile.split("x"))
    rast = Rasterizer(dev, tile=(tw, th), persistent=bool(a.persistent), pixels_per_thread=a.ppt,
                      front_fraction=FRONT_FRACTION if a.front is None else a.front, batch=a.batch)
    tuned = None
    if not a.no_tune:
        # the autotuner picks the launch options of the timed step (they never change a result)
        tuned = rast.autotune(g, cams, cache_path=os.path.join(out_dir, "autotune_cache.txt"))
    opts = rast.options()

    # sizes of the workload (outside the timed region)
    _, st = rast.render(g, cams)
    info = st.info()
    st.release()
    K, E, T = info["n_pairs"], info["n_evals"], info["n_tiles"]
    tile_bits = max(1, math.ceil(math.log2(max(T, 2))))
    tile_passes = (tile_bits + 7) // 8
    front = rast.front_fraction if rast.persistent else 0.0
    M = min(N * len(cams), max(1, math.ceil(front * N * len(cams)))) if front > 0 else 0

    # batched step, with the library's stage timers on
    adam = a.workload == "c5"
    graph = rast.contribution_graph(g, cams) if a.prune_record == "graph" else None
    step = TrainingStep(rast, g, cams, target, mask, per_view=False, adam=adam, graph=graph)
    for _ in range(a.warmup):
        step()
    rast.profile(True)
    launches0 = rast.kernel_launches()
    ms, wall_ms, clocks = timed(step, a.steps, 0, world, dev, os.path.join(out_dir, f"clocks_rank{rank}.csv"), local)
    launches = rast.kernel_launches() - launches0
    prof = rast.profile_read()
    rast.profile(False)
    kept = step.kept

    per_view = None
    if not a.no_per_view:
        pstep = TrainingStep(rast, g, cams, target, mask, per_view=True, adam=adam)
        pms, pwall, _ = timed(pstep, a.steps, a.warmup, world, dev)
        per_view = {"ms_per_step": pms, "value": P_job / (pms / 1e3) / 1e6,
                    "launch_sets": len(cams), "batched_speedup": pms / ms,
                    "front_fraction": rast.front_fraction if rast.persistent else 0.0}
        if rast.persistent and rast.front_fraction > 0:
            # the same per-view step with one-pass binning: no host read of the second pass's
            # pair count in the middle of each one-view render
            rast.set_options(**dict(opts, front_fraction=0.0))
            oms, _, _ = timed(pstep, a.steps, a.warmup, world, dev)
            rast.set_options(**opts)
            per_view["one_pass"] = {"ms_per_step": oms, "value": P_job / (oms / 1e3) / 1e6,
                                    "batched_speedup": oms / ms, "front_fraction": 0.0}

    # roofline of the dominant stage and of the whole step
    peaks = load_peaks()
    n_sm = torch.cuda.get_device_properties(dev).multi_processor_count
    fp32_peak = n_sm * 128 * 2 * peaks["sm_max_mhz"] * 1e6 / 1e12  # TFLOP/s: SMs x FP32 lanes x FMA x clock
    stages = {}
    step_bytes = 0
    for name, (tot_ms, cnt) in prof.items():
        if cnt == 0:
            continue  # a stage this workload does not run
        alg = algorithmic(name, N, len(cams), P, K, T, E, tile_passes, kept, 3 if adam else 1, M)
        step_bytes += alg["bytes"]
        per_ms = tot_ms / a.steps
        stages[name] = {"ms": per_ms, "launch_sets": cnt / a.steps,
                        "gbs": alg["bytes"] / (per_ms * 1e-3) / 1e9 if per_ms > 0 else None,
                        "tflops": (alg["flops"] / (per_ms * 1e-3) / 1e12) if alg["flops"] and per_ms > 0 else None}
    dom = max(stages, key=lambda k: stages[k]["ms"])
    dstage = stages[dom]
    per_launch_ms = prof[dom][0] / max(prof[dom][1], 1)
    alg = algorithmic(dom, N, len(cams), P, K, T, E, tile_passes, kept, 3 if adam else 1, M)
    stage_kernel = {"raster_fwd": "raster_fwd_kernel", "raster_bwd": "raster_bwd_kernel",
                    "preprocess": "preprocess_kernel", "preprocess_bwd": "preprocess_bwd_kernel"}
    traffic = None
    if dom in stage_kernel:
        traffic = measured_traffic(stage_kernel[dom], workload_args(a, opts))
    if alg["flops"]:
        ach = alg["flops"] / (per_launch_ms * 1e-3) / 1e12
        roofline = {"kernel": dom, "bound": "alu", "achieved": ach, "peak": fp32_peak, "unit": "TFLOP/s",
                    "frac": ach / fp32_peak, "traffic": traffic,
                    "peak_source": f"{n_sm} SMs (queried) x 128 FP32 lanes x 2 x {peaks['sm_max_mhz']:.0f} MHz "
                                   f"(maximum SM clock, {peaks['source']})"}
    else:
        ach = alg["bytes"] / (per_launch_ms * 1e-3) / 1e9
        roofline = {"kernel": dom, "bound": "hbm", "achieved": ach, "peak": peaks["hbm_gbs"], "unit": "GB/s",
                    "frac": ach / peaks["hbm_gbs"], "traffic": traffic, "peak_source": peaks["source"]}
    hbm_step = {"bytes_per_step": step_bytes, "achieved_gbs": step_bytes / (ms * 1e-3) / 1e9,
                "peak_gbs": peaks["hbm_gbs"], "frac": step_bytes / (ms * 1e-3) / 1e9 / peaks["hbm_gbs"],
                "mpix_s_at_roofline": P / (step_bytes / (peaks["hbm_gbs"] * 1e9)) / 1e6}

    # end to end through the public API with host buffers
    e2e = None
    if not a.no_e2e:
        pin = {k: v.cpu().pin_memory() for k, v in g.items()}
        tgt_h = torch.tensor(target_np).pin_memory()
        msk_h = torch.tensor(mask_np).pin_memory()
        pipe = E2EPipeline(rast, cams, pin, tgt_h, msk_h, adam, dev)
        ems, ewall, _ = timed(pipe, a.steps, 1, world, dev)
        h2d = sum(v.numel() * v.element_size() for v in pin.values()) + tgt_h.numel() * 4 + msk_h.numel()
        d2h = sum(v.numel() * v.element_size() for v in pipe.grads_h[0].values()) + pipe.loss_h[0].numel() * 8
        e2e = {"value": P_job / (max(ems, ewall) / 1e3) / 1e6, "unit": UNIT, "h2d_bytes_per_step": int(h2d),
               "d2h_bytes_per_step": int(d2h), "ms_per_step": max(ems, ewall),
               "overlap": "double-buffered: step i+1's upload and step i-1's download run on a copy "
                          "stream during step i"}
        del pipe

    cpu = None
    if rank == 0 and world == 1 and not a.no_cpu_baseline:
        cpu = time_oracle(sc, a.cpu_sample)

    if rank == 0:
        line = {"metric": metric_name(a), "value": P_job / (ms / 1e3) / 1e6, "unit": UNIT, "n_gpus": world,
                "steps": a.steps, "warmup": a.warmup, "ms_per_step": ms, "higher_is_better": True,
                "scaling": "weak", "vs_baseline": None, "dtype": "f32", "data": "synthetic",
                "config": {"workload": workload_name(a), "mode": "batched (one pass over all views)",
                           "prune_record": ("fused into the step's forward" if a.prune_record == "fused" else
                                            "captured CUDA-graph sweep over the step's views"),
                           "n_gaussians": N, "n_views": len(cams), "pixels_per_gpu": P,
                           "resolutions": [f"{c['width']}x{c['height']}" for c in cams],
                           "tile": f"{opts['tile'][0]}x{opts['tile'][1]}",
                           "pixels_per_thread": opts["pixels_per_thread"], "persistent": opts["persistent"],
                           "front_fraction": front, "gaussians_per_batch": opts["batch"],
                           "options_from": "autotuner" if tuned else "command line",
                           "autotune": tuned, "pairs": K, "evals": E,
                           "l2": f"inputs larger than L2: {step_bytes / 1e9:.1f} GB algorithmic traffic per step",
                           "parallelism": f"replicas x{world}" if world > 1 else "1 GPU"},
                "per_view": per_view, "stages": stages, "roofline": roofline, "hbm_roofline_step": hbm_step,
                "cpu_baseline": cpu, "e2e": e2e, "clocks": clocks, "gpu_launches": int(launches),
                "wall_ms_per_step": wall_ms, "kept_after_prune": kept}
        print(json.dumps(line), flush=True)
    rast.close()
    if world > 1:
        dist.destroy_process_group()


METRIC_EWA = "3DGS pruning-sweep Mpix/s at 500k Gaussians x 16 views (EWA forward + contribution record)"


def run_ewa(a, rank: int, world: int, local: int):
    """The 3DGS variant of the pruning record (Appendix B): the contribution sweep of
    500k 3D Gaussians (config 4's scene with a third scale axis) over config 4's views."""
    import torch
    import torch.distributed as dist

    import synthetic
    from paper_2501_08174_gb300 import FRONT_FRACTION, Rasterizer, n_pixels

    dev = torch.device("cuda", local)
    torch.cuda.set_device(dev)
    if world > 1:
        dist.init_process_group("nccl", device_id=dev)
    sc = synthetic.config4(seed=4 + rank, n=a.n, n_views=a.views)
    cams = sc["cameras"]
    P = n_pixels(cams)
    P_job = int(sum_over_ranks(P, world, dev))
    rng = np.random.default_rng(44 + rank)
    g_np = dict(sc["gaussians"])
    third = np.exp(rng.uniform(np.log(0.01), np.log(0.1), size=(a.n, 1)))
    g_np["scale"] = np.concatenate([np.asarray(g_np["scale"], np.float64), third], 1)
    g = {k: torch.tensor(np.asarray(g_np[k], np.float32), device=dev) for k in ("xyz", "quat", "scale", "opacity", "sh")}
    tw, th = (int(x) for x in a.tile.split("x"))
    rast = Rasterizer(dev, tile=(tw, th), persistent=bool(a.persistent), pixels_per_thread=a.ppt,
                      front_fraction=FRONT_FRACTION if a.front is None else a.front)
    score = torch.zeros(a.n, device=dev)

    def step():
        score.zero_()
        rast.accumulate_contribution_3d(g, cams, score)

    for _ in range(a.warmup):
        step()
    rast.profile(True)
    launches0 = rast.kernel_launches()
    out_dir = samples_dir()
    ms, wall_ms, clocks = timed(step, a.steps, 0, world, dev, os.path.join(out_dir, f"clocks_rank{rank}.csv"), local)
    launches = rast.kernel_launches() - launches0
    prof = rast.profile_read()
    rast.profile(False)
    kept = int((score > TAU).sum())
    if rank == 0:
        stages = {k: {"ms": v[0] / a.steps, "launch_sets": v[1] / a.steps} for k, v in prof.items() if v[1] > 0}
        line = {"metric": METRIC_EWA, "value": P_job / (ms / 1e3) / 1e6, "unit": UNIT, "n_gpus": world,
                "steps": a.steps, "warmup": a.warmup, "ms_per_step": ms, "higher_is_better": True,
                "scaling": "weak", "vs_baseline": None, "dtype": "f32", "data": "synthetic",
                "config": {"workload": f"3DGS pruning sweep: {a.n} Gaussians SH3, {a.views} hemisphere views of "
                                       f"uneven resolution, EWA forward with the contribution record",
                           "pixels_per_gpu": P, "tile": a.tile, "pixels_per_thread": a.ppt,
                           "parallelism": f"replicas x{world}" if world > 1 else "1 GPU"},
                "stages": stages, "clocks": clocks, "gpu_launches": int(launches), "wall_ms_per_step": wall_ms,
                "kept_at_tau": kept}
        print(json.dumps(line), flush=True)
    rast.close()
    if world > 1:
        dist.destroy_process_group()


def main():
    a = parse_args()
    rank, world, local = dist_info()
    if a.impl == "reference":
        run_reference(a, rank, world)
        return
    if a.workload == "ewa":
        run_ewa(a, rank, world, local)
        return
    run_ours(a, rank, world, local)


if __name__ == "__main__":
    main()
