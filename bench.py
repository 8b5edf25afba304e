#!/usr/bin/env python
"""Throughput of the differentiable ERP Gaussian rasterizer on one GB300 (and N replicas).

One step = one forward + backward iteration of the whole hot path on the headline workload:
1M Gaussians (SH degree 3, 20% near the poles, 20% on the longitude seam), one 2048x1024 ERP
view: preprocess -> depth sort + tile binning + tile sort -> forward blend -> L1 loss against a
noise target (torch) -> backward blend -> chain rule to all parameter gradients.

Prints ONE JSON line (rank 0). ``--impl reference`` times the FP64 CPU oracle on bounded pixel
samples of the same workload instead (the CPU baseline; it never touches the GPU).
Under torchrun (N > 1) every rank runs an independent replica of the workload (weak scaling; the
path has no data exchange between frames) and rank 0 reports the whole-job rate.
"""
from __future__ import annotations

import argparse
import json
import os
import subprocess
import sys
import threading
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "ERP fwd+bwd iter/s at 1M Gaussians 2048×1024 (1 GB300); batched views/s vs single"
UNIT = "iter/s"
WORKLOAD = "config2: 1,000,000 Gaussians (SH3; 20% within 10 deg of the poles, 20% within 5 deg of the seam), " \
           "one 2048x1024 ERP view, fwd+bwd with L1 loss"
CPU_SAMPLE_PIXELS = 8192  # about 10-15 s of oracle work on 16 cores


def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=200)
    ap.add_argument("--warmup", type=int, default=5)
    ap.add_argument("--impl", choices=["ours", "reference"], default="ours")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-e2e", action="store_true")
    ap.add_argument("--n", type=int, default=1_000_000, help="Gaussians (headline: 1M)")
    ap.add_argument("--width", type=int, default=2048)
    ap.add_argument("--tile", type=str, default="16x16")
    ap.add_argument("--batch", type=int, default=128)
    ap.add_argument("--ppt", type=int, default=0, help="pixels per thread in the forward blend (0 = auto)")
    ap.add_argument("--ppt-bwd", type=int, default=0, help="pixels per thread in the backward blend (0 = auto)")
    ap.add_argument("--no-batched", action="store_true", help="skip the 16-view batched measurement")
    ap.add_argument("--no-large", action="store_true", help="skip the 8 x 4096x2048 roaming-scale measurement")
    ap.add_argument("--batched-steps", type=int, default=10)
    ap.add_argument("--no-next", action="store_true", help="skip the measurements of the steps after the hot path")
    return ap.parse_args()


# ------------------------------------------------------------------ clocks

class ClockSampler:
    FIELDS = ["clocks.sm", "clocks.max.sm", "power.draw", "clocks_event_reasons.active",
              "clocks_event_reasons.hw_slowdown", "clocks_event_reasons.hw_thermal_slowdown",
              "clocks_event_reasons.sw_thermal_slowdown", "clocks_event_reasons.sw_power_cap"]

    def __init__(self, gpu_id: str):
        self.gpu_id = gpu_id
        self.proc = None
        self.lines = []

    def start(self):
        try:
            self.proc = subprocess.Popen(["nvidia-smi", "-i", self.gpu_id, "--query-gpu=" + ",".join(self.FIELDS),
                                          "--format=csv,noheader,nounits", "-lms", "100"],
                                         stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
            self.t = threading.Thread(target=self._read, daemon=True)
            self.t.start()
        except Exception:
            self.proc = None

    def _read(self):
        for line in self.proc.stdout:
            self.lines.append(line.strip())

    def stop(self):
        if self.proc is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        time.sleep(0.25)
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except Exception:
            self.proc.kill()
        return summarise_clocks(self.lines)


def summarise_clocks(lines):
    """Median and lowest SM clock, the maximum, the throttle reasons seen active and the peak
    power of ``nvidia-smi --format=csv,noheader,nounits`` lines of ``ClockSampler.FIELDS``."""
    sm, smax, reasons, power = [], [], set(), []
    names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
    for ln in lines:
        parts = [p.strip() for p in ln.split(",")]
        if len(parts) < 8:
            continue
        try:
            sm.append(float(parts[0]))
            smax.append(float(parts[1]))
            power.append(float(parts[2]))
        except ValueError:
            continue
        for nm, val in zip(names, parts[4:8]):
            if val.lower().startswith("active"):
                reasons.add(nm)
    if not sm:
        return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["no samples"]}
    sm.sort()
    return {"sm_mhz": sm[len(sm) // 2], "sm_min_mhz": sm[0], "sm_max_mhz": max(smax), "reasons": sorted(reasons),
            "samples": len(sm), "power_w_max": max(power) if power else None}


def _gpu_id(torch, dev):
    try:
        u = str(torch.cuda.get_device_properties(dev).uuid)
        return u if u.startswith("GPU-") else "GPU-" + u
    except Exception:
        return str(dev)


def _peaks():
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
            return json.load(f), "measured"
    except Exception:
        return {"hbm_gbs": 6800.0, "sm_max_mhz": 2070.0}, "fallback"


# ------------------------------------------------------------------ algorithmic work

# FP32 flops (FMA = 2) per (pixel, list entry) of the blend, as the method needs them:
#   every tested entry: pixel offset (2), quadratic form of Eq. 2 with log-opacity (8), test (1)
#   every blended entry, forward: exp (1), clamp (1), 1 - alpha (1), T' (1), test (1), alpha T (1),
#                                 colour accumulation (6)
#   every blended entry, backward: exp, clamp, 1 - alpha, T recovery, weight (5), rgb.g (5),
#                                 dL/dalpha (3), B update (2), dL/drgb (3), dL/dpower (1),
#                                 dL/do (1), dL/dconic (6), dL/d(u, v) (8)
FLOP_TESTED = 11
FLOP_BLEND_FWD = 12
FLOP_BLEND_BWD = 34


def fp32_peak_tflops(torch, dev, peaks):
    sms = torch.cuda.get_device_properties(dev).multi_processor_count
    mhz = float(peaks.get("sm_max_mhz", 2070.0))
    return sms * 128 * 2 * mhz * 1e6 / 1e12, sms, mhz


# Algorithmic bytes of the HBM-bound stages (each byte the stage must move once):
#   preprocess     per Gaussian its parameters (means 12, scales 12, quats 16, opacity 4, SH 48 x
#                  4 at degree 3 = 236 B); per visible item its record (ERP mean 8, conic 12,
#                  opacity 4, colour 12, depth key 4, tile rectangle 12 = 52 B)
#   bin_sort       per item: four 8-bit depth-sort passes over key + value (16 B each) and the
#                  digit counts' read of the keys (4 B); the pair count and the emission read the
#                  sorted index and the rectangle twice (40 B); the saturation bound's read of
#                  the rectangle and the conic (32 B); the sorted key read and the kept-pair word
#                  written and read (12 B). Per sorted pair (the kept prefixes of the tile lists):
#                  its key + value written (8 B), each tile-sort pass (16 B), the range scan's
#                  read of the key (4 B). Per tile its range (8 B) and its 32 depth-bucket sums
#                  and prefix counts zeroed, written and read (3 x 128 B)
#   preprocess_bwd per Gaussian its parameters read and their gradients written (2 x 236 B); per
#                  visible item the 9 accumulated screen-space gradients (36 B)
def param_bytes(sh_degree):
    return 4 * (3 + 3 + 4 + 1 + 3 * (sh_degree + 1) ** 2)


RECORD_BYTES = 52
ACC_BYTES = 36


def stage_rooflines(kern, stats, n, sh_degree, tiles, pair_passes, hbm_gbs, alu_tflops, alu_measured,
                    ex2_measured=None):
    items, vis, pairs = n, stats["visible"], stats["pairs_sorted"]
    hbm = {
        "preprocess": n * param_bytes(sh_degree) + vis * RECORD_BYTES,
        "bin_sort": items * (4 * 16 + 4 + 40 + 32 + 12) + pairs * (8 + 16 * pair_passes + 4) + tiles * (8 + 3 * 128),
        "preprocess_bwd": n * 2 * param_bytes(sh_degree) + vis * ACC_BYTES,
    }
    alu = {
        "render_fwd": FLOP_TESTED * stats["evals_fwd"] + FLOP_BLEND_FWD * stats["blended"],
        "render_bwd": FLOP_TESTED * stats["evals_bwd"] + FLOP_BLEND_BWD * stats["blended"],
    }
    out = {}
    for k, b in hbm.items():
        gbs = b / (kern[k] * 1e-3) / 1e9
        out[k] = {"ms": kern[k], "bound": "hbm", "bytes": b, "achieved": gbs, "unit": "GB/s", "peak": hbm_gbs,
                  "frac": gbs / hbm_gbs}
    for k, f in alu.items():
        tf = f / (kern[k] * 1e-3) / 1e12
        out[k] = {"ms": kern[k], "bound": "alu", "flops": f, "achieved": tf, "unit": "TFLOP/s", "peak": alu_tflops,
                  "frac": tf / alu_tflops}
        if alu_measured:
            out[k]["frac_of_measured_ffma"] = tf / alu_measured
        # SFU: one ex2 per blended entry (Eq. 2's exponential; the backward recomputes the forward's)
        ex2 = stats["blended"] / (kern[k] * 1e-3) / 1e9
        out[k]["ex2"] = stats["blended"]
        out[k]["ex2_gops"] = ex2
        if ex2_measured:
            out[k]["frac_of_measured_ex2"] = ex2 / ex2_measured
    return out


# DRAM bytes (read + write) of one k_render_bwd launch on this workload from an ncu capture
# (dram__bytes_read.sum + dram__bytes_write.sum), valid while the kernel's sources (its file, the
# shared device header and its argument struct) hash to the recorded value; after any change the
# bench reports null until it is captured again.
PROFILED_TRAFFIC = {"kernel": "k_render_bwd", "sources": ("render_bwd.cu", "odgs_common.cuh"),
                    "structs": ("odgs_internal.h", "BwdArgs"),
                    "sha256": "79548bc8d827a32d6196073bbce0fad16e61150ec889680e230c810e30ee5cfe",
                    "bytes": 171006208}


def kernel_sources_digest(spec=PROFILED_TRAFFIC):
    import hashlib
    import re
    h = hashlib.sha256()
    csrc = os.path.join(ROOT, "paper_2410_20686_gb300", "csrc")
    try:
        for f in spec["sources"]:
            with open(os.path.join(csrc, f), "rb") as fh:
                h.update(fh.read())
        header, name = spec["structs"]
        with open(os.path.join(csrc, header)) as fh:
            m = re.search(r"struct %s \{.*?\n\};" % name, fh.read(), re.S)
        if m is None:
            return None
        h.update(m.group(0).encode())
    except OSError:
        return None
    return h.hexdigest()


def profiled_traffic():
    d = kernel_sources_digest()
    if d is not None and PROFILED_TRAFFIC["sha256"] and d == PROFILED_TRAFFIC["sha256"]:
        return PROFILED_TRAFFIC["bytes"]
    return None


# ------------------------------------------------------------------ CPU oracle leg

def oracle_sample(scene, n_pix, seed=0):
    """Oracle forward and adjoint on n_pix seeded pixels, timed separately; returns the timings and
    the extrapolated full-frame times of each pass (per-Gaussian work once, per-pixel work times
    the frame's pixels)."""
    import numpy as np
    from oracle import oracle as O
    from paper_2410_20686_gb300 import scenes as S
    v = scene.views[0]
    p = O.Params.of(scene)
    st = O.Settings(sh_degree=scene.sh_degree, dilation=float(np.float32(0.3)), r_near=float(np.float32(0.2)),
                    r_far=float(np.float32(1e4)))
    pix = S.sample_pixels(v.width, v.height, n_pix, [], seed=seed)
    rng = np.random.default_rng(seed)
    g = rng.normal(size=(len(pix), 3))
    t0 = time.perf_counter()
    O.render(p, v, st, pix=pix[:1])
    t1 = time.perf_counter()
    O.render(p, v, st, pix=pix)
    t2 = time.perf_counter()
    O.backward(p, v, st, g[:1], pix=pix[:1])
    t3 = time.perf_counter()
    O.backward(p, v, st, g, pix=pix)
    t4 = time.perf_counter()
    px = v.width * v.height
    span = max(len(pix) - 1, 1)
    # the one-pixel call is the per-Gaussian cost (projection, sort; the adjoint's chain rule)
    fwd = (t1 - t0) + (t2 - t1) / span * px
    adj = (t3 - t2) + (t4 - t3) / span * px
    return {"sample_s": t4 - t0, "full_iter_s": fwd + adj, "forward_s": fwd, "adjoint_s": adj,
            "pixels": len(pix), "threads": O.num_threads()}


def cpu_baseline(scene):
    r = oracle_sample(scene, CPU_SAMPLE_PIXELS)
    return {"value": 1.0 / r["full_iter_s"], "unit": UNIT, "cores": r["threads"], "kind": "oracle",
            "forward_s_per_frame": r["forward_s"], "adjoint_s_per_frame": r["adjoint_s"],
            "sample": f"{r['pixels']} seeded pixels of the 2048x1024 view, forward and adjoint timed separately, "
                      f"per-pixel time extrapolated to all pixels plus the full per-Gaussian projection / adjoint "
                      f"({r['sample_s']:.1f} s of CPU work); extrapolated"}


def workload_config(args, world):
    """The workload both arms name in their JSON line (the same dict, so that their lines compare)."""
    return {"workload": WORKLOAD, "gaussians": args.n, "width": args.width, "height": args.width // 2,
            "sh_degree": 3, "tile": args.tile, "batch": args.batch, "pixels_per_thread": args.ppt,
            "pixels_per_thread_bwd": args.ppt_bwd,
            "l2": "inputs larger than L2 (236 MB of parameters read twice per step)",
            "parallelism": f"replicas x{world}"}


def run_reference(args):
    world, rank, _ = dist_env()
    if rank != 0:  # under torchrun only rank 0 times the oracle; the others exit without work
        return
    from paper_2410_20686_gb300 import scenes as S
    from oracle import oracle as O
    O.build()
    scene = S.config2(n=args.n, width=args.width)
    for w in range(args.warmup):
        oracle_sample(scene, 64, seed=100 + w)
    times, fwd, adj = [], [], []
    res = None
    for k in range(args.steps):
        res = oracle_sample(scene, 256, seed=k)
        times.append(res["full_iter_s"])
        fwd.append(res["forward_s"])
        adj.append(res["adjoint_s"])
    import statistics
    full = statistics.median(times)
    value = 1.0 / full
    out = {"metric": METRIC, "value": value, "unit": UNIT, "n_gpus": args.gpus, "steps": args.steps,
           "warmup": args.warmup, "ms_per_step": full * 1e3, "higher_is_better": True, "scaling": "weak",
           "vs_baseline": None, "dtype": "f64", "data": "synthetic", "impl": "reference",
           "config": workload_config(args, world),
           "timing": "the FP64 oracle on the host cores, one seeded pixel sample per step, extrapolated to the "
                     "full frame; value from the median step",
           "cpu_baseline": {"value": value, "unit": UNIT, "cores": res["threads"], "kind": "oracle",
                            "forward_s_per_frame": statistics.median(fwd),
                            "adjoint_s_per_frame": statistics.median(adj),
                            "sample": "each step: 256 seeded pixels, forward and adjoint timed separately, "
                                      "extrapolated to the full frame"},
           "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(out), flush=True)


# ------------------------------------------------------------------ batched views (config 3)

BATCHED_WORKLOAD = ("config3: 500,000 shared Gaussians (SH3), 16 ERP views (4x512x256, 4x1024x512, "
                    "8x2048x1024) on a 3 m path with random yaw, fwd+bwd with L1 loss, gradients of all "
                    "views summed into one buffer")


def run_batched(dev, rs, steps, warmup):
    """views/s of one CUDA-graph-replayed 16-view frame vs the same views one frame at a time."""
    import torch
    from dataclasses import replace
    from paper_2410_20686_gb300 import scenes as S
    from paper_2410_20686_gb300.graph import GraphedFrame, l1_grad
    from paper_2410_20686_gb300.rasterizer import Rasterizer

    sc = S.config3()
    params = [torch.tensor(a, device=dev) for a in (sc.means, sc.scales, sc.quats, sc.opacity, sc.sh)]
    targets = [torch.tensor(t, device=dev) for t in S.target_images(sc, 3)]
    V = len(sc.views)
    gf = GraphedFrame(params, sc.views, targets, rs)
    for _ in range(warmup):
        gf.replay()
    torch.cuda.synchronize(dev)
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record()
    for _ in range(steps):
        gf.replay()
    e1.record()
    torch.cuda.synchronize(dev)
    t_b = e0.elapsed_time(e1) / 1e3 / steps
    assert gf.status() == 0
    # the same views, one frame each (same kernels, no graph); gradients summed over the views
    rast = Rasterizer(dev, capacity_mode="query", headroom=1.3)
    grads = {k: torch.empty_like(t) for k, t in zip(("means", "scales", "quats", "opacity", "sh"), params)}
    acc = replace(rs, grad_accumulate=True)

    def single_round():
        for i, (v, tg) in enumerate(zip(sc.views, targets)):
            r = rs if i == 0 else acc
            imgs, _ = rast.forward(*params, [v], r, want_T=False)
            _, gi = l1_grad(imgs, [tg])
            rast.backward(gi, grads)

    single_round()  # sizes the buffers for the largest view
    torch.cuda.synchronize(dev)
    rast.capacity_mode = "fixed"
    for _ in range(warmup):
        single_round()
    torch.cuda.synchronize(dev)
    e0.record()
    for _ in range(steps):
        single_round()
    e1.record()
    torch.cuda.synchronize(dev)
    t_s = e0.elapsed_time(e1) / 1e3 / steps
    assert rast.status() == 0
    return {"workload": BATCHED_WORKLOAD, "views_per_s": V / t_b, "single_views_per_s": V / t_s,
            "speedup": t_s / t_b, "ms_per_frame": t_b * 1e3, "ms_per_views_one_at_a_time": t_s * 1e3,
            "kernel_launches_per_frame": gf.launches + 2 * V, "rasterizer_launches_per_frame": gf.launches,
            "steps": steps, "per_gpu": True}


LARGE_WORKLOAD = ("config4: 3,000,000 Gaussians (SH3) along a 50 m corridor (30% in 100 clusters), 8 ERP views "
                  "of 4096x2048 every 6 m, fwd+bwd with L1 loss, gradients of all views summed into one buffer")


def run_batched_large(dev, rs, steps, warmup, group_size=2):
    """views/s of the roaming-scale frame: GroupedFrame (groups of views sharing one pair buffer,
    tile lists rebuilt in each group's backward pass, as the configuration prescribes), and for
    comparison all 8 views in one CUDA-graph-replayed frame with the lists kept."""
    import torch
    from paper_2410_20686_gb300 import scenes as S
    from paper_2410_20686_gb300.graph import GraphedFrame, GroupedFrame

    sc = S.config4()
    params = [torch.tensor(a, device=dev) for a in (sc.means, sc.scales, sc.quats, sc.opacity, sc.sh)]
    targets = [torch.tensor(t, device=dev) for t in S.target_images(sc, 4)]
    V = len(sc.views)
    px = sum(v.width * v.height for v in sc.views)

    def timed(fn):
        for _ in range(warmup):
            fn()
        torch.cuda.synchronize(dev)
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record()
        for _ in range(steps):
            fn()
        e1.record()
        torch.cuda.synchronize(dev)
        return e0.elapsed_time(e1) / 1e3 / steps

    grouped = GroupedFrame(params, sc.views, targets, rs, group_size=group_size)
    t_g = timed(grouped.step)
    assert grouped.status() == 0
    pair_bytes = grouped.pair_buffer_bytes()
    del grouped
    torch.cuda.empty_cache()
    whole = GraphedFrame(params, sc.views, targets, rs)
    t_w = timed(whole.replay)
    assert whole.status() == 0
    whole_pairs = whole.rast.stats()["pairs"]
    return {"workload": LARGE_WORKLOAD, "views_per_s": V / t_g, "ms_per_frame": t_g * 1e3,
            "pixels_per_s": px / t_g, "mode": f"GroupedFrame, {group_size} views per group, lists rebuilt in "
                                              f"the backward pass", "pair_buffer_bytes": pair_bytes,
            "all_views_graphed": {"views_per_s": V / t_w, "ms_per_frame": t_w * 1e3, "pairs": whole_pairs},
            "steps": steps, "per_gpu": True}


# ------------------------------------------------------------------ densification (Sec. 3.3)

def timed_flushed(torch, dev, fn, iters):
    """Mean CUDA-event milliseconds of fn over iters calls, each after an L2 flush (a 256 MB write)."""
    flush = torch.empty(64 << 20, dtype=torch.float32, device=dev)
    total = 0.0
    for _ in range(iters):
        flush.zero_()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record()
        fn()
        e1.record()
        torch.cuda.synchronize(dev)
        total += e0.elapsed_time(e1)
    return total / iters


def run_densify(torch, dev, rast, params, view, rs, target, hbm_gbs, iters=20):
    """Statistics over a few frames, then the decision and the densified arrays, timed."""
    from paper_2410_20686_gb300.densify import DensifyParams, DensifyStats, apply, select
    n = params[0].shape[0]
    stats = DensifyStats(n, dev)
    grads = {k: torch.empty_like(t) for k, t in zip(("means", "scales", "quats", "opacity", "sh"), params)}
    for _ in range(4):
        imgs, _ = rast.forward(*params, [view], rs, want_T=False)
        g = torch.sign(imgs[0] - target) * (1.0 / imgs[0].numel())
        rast.render_bwd([g])
        rast.preprocess_bwd(grads, densify=stats)
    # the fused statistics' cost: the backward preprocess with and without them
    t_plain = timed_flushed(torch, dev, lambda: rast.preprocess_bwd(grads), iters)
    t_stats = timed_flushed(torch, dev, lambda: rast.preprocess_bwd(grads, densify=stats), iters)
    prm = DensifyParams(scene_extent=10.0)
    act = select(stats, params[1], params[3], prm)
    t_sel = timed_flushed(torch, dev, lambda: select(stats, params[1], params[3], prm), iters)
    noise = torch.randn((n, 2, 3), device=dev, generator=torch.Generator(device=dev).manual_seed(0))
    out = apply(*params, act, noise)
    t_app = timed_flushed(torch, dev, lambda: apply(*params, act, noise), max(3, iters // 4))
    a = act.cpu()
    kept, clone, split = int(((a == 0) | (a == 1)).sum()), int((a == 1).sum()), int((a == 2).sum())
    pbytes = param_bytes(3)
    # select: statistics 12 B, scales 12 B, opacity 4 B read, one action byte written
    sel_bytes = n * (12 + 12 + 4 + 1)
    # apply: actions read twice (count and scatter), each used Gaussian's parameters read once, the
    # noise of split ones, every output written
    used = kept + split
    app_bytes = 2 * n + used * pbytes + split * 24 + out[0].shape[0] * pbytes
    return {"workload": "statistics of 4 fwd+bwd frames of the 1M-Gaussian view, then one densification "
                        "(tau_min 2e-5, tau_max 1e-4, percent_dense 1e-3, scene extent 10)",
            "stats_overhead_ms": t_stats - t_plain, "preprocess_bwd_ms": t_plain,
            "select_ms": t_sel, "select_gbs": sel_bytes / (t_sel * 1e-3) / 1e9,
            "select_frac": sel_bytes / (t_sel * 1e-3) / 1e9 / hbm_gbs,
            "apply_ms": t_app, "apply_gbs": app_bytes / (t_app * 1e-3) / 1e9,
            "apply_frac": app_bytes / (t_app * 1e-3) / 1e9 / hbm_gbs,
            "kept": kept, "cloned": clone, "split": split, "pruned": n - kept - split, "n_out": int(out[0].shape[0]),
            "l2": "flushed before every timed call"}


def run_adam(torch, dev, params, hbm_gbs, iters=10):
    """One fused Adam step over all five parameter tensors of the 1M-Gaussian scene."""
    from paper_2410_20686_gb300.optim import GaussianAdam
    work = [t.clone() for t in params]
    grads = [torch.randn_like(t) * 1e-3 for t in params]
    opt = GaussianAdam(work, scene_extent=10.0)
    opt.step(grads)
    ms = timed_flushed(torch, dev, lambda: opt.step(grads), iters)
    floats = sum(t.numel() for t in work)
    nbytes = floats * 28  # p, g, m, v read; p, m, v written
    return {"workload": "Adam step over the 1M Gaussians' parameters (59 floats each, SH DC / rest rates)",
            "ms": ms, "params": floats, "bytes": nbytes, "gbs": nbytes / (ms * 1e-3) / 1e9,
            "frac": nbytes / (ms * 1e-3) / 1e9 / hbm_gbs, "l2": "inputs (1.65 GB) larger than L2, flushed too"}


def run_loss(torch, dev, image, target, hbm_gbs, alu_tflops, iters=20):
    """L1 + D-SSIM loss and gradient of the 2048x1024 view (cos-theta row weights, seam wrap)."""
    from paper_2410_20686_gb300.loss import l1_dssim
    # captured once in a CUDA graph, so that the time is the kernels', not the Python wrapper's
    s = torch.cuda.Stream(dev)
    s.wait_stream(torch.cuda.current_stream(dev))
    with torch.cuda.stream(s):
        l1_dssim([image], [target])
    torch.cuda.current_stream(dev).wait_stream(s)
    graph = torch.cuda.CUDAGraph()
    with torch.cuda.graph(graph):
        l1_dssim([image], [target])
    ms = timed_flushed(torch, dev, graph.replay, iters)
    px = image.numel() // 3
    # algorithmic: image and target read, gradient written (36 B per pixel); the kernels also write
    # and re-read three adjoint maps per channel (another 72 B per pixel)
    nbytes = px * 36
    # 11-tap separable passes: forward 5 moments x 11 taps x (26 / 16 halo rows + 1), backward 3 x 11
    # x (26 / 16 + 1), per channel, 2 flop each; the per-pixel SSIM terms are left out
    flops = px * 3 * 2 * (5 + 3) * 11 * (26.0 / 16.0 + 1.0)
    t = ms * 1e-3
    return {"workload": "L1 + D-SSIM (lambda 0.2, 11x11 window) and its gradient on one 2048x1024 ERP view",
            "ms": ms, "gbs": nbytes / t / 1e9, "hbm_frac": nbytes / t / 1e9 / hbm_gbs,
            "tflops": flops / t / 1e12, "alu_frac": flops / t / 1e12 / alu_tflops,
            "traffic_per_pixel_bytes": 108, "timing": "CUDA-graph replays of the call",
            "l2": "flushed before every timed call"}


def run_cubemap(torch, dev, params, target_erp, rs, steps=20, warmup=3):
    """The same Gaussians rendered as six 90-degree pinhole faces of equal total pixel count
    (6 x 592^2 = 2.10 Mpx vs 2048 x 1024 = 2.10 Mpx), fwd+bwd from one CUDA graph: the
    3DGS(P)-style cubemap alternative to the ERP view."""
    from paper_2410_20686_gb300 import scenes as S
    from paper_2410_20686_gb300.graph import GraphedFrame
    # faces of about the ERP view's pixel count, a multiple of the tile width
    face = max(rs.tile_w, int(round((2048 * 1024 / 6) ** 0.5 / rs.tile_w)) * rs.tile_w)
    faces = S.cubemap_views(face)
    targets = [torch.rand((3, face, face), device=dev, generator=torch.Generator(device=dev).manual_seed(k))
               for k in range(6)]
    gf = GraphedFrame(params, faces, targets, rs)
    for _ in range(warmup):
        gf.replay()
    torch.cuda.synchronize(dev)
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record()
    for _ in range(steps):
        gf.replay()
    e1.record()
    torch.cuda.synchronize(dev)
    assert gf.status() == 0
    ms = e0.elapsed_time(e1) / steps
    return {"workload": f"1M Gaussians, six {face}x{face} pinhole cube faces ({6 * face * face / 1e6:.2f} Mpx), "
                        "fwd+bwd with L1 loss, one graph",
            "ms_per_frame": ms, "iter_per_s": 1e3 / ms, "pixels": 6 * face * face}


# ------------------------------------------------------------------ end to end through the C ABI

GRAD_NAMES = ("means", "scales", "quats", "opacity", "sh")


def run_e2e_abi(torch, dev, rs, view, host_in, steps, warmup, barrier):
    """fwd+bwd iterations/s through the library's C ABI with host buffers: every step copies the
    five parameter arrays and the target from pinned host memory to the device, calls
    odgs_preprocess -> odgs_bin_sort -> odgs_render_fwd -> fused L1 loss -> odgs_render_bwd ->
    odgs_preprocess_bwd (eager calls, no graph), and copies all five gradient arrays and the loss
    back to pinned host memory, where the host reads them. Uploads of step i+1 (one copy stream) and
    downloads of step i (another) overlap step i+1's kernels through two device input and gradient
    sets."""
    from paper_2410_20686_gb300.loss import l1_dssim
    from paper_2410_20686_gb300.rasterizer import Rasterizer
    sets = [[torch.empty(h.shape, dtype=h.dtype, device=dev) for h in host_in] for _ in range(2)]
    gsets = [{k: torch.empty_like(t) for k, t in zip(GRAD_NAMES, st[:5])} for st in sets]
    host_g = [{k: torch.empty(t.shape, dtype=t.dtype).pin_memory() for k, t in g.items()} for g in gsets]
    loss_host = [torch.empty((), dtype=torch.float32).pin_memory() for _ in range(2)]
    image = torch.empty((3, view.height, view.width), dtype=torch.float32, device=dev)
    rast = Rasterizer(dev, capacity_mode="query", headroom=1.1)
    up, down = torch.cuda.Stream(dev), torch.cuda.Stream(dev)
    main = torch.cuda.current_stream(dev)
    loaded, freed, computed, downloaded = ([torch.cuda.Event() for _ in range(2)] for _ in range(4))

    def upload(j):
        with torch.cuda.stream(up):
            up.wait_event(freed[j])  # the step that last read input set j has finished
            for h, d in zip(host_in, sets[j]):
                d.copy_(h, non_blocking=True)
            loaded[j].record(up)

    def compute(j):
        main.wait_event(loaded[j])
        main.wait_event(downloaded[j])  # gradient set j has been copied out
        p = sets[j]
        rast.preprocess(*p[:5], [view], rs)
        rast.bin_sort()
        rast.render_fwd([image], want_T=False)
        loss, gl = l1_dssim([image], [p[5]], lam=0.0, area_weight=False)
        rast.render_bwd([gl[0]])
        rast.preprocess_bwd(gsets[j])
        freed[j].record(main)
        computed[j].record(main)
        loss.record_stream(down)
        with torch.cuda.stream(down):
            down.wait_event(computed[j])
            for k in GRAD_NAMES:
                host_g[j][k].copy_(gsets[j][k], non_blocking=True)
            loss_host[j].copy_(loss.reshape(()), non_blocking=True)
            downloaded[j].record(down)

    def consume(j, out):
        downloaded[j].synchronize()
        out.append((float(loss_host[j]), float(host_g[j]["opacity"][0])))

    def run(n):
        results = []
        for j in range(2):
            freed[j].record(main)
            downloaded[j].record(main)
        upload(0)
        for i in range(n):
            j = i % 2
            if i + 1 < n:
                upload(1 - j)
            compute(j)
            if i > 0:  # the previous step's gradients and loss, read while this step runs
                consume(1 - j, results)
        consume((n - 1) % 2, results)
        return results

    # size the pair buffer once (one host read of the pair count), then no host synchronisation
    upload(0)
    main.wait_event(loaded[0])
    rast.forward(*sets[0][:5], [view], rs, want_T=False)
    torch.cuda.synchronize(dev)
    rast.capacity_mode = "fixed"
    run(warmup)
    torch.cuda.synchronize(dev)
    barrier()
    t0 = time.perf_counter()
    res = run(steps)
    torch.cuda.synchronize(dev)
    seconds = time.perf_counter() - t0
    barrier()
    import math
    assert len(res) == steps and all(math.isfinite(a) and math.isfinite(b) for a, b in res)
    assert rast.status() == 0
    h2d = sum(h.numel() * h.element_size() for h in host_in)
    d2h = sum(t.numel() * t.element_size() for t in gsets[0].values()) + 4
    return {"seconds": seconds, "h2d_bytes_per_step": h2d, "d2h_bytes_per_step": d2h,
            "path": "C-ABI calls every step (odgs_preprocess, odgs_bin_sort, odgs_render_fwd, fused L1 loss, "
                    "odgs_render_bwd, odgs_preprocess_bwd) from pinned host parameters and target; all five "
                    "gradient arrays and the loss copied back to pinned host memory and read by the host",
            "overlap": "uploads of step i+1 and downloads of step i on two copy streams beside step i+1's kernels"}


# ------------------------------------------------------------------ multi-process plumbing

def dist_env():
    """(world, rank, local_rank) from the torchrun environment (1, 0, 0 without it)."""
    return (int(os.environ.get("WORLD_SIZE", "1")), int(os.environ.get("RANK", "0")),
            int(os.environ.get("LOCAL_RANK", "0")))


def max_over_ranks(x: float, world: int, device) -> float:
    """The largest x of all ranks (the job's wall time is its slowest rank's)."""
    if world == 1:
        return float(x)
    import torch
    import torch.distributed as dist
    t = torch.tensor([float(x)], device=device, dtype=torch.float64)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def job_rate(world: int, steps: int, seconds_max: float) -> float:
    """Whole-job iterations per second: every rank ran `steps` independent iterations."""
    return world * steps / seconds_max


# ------------------------------------------------------------------ GPU leg

def run_ours(args):
    import numpy as np
    import torch
    import torch.distributed as dist

    from paper_2410_20686_gb300 import build as B
    from paper_2410_20686_gb300 import scenes as S
    from paper_2410_20686_gb300.graph import GraphedFrame
    from paper_2410_20686_gb300.loss import l1_dssim
    from paper_2410_20686_gb300.rasterizer import Rasterizer, RenderSettings

    world, rank, local = dist_env()
    B.build()
    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)
    if world > 1:
        dist.init_process_group("nccl", init_method="env://")

    def barrier():
        if world > 1:
            dist.barrier()

    tw, th = (int(x) for x in args.tile.split("x"))
    rs = RenderSettings(sh_degree=3, tile_w=tw, tile_h=th, batch=args.batch, pixels_per_thread=args.ppt,
                        pixels_per_thread_bwd=args.ppt_bwd)
    scene = S.config2(n=args.n, width=args.width)
    target_np = S.target_images(scene, 2)[0]
    view = scene.views[0]
    params = [torch.tensor(a, device=dev) for a in (scene.means, scene.scales, scene.quats, scene.opacity, scene.sh)]
    target = torch.tensor(target_np, device=dev)
    grads = {k: torch.empty_like(t) for k, t in zip(("means", "scales", "quats", "opacity", "sh"), params)}
    rast = Rasterizer(dev, capacity_mode="query", headroom=1.1)

    evs = None

    def step(record=None, inputs=None):
        p, tgt = (params, target) if inputs is None else (inputs[:5], inputs[5])
        if record is not None:
            record[0].record()
        rast.preprocess(*p, [view], rs)
        if record is not None:
            record[1].record()
        rast.bin_sort()
        if record is not None:
            record[2].record()
        imgs, _ = rast.render_fwd(want_T=False)
        if record is not None:
            record[3].record()
        # mean absolute error and its gradient sign(C - target) / (3 W H), one fused kernel
        loss, gl = l1_dssim([imgs[0]], [tgt], lam=0.0, area_weight=False)
        g = gl[0]
        if record is not None:
            record[4].record()
        rast.render_bwd([g])
        if record is not None:
            record[5].record()
        rast.preprocess_bwd(grads)
        if record is not None:
            record[6].record()
        return loss

    # size the pair buffer once, then run without host synchronisation
    step()
    torch.cuda.synchronize()
    rast.capacity_mode = "fixed"
    stats = rast.stats()
    assert stats["status"] == 0, stats
    for _ in range(args.warmup):
        step()
    torch.cuda.synchronize()

    K = args.steps
    # per-stage times: an eager run of the step with CUDA events between the stages
    evs = [[torch.cuda.Event(enable_timing=True) for _ in range(7)] for _ in range(K)]
    stage_sampler = ClockSampler(_gpu_id(torch, local))
    stage_sampler.start()
    for i in range(K):
        step(evs[i])
    torch.cuda.synchronize()
    stage_clocks = stage_sampler.stop()
    stats = rast.stats()
    assert stats["status"] == 0, stats
    names = ["preprocess", "bin_sort", "render_fwd", "loss", "render_bwd", "preprocess_bwd"]
    kern = {nm: float(np.mean([evs[i][j].elapsed_time(evs[i][j + 1]) for i in range(K)])) for j, nm in enumerate(names)}
    eager_ms = float(np.mean([evs[i][0].elapsed_time(evs[i][6]) for i in range(K)]))

    # the timed steps: the same fwd+bwd step (same kernels, inputs and fused L1 loss) replayed from a
    # CUDA graph, as a training loop runs it (GraphedFrame), which removes the host launch gaps
    frames = [GraphedFrame(params, [view], [target], rs)]
    for _ in range(args.warmup):
        frames[0].replay()
    torch.cuda.synchronize()
    start, stop = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    sampler = ClockSampler(_gpu_id(torch, local))
    barrier()
    torch.cuda.synchronize()
    sampler.start()
    start.record()
    for i in range(K):
        frames[0].replay()
    stop.record()
    torch.cuda.synchronize()
    barrier()
    clocks = sampler.stop()
    elapsed = max_over_ranks(start.elapsed_time(stop) / 1e3, world, dev)
    assert frames[0].status() == 0
    # the rasterizer's kernels of one step plus the fused L1 loss's two (k_l1, k_loss_reduce)
    graph_launches = frames[0].launches + 2

    # end-to-end through host buffers: every step copies its parameters and target in from pinned
    # host memory and reads its loss back. The copies run on a second stream into the inputs of one
    # of two graphed frames, so step i+1's upload overlaps step i's kernels (a data loader's
    # prefetch); the first upload and the last loss read are inside the timed region.
    e2e = None
    if not args.no_e2e:
        host = [t_.cpu().pin_memory() for t_ in params] + [target.cpu().pin_memory()]
        second = [t_.clone() for t_ in params]
        frames.append(GraphedFrame(second, [view], [target.clone()], rs))
        sets = [f.params + f.targets for f in frames]
        h2d = sum(h.numel() * h.element_size() for h in host)
        copy_stream = torch.cuda.Stream(dev)
        main = torch.cuda.current_stream(dev)
        loaded = [torch.cuda.Event() for _ in sets]
        freed = [torch.cuda.Event() for _ in sets]
        loss_host = [torch.empty((), dtype=torch.float32).pin_memory() for _ in sets]
        read = [torch.cuda.Event() for _ in sets]

        def upload(j):
            with torch.cuda.stream(copy_stream):
                copy_stream.wait_event(freed[j])  # the step that last read set j has finished
                for h, d in zip(host, sets[j]):
                    d.copy_(h, non_blocking=True)
                loaded[j].record(copy_stream)

        def run_e2e(steps):
            losses = []
            for j in range(2):
                freed[j].record(main)
            upload(0)
            for i in range(steps):
                j = i % 2
                if i + 1 < steps:
                    upload(1 - j)
                main.wait_event(loaded[j])
                loss = frames[j].replay()
                freed[j].record(main)
                loss_host[j].copy_(loss.reshape(()), non_blocking=True)
                read[j].record(main)
                if i > 0:  # the previous step's loss, read while this step runs
                    read[1 - j].synchronize()
                    losses.append(float(loss_host[1 - j]))
            read[(steps - 1) % 2].synchronize()
            losses.append(float(loss_host[(steps - 1) % 2]))
            return losses
        run_e2e(max(3, args.warmup))
        torch.cuda.synchronize()
        barrier()
        t0 = time.perf_counter()
        losses = run_e2e(K)
        torch.cuda.synchronize()
        barrier()
        te = max_over_ranks(time.perf_counter() - t0, world, dev)
        assert len(losses) == K and all(np.isfinite(losses)), losses
        assert all(f.status() == 0 for f in frames)
        e2e_graph = {"value": job_rate(world, K, te), "unit": UNIT, "h2d_bytes_per_step": h2d,
                     "d2h_bytes_per_step": 4,
                     "overlap": "uploads on a second stream into the inputs of two graphed frames; losses read "
                                "one step behind; the gradients stay on the device (a training loop's reading)"}
        del frames[1:]
        torch.cuda.empty_cache()
        barrier()
        abi = run_e2e_abi(torch, dev, rs, view, host, K, max(3, args.warmup), barrier)
        te = max_over_ranks(abi.pop("seconds"), world, dev)
        e2e = dict(value=job_rate(world, K, te), unit=UNIT, **abi)
        e2e["graph_replay"] = e2e_graph

    if rank != 0:
        if world > 1:
            dist.destroy_process_group()
        return

    # FP32 FMA and exp2f throughput of this device (own microbenchmark), after the timed regions:
    # its seconds of full-rate FMA and MUFU work can leave the SM clock lower for a while
    from paper_2410_20686_gb300.rasterizer import measure_peaks
    measured = measure_peaks(dev)
    torch.cuda.synchronize()

    peaks, peak_src = _peaks()
    peak_tf, sms, mhz = fp32_peak_tflops(torch, dev, peaks)
    tiles = (view.width // tw) * ((view.height + th - 1) // th)
    pair_passes = (max(1, (tiles - 1).bit_length()) + 7) // 8  # 8-bit passes over the tile id
    kernels = stage_rooflines(kern, stats, args.n, 3, tiles, pair_passes, float(peaks["hbm_gbs"]), peak_tf,
                              measured["ffma_tflops"] if measured else None,
                              measured["ex2_gops"] if measured else None)
    dom = max(("render_fwd", "render_bwd"), key=lambda k: kern[k])
    d = kernels[dom]
    roofline = {"bound": "alu", "kernel": "k_render_fwd" if dom == "render_fwd" else "k_render_bwd",
                "achieved": d["achieved"], "peak": peak_tf, "unit": "TFLOP/s", "frac": d["frac"],
                "traffic": profiled_traffic() if dom == "render_bwd" else None,
                "peak_note": f"FP32 FMA peak {sms} SMs x 128 lanes x 2 flop x {mhz:.0f} MHz (max SM clock, "
                             f"{peak_src} peaks file)",
                "units": {"evals_fwd": stats["evals_fwd"], "evals_bwd": stats["evals_bwd"],
                          "blended": stats["blended"], "pairs": stats["pairs"], "pairs_sorted": stats["pairs_sorted"],
                          "entries_tile": stats["entries_tile"], "visible": stats["visible"]}}
    if measured:
        roofline["peak_measured"] = measured
        roofline["frac_of_measured_ffma"] = d.get("frac_of_measured_ffma")
        roofline["ex2_frac_of_measured"] = d.get("frac_of_measured_ex2")

    out = {"metric": METRIC, "value": job_rate(world, K, elapsed), "unit": UNIT, "n_gpus": world, "steps": K,
           "warmup": args.warmup, "ms_per_step": elapsed / K * 1e3, "higher_is_better": True, "scaling": "weak",
           "vs_baseline": None, "dtype": "f32", "data": "synthetic",
           "config": workload_config(args, world),
           "timing": "whole fwd+bwd step replayed from a CUDA graph (GraphedFrame), CUDA events around K "
                     "replays; kernels_ms from an eager run with events between the stages",
           "roofline": roofline, "kernels_ms": kern, "kernels": kernels, "gpu_launches": graph_launches * K,
           "eager_ms_per_step": eager_ms,
           "clocks": clocks, "stage_clocks": stage_clocks}
    if e2e:
        out["e2e"] = e2e
    if not args.no_batched:
        out["batched"] = run_batched(dev, rs, args.batched_steps, args.warmup)
    if not args.no_large:
        out["batched_large"] = run_batched_large(dev, rs, steps=5, warmup=2)
    if not args.no_next:
        imgs_last, _ = rast.forward(*params, [view], rs, want_T=False)
        imgs_last = imgs_last[0]
        out["next"] = {"densify": run_densify(torch, dev, rast, params, view, rs, target, float(peaks["hbm_gbs"])),
                       "adam": run_adam(torch, dev, params, float(peaks["hbm_gbs"])),
                       "loss": run_loss(torch, dev, imgs_last, target, float(peaks["hbm_gbs"]), peak_tf),
                       "cubemap": run_cubemap(torch, dev, params, target, rs)}
    if not args.no_cpu_baseline:
        out["cpu_baseline"] = cpu_baseline(scene)
    print(json.dumps(out), flush=True)
    if world > 1:
        dist.destroy_process_group()


def main():
    args = parse()
    if args.impl == "reference":
        run_reference(args)
    else:
        run_ours(args)


if __name__ == "__main__":
    main()
