"""Benchmark of the relativistic ray march on one GB300 (or N replicas).

A step is one pass of the whole hot path over one batch of views: the batch
render of every view of a workload, with the snapshot volume resident in HBM
(loaded and packed once, before timing).

Workloads (synthetic, seeded; see gen/):
  batched      384^3 x 32 turbulent jet, float32 j' and beta, 256 views of
               256^2 on a Fibonacci sphere (the largest single-GPU workload).
  time_delay   256^3 x 16 epochs, float32: a Gaussian blob (sigma = 8 cells)
               at beta = 0.95 z over a steady conical jet; 512^2 images at
               theta in {10, 45} deg x 9 observer times = 18 images per step.
  precision    512^3 x 8 turbulent jet stored as bfloat16 j' + float16
               four-velocity, one 1024^2 view.
  serving      a resident catalogue of six volumes under a Poisson stream of
               render requests.

Default run (no --workload): the suite.  The top-level line is the batched
workload's batch render; nested entries (key "configs") carry the batched
workload stored as bfloat16/float16 records, the time-delay workload in
float32 (lone march, and time groups) and as bfloat16/float16 records, the
precision workload in bfloat16/float16, the plain float32 per-image march of
each workload (one render call per view, default layout and launch), and a
short serving phase with p50/p99 latency.  Each entry has its own roofline
and its error against the FP64 oracle on sampled pixels.  Launch shapes and
layouts are fixed to the autotuner's picks on GB300 (``--tune`` re-runs the
tuner instead).

--workload X times one workload alone, optionally in another form:
  batch (default)  the batch render of every view, volume resident.
  streamed         the volume stays in pinned host memory and is uploaded slab
                   by slab with flexload, marched slab by slab (out-of-core).
  labelled         the volume given as two sub-domains (its halves along x).
  vector           three extra emissivity channels marched with j'.

Prints one JSON line.  --impl reference times the FP64 CPU oracle on a
bounded sample of the same workload instead.
"""
from __future__ import annotations

import argparse
import hashlib
import json
import math
import os
import re
import statistics
import subprocess
import sys
import threading
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

METRIC = "Gcell-samples/s and images/s at 1 GB300 (% HBM roofline); serving p50/p99 ms"
UNIT = "Gcell-samples/s"
# Algorithmic bytes per cell-sample: two snapshot records per sample under
# lookback (float32 record 16 B, bfloat16/float16 record 8 B), one without.
RECORD_BYTES = {"f32": 16, "bf16": 8}

# Launch (packet_w, packet_h, warps per CTA, cells ahead, capped registers
# [, region edge [, time-group size]]) and layout (brick, super-brick, paired)
# measured fastest on GB300 for each workload, within the autotuner's search
# space.
PINNED = {
    "batched": ("4,8,4,2,1,64", "8,4,0"),
    "batched_bf16": ("4,8,4,2,1,64", "4,4,1"),
    "time_delay": ("4,8,4,2,1,0,1", "4,4,0"),
    "time_delay_grouped": ("4,8,4,2,1,0,4", "4,2,1"),
    "time_delay_bf16": ("8,4,8,4,1,0,4", "4,2,1"),
    "precision": ("4,8,4,4,1,0,2", "8,4,1"),
}
L2_NOTE = "inputs larger than L2 (resident volume %.1f GB; L2 129 MB), no flush between steps"


# ------------------------------------------------------------------ inputs
def make_workload(name: str, scale: float = 1.0, device: str = "cpu"):
    import gen
    if name == "time_delay":
        n, size = int(round(256 * scale)), int(round(512 * scale))
        grid, j, beta, views = gen.config_time_delay(n=n, size=size, dtype=np.float32)
        desc = (f"time-delay path: {n}^3 grid x 16 epochs FP32 (j', beta), Gaussian blob sigma={8 * scale:g} "
                f"cells at beta=0.95 z over a steady conical jet, c*dt=4 cells; 18 images of {size}x{size} per "
                "step (theta in {10,45} deg x 9 observer times), retarded-time epoch lerp on")
        return dict(name=name, grid=grid, j=j, beta=beta, views=views, store="f32", desc=desc, lookback=True)
    if name == "precision":
        n, size = int(round(512 * scale)), int(round(1024 * scale))
        grid, j, beta, views = gen.config_precision_device(n=n, size=size, device=device)
        desc = (f"precision: {n}^3 grid x 8 epochs turbulent jet, stored bf16 j' + fp16 u=Gamma*beta, FP32 "
                f"accumulation; one {size}x{size} view at theta=30, phi=20, t_obs mid-window")
        return dict(name=name, grid=grid, j=j, beta=beta, views=views, store="bf16", desc=desc, lookback=True)
    if name == "batched":
        n, size = int(round(384 * scale)), int(round(256 * scale))
        grid, j, beta, views = gen.config_batched_device(n=n, size=size, device=device)
        desc = (f"batched views: {n}^3 grid x 32 epochs FP32 turbulent jet, 256 orientations on a Fibonacci "
                f"sphere, {size}x{size} each, graph-captured batch render")
        return dict(name=name, grid=grid, j=j, beta=beta, views=views, store="f32", desc=desc, lookback=True)
    raise SystemExit(f"unknown workload {name}")


def host_fields(wl):
    """The workload's fields as host numpy arrays (the oracle's inputs)."""
    for key in ("j", "beta"):
        if hasattr(wl[key], "cpu"):
            wl[key] = wl[key].cpu().numpy()
    return wl


def parse_launch(spec: str):
    vals = [int(x) for x in spec.split(",")]
    pw, ph, warps, depth, regcap = vals[:5]
    region = vals[5] if len(vals) > 5 else 0
    group = vals[6] if len(vals) > 6 else 0
    return {"packet": (pw, ph), "cta_warps": warps, "depth": depth, "persistent": 0 if region else 1,
            "regcap": regcap, "region": region, "group": group}


def parse_layout(spec: str):
    """brick, super-brick, paired[, Morton cell order] (0 where not given)."""
    return ([int(x) for x in spec.split(",")] + [0, 0])[:4] if spec else (0, 0, 0, 0)


# ------------------------------------------------------------------ clocks
class ClockSampler:
    """Samples nvidia-smi clocks and throttle reasons while running."""
    FIELDS = ["clocks.sm", "clocks.max.sm", "power.draw", "clocks_event_reasons.active",
              "clocks_event_reasons.hw_slowdown", "clocks_event_reasons.hw_thermal_slowdown",
              "clocks_event_reasons.sw_thermal_slowdown", "clocks_event_reasons.sw_power_cap"]
    INTERVAL_MS = 50

    def __init__(self, index: int):
        self.index = index
        self.rows = []
        self.proc = None
        self.thread = None

    def __enter__(self):
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", f"--id={self.index}", "--query-gpu=" + ",".join(self.FIELDS),
                 "--format=csv,noheader,nounits", "-lms", str(self.INTERVAL_MS)],
                stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
            self.thread = threading.Thread(target=self._read, daemon=True)
            self.thread.start()
        except (OSError, ValueError):
            self.proc = None
        return self

    def _read(self):
        for line in self.proc.stdout:
            parts = [p.strip() for p in line.split(",")]
            if len(parts) == len(self.FIELDS):
                self.rows.append([time.perf_counter()] + parts)

    def __exit__(self, *exc):
        if self.proc:
            self.proc.terminate()
            try:
                self.proc.wait(timeout=5)
            except subprocess.TimeoutExpired:
                self.proc.kill()
            self.thread.join(timeout=5)

    def summary(self, t_start: float, t_end: float):
        """Clocks of the samples inside [t_start, t_end] (widened by one
        interval at each end; the nearest sample if none falls inside)."""
        lo = t_start - self.INTERVAL_MS * 1e-3
        hi = t_end + self.INTERVAL_MS * 1e-3
        rows = [r[1:] for r in list(self.rows) if lo <= r[0] <= hi]
        if not rows and self.rows:
            rows = [min(self.rows, key=lambda r: abs(r[0] - lo))[1:]]
        if not rows:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["unavailable"], "samples": 0}

        def num(x):
            try:
                return float(x)
            except ValueError:
                return None
        sm = [num(r[0]) for r in rows if num(r[0]) is not None]
        mx = [num(r[1]) for r in rows if num(r[1]) is not None]
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        reasons = sorted({names[i] for r in rows for i in range(4) if r[4 + i].lower() == "active"})
        pw = [num(r[2]) for r in rows if num(r[2]) is not None]
        return {"sm_mhz": statistics.median(sm) if sm else None, "sm_max_mhz": max(mx) if mx else None,
                "reasons": reasons, "samples": len(rows), "power_w_max": max(pw) if pw else None}


# ------------------------------------------------------------------ peaks
def reduce_over_ranks(value: float, op: str, device: str) -> float:
    """``value`` combined over all ranks of the default process group ("max" or
    "sum"); the value itself on a single process."""
    import torch
    import torch.distributed as dist
    if not (dist.is_available() and dist.is_initialized()) or dist.get_world_size() == 1:
        return float(value)
    t = torch.tensor([float(value)], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX if op == "max" else dist.ReduceOp.SUM)
    return float(t.item())


def measured_peak_hbm():
    path = os.path.join(ROOT, "MEASURED_PEAKS.json")
    try:
        with open(path) as f:
            d = json.load(f)
        return float(d["hbm_gbs"]), "measured"
    except (OSError, KeyError, ValueError):
        return 6800.0, "fallback"


def recorded_traffic(tag: str, launch: dict | None, layout):
    """Per-launch DRAM bytes from the committed ncu summary ``profiles/march_<tag>.md``,
    or None when absent, taken on a different kernel source, or taken on
    another launch shape or layout than the one timed."""
    path = os.path.join(ROOT, "profiles", f"march_{tag}.md")
    src = os.path.join(ROOT, "paper_2609_09322_gb300", "csrc", "march.cu")
    try:
        text = open(path).read()
        digest = hashlib.sha256(open(src, "rb").read()).hexdigest()[:16]
        m_hash = re.search(r"march\.cu sha256\[:16\]:\s*([0-9a-f]{16})", text)
        m_traffic = re.search(r"traffic_bytes_per_launch:\s*([0-9.eE+]+)", text)
        m_cfg = re.search(r"timed configuration:\s*--launch\s+(\S+)\s+--layout\s+(\S+)", text)
        if not (m_hash and m_traffic and m_cfg and m_hash.group(1) == digest):
            return None
        if launch is None or parse_launch(m_cfg.group(1)) != launch or parse_layout(m_cfg.group(2)) != list(layout):
            return None
        return float(m_traffic.group(1))
    except OSError:
        return None


def roofline(samples: int, bytes_per_sample: int, kernel_ms: float, traffic=None, compulsory=None):
    peak, kind = measured_peak_hbm()
    achieved = samples * bytes_per_sample / (kernel_ms * 1e-3) / 1e9
    return {"bound": "hbm", "achieved": round(achieved, 1), "peak": peak, "unit": "GB/s",
            "frac": round(achieved / peak, 4), "traffic": traffic, "peak_source": f"{kind} hbm_gbs (burst copy)",
            "bytes_per_sample": bytes_per_sample, "compulsory_bytes_per_step": compulsory,
            "kernel_ms_median": round(kernel_ms, 4)}


# ------------------------------------------------------------------ GPU timing
def load_volume(ctx, wl, store: str, layout):
    import torch
    brick, sbrick, paired, morton = layout
    t0 = time.perf_counter()
    vol = ctx.load_snapshots(wl["grid"], wl["j"], wl["beta"], store=store, brick=brick, super_brick=sbrick,
                             paired=bool(paired), morton_cells=bool(morton))
    torch.cuda.synchronize()
    return vol, ctx.volume_info(vol), time.perf_counter() - t0


def count_samples(ctx, vol, views, launch, stream) -> int:
    import torch
    with torch.cuda.stream(stream):
        _, cnt = ctx.render_batch(vol, views, samples=True, launch=launch, stream=stream)
    stream.synchronize()
    return int(cnt.to(torch.int64).sum().item())


def time_steps(step, steps: int, warmup: int, stream, world: int, dev: int):
    """W untimed steps, then K steps between CUDA events on the launching
    stream (synchronised, barrier on both sides); returns (per-step ms,
    whole-run ms max over ranks, wall-clock start and end of the timed part)."""
    import torch
    import torch.distributed as dist
    for _ in range(warmup):
        step()
    stream.synchronize()
    if world > 1:
        dist.barrier()
    torch.cuda.synchronize()
    ev = [torch.cuda.Event(enable_timing=True) for _ in range(steps + 1)]
    t_start = time.perf_counter()
    ev[0].record(stream)
    for k in range(steps):
        step()
        ev[k + 1].record(stream)
    stream.synchronize()
    t_end = time.perf_counter()
    torch.cuda.synchronize()
    per_step = [ev[k].elapsed_time(ev[k + 1]) for k in range(steps)]
    total_ms = ev[0].elapsed_time(ev[-1])
    if world > 1:
        dist.barrier()
        total_ms = reduce_over_ranks(total_ms, "max", f"cuda:{dev}")
    return per_step, total_ms, t_start, t_end


def march_entry(ctx, wl, vol, info, launch, stream, steps, warmup, world, dev, *, per_image=False, clk=None,
                label=""):
    """Times the batch render (or, per_image, one render call per view) of
    the workload's views; returns the entry dict and the last step's images."""
    import torch
    views = wl["views"]
    n_views = len(views)
    samples = count_samples(ctx, vol, views, None if per_image else launch, stream)
    out = torch.empty((n_views, views[0].height, views[0].width), dtype=torch.float32, device=f"cuda:{dev}")
    if per_image:
        def step():
            for k, v in enumerate(views):
                ctx.render(vol, v, out=out[k], stream=stream)
    else:
        def step():
            ctx.render_batch(vol, views, out=out, launch=launch, stream=stream)
    per_step, total_ms, t0, t1 = time_steps(step, steps, warmup, stream, world, dev)
    ms = total_ms / steps
    step()
    stream.synchronize()
    launches = n_views if per_image else ctx.last_launch_count()
    store = "f32" if info["store"] == 0 else "bf16"
    bytes_per_sample = RECORD_BYTES[store] * (2 if wl["lookback"] else 1)
    kernel_ms = statistics.median(per_step)
    entry = {
        "value": round(world * samples / (ms * 1e-3) / 1e9, 4), "unit": UNIT, "ms_per_step": round(ms, 4),
        "steps": steps, "warmup": warmup, "images_per_s": round(world * n_views / (ms * 1e-3), 2),
        "dtype": "f32" if store == "f32" else "bf16/f16 storage, f32 math",
        "gpu_launches": steps * launches,
        "config": {"workload": wl["desc"] + ("; plain per-image renders (one call per view)" if per_image else ""),
                   "images_per_step": n_views, "cell_samples_per_step": samples, "volume_bytes": info["bytes"],
                   "l2": L2_NOTE % (info["bytes"] / 1e9),
                   "layout": f"brick {info['brick']}, super-brick {info['super_brick']}"
                             + (", paired snapshots" if info.get("paired") else "")
                             + (", Morton cell order" if info.get("morton_cells") else ""),
                   "launch": "default" if per_image else
                             {k: launch[k] for k in ("packet", "cta_warps", "depth", "persistent", "regcap",
                                                     "region", "group")}},
        "roofline": roofline(samples, bytes_per_sample, kernel_ms),
    }
    if clk is not None:
        entry["clocks"] = clk.summary(t0, t1)
    entry["_t"] = (t0, t1)
    return entry, out.cpu().numpy(), samples


def with_oracle_error(entry, wl, images, seconds: float):
    """Adds the GPU's error against the FP64 oracle on a bounded random sample
    of the workload's pixels (the oracle reads the float32 fields the volume
    was made from)."""
    errors = []
    wl = dict(wl, gpu_images=images)
    oracle_sample(wl, seconds, seed=7, errors=errors)
    if errors:
        entry["oracle_error"] = oracle_error(errors, "f32" if entry["dtype"] == "f32" else "bf16")
    return entry


# ------------------------------------------------------------------ suite
def run_suite(args, rank: int, world: int):
    import torch
    from paper_2609_09322_gb300 import Context

    dev = int(os.environ.get("LOCAL_RANK", "0"))
    torch.cuda.set_device(dev)
    ctx = Context(dev)
    stream = torch.cuda.Stream()
    nested = {}
    oracle_s = args.nested_oracle_seconds
    with ClockSampler(dev) as clk:
        # ---- batched views: the top-level line
        wl = make_workload("batched", args.scale, device=f"cuda:{dev}")
        launch_s, layout_s = PINNED["batched"]
        layout = parse_layout(layout_s)
        vol, info, t_load = load_volume(ctx, wl, "f32", layout)
        launch = parse_launch(launch_s)
        tuned = None
        if args.tune:
            tuned = ctx.tune(vol, wl["views"], launch=True, layout=True, stream=stream)
            launch = {k: tuned[k] for k in ("packet", "cta_warps", "depth", "persistent", "regcap", "region", "group")}
            info = ctx.volume_info(vol)
            layout = [info["brick"], info["super_brick"], info["paired"]]
        wl_dev = wl
        wl = host_fields(dict(wl))  # host copies for the oracle; the packed volume is resident
        del wl_dev
        torch.cuda.empty_cache()
        top, images, samples = march_entry(ctx, wl, vol, info, launch, stream, args.steps, args.warmup, world, dev,
                                           clk=clk)
        t_top = top.pop("_t")
        top["roofline"]["compulsory_bytes_per_step"] = ctx.touched_records(vol, wl["views"]) * RECORD_BYTES["f32"]
        top["roofline"]["traffic"] = recorded_traffic("batched", launch, layout)
        top["e2e"] = e2e_batch(ctx, vol, wl["views"], launch, stream, samples, world, args.steps)
        top["load_s"] = round(t_load, 3)
        if tuned:
            top["config"]["tuned"] = {k: tuned[k] for k in ("ms", "candidates")}
        batched_images = images
        ctx.unload(vol)
        # the same workload stored as bfloat16/float16 records, and the plain
        # float32 per-image march (default layout and launch)
        for key, store, form in (("batched_bf16", "bf16", "batched_bf16"), ("batched_f32_per_image", "f32", None)):
            launch = parse_launch(PINNED[form][0]) if form else None
            layout = parse_layout(PINNED[form][1]) if form else (0, 0, 0, 0)
            vol, info, _ = load_volume(ctx, wl, store, layout)
            e, img, _ = march_entry(ctx, wl, vol, info, launch, stream, args.steps if form else max(3, min(args.steps, 5)),
                                    args.warmup if form else 3, world, dev, per_image=form is None, clk=clk)
            e.pop("_t")
            if form:
                e["roofline"]["traffic"] = recorded_traffic(form, launch, layout)
                e["config"]["workload"] += "; stored as bf16 j' + fp16 u"
            nested[key] = with_oracle_error(e, wl, img, oracle_s)
            ctx.unload(vol)
        torch.cuda.empty_cache()
        cpu = None
        if rank == 0 and world == 1 and not args.no_cpu_baseline:
            errors = []
            rate, pix, threads, el = oracle_sample(dict(wl, gpu_images=batched_images), args.cpu_seconds,
                                                   errors=errors)
            cpu = {"value": round(rate, 6), "unit": UNIT, "cores": threads, "kind": "oracle",
                   "sample": f"{pix} random pixels of the batched workload's views, {el:.1f} s"}
            top["oracle_error"] = oracle_error(errors, "f32")
        del wl, batched_images

        # ---- time-delay: float32 time groups, bfloat16/float16 records, per-image
        wl = make_workload("time_delay", args.scale)
        for key, store, form in (("time_delay_f32", "f32", "time_delay"),
                                 ("time_delay_f32_grouped", "f32", "time_delay_grouped"),
                                 ("time_delay_bf16", "bf16", "time_delay_bf16"),
                                 ("time_delay_f32_per_image", "f32", None)):
            launch = parse_launch(PINNED[form][0]) if form else None
            layout = parse_layout(PINNED[form][1]) if form else (0, 0, 0, 0)
            vol, info, _ = load_volume(ctx, wl, store, layout)
            e, img, _ = march_entry(ctx, wl, vol, info, launch, stream, args.steps if form else 10, args.warmup,
                                    world, dev, per_image=form is None, clk=clk)
            e.pop("_t")
            if form:
                e["roofline"]["traffic"] = recorded_traffic(form, launch, layout)
            nested[key] = with_oracle_error(e, wl, img, oracle_s)
            ctx.unload(vol)
        del wl
        torch.cuda.empty_cache()

        # ---- precision: bfloat16/float16 records, and the float32 per-image march
        wl = make_workload("precision", args.scale, device=f"cuda:{dev}")
        wl_host = None
        for key, store, form in (("precision_bf16", "bf16", "precision"), ("precision_f32_per_image", "f32", None)):
            launch = parse_launch(PINNED[form][0]) if form else None
            layout = parse_layout(PINNED[form][1]) if form else (0, 0, 0, 0)
            vol, info, _ = load_volume(ctx, wl, store, layout)
            e, img, _ = march_entry(ctx, wl, vol, info, launch, stream, args.steps if form else 10, args.warmup,
                                    world, dev, per_image=form is None, clk=clk)
            e.pop("_t")
            if form:
                e["roofline"]["traffic"] = recorded_traffic(form, launch, layout)
            if wl_host is None:
                wl_host = host_fields(dict(wl))
            nested[key] = with_oracle_error(e, wl_host, img, oracle_s)
            ctx.unload(vol)
        del wl, wl_host
        torch.cuda.empty_cache()

    # ---- serving: a short phase of continuous batching
    ctx.close()
    sargs = argparse.Namespace(**vars(args))
    sargs.serve_requests, sargs.serve_warmup = args.suite_serve_requests, args.suite_serve_warmup
    srv = run_serving(sargs, rank, world)
    nested["serving"] = {k: srv[k] for k in ("value", "unit", "p50_ms", "p99_ms", "serving", "config", "load_s")}
    nested["serving"]["note"] = "value: Gcell-samples/s at 0.95 of the saturated request rate"

    result = {
        "metric": METRIC, "value": top["value"], "unit": UNIT, "n_gpus": world, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": top["ms_per_step"], "higher_is_better": True, "scaling": "weak",
        "vs_baseline": None, "dtype": "f32", "data": "synthetic (seeded generators in gen/)",
        "config": dict(top["config"], parallelism="replicas" if world > 1 else "single GPU"),
        "images_per_s": top["images_per_s"],
        "rays_per_s": round(top["images_per_s"] * 256 * 256 * args.scale * args.scale, 1),
        "roofline": top["roofline"], "e2e": top["e2e"], "gpu_launches": top["gpu_launches"],
        "clocks": clk.summary(*t_top), "load_s": top["load_s"],
    }
    if "oracle_error" in top:
        result["oracle_error"] = top["oracle_error"]
    if cpu:
        result["cpu_baseline"] = cpu
    result["configs"] = nested
    return result


def e2e_batch(ctx, vol, views, launch, stream, samples, world, steps):
    """The batch render end to end through the public call with host output:
    per-view constants travel to the device in the launch parameters, every
    step's images come back into pinned host memory.  Two pinned buffers on two
    streams: step k's images are copied back while step k + 1 marches."""
    import torch
    n = len(views)
    streams = [stream, torch.cuda.Stream()]
    hosts = [torch.empty((n, views[0].height, views[0].width), dtype=torch.float32, pin_memory=True)
             for _ in range(2)]
    k = [0]

    def e2e_step():
        i = k[0] % 2
        k[0] += 1
        ctx.render_batch_host(vol, views, hosts[i], launch=launch, stream=streams[i])
    for _ in range(4):
        e2e_step()
    torch.cuda.synchronize()
    n_steps = max(4, min(steps, 40))
    t0 = time.perf_counter()
    for _ in range(n_steps):
        e2e_step()
    torch.cuda.synchronize()
    sec = (time.perf_counter() - t0) / n_steps
    return {"value": round(world * samples / sec / 1e9, 4), "unit": UNIT,
            "h2d_bytes_per_step": 216 * n, "d2h_bytes_per_step": hosts[0].numel() * 4,
            "note": "render_batch with host output on two streams, double-buffered (two steps in flight, so one "
                    "step's launch tail overlaps the next step's march); per-view constants H2D in the launch "
                    "parameters, images D2H into pinned memory, volume resident"}


# ------------------------------------------------------------------ one workload
def run_gpu(args, rank: int, world: int):
    import torch

    from paper_2609_09322_gb300 import Context

    dev = int(os.environ.get("LOCAL_RANK", "0"))
    torch.cuda.set_device(dev)
    wl = make_workload(args.workload, args.scale, device=f"cuda:{dev}")
    if args.store:
        wl["store"] = args.store
        wl["desc"] += f"; stored as {'bf16 j + fp16 u' if args.store == 'bf16' else 'fp32'}"
    views = wl["views"]
    n_views = len(views)
    ctx = Context(dev)
    layout = parse_layout(args.layout)
    vol, info, t_load = load_volume(ctx, wl, wl["store"], layout)
    host_fields(wl)
    torch.cuda.empty_cache()
    stream = torch.cuda.Stream()
    launch = None
    tuned = None
    if args.launch:
        launch = parse_launch(args.launch)
        tuned = dict(launch)
    elif args.tune and not args.per_image:
        # autotune the launch (and, with --tune-layout, the volume layout) before timing
        tuned = ctx.tune(vol, views, launch=True, layout=args.tune_layout, stream=stream)
        info = ctx.volume_info(vol)

    samples_per_step = count_samples(ctx, vol, views, launch, stream)
    out = torch.empty((n_views, views[0].height, views[0].width), dtype=torch.float32, device=f"cuda:{dev}")

    form_note = {}
    extra_bytes_per_sample = 0
    if args.form == "streamed":
        # the series in pinned host memory; each step uploads and marches it slab by slab
        j_h = torch.from_numpy(np.ascontiguousarray(wl["j"], dtype=np.float32)).pin_memory()
        b_h = torch.from_numpy(np.ascontiguousarray(wl["beta"], dtype=np.float32)).pin_memory()
        ctx.unload(vol)
        s_launch = launch or {"packet": (4, 8), "cta_warps": 4, "depth": 2, "persistent": 1, "regcap": 1}
        s_info = {}

        def step():
            _, s = ctx.render_streamed(wl["grid"], j_h.numpy(), b_h.numpy(), views, out=out, store=wl["store"],
                                       slab=args.slab, flexload=True, launch=s_launch, stream=stream)
            s_info.update(s)
        step()
        # the host link's measured rate: a 1 GiB pinned host-to-device copy
        probe_h = torch.empty(1 << 30, dtype=torch.uint8, pin_memory=True)
        probe_d = torch.empty(1 << 30, dtype=torch.uint8, device=f"cuda:{dev}")
        probe_d.copy_(probe_h, non_blocking=True)
        torch.cuda.synchronize()
        t_p = time.perf_counter()
        for _ in range(4):
            probe_d.copy_(probe_h, non_blocking=True)
        torch.cuda.synchronize()
        h2d_peak = 4 * (1 << 30) / (time.perf_counter() - t_p) / 1e9
        del probe_h, probe_d
        form_note = {"form": "streamed", "slab": args.slab, "flexload": True,
                     "h2d_peak_gb_per_s": round(h2d_peak, 1)}
    elif args.form == "labelled":
        g = wl["grid"]
        cut = g.n[0] // 2
        halves = []
        brick, sbrick, paired, morton = layout
        for lo, hi in ((0, cut), (cut, g.n[0])):
            sub = type(g)(n=(hi - lo, g.n[1], g.n[2]), origin=(g.origin[0] + lo * g.dx[0], g.origin[1], g.origin[2]),
                          dx=g.dx, n_epochs=g.n_epochs, t0=g.t0, dt=g.dt)
            halves.append(ctx.load_snapshots(sub, np.ascontiguousarray(wl["j"][..., lo:hi]),
                                             np.ascontiguousarray(wl["beta"][..., lo:hi, :]), store=wl["store"],
                                             brick=brick, super_brick=sbrick, paired=bool(paired),
                                             morton_cells=bool(morton)))

        def step():
            ctx.render_labelled(halves, views, out=out, launch=launch, stream=stream)
        form_note = {"form": "labelled", "sub_domains": 2}
    elif args.form == "vector":
        jj = np.ascontiguousarray(wl["j"], dtype=np.float32)
        ctx.load_channels(vol, np.stack([2.0 * jj, jj * jj, -jj]))
        vout = torch.empty((n_views, 4, views[0].height, views[0].width), dtype=torch.float32, device=f"cuda:{dev}")
        extra_bytes_per_sample = 3 * 4 * (2 if wl["lookback"] else 1)

        def step():
            ctx.render_vector(vol, views, out=vout, launch=launch, stream=stream)
        form_note = {"form": "vector", "channels": 1 + 3}
    elif args.per_image:
        # the plain per-image march: one render call per view, no batching
        def step():
            for k, v in enumerate(views):
                ctx.render(vol, v, out=out[k], launch=launch, stream=stream)
    else:
        def step():
            ctx.render_batch(vol, views, out=out, launch=launch, stream=stream)

    with ClockSampler(dev) as clk:
        # keep the GPU busy while the sampler starts (untimed)
        t_busy = time.perf_counter()
        while time.perf_counter() - t_busy < 0.3:
            step()
            stream.synchronize()
        per_step, total_ms, t0, t1 = time_steps(step, args.steps, args.warmup, stream, world, dev)
    ms_per_step = total_ms / args.steps
    step()  # one more, untimed, to read how many march kernels a step launches
    stream.synchronize()
    launches = args.steps * (n_views if args.per_image else ctx.last_launch_count())

    # end to end through the public API with host buffers
    if args.form == "batch" and not args.per_image:
        e2e = e2e_batch(ctx, vol, views, launch, stream, samples_per_step, world, args.steps)
    else:
        dev_img = vout if args.form == "vector" else out
        host = torch.empty(dev_img.shape, dtype=torch.float32, pin_memory=True)

        def e2e_step():
            step()
            with torch.cuda.stream(stream):
                host.copy_(dev_img, non_blocking=True)
        for _ in range(4):
            e2e_step()
        torch.cuda.synchronize()
        e2e_steps = max(4, min(args.steps, 40))
        t_e = time.perf_counter()
        for _ in range(e2e_steps):
            e2e_step()
            stream.synchronize()
        e2e_s = (time.perf_counter() - t_e) / e2e_steps
        view_bytes = 216 * n_views
        if args.form == "streamed":
            view_bytes += int(s_info.get("bytes_uploaded", 0))  # the series itself, slab by slab
        e2e = {"value": round(world * samples_per_step / e2e_s / 1e9, 4), "unit": UNIT,
               "h2d_bytes_per_step": view_bytes, "d2h_bytes_per_step": host.numel() * 4,
               "note": ("one render call per view" if args.per_image else f"the {args.form} form's call")
                       + ", then the images D2H into pinned memory; per-view constants H2D in the launch parameters"}

    rec = RECORD_BYTES[wl["store"]]
    bytes_per_sample = rec * (2 if wl["lookback"] else 1) + extra_bytes_per_sample
    compulsory = ctx.touched_records(vol, views) * rec if args.form == "batch" else None
    kernel_ms = statistics.median(per_step)
    tag = args.workload + ("_bf16" if args.store == "bf16" and args.workload != "precision" else "")
    traffic = (recorded_traffic(tag, launch, parse_layout(args.layout))
               if args.form == "batch" and not args.per_image else None)
    value = world * samples_per_step / (ms_per_step * 1e-3) / 1e9
    result = {
        "metric": METRIC, "value": round(value, 4), "unit": UNIT, "n_gpus": world, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": round(ms_per_step, 4), "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None, "dtype": "f32" if wl["store"] == "f32" else "bf16/f16 storage, f32 math",
        "data": "synthetic (seeded generators in gen/)",
        "config": {"workload": wl["desc"] + ("; plain per-image renders" if args.per_image else "")
                   + {"batch": "", "streamed": f"; out-of-core: series in pinned host memory, {args.slab}-cell "
                                                f"slabs uploaded with flexload each step",
                      "labelled": "; labelled: two sub-domains (halves along x)",
                      "vector": "; vector: j' and three extra emissivity channels per ray"}[args.form],
                   "images_per_step": n_views,
                   "cell_samples_per_step": samples_per_step,
                   "volume_bytes": info["bytes"], "l2": L2_NOTE % (info["bytes"] / 1e9),
                   "parallelism": "replicas" if world > 1 else "single GPU",
                   "layout": f"brick {info['brick']}, super-brick {info['super_brick']}"
                             + (", paired snapshots" if info.get("paired") else "")
                             + (", Morton cell order" if info.get("morton_cells") else ""),
                   "launch": ({k: tuned[k] for k in ("packet", "cta_warps", "depth", "persistent", "regcap", "region", "group") if k in tuned}
                              if tuned else "default")},
        "images_per_s": round(world * n_views / (ms_per_step * 1e-3), 2),
        "rays_per_s": round(world * n_views * views[0].width * views[0].height / (ms_per_step * 1e-3), 1),
        "roofline": dict(roofline(samples_per_step, bytes_per_sample, kernel_ms, traffic, compulsory)),
        "e2e": e2e,
        "gpu_launches": launches,
        **({"form": form_note} if form_note else {}),
        **({"streamed": {"bytes_uploaded_per_step": int(s_info.get("bytes_uploaded", 0)),
                         "bytes_of_series": int(s_info.get("bytes_total", 0)), "slabs": int(s_info.get("slabs", 0)),
                         "upload_gb_per_s": round(s_info.get("bytes_uploaded", 0) / (ms_per_step * 1e-3) / 1e9, 1),
                         "link_frac": round(s_info.get("bytes_uploaded", 0) / (ms_per_step * 1e-3) / 1e9
                                            / max(form_note.get("h2d_peak_gb_per_s", 1.0), 1e-9), 3)}}
           if args.form == "streamed" else {}),
        "load_s": round(t_load, 3),
        "clocks": clk.summary(t0, t1),
    }
    ctx.close()
    # the last step's images, for the oracle comparison of the CPU-baseline leg
    wl["gpu_images"] = (vout[:, 0] if args.form == "vector" else out).cpu().numpy()
    return result, wl


# ------------------------------------------------------------------ serving
SERVING_CATALOGUE = [  # (n, epochs, store)
    (64, 32, "f32"), (128, 16, "bf16"), (256, 32, "f32"), (384, 8, "bf16"), (512, 8, "f32"), (512, 32, "bf16")]


def run_serving(args, rank: int, world: int):
    """Continuous batching under Poisson load: p50/p99 latency (submission to
    completion on the GPU), throughput and cell-samples/s at 0.5, 0.8 and
    0.95 of the saturated request rate."""
    import torch
    import gen
    from paper_2609_09322_gb300 import Context

    dev = int(os.environ.get("LOCAL_RANK", "0"))
    torch.cuda.set_device(dev)
    device = f"cuda:{dev}"
    ctx = Context(dev)
    vols, grids = [], []
    t_load = time.perf_counter()
    for k, (n, m, store) in enumerate(SERVING_CATALOGUE):
        n = max(8, int(round(n * args.scale)))
        grid = gen.Grid(n=(n, n, n), n_epochs=m, t0=0.0, dt=n / 16.0)
        j, beta = gen.turbulent_jet_torch(grid, 50 + k, device)
        vols.append(ctx.load_snapshots(grid, j, beta, store=store))
        grids.append(grid)
        del j, beta
        torch.cuda.empty_cache()
    t_load = time.perf_counter() - t_load
    resident = sum(ctx.volume_info(v)["bytes"] for v in vols)
    rng = np.random.default_rng(args.seed)

    def make_requests(count):
        reqs = []
        for _ in range(count):
            k = int(rng.integers(len(vols)))
            grid = grids[k]
            size = max(8, int(round(int(rng.choice([128, 256, 512, 1024])) * args.scale)))
            d = rng.normal(size=3)
            t_obs = float(rng.uniform(0.0, (grid.n_epochs - 1) * grid.dt))
            reqs.append((vols[k], gen.view_from_direction(grid, -d, size=size, c=1.0, t_obs=t_obs)))
        return reqs

    reqs = make_requests(args.serve_requests + args.serve_warmup)
    outs = [torch.empty((v.height, v.width), dtype=torch.float32, device=device) for _, v in reqs]
    # cell-samples of every request, counted once outside the timed phases
    samples = []
    for vol, view in reqs:
        _, cnt = ctx.render(vol, view, samples=True)
        samples.append(cnt)
    torch.cuda.synchronize()
    samples = [int(c.to(torch.int64).sum().item()) for c in samples]
    ctx.serve_start(max_waves=args.serve_waves, max_requests_per_wave=args.serve_wave_size)

    def run_phase(rate, lo, hi):
        """Submit requests lo..hi-1 (Poisson at `rate` per second, or all at
        once when rate is None); returns stats of the measured part."""
        ctx.serve_stats(reset=True)
        tickets = []
        t = time.perf_counter()
        next_t = t
        warm = min(args.serve_warmup, hi - lo)
        for i in range(lo, hi):
            if rate:
                next_t += float(rng.exponential(1.0 / rate))
                while time.perf_counter() < next_t:
                    pass
            if i == lo + warm:
                for tk in tickets:
                    ctx.wait(tk, 120000)
                tickets = []
                ctx.serve_stats(reset=True)
                t_meas = time.perf_counter()
                s_meas = 0
            tickets.append(ctx.submit(reqs[i][0], reqs[i][1], outs[i]))
            if i >= lo + warm:
                s_meas += samples[i]
        for tk in tickets:
            ctx.wait(tk, 120000)
        st = ctx.serve_stats()
        span = time.perf_counter() - t_meas
        return dict(offered_per_s=round(rate, 1) if rate else None, completed=st["completed"],
                    p50_ms=round(st["p50_ms"], 3), p99_ms=round(st["p99_ms"], 3), max_ms=round(st["max_ms"], 3),
                    requests_per_s=round(st["completed"] / span, 1),
                    gcell_samples_per_s=round(s_meas / span / 1e9, 3),
                    mean_requests_per_wave=round(st["mean_requests_per_wave"], 2),
                    max_waves_in_flight=st["max_waves_in_flight"])

    total = len(reqs)
    sat = run_phase(None, 0, total)
    r_sat = sat["requests_per_s"]
    points = [run_phase(f * r_sat, 0, total) for f in (0.5, 0.8, 0.95)]
    # replicas: every rank serves its own stream; rates add up over the ranks
    # and latencies are the worst rank's
    for ph in [sat] + points:
        for k in ("requests_per_s", "gcell_samples_per_s", "completed"):
            ph[k] = round(reduce_over_ranks(ph[k], "sum", device), 3)
        for k in ("p50_ms", "p99_ms", "max_ms"):
            ph[k] = round(reduce_over_ranks(ph[k], "max", device), 3)
    top = points[-1]
    result = {
        "metric": METRIC, "value": top["gcell_samples_per_s"], "unit": UNIT, "n_gpus": world,
        "steps": args.serve_requests, "warmup": args.serve_warmup, "higher_is_better": True, "scaling": "weak",
        "vs_baseline": None, "dtype": "f32 / bf16+f16 storage, f32 math", "data": "synthetic (seeded generators in gen/)",
        "config": {"workload": "serving: Poisson stream of render requests over a resident catalogue of "
                               + ", ".join(f"{n}^3x{m} {st}" for n, m, st in SERVING_CATALOGUE)
                               + "; images 128^2-1024^2, random orientations and observer times",
                   "resident_bytes": resident, "max_waves": args.serve_waves,
                   "max_requests_per_wave": args.serve_wave_size},
        "serving": {"saturated": sat, "load_points": points},
        "p50_ms": top["p50_ms"], "p99_ms": top["p99_ms"],
        "load_s": round(t_load, 1),
    }
    ctx.close()
    return result


# ------------------------------------------------------------------ CPU oracle
def oracle_sample(wl, seconds: float, seed: int = 0, errors: list | None = None):
    """Times the oracle on a random sample of the workload's pixels until
    about ``seconds`` of work; returns (cell-samples/s, pixels, threads).
    With ``errors`` (and the GPU's images in wl), appends per batch the
    oracle's values with the GPU's values of the same pixels."""
    import oracle
    rng = np.random.default_rng(seed)
    views = wl["views"]
    threads = oracle.max_threads()
    done_samples, done_pix, elapsed = 0, 0, 0.0
    batch = 256
    while elapsed < seconds:
        vi = int(rng.integers(len(views)))
        v = views[vi]
        pix = np.stack([rng.integers(0, v.width, batch), rng.integers(0, v.height, batch)], axis=1)
        t0 = time.perf_counter()
        val, cnt = oracle.render_pixels(wl["grid"], wl["j"], wl["beta"], v, pix, counts=True)
        dt = time.perf_counter() - t0
        elapsed += dt
        done_samples += int(cnt.sum())
        done_pix += batch
        if errors is not None and "gpu_images" in wl:
            errors.append((val, wl["gpu_images"][vi][pix[:, 1], pix[:, 0]].astype(np.float64)))
        if dt < 0.5 * seconds / 4 and batch < 65536:
            batch *= 2
    return done_samples / elapsed / 1e9, done_pix, threads, elapsed


def oracle_error(errors, store: str):
    """The GPU's error on the oracle's sampled pixels, per pixel relative to
    |I_ref| + 1e-3 max(I_ref) (the parity tests' floor).  For float32 storage
    the oracle reads the same float32 fields as the GPU (kernel arithmetic);
    for BF16/FP16 storage it reads the float32 fields the records were made
    from (storage and arithmetic together)."""
    ref = np.concatenate([e[0] for e in errors])
    gpu = np.concatenate([e[1] for e in errors])
    peak = float(np.abs(ref).max()) if ref.size else 0.0
    rel = np.abs(gpu - ref) / (np.abs(ref) + 1e-3 * peak + 1e-300)
    tol = 1e-5 if store == "f32" else 1e-2
    return {"pixels": int(ref.size), "max_rel": float(f"{rel.max():.3g}"), "p99_rel": float(f"{np.quantile(rel, 0.99):.3g}"),
            "within_tolerance": round(float((rel <= tol).mean()), 6), "tolerance": tol,
            "flux_rel": float(f"{abs(gpu.sum() - ref.sum()) / max(abs(ref.sum()), 1e-300):.3g}"),
            "reference": "FP64 oracle on the stored float32 fields" if store == "f32"
                         else "FP64 oracle on the float32 fields the BF16/FP16 records were made from"}


def run_reference(args, rank: int):
    """The FP64 oracle timed on the machine's host cores on bounded random pixel
    samples of the workload the GPU arm's top-level line times.  The fields
    are built on the GPU when one is present (input generation only; the
    oracle never touches the device), else on the host."""
    name = args.workload or "batched"
    device = "cpu"
    try:
        import torch
        if torch.cuda.is_available() and name in ("precision", "batched"):
            device = "cuda:0"
    except ImportError:
        pass
    wl = host_fields(make_workload(name, args.scale, device=device))
    per_step = []
    n_pix = 0
    threads = 1
    budget = max(2.0, min(10.0, 150.0 / max(1, args.steps + args.warmup)))
    for k in range(args.warmup + args.steps):
        rate, pix, threads, _ = oracle_sample(wl, budget, seed=k)
        if k >= args.warmup:
            per_step.append(rate)
            n_pix += pix
    value = statistics.mean(per_step)
    return {
        "impl": "reference", "metric": METRIC, "value": round(value, 6), "unit": UNIT, "n_gpus": 1,
        "steps": args.steps, "warmup": args.warmup, "higher_is_better": True, "scaling": "weak",
        "vs_baseline": None, "dtype": "f64", "data": "synthetic (seeded generators in gen/)",
        "config": {"workload": wl["desc"]},
        "cpu_baseline": {"value": round(value, 6), "unit": UNIT, "cores": threads, "kind": "oracle",
                         "sample": f"{n_pix} random pixels of the workload's views over {args.steps} steps"},
        "e2e": {"value": round(value, 6), "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }


def main():
    ap = argparse.ArgumentParser(description=__doc__, formatter_class=argparse.RawDescriptionHelpFormatter)
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=20)
    ap.add_argument("--warmup", type=int, default=5)
    ap.add_argument("--impl", default="gbdart", choices=["gbdart", "reference"])
    ap.add_argument("--workload", default="", choices=["", "time_delay", "precision", "batched", "serving"],
                    help="one workload alone (default: the suite, see above)")
    ap.add_argument("--serve-requests", type=int, default=2000)
    ap.add_argument("--serve-warmup", type=int, default=200)
    ap.add_argument("--suite-serve-requests", type=int, default=600)
    ap.add_argument("--suite-serve-warmup", type=int, default=100)
    ap.add_argument("--serve-waves", type=int, default=3)
    ap.add_argument("--serve-wave-size", type=int, default=64)
    ap.add_argument("--seed", type=int, default=5)
    ap.add_argument("--scale", type=float, default=1.0,
                    help="linear size factor of the workload's grid and images (1 = the stated "
                         "configuration; smaller cases are for profiling)")
    ap.add_argument("--cpu-seconds", type=float, default=12.0, help="oracle work for the cpu_baseline key")
    ap.add_argument("--nested-oracle-seconds", type=float, default=2.0,
                    help="oracle work for each nested entry's oracle_error")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--tune", action="store_true", help="run the autotuner instead of the fixed launch and layout")
    ap.add_argument("--tune-layout", action="store_true", help="with --tune and --workload: also tune the layout")
    ap.add_argument("--store", default="", choices=["", "f32", "bf16"], help="override the workload's storage")
    ap.add_argument("--form", default="batch", choices=["batch", "streamed", "labelled", "vector"],
                    help="form of the march (see the module docstring)")
    ap.add_argument("--slab", type=int, default=64, help="z cells per slab of the streamed form")
    ap.add_argument("--per-image", action="store_true",
                    help="plain per-image march: one render call per view, default layout, no tuning")
    ap.add_argument("--launch", default="", help="fixed launch: packet_w,packet_h,warps,depth,regcap[,region[,group]]")
    ap.add_argument("--layout", default="", help="fixed volume layout: brick,super_brick[,paired]")
    args = ap.parse_args()
    if args.warmup < 3:
        raise SystemExit("--warmup must be >= 3")
    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))

    if args.impl == "reference":
        if rank == 0:
            print(json.dumps(run_reference(args, rank)), flush=True)
        return

    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl")
        import torch
        torch.cuda.set_device(int(os.environ.get("LOCAL_RANK", "0")))
    if args.workload == "serving":
        result = run_serving(args, rank, world)
    elif not args.workload:
        result = run_suite(args, rank, world)
    else:
        if args.workload in PINNED and not args.launch and not args.tune and not args.per_image:
            key = args.workload + ("_bf16" if args.store == "bf16" and args.workload != "precision" else "")
            args.launch = PINNED[key][0]
            args.layout = args.layout or PINNED[key][1]
        result, wl = run_gpu(args, rank, world)
        if rank == 0 and world == 1 and not args.no_cpu_baseline:
            errors = []
            rate, pix, threads, el = oracle_sample(wl, args.cpu_seconds, errors=errors)
            result["cpu_baseline"] = {"value": round(rate, 6), "unit": UNIT, "cores": threads, "kind": "oracle",
                                      "sample": f"{pix} random pixels of the workload's views, {el:.1f} s"}
            if errors:
                result["oracle_error"] = oracle_error(errors, wl["store"])
    if rank == 0:
        print(json.dumps(result), flush=True)
    if world > 1:
        import torch.distributed as dist
        dist.destroy_process_group()


if __name__ == "__main__":
    main()
