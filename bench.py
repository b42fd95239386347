"""Benchmark of the relativistic ray march on one GB300 (or N replicas).

A step is one pass of the whole hot path over one batch of views: the
persistent, graph-captured batch render of every view of the workload, with
the snapshot volume resident in HBM (loaded and packed once, before timing).

Workloads (synthetic, seeded; see gen/):
  time_delay (default)  256^3 x 16 epochs, float32 j' and beta: a Gaussian
                        blob (sigma = 8 cells) at beta = 0.95 z over a steady
                        conical jet; 512^2 images at theta in {10, 45} deg x 9
                        observer times = 18 images per step, lookback on.
  precision             512^3 x 8 turbulent jet stored as bfloat16 j' +
                        float16 four-velocity, one 1024^2 view.
  batched               384^3 x 32 turbulent jet, float32, 256 views of 256^2
                        on a Fibonacci sphere in one persistent launch.

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


# ------------------------------------------------------------------ inputs
def make_workload(name: str, scale: float = 1.0, device: str = "cpu"):
    import gen
    if name == "time_delay":
        n, size = int(round(256 * scale)), int(round(512 * scale))
        grid, j, beta, views = gen.config_time_delay(n=n, size=size, dtype=np.float32)
        desc = (f"time-delay path: {n}^3 grid x 16 epochs FP32 (j', beta), Gaussian blob sigma={8 * scale:g} "
                f"cells at beta=0.95 z over a steady conical jet, c*dt=4 cells; 18 images of {size}x{size} per "
                "step (theta in {10,45} deg x 9 observer times), retarded-time epoch lerp on")
        return dict(grid=grid, j=j, beta=beta, views=views, store="f32", desc=desc, lookback=True)
    if name == "precision":
        grid, j, beta, views = gen.config_precision_device(device=device)
        desc = ("precision: 512^3 grid x 8 epochs turbulent jet, stored bf16 j' + fp16 u=Gamma*beta, FP32 "
                "accumulation; one 1024x1024 view at theta=30, phi=20, t_obs mid-window")
        return dict(grid=grid, j=j, beta=beta, views=views, store="bf16", desc=desc, lookback=True)
    if name == "batched":
        grid, j, beta, views = gen.config_batched_device(device=device)
        desc = ("batched views: 384^3 grid x 32 epochs FP32 turbulent jet, 256 orientations on a Fibonacci "
                "sphere, 256x256 each, one persistent graph-captured launch")
        return dict(grid=grid, j=j, beta=beta, views=views, store="f32", desc=desc, lookback=True)
    raise SystemExit(f"unknown workload {name}")


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

    def mark(self, name: str):
        setattr(self, name, time.perf_counter())

    def __exit__(self, *exc):
        if self.proc:
            self.proc.terminate()
            try:
                self.proc.wait(timeout=5)
            except subprocess.TimeoutExpired:
                self.proc.kill()
            self.thread.join(timeout=5)

    def summary(self):
        # samples inside the timed region (widened by one interval at each end)
        lo = getattr(self, "t_start", -math.inf) - self.INTERVAL_MS * 1e-3
        hi = getattr(self, "t_end", math.inf) + self.INTERVAL_MS * 1e-3
        rows = [r[1:] for r in self.rows if lo <= r[0] <= hi]
        if not rows and self.rows:
            rows = [min(self.rows, key=lambda r: abs(r[0] - lo))[1:]]
        self.rows = rows
        if not self.rows:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["unavailable"], "samples": 0}
        def num(x):
            try:
                return float(x)
            except ValueError:
                return None
        sm = [num(r[0]) for r in self.rows if num(r[0]) is not None]
        mx = [num(r[1]) for r in self.rows if num(r[1]) is not None]
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        reasons = sorted({names[i] for r in self.rows for i in range(4) if r[4 + i].lower() == "active"})
        pw = [num(r[2]) for r in self.rows if num(r[2]) is not None]
        return {"sm_mhz": statistics.median(sm) if sm else None, "sm_max_mhz": max(mx) if mx else None,
                "reasons": reasons, "samples": len(self.rows), "power_w_max": max(pw) if pw else None}


# ------------------------------------------------------------------ peaks
def measured_peak_hbm():
    path = os.path.join(ROOT, "MEASURED_PEAKS.json")
    try:
        with open(path) as f:
            d = json.load(f)
        return float(d["hbm_gbs"]), "measured"
    except (OSError, KeyError, ValueError):
        return 6800.0, "fallback"


def recorded_traffic(kernel_tag: str):
    """Per-launch DRAM bytes from the committed ncu summary of this workload,
    or None when absent or taken on a different kernel source."""
    path = os.path.join(ROOT, "profiles", f"march_{kernel_tag}.md")
    src = os.path.join(ROOT, "paper_2609_09322_gb300", "csrc", "march.cu")
    try:
        text = open(path).read()
        digest = hashlib.sha256(open(src, "rb").read()).hexdigest()[:16]
        m_hash = re.search(r"march\.cu sha256\[:16\]:\s*([0-9a-f]{16})", text)
        m_traffic = re.search(r"traffic_bytes_per_launch:\s*([0-9.eE+]+)", text)
        if m_hash and m_traffic and m_hash.group(1) == digest:
            return float(m_traffic.group(1))
    except OSError:
        pass
    return None


# ------------------------------------------------------------------ GPU arm
def run_gpu(args, rank: int, world: int):
    import torch
    import torch.distributed as dist

    from paper_2609_09322_gb300 import Context

    dev = int(os.environ.get("LOCAL_RANK", "0"))
    torch.cuda.set_device(dev)
    wl = make_workload(args.workload, args.scale, device=f"cuda:{dev}")
    views = wl["views"]
    n_views = len(views)
    ctx = Context(dev)
    t_load = time.perf_counter()
    vol = ctx.load_snapshots(wl["grid"], wl["j"], wl["beta"], store=wl["store"])
    torch.cuda.synchronize()
    t_load = time.perf_counter() - t_load
    info = ctx.volume_info(vol)
    if isinstance(wl["j"], torch.Tensor) and wl["j"].is_cuda:
        # the packed volume is resident; keep host copies of the inputs only
        # for the CPU oracle baseline
        wl["j"] = wl["j"].cpu().numpy()
        wl["beta"] = wl["beta"].cpu().numpy()
        torch.cuda.empty_cache()
    stream = torch.cuda.Stream()
    launch = None
    tuned = None
    if not args.no_tune:
        # autotune the launch (and, with --tune-layout, the volume layout) before timing
        tuned = ctx.tune(vol, views, launch=True, layout=args.tune_layout, stream=stream)
        info = ctx.volume_info(vol)

    # cell-samples of one step (counted once, outside the timed region)
    with torch.cuda.stream(stream):
        _, cnt = ctx.render_batch(vol, views, samples=True, launch=launch, stream=stream)
    stream.synchronize()
    samples_per_step = int(cnt.to(torch.int64).sum().item())
    del cnt
    out = torch.empty((n_views, views[0].height, views[0].width), dtype=torch.float32, device=f"cuda:{dev}")

    def step():
        ctx.render_batch(vol, views, out=out, launch=launch, stream=stream)

    for _ in range(args.warmup):
        step()
    stream.synchronize()
    if world > 1:
        dist.barrier()
    torch.cuda.synchronize()
    ev = [torch.cuda.Event(enable_timing=True) for _ in range(args.steps + 1)]
    with ClockSampler(dev) as clk:
        # keep the GPU busy while the sampler starts (untimed)
        t_busy = time.perf_counter()
        while time.perf_counter() - t_busy < 0.3:
            step()
            stream.synchronize()
        clk.mark("t_start")
        ev[0].record(stream)
        for k in range(args.steps):
            step()
            ev[k + 1].record(stream)
        stream.synchronize()
        clk.mark("t_end")
    torch.cuda.synchronize()
    per_step = [ev[k].elapsed_time(ev[k + 1]) for k in range(args.steps)]
    total_ms = ev[0].elapsed_time(ev[-1])
    if world > 1:
        dist.barrier()
        t = torch.tensor([total_ms], device=f"cuda:{dev}")
        dist.all_reduce(t, op=dist.ReduceOp.MAX)
        total_ms = float(t.item())
    ms_per_step = total_ms / args.steps
    launches = args.steps * 1  # one march kernel per graph replay

    # end to end through the public API with host buffers
    host = torch.empty((n_views, views[0].height, views[0].width), dtype=torch.float32, pin_memory=True)
    for _ in range(2):
        ctx.render_batch_host(vol, views, host, stream=stream)
    stream.synchronize()
    e2e_steps = max(3, min(args.steps, 20))
    t0 = time.perf_counter()
    for _ in range(e2e_steps):
        ctx.render_batch_host(vol, views, host, stream=stream)
        stream.synchronize()
    e2e_s = (time.perf_counter() - t0) / e2e_steps
    view_bytes = 208 * n_views  # float64/float32 view record copied per step
    img_bytes = host.numel() * 4

    rec = RECORD_BYTES[wl["store"]]
    bytes_per_sample = rec * (2 if wl["lookback"] else 1)
    alg_bytes = samples_per_step * bytes_per_sample
    kernel_ms = statistics.median(per_step)
    achieved = alg_bytes / (kernel_ms * 1e-3) / 1e9
    peak, peak_kind = measured_peak_hbm()
    traffic = recorded_traffic(args.workload)
    value = world * samples_per_step / (ms_per_step * 1e-3) / 1e9
    result = {
        "metric": METRIC, "value": round(value, 4), "unit": UNIT, "n_gpus": world, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": round(ms_per_step, 4), "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None, "dtype": "f32" if wl["store"] == "f32" else "bf16/f16 storage, f32 math",
        "data": "synthetic (seeded generators in gen/)",
        "config": {"workload": wl["desc"], "images_per_step": n_views,
                   "cell_samples_per_step": samples_per_step,
                   "volume_bytes": info["bytes"], "l2": "inputs larger than L2 (resident volume %.1f GB)"
                   % (info["bytes"] / 1e9), "parallelism": "replicas" if world > 1 else "single GPU",
                   "layout": f"brick {info['brick']}, super-brick {info['super_brick']}",
                   "launch": ({k: tuned[k] for k in ("packet", "cta_warps", "depth", "persistent", "regcap")}
                              if tuned else "default")},
        "images_per_s": round(world * n_views / (ms_per_step * 1e-3), 2),
        "rays_per_s": round(world * n_views * views[0].width * views[0].height / (ms_per_step * 1e-3), 1),
        "roofline": {"bound": "hbm", "achieved": round(achieved, 1), "peak": peak, "unit": "GB/s",
                     "frac": round(achieved / peak, 4), "traffic": traffic,
                     "peak_source": f"{peak_kind} hbm_gbs", "bytes_per_sample": bytes_per_sample,
                     "kernel_ms_median": round(kernel_ms, 4)},
        "e2e": {"value": round(world * samples_per_step / e2e_s / 1e9, 4), "unit": UNIT,
                "h2d_bytes_per_step": view_bytes, "d2h_bytes_per_step": img_bytes,
                "note": "render_batch with host output: view table H2D, images D2H into pinned memory, "
                        "volume resident"},
        "gpu_launches": launches,
        "load_s": round(t_load, 3),
    }
    ctx.close()
    return result, clk.summary(), wl


# ------------------------------------------------------------------ CPU oracle
def oracle_sample(wl, seconds: float, seed: int = 0):
    """Times the oracle on a random sample of the workload's pixels until
    about ``seconds`` of work; returns (cell-samples/s, pixels, threads)."""
    import oracle
    rng = np.random.default_rng(seed)
    views = wl["views"]
    threads = oracle.max_threads()
    done_samples, done_pix, elapsed = 0, 0, 0.0
    batch = 256
    while elapsed < seconds:
        v = views[int(rng.integers(len(views)))]
        pix = np.stack([rng.integers(0, v.width, batch), rng.integers(0, v.height, batch)], axis=1)
        t0 = time.perf_counter()
        _, cnt = oracle.render_pixels(wl["grid"], wl["j"], wl["beta"], v, pix, counts=True)
        dt = time.perf_counter() - t0
        elapsed += dt
        done_samples += int(cnt.sum())
        done_pix += batch
        if dt < 0.5 * seconds / 4 and batch < 65536:
            batch *= 2
    return done_samples / elapsed / 1e9, done_pix, threads, elapsed


def run_reference(args, rank: int):
    wl = make_workload(args.workload, args.scale, device="cpu")
    for key in ("j", "beta"):
        if hasattr(wl[key], "numpy"):
            wl[key] = wl[key].numpy()
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
    ap.add_argument("--steps", type=int, default=200)
    ap.add_argument("--warmup", type=int, default=10)
    ap.add_argument("--impl", default="gbdart", choices=["gbdart", "reference"])
    ap.add_argument("--workload", default="time_delay", choices=["time_delay", "precision", "batched"])
    ap.add_argument("--scale", type=float, default=1.0,
                    help="linear size factor of the time_delay workload (1 = the stated configuration; "
                         "smaller cases are for profiling)")
    ap.add_argument("--cpu-seconds", type=float, default=12.0, help="oracle work for the cpu_baseline key")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-tune", action="store_true", help="skip the launch autotuner (default configuration)")
    ap.add_argument("--tune-layout", action="store_true", help="also autotune the volume's brick layout")
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
    result, clocks, wl = run_gpu(args, rank, world)
    result["clocks"] = clocks
    if rank == 0 and world == 1 and not args.no_cpu_baseline:
        rate, pix, threads, el = oracle_sample(wl, args.cpu_seconds)
        result["cpu_baseline"] = {"value": round(rate, 6), "unit": UNIT, "cores": threads, "kind": "oracle",
                                  "sample": f"{pix} random pixels of the workload's views, {el:.1f} s"}
    if rank == 0:
        print(json.dumps(result), flush=True)
    if world > 1:
        import torch.distributed as dist
        dist.destroy_process_group()


if __name__ == "__main__":
    main()
