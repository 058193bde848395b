#!/usr/bin/env python
"""Benchmark of the stixel pipeline on GB300.

Default workload: one 1024 x 440 FP32 disparity frame, stixel width 5,
dmax 128 (the paper's headline size), through the plain per-frame launch:
column reduction -> prefix LUTs -> DP + backtracking.  One step = one frame.
Prints one JSON line (rank 0).

  python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference]

--impl reference times the CPU oracle (oracle/) on the host cores for the same
workload and metric.  With N > 1 (torchrun) every rank runs an independent
replica on its own GPU; there is no data exchange between ranks.
"""
from __future__ import annotations

import argparse
import hashlib
import json
import math
import os
import statistics
import subprocess
import sys
import tempfile
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

METRIC = "frames/s @1024x440 w=5"
PAPER_FPS = 413.0          # Titan X (Maxwell), 1024x440, s = 5 (paper Sec. 6): context only
# algorithmic integer ops per object DP candidate: S (1), rounded mean by a
# multiply-high (3), two LUT reads and their difference (3), three prior
# candidates (6), their minimum (2), plus the data term (1), running argmin (3)
OPS_PER_CELL = 20
L2_FLUSH_BYTES = 256 << 20

# DRAM traffic per launch from ncu (dram__bytes_read.sum + dram__bytes_write.sum),
# keyed by the sha1 of the kernel's source file at the time of the capture.  A
# kernel whose source changed since reports null.
NCU_TRAFFIC = {
    "kernels_dp.cu": ("d202414b4fa3", 25510144),
    "kernels_luts.cu": ("799b26e901fe", 582656),
    "kernels_reduce.cu": ("15f7465702e2", 1809024),
}


def _sha(path):
    with open(path, "rb") as fh:
        return hashlib.sha1(fh.read()).hexdigest()[:12]


def _traffic(kernel_file):
    rec = NCU_TRAFFIC.get(os.path.basename(kernel_file))
    if not rec:
        return None
    sha, nbytes = rec
    return nbytes if sha == _sha(kernel_file) else None


def parse_args():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=300)
    ap.add_argument("--warmup", type=int, default=20)
    ap.add_argument("--impl", choices=["ours", "reference"], default="ours")
    ap.add_argument("--cpu-seconds", type=float, default=10.0, help="CPU-baseline sample budget")
    ap.add_argument("--no-e2e", action="store_true")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-batched", action="store_true")
    ap.add_argument("--no-served", action="store_true")
    ap.add_argument("--no-variants", action="store_true", help="skip the model-variant timings")
    ap.add_argument("--no-sweep", action="store_true", help="skip the frame-size sweep")
    ap.add_argument("--served-seconds", type=float, default=2.0, help="length of the Poisson arrival trace")
    ap.add_argument("--only", choices=["all", "batched", "served"], default="all",
                    help="run one secondary workload alone and print its record (for profiling); "
                         "the default prints the full benchmark line")
    return ap.parse_args()


def dist_info():
    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return world, rank, local


def max_over_ranks(x, world, device):
    """The largest of every rank's x (the job's time is its slowest replica's)."""
    if world <= 1:
        return float(x)
    import torch
    import torch.distributed as dist
    t = torch.tensor([float(x)], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def job_rate(units_per_rank, world, seconds):
    """Whole-job throughput: the units all ranks processed over the slowest rank's time."""
    return units_per_rank * world / seconds


def host_cores():
    try:
        return len(os.sched_getaffinity(0))
    except Exception:
        return os.cpu_count() or 1


class ClockSampler:
    """nvidia-smi sampling of SM clock and throttle reasons during the timed region."""

    FIELDS = ("clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_index):
        self.gpu = gpu_index
        self.proc = None
        self.path = None

    def start(self):
        fd, self.path = tempfile.mkstemp(suffix=".csv")
        os.close(fd)
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", "-i", str(self.gpu), f"--query-gpu={self.FIELDS}", "--format=csv,noheader,nounits",
                 "-lms", "100"], stdout=open(self.path, "w"), stderr=subprocess.DEVNULL)
        except Exception:
            self.proc = None
        time.sleep(0.3)

    def stop(self):
        if self.proc is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except Exception:
            self.proc.kill()
        rows = []
        for line in open(self.path):
            parts = [x.strip() for x in line.split(",")]
            if len(parts) >= 8:
                rows.append(parts)
        os.unlink(self.path)
        if not rows:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["no samples"]}
        sm = [float(r[0]) for r in rows if r[0].replace(".", "").isdigit()]
        mx = [float(r[1]) for r in rows if r[1].replace(".", "").isdigit()]
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        reasons = sorted({names[i] for r in rows for i in range(4) if r[4 + i].lower() == "active"})
        return {"sm_mhz": statistics.median(sm) if sm else None, "sm_max_mhz": max(mx) if mx else None,
                "reasons": reasons, "samples": len(rows)}


def measured_peaks():
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as fh:
            return json.load(fh), "measured"
    except Exception:
        return {"hbm_gbs": 6800.0, "sm_max_mhz": 2070.0}, "fallback"


# ----------------------------------------------------------------------------- CPU oracle

def oracle_rate(cam, scene_fn, seconds, max_frames=1024, nthreads=0):
    """Frames/s of the CPU oracle on host cores (nthreads = 0: all of them,
    OpenMP over columns), over a bounded sample: each frame is generated
    outside the timed call, and the sample ends once the oracle's own time
    reaches `seconds`."""
    import oracle
    p = oracle.make_params(cam)
    frames, busy = 0, 0.0
    while True:
        sc = scene_fn(frames)
        t0 = time.perf_counter()
        oracle.frame(p, sc.disparity, cap=64, nthreads=nthreads)
        busy += time.perf_counter() - t0
        frames += 1
        if busy >= seconds or frames >= max_frames:
            return frames / busy, frames, busy


# ----------------------------------------------------------------------------- batched / served

def _cells(cam):
    return (cam.width // cam.stixel_width) * cam.height * (cam.height + 1) // 2


def bench_batched(S, scenes, torch, dev, cams, seed0, launches, label, **kw):
    """One graph-captured batch over `cams` (one frame each, parameter overrides `kw`),
    autotuned; frames/s over `launches` back-to-back launches (inputs and LUTs far exceed
    L2, so no flush is needed)."""
    hs = [S.Stixels(S.default_params(c, **kw)) for c in cams]
    b = S.Batch([(h, c.height, c.width) for h, c in zip(hs, cams)])
    for i, c in enumerate(cams):
        sc = scenes.make_scene(c, seed0 + i, n_obstacles=(8, 20))
        b.set_input(i, torch.from_numpy(sc.disparity).to(dev))
    torch.cuda.synchronize()
    stream = torch.cuda.current_stream()
    chosen = b.tune(None, stream)
    for _ in range(3):
        b.launch(stream)
    torch.cuda.synchronize()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    for _ in range(launches):
        b.launch(stream)
    e1.record(stream)
    torch.cuda.synchronize()
    ms = e0.elapsed_time(e1) / launches
    cells = sum(_cells(c) for c in cams)
    b.close()
    for h in hs:
        h.close()
    return {"workload": label, "frames": len(cams), "launches_timed": launches, "ms_per_launch": ms,
            "frames_per_s": len(cams) / (ms / 1000.0), "dp_cells_per_s": cells / (ms / 1000.0),
            "tuned_config": {"dp_warps": chosen[0], "dp_ctas_per_sm": chosen[1]},
            "kernels_per_launch": "reduce (one per stixel-width/mode group) + LUT + persistent DP, one CUDA graph"}


def bench_served(S, scenes, torch, seconds, rate=2000.0, budget=20 << 30, seed=5000, cams=None, label=None):
    """8 cameras (the serving workload's, or `cams`), Poisson arrivals at `rate` frames/s in
    aggregate, host frames in pinned memory, submitted by one client thread at their arrival
    times and polled by another; latency = completion of poll (results in host memory) -
    scheduled arrival."""
    import queue
    import threading

    import numpy as np

    cams = cams or scenes.serving_cameras(seed)
    hs = [S.Stixels(S.default_params(c)) for c in cams]
    per_cam = 3
    frames = []
    for k, c in enumerate(cams):
        fr = []
        for j in range(per_cam):
            d = scenes.make_scene(c, seed + 100 * k + j, n_obstacles=(8, 20)).disparity
            fr.append(torch.from_numpy(d).pin_memory().numpy())
        frames.append(fr)
    outs = [hs[k].alloc_host_output(c.height, c.width, pinned=True) for k, c in enumerate(cams)]
    srv = S.Server(budget, max_slots=1024)
    # warm-up: one frame per camera
    for k in range(8):
        t = srv.submit(hs[k], frames[k][0])
        srv.poll(t, outs[k], timeout_us=10_000_000)

    rng = np.random.default_rng(seed)
    n = int(rate * seconds)
    arrivals = np.cumsum(rng.exponential(1.0 / rate, size=n))
    which = rng.integers(0, 8, size=n)
    pending = queue.Queue()
    lat = np.zeros(n)
    done_at = np.zeros(n)
    retries = [0]
    t0 = time.perf_counter() + 0.05

    def client():
        for i in range(n):
            k = int(which[i])
            # sleep to 0.2 ms before the arrival, then yield until it (a
            # plain sleep overshoots by tens of microseconds)
            wait = t0 + arrivals[i] - time.perf_counter()
            if wait > 2e-4:
                time.sleep(wait - 2e-4)
            while time.perf_counter() < t0 + arrivals[i]:
                time.sleep(0)
            while True:
                t = srv.submit(hs[k], frames[k][i % per_cam])
                if t is not None:
                    break
                retries[0] += 1
                time.sleep(50e-6)
            pending.put((i, k, t))
        pending.put(None)

    def poller():
        live = []
        finished = False
        while not finished or live:
            try:
                while True:
                    item = pending.get_nowait()
                    if item is None:
                        finished = True
                        break
                    live.append(item)
            except queue.Empty:
                pass
            progressed = False
            keep = []
            for (i, k, t) in live:
                rc = srv.poll(t, outs[k], timeout_us=0)
                if rc == S.E_NOT_READY:
                    keep.append((i, k, t))
                    continue
                now = time.perf_counter()
                done_at[i] = now
                lat[i] = now - (t0 + arrivals[i])
                progressed = True
            live = keep
            if not progressed:
                if live:
                    # wait (in the library, without the interpreter lock) on
                    # the oldest frame for up to 0.1 ms, then sweep again
                    i, k, t = live[0]
                    rc = srv.poll(t, outs[k], timeout_us=100)
                    if rc not in (S.E_NOT_READY, S.E_TIMEOUT):
                        now = time.perf_counter()
                        done_at[i] = now
                        lat[i] = now - (t0 + arrivals[i])
                        live = live[1:]
                else:
                    time.sleep(20e-6)

    th = [threading.Thread(target=client), threading.Thread(target=poller)]
    # hand the interpreter lock between the two threads every 0.1 ms, not 5 ms
    switch = sys.getswitchinterval()
    sys.setswitchinterval(1e-4)
    for x in th:
        x.start()
    for x in th:
        x.join()
    sys.setswitchinterval(switch)
    st = srv.stats()
    srv.close()
    for h in hs:
        h.close()
    span = float(done_at.max() - t0)
    lat_ms = np.sort(lat) * 1000.0
    return {"workload": (label or "8 cameras (3x 640x240 dmax 64, 3x 1024x440, 2x 2048x880 dmax 128; s=5)") +
                        f", Poisson arrivals {rate:.0f} frames/s aggregate, {budget >> 30} GB arena budget, host "
                        "frames (pinned) in, results in host memory out",
            "offered_fps": rate, "frames": n, "achieved_fps": n / span,
            "p50_ms": float(np.percentile(lat_ms, 50)), "p99_ms": float(np.percentile(lat_ms, 99)),
            "max_ms": float(lat_ms[-1]), "mean_batch": st["frames_in_iterations"] / max(st["iterations"], 1),
            "iterations": st["iterations"], "rejected_retries": retries[0],
            "latency": "scheduled arrival -> poll returned with results in host memory"}


def bench_served_saturated(S, scenes, torch, frames_total=2000, budget=20 << 30, seed=5000, cams=None):
    """Serving capacity: all frames submitted as fast as admission allows (no arrival pacing)."""
    import threading

    cams = cams or scenes.serving_cameras(seed)
    hs = [S.Stixels(S.default_params(c)) for c in cams]
    frames = [torch.from_numpy(scenes.make_scene(c, seed + 100 * k, n_obstacles=(8, 20)).disparity)
              .pin_memory().numpy() for k, c in enumerate(cams)]
    outs = [hs[k].alloc_host_output(c.height, c.width, pinned=True) for k, c in enumerate(cams)]
    srv = S.Server(budget, max_slots=1024)
    for k in range(8):
        srv.poll(srv.submit(hs[k], frames[k]), outs[k], timeout_us=10_000_000)
    import queue
    pending = queue.Queue()

    def client():
        for i in range(frames_total):
            k = i % 8
            while True:
                t = srv.submit(hs[k], frames[k])
                if t is not None:
                    break
                time.sleep(50e-6)
            pending.put((k, t))
        pending.put(None)

    t0 = time.perf_counter()
    th = threading.Thread(target=client)
    th.start()
    while True:
        item = pending.get()
        if item is None:
            break
        k, t = item
        srv.poll(t, outs[k], timeout_us=60_000_000)
    el = time.perf_counter() - t0
    th.join()
    st = srv.stats()
    srv.close()
    for h in hs:
        h.close()
    return {"frames": frames_total, "fps": frames_total / el,
            "mean_batch": st["frames_in_iterations"] / max(st["iterations"], 1)}


# ----------------------------------------------------------------------------- sweep

def bench_sweep(S, scenes, torch, dev, flush, stream, steps):
    """The small frame (320x120 s=5 dmax 64) and the width / height sweep (1024x440 at s = 3, 5, 7,
    11; 2048x880 s=5), each one frame per step through stixels_compute (frames/s) and through the
    staged entry points (the DP's time, per column): the method's work grows with the columns W/s
    and with H^2 per column (Sec. 3.3)."""
    import statistics as st
    out = []
    for wl, i, cam in [(1, 0, scenes.CONFIG1)] + [(3, j, c) for j, c in enumerate(scenes.CONFIG3)]:
        sc = scenes.make_scene(cam, 1000 * wl + i, n_obstacles=scenes.OBSTACLES[wl])
        disp = torch.from_numpy(sc.disparity).to(dev)
        h = S.Stixels(S.default_params(cam))
        t_c = time_compute(torch, h, disp, flush, stream, 5, steps)
        _, _, _, t_dp, _ = time_stages(S, torch, h, disp, flush, stream, 5, steps)
        ncols = cam.width // cam.stixel_width
        cells = ncols * cam.height * (cam.height + 1) // 2
        dp = st.median(t_dp)
        out.append({"frame": f"{cam.width}x{cam.height} s={cam.stixel_width} dmax={cam.dmax}", "columns": ncols,
                    "frames_per_s": len(t_c) / (sum(t_c) / 1000.0), "ms_per_frame_median": st.median(t_c),
                    "dp_ms_median": dp, "dp_us_per_column": 1000.0 * dp / ncols,
                    "dp_cells_per_s": cells / (dp / 1000.0), "device_error_word": h.get_error(stream)})
        h.close()
    by = {r["frame"]: r for r in out}
    base, tall = by["1024x440 s=5 dmax=128"], by["2048x880 s=5 dmax=128"]
    return {"frames": out,
            "h_doubling": {"note": "2048x880 vs 1024x440 at s=5: 2.0x columns, 4.0x cells per column (H^2)",
                           "dp_time_ratio": tall["dp_ms_median"] / base["dp_ms_median"],
                           "dp_per_column_ratio": tall["dp_us_per_column"] / base["dp_us_per_column"],
                           "frame_time_ratio": tall["ms_per_frame_median"] / base["ms_per_frame_median"]},
            "width_sweep": {"note": "1024x440 at s = 3, 5, 7, 11: DP time against columns (linear in W/s)",
                            "columns": [by[f"1024x440 s={w} dmax=128"]["columns"] for w in (3, 5, 7, 11)],
                            "dp_ms": [by[f"1024x440 s={w} dmax=128"]["dp_ms_median"] for w in (3, 5, 7, 11)]}}


# ----------------------------------------------------------------------------- ours

def time_stages(S, torch, h, disp, flush, stream, warmup, steps):
    """The per-frame pipeline (reduce -> LUTs -> DP) for `steps` steps after
    `warmup`, each stage between CUDA events on the launching stream and the L2
    flushed (untimed) before every step.  Returns per-step times (ms): step,
    reduce, LUTs, DP, and the last output."""
    H, W = disp.shape
    h.reserve(H, W)
    ncols, cap = h.output_shape(H, W)
    P, F = S.lut_pitch(H), h.params.dmax + 1
    dev = disp.device
    q = torch.zeros((ncols, H), dtype=torch.int16, device=dev)
    pd = torch.zeros((ncols, P), dtype=torch.int32, device=dev)
    pg, ps = torch.zeros_like(pd), torch.zeros_like(pd)
    po = torch.zeros((ncols, F, P), dtype=torch.int32, device=dev)
    out = h.alloc_output(H, W, dev)

    def luts():
        S._check(S.lib().stixels_build_luts(h.handle, S._ptr(q), H, ncols, S._stream_ptr(stream), S._ptr(pd),
                                            S._ptr(pg), S._ptr(ps), S._ptr(po)), "build_luts")

    for i in range(warmup):
        flush.fill_(float(i))
        h.reduce(disp, q, stream)
        luts()
        h.solve(pd, pg, ps, po, H, ncols, out, stream)
    torch.cuda.synchronize()
    ev = [[torch.cuda.Event(enable_timing=True) for _ in range(4)] for _ in range(steps)]
    for i in range(steps):
        flush.fill_(float(i))                   # L2 flush between steps (not timed)
        e = ev[i]
        e[0].record(stream)
        h.reduce(disp, q, stream)
        e[1].record(stream)
        luts()
        e[2].record(stream)
        h.solve(pd, pg, ps, po, H, ncols, out, stream)
        e[3].record(stream)
    torch.cuda.synchronize()
    return ([e[0].elapsed_time(e[3]) for e in ev], [e[0].elapsed_time(e[1]) for e in ev],
            [e[1].elapsed_time(e[2]) for e in ev], [e[2].elapsed_time(e[3]) for e in ev], out)


def workload_config(cam, world):
    """The workload both arms name in `config` (the same dict)."""
    return {"workload": f"{cam.width}x{cam.height} s={cam.stixel_width} dmax={cam.dmax}, one frame per step "
                        f"(paper-sized frame)",
            "H": cam.height, "W": cam.width, "stixel_width": cam.stixel_width, "dmax": cam.dmax,
            "frames_per_step": 1, "l2": "flushed between steps (256 MB write, untimed) on the GPU arm",
            "parallelism": f"replicas x{world}" if world > 1 else "single GPU"}


def time_compute(torch, h, disp, flush, stream, warmup, steps):
    """The per-frame entry point (stixels_compute: the whole hot path in one
    call) for `steps` steps after `warmup`, each between CUDA events on the
    launching stream, the L2 flushed (untimed) before every step.  Returns the
    per-step times (ms)."""
    H, W = disp.shape
    out = h.alloc_output(H, W, disp.device)
    for i in range(warmup):
        flush.fill_(float(i))
        h.compute(disp, out, stream)
    torch.cuda.synchronize()
    ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(steps)]
    for i in range(steps):
        flush.fill_(float(i))
        ev[i][0].record(stream)
        h.compute(disp, out, stream)
        ev[i][1].record(stream)
    torch.cuda.synchronize()
    return [a.elapsed_time(b) for a, b in ev]


def compute_launches(p):
    """Kernel launches of one stixels_compute call: reduce, LUTs, DP, and the
    ground estimate's three kernels when it is on."""
    return 3 + (3 if p.ground_estimate else 0)


def bench_ours(args, world, rank, local):
    import numpy as np
    import torch

    import paper_1610_04124_gb300 as S
    import scenes

    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl", device_id=dev)

    cam = scenes.CONFIG2
    H, W, s, dmax = cam.height, cam.width, cam.stixel_width, cam.dmax
    sc = scenes.make_scene(cam, 2000 + rank, n_obstacles=(8, 20))
    disp = torch.from_numpy(sc.disparity).to(dev)
    flush = torch.empty(L2_FLUSH_BYTES // 4, dtype=torch.float32, device=dev)
    stream = torch.cuda.current_stream()
    h = S.Stixels(S.default_params(cam))
    ncols, cap = h.output_shape(H, W)
    P, F = S.lut_pitch(H), dmax + 1

    if world > 1:
        torch.distributed.barrier()
    # per-kernel times through the staged entry points (reduce, build_luts,
    # solve): the rooflines and the stage breakdown
    t_stage_step, t_red, t_lut, t_dp, out = time_stages(S, torch, h, disp, flush, stream, args.warmup, args.steps)
    if world > 1:
        torch.distributed.barrier()
    # the headline: the per-frame entry point, one call per step
    clocks = ClockSampler(local)
    clocks.start()
    t_step = time_compute(torch, h, disp, flush, stream, args.warmup, args.steps)
    K = args.steps
    torch.cuda.synchronize()
    clk = clocks.stop()
    if world > 1:
        torch.distributed.barrier()
    torch.cuda.synchronize()
    total_ms = max_over_ranks(sum(t_step), world, dev)
    value = job_rate(K, world, total_ms / 1000.0)
    err = h.get_error(stream)

    # end to end through the C ABI, host buffers (pinned), copies inside the timed region
    e2e = None
    if not args.no_e2e:
        host_in = torch.from_numpy(sc.disparity).pin_memory().numpy()
        host_out = h.alloc_host_output(H, W, pinned=True)
        for _ in range(3):
            h.compute_host(host_in, host_out)
        n_e2e = max(10, min(K, 200))
        if world > 1:
            torch.distributed.barrier()
        t0 = time.perf_counter()
        for _ in range(n_e2e):
            h.compute_host(host_in, host_out)
        el = max_over_ranks(time.perf_counter() - t0, world, dev)
        e2e = {"value": job_rate(n_e2e, world, el), "unit": "frames/s", "h2d_bytes_per_step": H * W * 4,
               "d2h_bytes_per_step": ncols * cap * 12 + ncols * 4 + ncols * 4, "steps": n_e2e}

    # model variants on the same frame: the paper's LUT_cost variant (Sec. 3.4:
    # whole-pixel disparities, mean reduction, object pixel costs from the
    # off-line (f, d) table) and the disparity-dependent noise model (Eq. 3's
    # sigma^c(f, v)), each through the same staged loop
    variants = None
    if rank == 0 and not args.no_variants:
        variants = {}
        for name, kw, label in [
                ("lut_cost", dict(pixel_grid=1, reduce_mode=1),
                 "same 1024x440 frame; whole-pixel grid + mean reduction + off-line LUT_cost table"),
                ("variable_sigma", dict(sigma_gain=1.0, sigma_mid=40.0, sigma_width=10.0),
                 "same 1024x440 frame; sigma(f) = sigma (1 + logistic((f - 40) / 10)), per-f / per-row tables")]:
            # capacity H: no column's output is cut short (the whole-pixel grid
            # over-segments some columns of this scene past the default 64)
            hv = S.Stixels(S.default_params(cam, max_stixels_per_col=H, **kw))
            vs, vr, vl, vd, _ = time_stages(S, torch, hv, disp, flush, stream, 5, min(K, 100))
            lut_bytes_v = ncols * (F + 3) * P * 4 + ncols * H * 2
            variants[name] = {
                "workload": label, "frames_per_s": len(vs) / (sum(vs) / 1000.0),
                "stages_ms": {"reduce": statistics.mean(vr), "luts": statistics.mean(vl), "dp": statistics.mean(vd)},
                "luts_gbs": lut_bytes_v / (statistics.mean(vl) / 1000.0) / 1e9,
                "device_error_word": hv.get_error(stream)}
            hv.close()
        def compute_loop(hx, nk):
            outx = hx.alloc_output(H, W, dev)
            for i in range(5):
                flush.fill_(float(i))
                hx.compute(disp, outx, stream)
            evx = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(nk)]
            for i in range(nk):
                flush.fill_(float(i))
                evx[i][0].record(stream)
                hx.compute(disp, outx, stream)
                evx[i][1].record(stream)
            torch.cuda.synchronize()
            return [a.elapsed_time(b) for a, b in evx]

        # the per-frame ground estimate (v-disparity) runs inside stixels_compute
        hg = S.Stixels(S.default_params(cam, ground_estimate=1))
        nk = min(K, 100)
        tg = compute_loop(hg, nk)
        q0 = hg.reduce(disp)
        line = hg.estimate_ground(q0, H, ncols)
        variants["ground_estimate"] = {
            "workload": "same 1024x440 frame; ground line estimated per frame from its v-disparity "
                        "(stixels_compute: reduce, estimate, LUTs, DP)",
            "frames_per_s": nk / (sum(tg) / 1000.0), "ms_per_frame": statistics.mean(tg),
            "line": {"slope_px_per_row": line[0] / 256.0, "horizon_row": line[1], "votes": line[2],
                     "camera": {"slope_px_per_row": cam.alpha, "horizon_row": cam.horizon_row}},
            "device_error_word": hg.get_error(stream)}
        hg.close()
        # the exact MAP with the ordering prior: object states carry their
        # disparity, so the recursion runs over (row, class, f)
        hm = S.Stixels(S.default_params(cam, global_map=1))
        nm = min(K, 20)
        tm = compute_loop(hm, nm)
        variants["global_map"] = {
            "workload": "same 1024x440 frame; exact MAP over (row, class, disparity) states "
                        "(stixels_compute: reduce, LUTs, global-MAP DP)",
            "frames_per_s": nm / (sum(tm) / 1000.0), "ms_per_frame": statistics.mean(tm),
            "device_error_word": hm.get_error(stream)}
        hm.close()

    batched = served = None
    if rank == 0 and not args.no_batched:
        batched = {
            "mixed64": bench_batched(S, scenes, torch, dev, scenes.CONFIG4, 4000, 10,
                                     "64 frames: 24x 640x240, 32x 1024x440, 8x 2048x880; s in {5,7}; dmax {64,128}"),
            "paper32": bench_batched(S, scenes, torch, dev, [cam] * 32, 4100, 20,
                                     "32 frames of 1024x440 s=5 dmax=128 in one launch"),
            "paper32_ground_estimate": bench_batched(
                S, scenes, torch, dev, [cam] * 32, 4100, 10,
                "32 frames of 1024x440 s=5 dmax=128 in one launch, ground line estimated per frame",
                ground_estimate=1),
            "paper32_global_map": bench_batched(
                S, scenes, torch, dev, [cam] * 32, 4100, 10,
                "32 frames of 1024x440 s=5 dmax=128 in one launch, global MAP (one launch over all columns)",
                global_map=1),
        }
    if rank == 0 and not args.no_served:
        served = bench_served(S, scenes, torch, args.served_seconds)
        served["saturated"] = bench_served_saturated(S, scenes, torch)
        # the paper's frame alone: 8 streams of 1024x440 s=5, against the per-frame launch
        paper8 = [cam] * 8
        served_paper = bench_served(S, scenes, torch, args.served_seconds, rate=6000.0, seed=5100, cams=paper8,
                                    label="8 streams of 1024x440 s=5 dmax=128")
        served_paper["saturated"] = bench_served_saturated(S, scenes, torch, seed=5100, cams=paper8)
        served["paper_frames_only"] = served_paper
    sweep = None
    if rank == 0 and not args.no_sweep:
        sweep = bench_sweep(S, scenes, torch, dev, flush, stream, min(K, 50))

    if rank != 0:
        h.close()
        return None

    peaks, peak_src = measured_peaks()
    props = torch.cuda.get_device_properties(dev)
    sms = props.multi_processor_count
    sm_max = float(peaks.get("sm_max_mhz") or 2070.0)
    alu_peak = sms * 128 * sm_max * 1e6 / 1e12          # Tops/s, 128 INT32/FP32 lanes per SM
    cells = ncols * H * (H + 1) // 2
    dp_ms = statistics.mean(t_dp)
    dp_tops = cells * OPS_PER_CELL / (dp_ms / 1000.0) / 1e12
    lut_bytes = ncols * (F + 3) * P * 4 + ncols * H * 2
    lut_ms = statistics.mean(t_lut)
    lut_gbs = lut_bytes / (lut_ms / 1000.0) / 1e9
    red_bytes = H * W * 4 + ncols * H * 2
    red_ms = statistics.mean(t_red)
    hbm = float(peaks.get("hbm_gbs") or 6800.0)
    kdir = os.path.join(ROOT, "paper_1610_04124_gb300", "csrc")

    cpu = None
    if not args.no_cpu_baseline and args.cpu_seconds > 0:
        fps, nfr, el = oracle_rate(cam, lambda i: scenes.make_scene(cam, 2100 + i, n_obstacles=(8, 20)),
                                   args.cpu_seconds)
        fps1, nfr1, el1 = oracle_rate(cam, lambda i: scenes.make_scene(cam, 2100 + i, n_obstacles=(8, 20)),
                                      max(1.0, args.cpu_seconds / 2), nthreads=1)
        cpu = {"value": fps, "unit": "frames/s", "cores": host_cores(), "kind": "oracle",
               "sample": f"{nfr} frames of 1024x440 s=5 dmax=128 (seeds 2100..{2100 + nfr - 1}), "
                         f"columns spread over all host cores with OpenMP, {el:.1f} s in the oracle",
               "single_thread": {"value": fps1, "unit": "frames/s", "cores": 1,
                                 "sample": f"{nfr1} frames (seeds 2100..{2100 + nfr1 - 1}), one thread, "
                                           f"{el1:.1f} s in the oracle"}}

    rec = {
        "metric": METRIC, "value": value, "unit": "frames/s", "n_gpus": world, "steps": K,
        "warmup": args.warmup, "ms_per_step": total_ms / K, "higher_is_better": True, "scaling": "weak",
        "vs_baseline": value / PAPER_FPS,
        "vs_baseline_ref": "paper: 413 fps on a Titan X (Maxwell) at 1024x440, s=5 (other hardware; context)",
        "dtype": "int32", "data": "synthetic",
        "config": workload_config(cam, world),
        "roofline": {"kernel": "stixel_dp_kernel", "bound": "alu", "achieved": dp_tops, "peak": alu_peak,
                     "unit": "Tops/s", "frac": dp_tops / alu_peak,
                     "traffic": _traffic(os.path.join(kdir, "kernels_dp.cu")),
                     "peak_source": f"{sms} SMs x 128 int32/fp32 lanes x {sm_max:.0f} MHz (max SM clock, {peak_src})",
                     "work": f"{cells} object DP cells x {OPS_PER_CELL} ops"},
        "roofline_luts": {"kernel": "prefix_lut_kernel", "bound": "hbm", "achieved": lut_gbs, "peak": hbm,
                          "unit": "GB/s", "frac": lut_gbs / hbm, "traffic": _traffic(os.path.join(kdir, "kernels_luts.cu")),
                          "peak_source": f"hbm_gbs ({peak_src})", "bytes": lut_bytes},
        "roofline_reduce": {"kernel": "reduce_transpose_kernel", "bound": "hbm",
                            "achieved": red_bytes / (red_ms / 1000.0) / 1e9, "peak": hbm, "unit": "GB/s",
                            "frac": red_bytes / (red_ms / 1000.0) / 1e9 / hbm, "bytes": red_bytes,
                            "traffic": _traffic(os.path.join(kdir, "kernels_reduce.cu"))},
        "ms_per_step_median": statistics.median(t_step),
        "stages_ms": {"reduce": red_ms, "luts": lut_ms, "dp": dp_ms,
                      "reduce_median": statistics.median(t_red), "luts_median": statistics.median(t_lut),
                      "dp_median": statistics.median(t_dp),
                      "staged_step_median": statistics.median(t_stage_step),
                      "step_median": statistics.median(t_step), "step_p99": sorted(t_step)[int(0.99 * (K - 1))],
                      "note": "reduce / luts / dp from the staged entry points (stixels_reduce, stixels_build_luts, "
                              "stixels_solve); step times from stixels_compute (the same three kernels)"},
        "dp_cells_per_s": cells / (dp_ms / 1000.0),
        "gpu_launches": compute_launches(h.params) * K,
        "clocks": clk,
        "device_error_word": err,
        "cpu_baseline": cpu,
        "e2e": e2e,
        "batched": batched,
        "served": served,
        "sweep": sweep,
        "model_variants": variants,
    }
    h.close()
    return rec


# ----------------------------------------------------------------------------- reference arm

def bench_reference(args, world, rank):
    """The CPU oracle as the reference arm: same workload and metric, host cores."""
    if rank != 0:
        return None
    import oracle
    import scenes
    cam = scenes.CONFIG2
    p = oracle.make_params(cam)
    sc = scenes.make_scene(cam, 2000, n_obstacles=(8, 20))
    ncols = cam.width // cam.stixel_width
    t0 = time.perf_counter()
    oracle.frame(p, sc.disparity, cap=64)
    t_frame = time.perf_counter() - t0
    total = args.steps + args.warmup
    budget = 150.0                                     # seconds for the whole run
    frac = min(1.0, budget / max(total * t_frame, 1e-9))
    sample_cols = max(1, min(ncols, int(math.ceil(frac * ncols))))
    W_s = sample_cols * cam.stixel_width
    sub = sc.disparity[:, :W_s].copy()
    for _ in range(args.warmup):
        oracle.frame(p, sub, cap=64)
    t0 = time.perf_counter()
    for _ in range(args.steps):
        oracle.frame(p, sub, cap=64)
    el = time.perf_counter() - t0
    frames = args.steps * sample_cols / ncols
    value = frames / el
    sample = (f"each step: {sample_cols} of the {ncols} columns of a 1024x440 s=5 dmax=128 frame "
              f"(seed 2000), scaled to frames; all host cores (OpenMP)")
    return {"impl": "reference", "metric": METRIC, "value": value, "unit": "frames/s", "n_gpus": world,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1000.0 * el / args.steps,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": value / PAPER_FPS, "dtype": "f64",
            "data": "synthetic",
            "config": workload_config(cam, world),
            "cpu_baseline": {"value": value, "unit": "frames/s", "cores": host_cores(), "kind": "oracle",
                             "sample": sample},
            "e2e": {"value": value, "unit": "frames/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}


def main():
    args = parse_args()
    world, rank, local = dist_info()
    if args.only != "all" and args.impl == "ours":
        import torch
        import paper_1610_04124_gb300 as S
        import scenes
        torch.cuda.set_device(local)
        dev = torch.device("cuda", local)
        if args.only == "batched":
            rec = {"batched": {
                "mixed64": bench_batched(S, scenes, torch, dev, scenes.CONFIG4, 4000, max(1, args.steps),
                                         "64 frames: 24x 640x240, 32x 1024x440, 8x 2048x880; s in {5,7}; dmax {64,128}"),
                "paper32": bench_batched(S, scenes, torch, dev, [scenes.CONFIG2] * 32, 4100, max(1, args.steps),
                                         "32 frames of 1024x440 s=5 dmax=128 in one launch"),
                "paper32_global_map": bench_batched(
                    S, scenes, torch, dev, [scenes.CONFIG2] * 32, 4100, max(1, args.steps),
                    "32 frames of 1024x440 s=5 dmax=128 in one launch, global MAP", global_map=1)}}
        else:
            rec = {"served": bench_served(S, scenes, torch, args.served_seconds)}
        if rank == 0:
            print(json.dumps(rec), flush=True)
        return
    if args.impl == "reference":
        rec = bench_reference(args, world, rank)
    else:
        rec = bench_ours(args, world, rank, local)
    if rec is not None and rank == 0:
        print(json.dumps(rec), flush=True)


if __name__ == "__main__":
    main()
