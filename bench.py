"""Throughput of the stereo pipeline on the paper's workload shape.

Workload: one RGB pair of 1436 x 992 with Dmax 145 per step (the paper's
Adirondack(H) shape, Table II), downscaled 2x to 718 x 496 with D = 73, the
whole pipeline of Sec. III including the bilateral upscale. Inputs are seeded
synthetic piecewise-planar scenes (the Middlebury images are not available).

value: frames per second over K back-to-back steps with inputs resident in
HBM, timed with CUDA events on the stream the library launches on; the inputs
rotate over a pool of pairs larger than the L2 cache. e2e: the same metric
through the host-buffer entry point (host-to-device copies of both images and
the device-to-host copy of the float map inside the timed region).
roofline: the fused cost + aggregation + WTA kernel against the SM issue
limit (ALU-bound: 13 integer operations per (x, y, d) cell for both bases on
the prefix formulation of Eqs. 3-9), and against its shared-memory pipe.

Multi-GPU (torchrun): one independent replica per GPU on its own frames
(weak scaling); a barrier and a max over ranks bracket the timed region.
"""
from __future__ import annotations

import argparse
import json
import os
import statistics
import subprocess
import sys
import threading
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "fps & W·H·D/s at 1436×992, Dmax 145 on 1 GB300; % of HBM/ALU roofline"
W_FULL, H_FULL, DMAX = 1436, 992, 145
PLANES, SEED = 40, 0
POOL = 20                       # 20 pairs x 8.5 MB = 171 MB > 126 MB of L2
PROFILE_EVERY = 10              # per-stage CUDA events on every 10th timed frame
PAPER_FPS = 40.0                # Table II, GTX 780 Ti (context only)
OPS_PER_CELL = 13               # algorithmic integer operations per (x, y, d) cell, both bases
DIFF_EXPS_PER_CELL = 9          # differentiable form, forward + backward: exp per cell
DIFF_FLOPS_PER_CELL = 48        # differentiable form: flops per cell besides the window sums
SFU_PER_SM = 16                 # exp (MUFU) results per SM and clock
SM_COUNT_NOMINAL = 152
LANES_PER_SM = 128              # 4 SM sub-partitions x 32 lanes issue one warp instruction per clock each


TRAFFIC_RECORD = os.path.join(ROOT, "profiles", "costagg_wta_kernel_1436x992_d145_traffic.txt")
COSTAGG_SRC = os.path.join(ROOT, "paper_2212_00488_gb300", "csrc", "costagg.cu")


def _recorded_counters():
    """The fused kernel's last ncu capture (DRAM bytes and shared-memory
    wavefronts per launch), or {} when the kernel source has changed since the
    counters were taken."""
    import hashlib
    try:
        with open(TRAFFIC_RECORD) as f:
            rec = json.load(f)
        with open(COSTAGG_SRC, "rb") as f:
            h = hashlib.sha256(f.read()).hexdigest()
    except (OSError, ValueError):
        return {}
    return rec if rec.get("source_sha256") == h else {}


def _recorded_traffic():
    """DRAM bytes per launch of the fused kernel, or None (see _recorded_counters)."""
    return _recorded_counters().get("traffic_bytes_per_launch")


def _shared_pipe(kernel_ms, sm_count, sm_mhz):
    """The fused kernel against its other limit, the shared-memory pipe: the
    wavefronts one launch issues (ncu) over its one-lane CUDA-event time,
    against one wavefront per SM and clock."""
    wf = _recorded_counters().get("shared_wavefronts_per_launch")
    if not wf or not kernel_ms:
        return None
    achieved = wf / (kernel_ms / 1e3)
    peak = sm_count * sm_mhz * 1e6
    return {"wavefronts_per_launch": wf, "achieved_per_s": achieved, "peak_per_s": peak,
            "frac": achieved / peak, "peak_source": f"{sm_count} SMs x 1 wavefront x {sm_mhz:.0f} MHz",
            "timer": "kernel_ms_one_lane"}


def _peaks():
    path = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(path):
        with open(path) as f:
            return json.load(f), "measured"
    return {"hbm_gbs": 6800.0, "sm_max_mhz": 2070.0}, "fallback"


class ClockSampler:
    """nvidia-smi samples of SM clock and throttle reasons during the timed region."""

    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_index: int):
        self.gpu = gpu_index
        self.proc = None
        self.lines = []

    def start(self):
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", f"--query-gpu={self.FIELDS}", "--format=csv,noheader,nounits", "-lms", "200",
                 "-i", str(self.gpu)], stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
        except OSError:
            self.proc = None
            return
        self.thread = threading.Thread(target=self._read, daemon=True)
        self.thread.start()

    def _read(self):
        for line in self.proc.stdout:
            self.lines.append(line.strip())

    def stop(self):
        if self.proc is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except subprocess.TimeoutExpired:
            self.proc.kill()
        self.thread.join(timeout=2)
        sm, smax, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for ln in self.lines:
            parts = [p.strip() for p in ln.split(",")]
            if len(parts) < 9:
                continue
            try:
                sm.append(float(parts[1]))
                smax.append(float(parts[2]))
            except ValueError:
                continue
            for name, val in zip(names, parts[5:9]):
                if val.lower() == "active":
                    reasons.add(name)
        return {"sm_mhz": statistics.median(sm) if sm else None, "sm_max_mhz": max(smax) if smax else None,
                "reasons": sorted(reasons), "samples": len(sm)}


def _dist():
    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return world, rank, local


def run_reference(args):
    """The CPU oracle, as it stands, on the host cores (OpenMP over rows on
    every core): a bounded sample per step, scaled to whole frames."""
    world, rank, _ = _dist()
    if rank != 0:
        return
    import numpy as np

    import oracle
    from paper_2212_00488_gb300 import scenes
    oracle.build.build()
    cores = oracle.set_threads(0)
    s = scenes.make_scene(W_FULL, H_FULL, DMAX, PLANES, SEED)
    band = H_FULL // 8                            # 124 full-res rows per step
    fracs, times = [], []
    for i in range(args.warmup + args.steps):
        y0 = (i * band) % (H_FULL - band)
        l, r = s.left[y0:y0 + band], s.right[y0:y0 + band]
        t0 = time.perf_counter()
        oracle.pipeline(np.ascontiguousarray(l), np.ascontiguousarray(r), DMAX, oracle.Params())
        dt = time.perf_counter() - t0
        if i >= args.warmup:
            times.append(dt)
            fracs.append(band / H_FULL)
    total = sum(times)
    fps = sum(fracs) / total
    line = {
        "impl": "reference", "metric": METRIC, "value": fps, "unit": "frames/s", "n_gpus": world,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1e3 * total / len(times),
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "int64",
        "data": "synthetic",
        "config": {"workload": "1436x992 RGB, Dmax 145, downscale 2x (718x496, D 73), full pipeline",
                   "sample": f"{band}-row band of the frame per step"},
        "cpu_baseline": {"value": fps, "unit": "frames/s", "cores": cores, "kind": "oracle",
                         "sample": f"one {band}x{W_FULL} row band (1/8 frame) per step, OpenMP over rows on "
                                   f"{cores} threads, scaled to frames/s"},
        "e2e": {"value": fps, "unit": "frames/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }
    print(json.dumps(line), flush=True)


def cpu_baseline_leg():
    """The oracle timed on this host (rank 0, N = 1), as it stands: integer
    mode with OpenMP over rows on every core (the line's value), integer mode
    on one thread, and the FP64 mode (Eqs. 3-9 in double for both bases, on
    every core)."""
    import numpy as np

    import oracle
    from paper_2212_00488_gb300 import scenes
    oracle.build.build()
    s = scenes.make_scene(W_FULL, H_FULL, DMAX, PLANES, SEED)
    left, right = np.ascontiguousarray(s.left), np.ascontiguousarray(s.right)

    def rate(n, fn):
        t0 = time.perf_counter()
        for _ in range(n):
            fn()
        return n / (time.perf_counter() - t0)

    cores = oracle.set_threads(0)
    whole = lambda: oracle.pipeline(left, right, DMAX, oracle.Params())   # noqa: E731
    all_cores = rate(6, whole)
    oracle.set_threads(1)
    one = rate(2, whole)
    oracle.set_threads(0)
    fp64 = rate(2, lambda: oracle.wta_pair_f64(left, right, DMAX, oracle.Params()))
    # the small configuration: 360x248, Dmax 36, no downscaling
    s0 = scenes.make_scene(360, 248, 36, 12, SEED)
    p0 = oracle.Params()
    p0.downscale = 0
    small = lambda: oracle.pipeline(s0.left, s0.right, 36, p0)   # noqa: E731
    small_all = rate(20, small)
    oracle.set_threads(1)
    small_one = rate(5, small)
    oracle.set_threads(0)
    return {"value": all_cores, "unit": "frames/s", "cores": cores, "kind": "oracle",
            "sample": f"6 full 1436x992/145 frames, whole pipeline, integer mode, OpenMP over rows on "
                      f"{cores} threads",
            "single_thread": {"value": one, "unit": "frames/s", "cores": 1,
                              "sample": "2 full frames, whole pipeline, integer mode, one thread"},
            "fp64": {"value": fp64, "unit": "frames/s", "cores": cores,
                     "sample": f"2 full frames: grey, downscale, census and arms, then the cost, both "
                               f"aggregations and the WTA of both bases in FP64 on {cores} threads"},
            "small_config": {"workload": "360x248 RGB pair, Dmax 36, no downscaling, whole pipeline, integer mode",
                             "value": small_all, "unit": "frames/s", "cores": cores,
                             "single_thread": small_one, "sample": "20 frames on every core, 5 on one thread"}}


BATCH_MENU = [(640, 480, 64), (1024, 768, 96), (1436, 992, 145), (1920, 1080, 192)]


def measure_batch(dev, stream, steps=20, warmup=3, seed=2):
    """Batched form: 16 pairs drawn by seed from the menu, one stereo_compute_batch
    call per step (persistent fused kernel, CUDA graph, autotuned tile)."""
    import numpy as np
    import torch

    from paper_2212_00488_gb300 import Stereo, _lib, scenes
    from paper_2212_00488_gb300.stereo import stream_handle
    rng = np.random.default_rng(seed)
    picks = [BATCH_MENU[i] for i in rng.integers(0, len(BATCH_MENU), size=16)]
    frames = []
    for shape in sorted(set(picks)):
        W, H, dmax = shape
        pool = scenes.scene_pool(W, H, dmax, 12, seed, picks.count(shape))
        for sc in pool:
            frames.append((torch.from_numpy(sc.left).to(dev), torch.from_numpy(sc.right).to(dev), W, H, dmax))
    outs = [torch.empty((H, W), dtype=torch.float32, device=dev) for _, _, W, H, _ in frames]
    jobs = [_lib.stereo_job(lt.data_ptr(), rt.data_ptr(), W, H, dmax, o.data_ptr(), None, None, None)
            for (lt, rt, W, H, dmax), o in zip(frames, outs)]
    st = Stereo(dev.index)
    h = stream_handle(stream)
    for _ in range(warmup):
        _lib.stereo_compute_batch(st.ctx, jobs, h)
    torch.cuda.synchronize()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    for _ in range(steps):
        _lib.stereo_compute_batch(st.ctx, jobs, h)
    e1.record(stream)
    torch.cuda.synchronize()
    _lib.stereo_sync(st.ctx)
    ms = e0.elapsed_time(e1) / steps
    tile, tune_ms = _lib.stereo_batch_tile(st.ctx)
    launches = _lib.stereo_last_launch_count(st.ctx)
    st.close()
    whd = sum(W * H * dmax for _, _, W, H, dmax in frames)
    return {"workload": "16 pairs drawn by seed from 640x480/64, 1024x768/96, 1436x992/145, 1920x1080/192",
            "shapes": [list(p) for p in picks], "value": 16 / (ms / 1e3), "unit": "frames/s",
            "mde_per_s": whd / (ms / 1e3), "ms_per_batch": ms, "steps": steps, "warmup": warmup,
            "tile": tile, "autotune_ms": [round(t, 4) for t in tune_ms], "gpu_launches_per_batch": launches}


SERVE_MENU = [(640, 480, 64), (1436, 992, 145), (1920, 1080, 192)]


def measure_serve(dev, seconds=60.0, rate=120.0, seed=4):
    """Serving form: Poisson arrivals at `rate` per second for `seconds`, each a
    single pair of a resolution drawn uniformly from the menu, device-resident
    inputs, continuous batching with an 8 GB admission cap."""
    import numpy as np
    import torch

    from paper_2212_00488_gb300 import scenes
    from paper_2212_00488_gb300.serve import StereoServer
    rng = np.random.default_rng(seed)
    pool = []
    for W, H, dmax in SERVE_MENU:
        for sc in scenes.scene_pool(W, H, dmax, 12, seed, 2):
            pool.append((torch.from_numpy(sc.left).to(dev), torch.from_numpy(sc.right).to(dev), W, H, dmax))
    torch.cuda.synchronize()
    # one autotuning run on the largest frame of the menu picks the tile shape
    # the server then keeps, so no request pays for tuning
    from paper_2212_00488_gb300 import Stereo, _lib
    from paper_2212_00488_gb300.stereo import stream_handle
    lt, rt, W, H, dmax = pool[-1]
    tuner = Stereo(dev.index)
    out = torch.empty((H, W), dtype=torch.float32, device=dev)
    _lib.stereo_compute_batch(tuner.ctx, [_lib.stereo_job(lt.data_ptr(), rt.data_ptr(), W, H, dmax, out.data_ptr(),
                                                          None, None, None)],
                              stream_handle(torch.cuda.current_stream(dev)))
    torch.cuda.synchronize()
    tile, _ = _lib.stereo_batch_tile(tuner.ctx)
    tuner.close()
    srv = StereoServer(dev.index, mem_cap_bytes=8 << 30, lanes=2, max_batch=16, tile=tile)
    for lt, rt, _, _, dmax in pool:                # warm-up: graphs, autotuning
        srv.submit(lt, rt, dmax).result(timeout=120)
    srv.latencies.clear()
    done0 = srv.completed
    futs, whd = [], 0
    t0 = time.perf_counter()
    t_next = t0
    while True:
        t_next += rng.exponential(1.0 / rate)
        if t_next - t0 > seconds:
            break
        delay = t_next - time.perf_counter()
        if delay > 0:
            time.sleep(delay)
        lt, rt, W, H, dmax = pool[2 * int(rng.integers(0, len(SERVE_MENU))) + int(rng.integers(0, 2))]
        futs.append(srv.submit(lt, rt, dmax))
        whd += W * H * dmax
    for f in futs:
        f.result(timeout=120)
    wall = time.perf_counter() - t0
    st = srv.stats()
    srv.close()
    n = st["completed"] - done0
    return {"workload": f"Poisson {rate:.0f} req/s for {seconds:.0f} s, single pairs from "
                        "640x480/64, 1436x992/145, 1920x1080/192, device-resident, 8 GB admission cap",
            "requests": n, "value": n / wall, "unit": "frames/s", "mde_per_s": whd / wall,
            "p50_ms": st["p50_ms"], "p99_ms": st["p99_ms"], "batches": st["batches"],
            "peak_admitted_bytes": st["peak_admitted_bytes"], "seconds": wall, "tile": tile}


def measure_diff(dev, steps=5, warmup=2, seed=6):
    """Differentiable form: a batch of 4 pairs of 718x496 (FP32 on [0, 1]),
    73 disparities, soft-argmin at temperature 0.1, L1 loss to the known
    disparity, forward and backward through the cross aggregation."""
    import numpy as np
    import torch

    from paper_2212_00488_gb300 import Stereo
    from paper_2212_00488_gb300.diff import soft_argmin_disparity
    from paper_2212_00488_gb300 import scenes
    W, H, D, B = 718, 496, 73, 4
    sc = [scenes.make_scene(W, H, D, planes=40, seed=seed + b) for b in range(B)]
    UL = torch.from_numpy(np.stack([s.left for s in sc])).to(dev)
    UR = torch.from_numpy(np.stack([s.right for s in sc])).to(dev)
    L = (UL.float() / 255.0).contiguous().requires_grad_(True)
    R = (UR.float() / 255.0).contiguous().requires_grad_(True)
    GT = torch.from_numpy(np.stack([s.disp for s in sc]).astype(np.float32)).to(dev)
    T = torch.tensor([1.0, 1.0, 0.3, 2.3], device=dev, requires_grad=True)
    st = Stereo(dev.index, downscale=0)

    def step():
        dh = soft_argmin_disparity(L, R, T, UL, UR, D, 0.1, st)
        loss = (dh - GT).abs().mean()
        loss.backward()
        return loss
    for _ in range(warmup):
        step()
    torch.cuda.synchronize()
    stream = torch.cuda.current_stream(dev)
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    for _ in range(steps):
        loss = step()
    e1.record(stream)
    torch.cuda.synchronize()
    ms = e0.elapsed_time(e1) / steps
    # mean spans of the frozen supports (the library's own arms of each pair)
    sx = sy = 0.0
    for b in range(B):
        st(UL[b].contiguous(), UR[b].contiguous(), D)
        arms = st.debug_planes(W, H)["arms_l"].cpu().numpy().view(np.uint32)
        sx += float(((arms & 0xFF) + ((arms >> 8) & 0xFF) + 1).mean()) / B
        sy += float((((arms >> 16) & 0xFF) + (arms >> 24) + 1).mean()) / B
    st.close()
    cells = B * W * H * D
    exps = DIFF_EXPS_PER_CELL * cells
    adds = (DIFF_FLOPS_PER_CELL + 3 * (sx + sy)) * cells
    props = torch.cuda.get_device_properties(dev)
    peaks, _ = _peaks()
    clk = float(peaks.get("sm_max_mhz", 2070.0)) * 1e6
    alu_peak = props.multi_processor_count * LANES_PER_SM * clk
    sfu_peak = props.multi_processor_count * SFU_PER_SM * clk
    floor_s = max(adds / alu_peak, exps / sfu_peak)
    return {"workload": "4 pairs 718x496 FP32, D 73, soft-argmin tau 0.1, L1 loss, forward + backward",
            "value": B / (ms / 1e3), "unit": "pairs/s (forward + backward)", "ms_per_step": ms,
            "mde_per_s": B * W * H * D / (ms / 1e3), "loss": float(loss.item()),
            "grad_theta": [float(v) for v in T.grad.cpu()], "steps": steps, "warmup": warmup,
            "roofline": {"bound": "alu", "unit": "ms per step", "achieved_ms": ms, "floor_ms": floor_s * 1e3,
                         "frac": floor_s * 1e3 / ms, "cells": cells, "exps_per_cell": DIFF_EXPS_PER_CELL,
                         "flops_per_cell": DIFF_FLOPS_PER_CELL + 3 * (sx + sy), "mean_x_span": sx,
                         "mean_y_span": sy,
                         "peak_source": f"{props.multi_processor_count} SMs x ({LANES_PER_SM} lanes for adds and "
                                        f"multiplies, {SFU_PER_SM} for exp) x {clk / 1e6:.0f} MHz",
                         "work": "per (x, y, d) cell, forward and backward: 9 exp, "
                                 f"{DIFF_FLOPS_PER_CELL} other flops, and the window sums three times along "
                                 "x and y (forward, the backward's recompute, the adjoint)"}}


TABLE_I_WX = (5, 9, 21, 41, 61, 141)      # Table I rows (per side)
TABLE_I_WY = (9, 11, 15, 21, 27, 31)      # Table I columns (per side)


def _max_cost_scale(wx, wy, lad=0.3, lmc=2.3, scale=512):
    """The default cost scale, lowered only where (2 wx + 1)(2 wy + 1) P would
    reach 2^24 (the aggregated cost's field of the WTA key)."""
    import math
    unit = (1 - math.exp(-1 / lad)) + (1 - math.exp(-6 / lmc))
    while (2 * wx + 1) * (2 * wy + 1) * (scale * unit + 1) >= 2 ** 24:
        scale -= 16
    return scale


def measure_sweep(dev, frames=10, warmup=3):
    """Timings beyond the headline workload (fused kernel and whole frame, one
    library context): the (W_x, W_y) grid of Table I at 1436x992/145, the other
    Middlebury-like shapes of Sec. V, and Dmax at 1436x992."""
    import torch
    from paper_2212_00488_gb300 import Stereo, _lib, scenes

    pools = {}

    def pool(W, H, Dmax):
        if (W, H, Dmax) not in pools:
            ps = [scenes.make_scene(W, H, Dmax, planes=PLANES, seed=SEED + 7 * k) for k in range(2)]
            pools[(W, H, Dmax)] = ([torch.from_numpy(q.left).to(dev) for q in ps],
                                   [torch.from_numpy(q.right).to(dev) for q in ps])
        return pools[(W, H, Dmax)]

    def time_cfg(W, H, Dmax, **params):
        L, R = pool(W, H, Dmax)
        st = Stereo(dev.index, **params)
        out = st(L[0], R[0], Dmax)
        for i in range(warmup):
            st(L[i % 2], R[i % 2], Dmax, out=out)
        torch.cuda.synchronize()
        _lib.stereo_set_profiling(st.ctx, True)
        stream = torch.cuda.current_stream(dev)
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        for i in range(frames):
            st(L[i % 2], R[i % 2], Dmax, out=out)
        e1.record(stream)
        torch.cuda.synchronize()
        ms, _ = _lib.stereo_stage_ms(st.ctx)
        tile = _lib.stereo_get_tile(st.ctx, W, H, Dmax)
        st.close()
        frame_ms = e0.elapsed_time(e1) / frames
        return {"W": W, "H": H, "Dmax": Dmax, **params, "frame_ms": round(frame_ms, 4),
                "fps": round(1e3 / frame_ms, 1), "kernel_ms": round(ms[_lib.STAGE_COSTAGG], 4), "tile": tile}

    window = [time_cfg(W_FULL, H_FULL, DMAX, wx=wx, wy=wy, cost_scale=_max_cost_scale(wx, wy))
              for wx in TABLE_I_WX for wy in TABLE_I_WY]
    shapes = [time_cfg(W, H, D) for W, H, D in ((1436, 992, 145), (1482, 994, 128), (1444, 960, 380))]
    dmax = [time_cfg(W_FULL, H_FULL, D) for D in (64, 128, 145, 256, 380, 511)]
    scale = [time_cfg(W_FULL, H_FULL, DMAX, cost_scale=cs) for cs in (512, 2048)]
    return {"frames": frames, "warmup": warmup, "window": window, "shapes": shapes, "dmax": dmax,
            "cost_scale": scale,
            "note": "arm caps per side (Table I grid); cost_scale lowered from 512 only where a window sum "
                    "could reach 2^24: " + ", ".join(f"wx {w['wx']} wy {w['wy']} -> {w['cost_scale']}"
                                                     for w in window if w["cost_scale"] != 512)}


def run_ours(args):
    import numpy as np
    import torch

    world, rank, local = _dist()
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl")
    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)

    from paper_2212_00488_gb300 import Stereo, _lib, build, scenes
    build.build()

    pool = scenes.scene_pool(W_FULL, H_FULL, DMAX, PLANES, SEED + rank, POOL)
    left = [torch.from_numpy(p.left).to(dev) for p in pool]
    right = [torch.from_numpy(p.right).to(dev) for p in pool]
    # Several contexts, each on its own stream, take frames in turn, so the
    # small kernels of one frame fill the SMs the other frames' kernels leave
    # idle.
    nl = args.lanes
    ctxs = [Stereo(local) for _ in range(nl)]
    if args.tile >= 0:
        for c_ in ctxs:
            _lib.stereo_set_tile(c_.ctx, args.tile)
    streams = [torch.cuda.Stream(dev) for _ in range(nl)]
    st, stream = ctxs[0], streams[0]
    lanes = list(zip(ctxs, streams))
    outs = []
    for ctx_, s_ in lanes:
        with torch.cuda.stream(s_):
            outs.append(ctx_(left[0], right[0], DMAX))
    torch.cuda.synchronize()

    isolate = {"on": False}

    def frame(i):
        ctx_, s_ = lanes[i % nl]
        # a profiled frame (lane 0, every PROFILE_EVERY-th of its frames) runs
        # with the other lanes held back, so its per-stage events time the
        # kernels rather than their wait for SMs the other lanes hold
        alone = isolate["on"] and i % nl == 0 and (i // nl) % PROFILE_EVERY == 0
        if alone:
            for s2 in streams[1:]:
                s_.wait_stream(s2)
        with torch.cuda.stream(s_):
            ctx_(left[i % POOL], right[i % POOL], DMAX, out=outs[i % nl])
        if alone:
            for s2 in streams[1:]:
                s2.wait_stream(s_)
        return _lib.stereo_last_launch_count(ctx_.ctx)

    for i in range(args.warmup):
        frame(i)
    torch.cuda.synchronize()
    torch.cuda.set_stream(stream)

    # the fused kernel's time comes from CUDA events around the stages of every
    # PROFILE_EVERY-th frame of the timed loop (events between kernels cost a
    # few us, so they are kept off most frames)
    _lib.stereo_set_profiling(st.ctx, PROFILE_EVERY)
    clocks = ClockSampler(local)
    clocks.start()
    time.sleep(0.3)
    if world > 1:
        dist.barrier()
    torch.cuda.synchronize()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    launches = 0
    e0.record(stream)
    for s_ in streams[1:]:
        s_.wait_event(e0)
    isolate["on"] = nl > 1
    for i in range(args.steps):
        launches += frame(i)
    isolate["on"] = False
    for s_ in streams[1:]:
        stream.wait_stream(s_)
    e1.record(stream)
    torch.cuda.synchronize()
    if world > 1:
        dist.barrier()
    clk = clocks.stop()
    ms_total = e0.elapsed_time(e1)
    stage_ms, nframes = _lib.stereo_stage_ms(st.ctx)
    _lib.stereo_set_profiling(st.ctx, False)
    # the same stages with one lane only (no frame of another lane competing
    # for SMs), after the timed region
    _lib.stereo_set_profiling(st.ctx, 1)
    for i in range(20):
        frame(nl * i)
    torch.cuda.synchronize()
    stage_alone, _ = _lib.stereo_stage_ms(st.ctx)
    _lib.stereo_set_profiling(st.ctx, False)

    from paper_2212_00488_gb300 import replicas
    agg = replicas.aggregate(float(args.steps), ms_total / 1e3)
    ms_max = agg.seconds_max * 1e3
    fps = agg.throughput

    # e2e through the host-buffer entry point, pinned host memory
    hl = [torch.from_numpy(p.left).pin_memory() for p in pool[:4]]
    hr = [torch.from_numpy(p.right).pin_memory() for p in pool[:4]]
    hdisp = [torch.empty((H_FULL, W_FULL), dtype=torch.float32).pin_memory() for _ in range(nl)]
    e2e_steps = max(10, min(args.steps, 100))
    # (1) one synchronous call per frame: copy in, pipeline, copy out, wait
    for i in range(3):
        st.compute_host(hl[i % 4], hr[i % 4], DMAX, hdisp[0])
    if world > 1:
        dist.barrier()
    t0 = time.perf_counter()
    for i in range(e2e_steps):
        st.compute_host(hl[i % 4], hr[i % 4], DMAX, hdisp[0])
    sync_fps = replicas.aggregate(float(e2e_steps), time.perf_counter() - t0).throughput
    # (2) the asynchronous call taking the contexts (streams) in turn, so one
    # frame's host copies overlap the others' compute; every frame still
    # copies its pair in and its map out inside the timed region
    for i in range(2 * nl):
        ctxs[i % nl].compute_host(hl[i % 4], hr[i % 4], DMAX, hdisp[i % nl], wait=False)
    for c_ in ctxs:
        c_.sync()
    if world > 1:
        dist.barrier()
    t0 = time.perf_counter()
    for i in range(e2e_steps):
        ctxs[i % nl].compute_host(hl[i % 4], hr[i % 4], DMAX, hdisp[i % nl], wait=False)
    for c_ in ctxs:
        c_.sync()
    e2e_dt = time.perf_counter() - t0
    e2e_fps = replicas.aggregate(float(e2e_steps), e2e_dt).throughput

    if rank == 0:
        peaks, src = _peaks()
        X, Y, D = W_FULL // 2, H_FULL // 2, (DMAX + 1) // 2
        cells = X * Y * D
        t_hot = stage_ms[_lib.STAGE_COSTAGG] / 1e3
        sm_count = torch.cuda.get_device_properties(dev).multi_processor_count
        sm_mhz = float(peaks.get("sm_max_mhz", 2070.0))
        peak_ops = sm_count * LANES_PER_SM * sm_mhz * 1e6
        achieved = OPS_PER_CELL * cells / t_hot
        # measured rates of the operations the count is made of (after the timed region)
        int_ops, popc_s, lds_bps = _lib.stereo_measure_peaks(dev.index)
        line = {
            "metric": METRIC,
            "value": fps,
            "unit": "frames/s",
            "n_gpus": world,
            "steps": args.steps,
            "warmup": args.warmup,
            "ms_per_step": ms_max / args.steps,
            "higher_is_better": True,
            "scaling": "weak",
            "vs_baseline": fps / world / PAPER_FPS,
            "dtype": "u32",
            "data": "synthetic",
            "config": {"workload": "1436x992 RGB pair, Dmax 145, downscaled 2x to 718x496 with D 73, "
                                   "full pipeline (grey, downscale, census+arms, cost+aggregation+WTA both "
                                   "bases, cross-check, median, bilateral fill, upscale)",
                       "scene": "seeded piecewise-planar, 40 planes, texture sigma 20, sensor sigma 2",
                       "l2": f"inputs rotate over {POOL} pairs ({POOL * W_FULL * H_FULL * 6 / 1e6:.0f} MB > L2)",
                       "parallelism": f"replicas x{world}",
                       "lanes": f"{nl} library contexts on {nl} CUDA streams take frames in turn",
                       "vs_baseline_ref": "paper Table II: 40 fps on a GTX 780 Ti (context, other hardware)"},
            "mde_per_s": fps * W_FULL * H_FULL * DMAX,
            "stage_ms": dict(zip(_lib.STAGE_NAMES, [round(t, 5) for t in stage_ms])),
            "stage_ms_one_lane": dict(zip(_lib.STAGE_NAMES, [round(t, 5) for t in stage_alone])),
            "roofline": {"bound": "alu", "kernel": "costagg_wta_kernel", "achieved": achieved / 1e12,
                         "peak": peak_ops / 1e12, "unit": "Tops/s", "frac": achieved / peak_ops,
                         "traffic": _recorded_traffic(),
                         "traffic_unit": "bytes per launch (dram read + write, ncu)",
                         "peak_source": f"{sm_count} SMs x {LANES_PER_SM} lanes x {sm_mhz:.0f} MHz (issue limit, "
                                        f"max clock from {src} peaks)",
                         "measured": {"int32_add_xor_min_tops": int_ops / 1e12, "popc_tops": popc_s / 1e12,
                                      "lds_tb_per_s": lds_bps / 1e12,
                                      "frac_of_measured_int32": achieved / int_ops,
                                      "source": "stereo_measure_peaks microbenchmarks on this GPU"},
                         "shared_pipe": _shared_pipe(stage_alone[_lib.STAGE_COSTAGG], sm_count, sm_mhz),
                         "ops_per_cell": OPS_PER_CELL, "cells_per_launch": cells,
                         "kernel_ms": stage_ms[_lib.STAGE_COSTAGG], "frames_timed": nframes,
                         "kernel_timer": f"CUDA events around each stage of every {PROFILE_EVERY}th frame of "
                                         f"lane 0 in the timed loop, on the stream the kernels run on; those "
                                         f"frames run with the other lanes' streams held back (cross-stream "
                                         f"waits), so the events time the kernels, not a wait for SMs",
                         "kernel_ms_one_lane": stage_alone[_lib.STAGE_COSTAGG],
                         "frac_one_lane": OPS_PER_CELL * cells / (stage_alone[_lib.STAGE_COSTAGG] / 1e3) / peak_ops,
                         "tile": _lib.stereo_get_tile(st.ctx, W_FULL, H_FULL, DMAX)},
            "e2e": {"value": e2e_fps, "unit": "frames/s", "h2d_bytes_per_step": 2 * W_FULL * H_FULL * 3,
                    "d2h_bytes_per_step": W_FULL * H_FULL * 4, "steps": e2e_steps,
                    "timer": "host wall clock around K stereo_compute_host_async calls from pinned host buffers, "
                             f"taking the {nl} contexts in turn, then a sync of all",
                    "synchronous_call_value": sync_fps},
            "gpu_launches": launches,
            "clocks": clk,
        }
        forms = [] if args.no_forms else [f for f in args.forms.split(",") if f]
        if forms:
            line["forms"] = {}
            if "batch" in forms:
                line["forms"]["batch"] = measure_batch(dev, stream)
            if "serve" in forms:
                line["forms"]["serve"] = measure_serve(dev, seconds=args.serve_seconds)
            if "diff" in forms:
                line["forms"]["diff"] = measure_diff(dev)
        if not args.no_sweep:
            line["sweep"] = measure_sweep(dev)
        if world == 1 and not args.no_cpu_baseline:
            line["cpu_baseline"] = cpu_baseline_leg()
        print(json.dumps(line), flush=True)
    for c_ in ctxs:
        c_.close()
    if world > 1:
        dist.destroy_process_group()


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=200)
    ap.add_argument("--warmup", type=int, default=20)
    ap.add_argument("--impl", choices=["ours", "reference"], default="ours")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-forms", action="store_true", help="skip the batched/served/differentiable forms")
    ap.add_argument("--forms", default="batch,serve,diff",
                    help="comma-separated forms to measure after the pipeline (batch, serve, diff)")
    ap.add_argument("--serve-seconds", type=float, default=60.0, help="length of the served request stream")
    ap.add_argument("--tile", type=int, default=-1, help="force a tile shape of the fused kernel (-1: automatic)")
    ap.add_argument("--lanes", type=int, default=6,
                    help="library contexts (each on its own stream) that take frames in turn, so the small "
                         "kernels of some frames run while another frame's fused kernel finishes")
    ap.add_argument("--no-sweep", action="store_true",
                    help="skip the timings of the Table I arm-cap grid, other frame shapes and Dmax (about 20 s)")
    args = ap.parse_args()
    if args.warmup < 3:
        ap.error("--warmup must be >= 3")
    if args.lanes < 1:
        ap.error("--lanes must be >= 1")
    if any(f not in ("batch", "serve", "diff") for f in args.forms.split(",") if f):
        ap.error("--forms takes batch, serve and diff")
    if args.impl == "reference":
        run_reference(args)
    else:
        run_ours(args)


if __name__ == "__main__":
    main()
