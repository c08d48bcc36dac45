#!/usr/bin/env python3
"""Throughput benchmark of the stereo hot path (Eq. 13 metric, Mde/s).

One step = one sr_match over a seeded synthetic 1280x720 road pair with 64
residual disparities, NCC 7x7, bilateral 11x11 (warp -> NCC volumes ->
aggregation + WTA -> L-R check + post-processing), inputs resident in HBM.
Prints ONE JSON line on rank 0.

  python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference]

--impl reference times the FP64 CPU oracle on the host cores on a bounded
band of rows of the same workload (the reference arm of this comparison).
Under torchrun (N > 1) every rank matches its own frame (weak scaling, no
collective on the data path); the step time is the max over ranks.
"""
from __future__ import annotations

import argparse
import hashlib
import json
import os
import re
import statistics
import subprocess
import sys
import threading
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

METRIC = "Mpix·disp/s + fps at 720p×64 disp; fp16-volume/batched vs fp32 at stated error"
UNIT = "Mpix·disp/s"
FP32_PEAK_TFLOPS = 152 * 128 * 2 * 2.070e9 / 1e12   # SMs x FP32 lanes x FMA x max SM clock
L2_FLUSH_BYTES = 256 << 20


def mdes(W: int, H: int, D: int, seconds: float) -> float:
    """Eq. 13: millions of disparity evaluations per second."""
    return W * H * D / seconds * 1e-6


def agg_flops_per_launch(W, H, D, agg_r):
    """Algorithmic work of one aggregation launch: one multiply and one add per
    window tap per (u, v, d) (Eq. 8 numerator)."""
    return 2 * (2 * agg_r + 1) ** 2 * W * H * D


AGG_SOURCES = ("k_agg.cuh", "k_agg_d64_f32.cu")


def _code_only(text: str) -> str:
    """C++ source without // and /* */ comments and without blank space, so
    that an edit of a comment leaves the hash of the code alone."""
    text = re.sub(r"/\*.*?\*/", " ", text, flags=re.S)
    text = re.sub(r"//[^\n]*", " ", text)
    return re.sub(r"\s+", "", text)


def _kernel_sha() -> str:
    """Hash of the code (comments dropped) of the 1280x720x64 FP32
    aggregation kernel's sources."""
    h = hashlib.sha256()
    for name in AGG_SOURCES:
        path = os.path.join(ROOT, "paper_1807_07433_gb300", "csrc", name)
        if not os.path.exists(path):
            return "missing"
        with open(path) as f:
            h.update(_code_only(f.read()).encode())
    return h.hexdigest()[:16]


def _stored_traffic():
    """DRAM bytes per aggregation launch from the committed ncu summary, or
    None when the kernel source changed since that capture."""
    path = os.path.join(ROOT, "profiles", "agg_wta_1280x720x64.md")
    try:
        text = open(path).read()
    except OSError:
        return None
    m = re.search(r"traffic_bytes_per_launch:\s*([0-9.eE+]+)\s*;\s*kernel_sha:\s*([0-9a-f]+)", text)
    if not m or m.group(2) != _kernel_sha():
        return None
    return float(m.group(1))


class ClockSampler:
    """Samples SM clocks and throttle reasons with nvidia-smi while running."""
    Q = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
         "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
         "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_index: int):
        self.idx = gpu_index
        self.proc = None
        self.lines: list[str] = []
        self.t = None

    def __enter__(self):
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", "-i", str(self.idx), f"--query-gpu={self.Q}",
                 "--format=csv,noheader,nounits", "-lms", "200"],
                stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
            self.t = threading.Thread(target=self._read, daemon=True)
            self.t.start()
            time.sleep(0.3)
        except (OSError, ValueError):
            self.proc = None
        return self

    def _read(self):
        for line in self.proc.stdout:
            self.lines.append(line.strip())

    def __exit__(self, *exc):
        if self.proc is not None:
            self.proc.terminate()
            try:
                self.proc.wait(timeout=5)
            except subprocess.TimeoutExpired:
                self.proc.kill()

    def summary(self):
        sm, smax, reasons = [], [], set()
        names = ("hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap")
        for ln in self.lines:
            f = [x.strip() for x in ln.split(",")]
            if len(f) < 9:
                continue
            try:
                sm.append(float(f[1]))
                smax.append(float(f[2]))
            except ValueError:
                continue
            for n, val in zip(names, f[5:9]):
                if val.lower() == "active":
                    reasons.add(n)
        if not sm:
            return None
        return {"sm_mhz": statistics.median(sm), "sm_max_mhz": max(smax),
                "reasons": sorted(reasons), "samples": len(sm)}


class NvmlSampler:
    """Samples SM clock, its maximum, power and clock-event (throttle)
    reasons through NVML (libnvidia-ml, loaded with ctypes) every ~2 ms on a
    background thread while running, so that even a timed region of a few
    tens of milliseconds gets several samples.  Falls back to ClockSampler
    (nvidia-smi every 200 ms) when NVML cannot be loaded."""
    REASONS = {0x4: "sw_power_cap", 0x8: "hw_slowdown", 0x20: "sw_thermal_slowdown",
               0x40: "hw_thermal_slowdown", 0x80: "hw_power_brake_slowdown"}

    def __init__(self, device_index: int, period_s: float = 0.002):
        self.idx = device_index
        self.period = period_s
        self.samples: list[tuple[float, float, int, float]] = []
        self.h = None
        self.lib = None
        self.stop = threading.Event()
        self.t = None
        self.fallback = None

    def _open(self):
        import ctypes
        lib = ctypes.CDLL("libnvidia-ml.so.1")
        if lib.nvmlInit_v2() != 0:
            raise OSError("nvmlInit failed")
        h = ctypes.c_void_p()
        ok = False
        try:   # the same GPU as the CUDA device: match the PCI bus id, else the UUID
            import torch
            props = torch.cuda.get_device_properties(self.idx)
            bus = getattr(props, "pci_bus_id", None)
            dom = getattr(props, "pci_domain_id", 0)
            dv = getattr(props, "pci_device_id", 0)
            if bus is not None:
                busid = f"{dom:08x}:{bus:02x}:{dv:02x}.0".encode()
                ok = lib.nvmlDeviceGetHandleByPciBusId_v2(busid, ctypes.byref(h)) == 0
            if not ok and getattr(props, "uuid", None) is not None:
                uu = f"GPU-{props.uuid}".encode()
                ok = lib.nvmlDeviceGetHandleByUUID(uu, ctypes.byref(h)) == 0
        except Exception:
            ok = False
        if not ok:
            vis = os.environ.get("CUDA_VISIBLE_DEVICES", "")
            order = [x for x in vis.split(",") if x.strip().isdigit()]
            nidx = int(order[self.idx]) if self.idx < len(order) else self.idx
            if lib.nvmlDeviceGetHandleByIndex_v2(nidx, ctypes.byref(h)) != 0:
                raise OSError("no NVML handle")
        self.lib, self.h = lib, h

    def _read(self):
        import ctypes
        clk, mx, pw = ctypes.c_uint(), ctypes.c_uint(), ctypes.c_uint()
        reasons = ctypes.c_ulonglong()
        get_reasons = getattr(self.lib, "nvmlDeviceGetCurrentClocksEventReasons", None) or \
            self.lib.nvmlDeviceGetCurrentClocksThrottleReasons
        while not self.stop.is_set():
            if self.lib.nvmlDeviceGetClockInfo(self.h, 1, ctypes.byref(clk)) == 0 and \
                    self.lib.nvmlDeviceGetMaxClockInfo(self.h, 1, ctypes.byref(mx)) == 0:
                r = get_reasons(self.h, ctypes.byref(reasons))
                p = self.lib.nvmlDeviceGetPowerUsage(self.h, ctypes.byref(pw))
                self.samples.append((float(clk.value), float(mx.value),
                                     int(reasons.value) if r == 0 else 0,
                                     pw.value / 1000.0 if p == 0 else float("nan")))
            time.sleep(self.period)

    def __enter__(self):
        try:
            self._open()
            self.t = threading.Thread(target=self._read, daemon=True)
            self.t.start()
            time.sleep(0.01)
        except Exception:
            self.fallback = ClockSampler(self.idx).__enter__()
        return self

    def __exit__(self, *exc):
        if self.fallback is not None:
            self.fallback.__exit__(*exc)
            return
        self.stop.set()
        if self.t is not None:
            self.t.join(timeout=2)

    def summary(self):
        if self.fallback is not None:
            out = self.fallback.summary()
            if out is not None:
                out["source"] = "nvidia-smi every 200 ms"
            return out
        if not self.samples:
            return None
        sm = [x[0] for x in self.samples]
        reasons = set()
        for _, _, mask, _ in self.samples:
            for bit, name in self.REASONS.items():
                if mask & bit:
                    reasons.add(name)
        pw = [x[3] for x in self.samples if x[3] == x[3]]
        return {"sm_mhz": statistics.median(sm), "sm_max_mhz": max(x[1] for x in self.samples),
                "sm_mhz_min": min(sm), "reasons": sorted(reasons), "samples": len(sm),
                "power_w_max": round(max(pw), 1) if pw else None,
                "source": "NVML every ~2 ms"}


def step_stats(ms: list[float]) -> dict:
    """Median, mean and 10th / 90th percentiles of per-step times (ms)."""
    q = statistics.quantiles(ms, n=10, method="inclusive") if len(ms) >= 2 else [ms[0]] * 9
    return {"median": round(statistics.median(ms), 5), "mean": round(sum(ms) / len(ms), 5),
            "p10": round(q[0], 5), "p90": round(q[8], 5), "n": len(ms)}


def _dist():
    ws = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return ws, rank, local


def max_over_ranks(x: float, ws: int, device) -> float:
    """Maximum of x over the ranks of the default process group (x for one rank)."""
    if ws == 1:
        return float(x)
    import torch
    import torch.distributed as dist
    t = torch.tensor([float(x)], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def whole_job(W: int, H: int, D: int, ms_step_max: float, ws: int):
    """Whole-job (Mde/s, fps) when each of ws ranks matches one W x H x D frame
    per step and the slowest rank takes ms_step_max per step (weak scaling)."""
    return mdes(W, H, D, ms_step_max * 1e-3) * ws, 1000.0 / ms_step_max * ws


def run_ours(args, w):
    import numpy as np
    import torch
    import torch.distributed as dist

    from paper_1807_07433_gb300 import sr, synth

    ws, rank, local = _dist()
    if ws > 1:
        dist.init_process_group("nccl", init_method="env://")
    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)
    W, H, D = w.scene.W, w.scene.H, w.D
    left, right, _ = synth.make_pair(w.scene)
    stream = torch.cuda.current_stream(dev)

    dl = torch.from_numpy(left).to(dev)
    dr = torch.from_numpy(right).to(dev)
    disp = torch.empty((H, W), dtype=torch.float32, device=dev)
    flush = torch.empty(L2_FLUSH_BYTES, dtype=torch.uint8, device=dev)

    vol = {"f32": sr.SR_VOL_F32, "f16": sr.SR_VOL_F16, "bf16": sr.SR_VOL_BF16}[args.volume]
    m = sr.Matcher(W, H, D, w.ncc_r, w.agg_r, w.gamma_d, w.gamma_r, w.lr_thresh, vol_dtype=vol,
                   stream=stream)
    m.set_plane(w.scene.alpha0, w.scene.alpha1, w.delta)
    kpm = sr.sr_kernels_per_match(m.ctx)

    for _ in range(args.warmup):
        flush.zero_()
        m.match(dl, dr, disp)
    torch.cuda.synchronize()

    # Timed region: K matches, each bracketed by CUDA events on the context's
    # stream; the L2 flush runs between them, outside the events.  The
    # library's stage events are off here: recorded between the kernels
    # they would stop each aggregation from starting while its predecessor
    # drains.  The stage times come from a second pass of K matches with
    # them on (the library records them into a ring, read after the pass).
    starts = [torch.cuda.Event(enable_timing=True) for _ in range(args.steps)]
    ends = [torch.cuda.Event(enable_timing=True) for _ in range(args.steps)]
    if ws > 1:
        dist.barrier()
    torch.cuda.synchronize()
    wall0 = time.perf_counter()
    with NvmlSampler(local) as clk:
        for k in range(args.steps):
            flush.zero_()                       # L2 flush outside the timed events
            starts[k].record(stream)
            m.match(dl, dr, disp)
            ends[k].record(stream)
        torch.cuda.synchronize()
    wall = time.perf_counter() - wall0
    if ws > 1:
        dist.barrier()
    step_ms = [s.elapsed_time(e) for s, e in zip(starts, ends)]
    total_ms_max = max_over_ranks(sum(step_ms), ws, dev)
    sr.sr_set_profiling(m.ctx, True)     # the stage pass
    for k in range(args.steps):
        flush.zero_()
        m.match(dl, dr, disp)
    torch.cuda.synchronize()
    stage_rows = sr.sr_stage_times_history(m.ctx, args.steps)
    sr.sr_set_profiling(m.ctx, False)

    # End to end through the public C ABI with pinned host buffers: every
    # frame's upload of both images and download of its disparity map are
    # inside the timed region.  sr_match_host_async (the streaming call)
    # overlaps them with the kernels of the neighbouring frames;
    # sr_match_host (one synchronous call per frame) is timed beside it.
    hl = torch.from_numpy(left).pin_memory()
    hr = torch.from_numpy(right).pin_memory()
    hd = [torch.empty((H, W), dtype=torch.float32).pin_memory() for _ in range(2)]
    for i in range(max(2, args.warmup)):
        sr.sr_match_host_async(m.ctx, hl, hr, hd[i % 2])
    sr.sr_synchronize(m.ctx)
    if ws > 1:
        dist.barrier()
    e0 = time.perf_counter()
    for i in range(args.steps):
        sr.sr_match_host_async(m.ctx, hl, hr, hd[i % 2])
    sr.sr_synchronize(m.ctx)
    e_s = max_over_ranks(time.perf_counter() - e0, ws, dev)
    valid_frac = float(np.isfinite(hd[(args.steps - 1) % 2].numpy()).mean())
    for _ in range(2):
        sr.sr_match_host(m.ctx, hl, hr, hd[0])
    if ws > 1:
        dist.barrier()
    e0 = time.perf_counter()
    for _ in range(args.steps):
        sr.sr_match_host(m.ctx, hl, hr, hd[0])
    torch.cuda.synchronize()
    e_sync_s = max_over_ranks(time.perf_counter() - e0, ws, dev)
    m.close()

    if rank != 0:
        if ws > 1:
            dist.destroy_process_group()
        return None

    ms_step = total_ms_max / args.steps
    agg_ms = [r["agg_ref"] for r in stage_rows]
    agg_avg_ms = sum(agg_ms) / len(agg_ms)
    flops = agg_flops_per_launch(W, H, D, w.agg_r)
    achieved = flops / (agg_avg_ms * 1e-3) / 1e12
    stages = {k: round(sum(r[k] for r in stage_rows) / len(stage_rows), 5) for k in stage_rows[0]}
    value, fps = whole_job(W, H, D, ms_step, ws)
    e2e_value, _ = whole_job(W, H, D, e_s / args.steps * 1e3, ws)
    e2e_sync_value, _ = whole_job(W, H, D, e_sync_s / args.steps * 1e3, ws)
    line = {
        "metric": METRIC, "value": round(value, 2), "unit": UNIT, "fps": round(fps, 2),
        "n_gpus": ws, "steps": args.steps, "warmup": args.warmup,
        "ms_per_step": round(ms_step, 5), "step_ms": step_stats(step_ms),
        "higher_is_better": True, "scaling": "weak",
        "vs_baseline": None, "dtype": "f32",
        "data": "synthetic: seeded textured road plane with potholes and grooves (generator "
                "paper_1807_07433_gb300/synth.py, seed 2); stands in for the paper's ZED road data",
        "config": {"workload": w.name, "W": W, "H": H, "D": D, "ncc_window": 2 * w.ncc_r + 1,
                   "bilateral_window": 2 * w.agg_r + 1, "gamma_d": w.gamma_d,
                   "gamma_r": w.gamma_r, "delta": w.delta,
                   "form": "staged " + {"f32": "fp32", "f16": "fp16", "bf16": "bf16"}[args.volume] + " volumes",
                   "l2": f"flushed between timed steps ({L2_FLUSH_BYTES >> 20} MiB memset)",
                   "parallelism": f"replicas x{ws} (independent frames)"},
        "roofline": {"bound": "alu", "kernel": "k_agg_wta (reference view)",
                     "achieved": round(achieved, 3), "peak": round(FP32_PEAK_TFLOPS, 2),
                     "unit": "TFLOP/s", "frac": round(achieved / FP32_PEAK_TFLOPS, 4),
                     "peak_source": "derived: 152 SMs x 128 FP32 lanes x 2 flop x 2070 MHz",
                     "flops_per_launch": flops, "launch_ms": round(agg_avg_ms, 5),
                     "traffic": _stored_traffic() if args.volume == "f32" else None},
        "stages_ms": stages,
        "e2e": {"value": round(e2e_value, 2), "unit": UNIT,
                "h2d_bytes_per_step": 2 * W * H, "d2h_bytes_per_step": 4 * W * H,
                "api": "sr_match_host_async (pinned host buffers; uploads and downloads on "
                       "copy streams overlap the neighbouring frames' kernels)",
                "value_sync_api": round(e2e_sync_value, 2)},
        "gpu_launches": kpm * args.steps,
        "valid_fraction": round(valid_frac, 4),
        "wall_s_timed_region": round(wall, 3),
    }
    clk_sum = clk.summary()
    line["clocks"] = clk_sum
    return line


def _timed_steps(fn, steps: int, warmup: int, stream, flush):
    """Per-step device times (ms) of fn: CUDA events on stream around each
    call, L2 flushed before each (outside the events), no synchronisation
    between steps."""
    import torch
    for _ in range(warmup):
        fn()
    torch.cuda.synchronize()
    ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True))
          for _ in range(steps)]
    for e0, e1 in ev:
        flush.zero_()
        e0.record(stream)
        fn()
        e1.record(stream)
    torch.cuda.synchronize()
    return [e0.elapsed_time(e1) for e0, e1 in ev]


def _faster_beyond_spread(form: dict, base: dict) -> bool:
    """The form's 90th-percentile step time lies below the base form's 10th."""
    return form["step_ms"]["p90"] < base["step_ms"]["p10"]


def forms_720p(w, steps: int, warmup: int, dev) -> dict:
    """The 1280x720x64 workload in each volume type (FP32, FP16, BF16 storage,
    FP32 arithmetic), steps steps each, and the FP32 step followed by
    sr_reconstruct (Sec. II-D)."""
    import torch
    from paper_1807_07433_gb300 import sr, synth
    W, H, D = w.scene.W, w.scene.H, w.D
    left, right, _ = synth.make_pair(w.scene)
    stream = torch.cuda.current_stream(dev)
    dl, dr = torch.from_numpy(left).to(dev), torch.from_numpy(right).to(dev)
    disp = torch.empty((H, W), dtype=torch.float32, device=dev)
    xyz = torch.empty((3, H, W), dtype=torch.float32, device=dev)
    flush = torch.empty(L2_FLUSH_BYTES, dtype=torch.uint8, device=dev)
    out = {}
    for name, vt in (("fp32", sr.SR_VOL_F32), ("fp16", sr.SR_VOL_F16), ("bf16", sr.SR_VOL_BF16)):
        with sr.Matcher(W, H, D, w.ncc_r, w.agg_r, w.gamma_d, w.gamma_r, w.lr_thresh,
                        vol_dtype=vt, stream=stream) as m:
            m.set_plane(w.scene.alpha0, w.scene.alpha1, w.delta)
            m.set_camera(w.f_px, w.baseline_mm)
            ms = _timed_steps(lambda: m.match(dl, dr, disp), steps, warmup, stream, flush)
            st = step_stats(ms)
            out[name] = {"mdes": round(mdes(W, H, D, st["median"] * 1e-3), 1),
                         "fps": round(1e3 / st["median"], 1), "step_ms": st}
            if name == "fp32":
                ms = _timed_steps(lambda: (m.match(dl, dr, disp), m.reconstruct(disp, xyz)),
                                  steps, warmup, stream, flush)
                out["fp32_with_reconstruct"] = {"step_ms": step_stats(ms)}
    for name in ("fp16", "bf16"):
        out[name]["vs_fp32_median"] = round(out["fp32"]["step_ms"]["median"] /
                                            out[name]["step_ms"]["median"], 4)
        out[name]["faster_beyond_spread"] = _faster_beyond_spread(out[name], out["fp32"])
    return out


def _gen_pairs_spawn(scenes):
    import multiprocessing as mp
    with mp.get_context("spawn").Pool(min(16, os.cpu_count() or 1)) as pool:
        return pool.map(_gen_pair, scenes)


def forms_batch(steps: int, warmup: int, dev, data=None) -> dict:
    """The 64-pair workload (16 each of 672x376, 1280x720, 1920x1080,
    2208x1242, D = 64, NCC 7x7, bilateral 11x11): 64 sequential plain FP32
    sr_match calls, and sr_match_batch (autotuned schedule in a CUDA graph)
    with FP32 and FP16 volumes; per-step times of the whole batch."""
    import torch
    from paper_1807_07433_gb300 import sr, synth
    ws = synth.batch_workloads()
    if data is None:
        data = _gen_pairs_spawn([w.scene for w in ws])
    D = ws[0].D
    stream = torch.cuda.current_stream(dev)
    ins, outs = [], []
    for left, right in data:
        H, W = left.shape
        ins.append((torch.from_numpy(left).to(dev), torch.from_numpy(right).to(dev)))
        outs.append(torch.empty((H, W), dtype=torch.float32, device=dev))
    total_de = sum(w.scene.W * w.scene.H * D for w in ws)
    flush = torch.empty(L2_FLUSH_BYTES, dtype=torch.uint8, device=dev)
    res = {}
    ctxs = {}
    for w in ws:
        key = (w.scene.W, w.scene.H)
        if key not in ctxs:
            ctxs[key] = sr.Matcher(w.scene.W, w.scene.H, D, w.ncc_r, w.agg_r, w.gamma_d,
                                   w.gamma_r, w.lr_thresh, stream=stream)

    def seq():
        for w, (dl, dr), out in zip(ws, ins, outs):
            m = ctxs[(w.scene.W, w.scene.H)]
            m.set_plane(w.scene.alpha0, w.scene.alpha1, w.delta)
            m.match(dl, dr, out)
    st = step_stats(_timed_steps(seq, steps, warmup, stream, flush))
    res["sequential_fp32"] = {"mdes": round(total_de / (st["median"] * 1e-3) * 1e-6, 1),
                              "step_ms": st}
    for m in ctxs.values():
        m.close()
    w0 = ws[0]
    for name, vt in (("batched_fp32", sr.SR_VOL_F32), ("batched_fp16", sr.SR_VOL_F16)):
        with sr.Matcher(8, 8, D, w0.ncc_r, w0.agg_r, w0.gamma_d, w0.gamma_r, w0.lr_thresh,
                        vol_dtype=vt, stream=stream) as m:
            sr.sr_set_autotune(m.ctx, True)
            descs = [sr.make_pair_desc(dl, dr, out, w.scene.alpha0, w.scene.alpha1, w.delta)
                     for w, (dl, dr), out in zip(ws, ins, outs)]
            sr.sr_match_batch(m.ctx, descs)        # tunes on first use
            torch.cuda.synchronize()
            st = step_stats(_timed_steps(lambda: sr.sr_match_batch(m.ctx, descs), steps,
                                         warmup, stream, flush))
            res[name] = {"mdes": round(total_de / (st["median"] * 1e-3) * 1e-6, 1),
                         "step_ms": st, "schedule": sr.sr_batch_info(m.ctx)}
        torch.cuda.empty_cache()
    for name in ("batched_fp32", "batched_fp16"):
        res[name]["vs_sequential_fp32_median"] = round(
            res["sequential_fp32"]["step_ms"]["median"] / res[name]["step_ms"]["median"], 4)
        res[name]["faster_beyond_spread"] = _faster_beyond_spread(res[name],
                                                                  res["sequential_fp32"])
    return {"pairs": len(ws), "total_disparity_evaluations": total_de, "forms": res}


def cpu_baseline_protocol(w2, target_s: float = 8.0) -> dict:
    """The FP64 oracle on the host cores: the 1280x720x64 frame on a band of
    rows with all cores and with one core, the 160x120x16 frame whole, and a
    band of the 1920x1080x64 frame, each sized to about target_s seconds."""
    import oracle
    from paper_1807_07433_gb300 import synth
    cores = os.cpu_count() or 1
    out = {}
    val, dt, rows, n = oracle_sample(w2, target_s=target_s)
    out["c2_all_cores"] = {"value": round(val, 4), "cores": n, "seconds": round(dt, 2),
                           "rows": list(rows)}
    oracle.set_num_threads(1)
    val1, dt1, rows1, _ = oracle_sample(w2, target_s=target_s, threads=1)
    out["c2_one_core"] = {"value": round(val1, 4), "cores": 1, "seconds": round(dt1, 2),
                          "rows": list(rows1)}
    oracle.set_num_threads(cores)
    val, dt, rows, n = oracle_sample(synth.C1, target_s=min(target_s, 2.0))
    out["c1_all_cores"] = {"value": round(val, 4), "cores": n, "seconds": round(dt, 2),
                           "rows": list(rows)}
    val, dt, rows, n = oracle_sample(synth.C3, target_s=target_s)
    out["c3_all_cores"] = {"value": round(val, 4), "cores": n, "seconds": round(dt, 2),
                           "rows": list(rows)}
    return out


def oracle_sample(w, target_s: float, rows_hint: int | None = None, threads: int | None = None):
    """Time the FP64 oracle on a band of output rows sized for about
    target_s seconds, on threads host cores (default: all); returns (Mde/s,
    seconds, rows, cores)."""
    import oracle
    from paper_1807_07433_gb300 import synth
    oracle.build()
    cores = threads or os.cpu_count() or 1
    oracle.set_num_threads(cores)
    left, right, _ = synth.make_pair(w.scene)
    p = oracle.Params(W=w.scene.W, H=w.scene.H, D=w.D, ncc_r=w.ncc_r, agg_r=w.agg_r,
                      gamma_d=w.gamma_d, gamma_r=w.gamma_r, lr_thresh=w.lr_thresh,
                      alpha0=w.scene.alpha0, alpha1=w.scene.alpha1, delta=w.delta)
    r0 = 0
    if rows_hint is None:
        probe = min(16, w.scene.H)
        t0 = time.perf_counter()
        oracle.match(p, left, right, rows=(0, probe), want=("dfull",))
        t_probe = time.perf_counter() - t0
        rows = int(max(probe, min(w.scene.H, probe * target_s / max(t_probe, 1e-6))))
    else:
        rows = rows_hint
    reps, t0 = 0, time.perf_counter()
    while True:   # repeat the band until about target_s of CPU work has run
        oracle.match(p, left, right, rows=(r0, r0 + rows), want=("dfull",))
        reps += 1
        dt = time.perf_counter() - t0
        if rows_hint is not None or dt >= target_s:
            break
    return mdes(w.scene.W, rows * reps, w.D, dt), dt, (r0, r0 + rows), oracle.num_threads()


def run_reference(args, w):
    ws, rank, _ = _dist()
    if rank != 0:
        return None
    # one probe sizes the band; each timed step re-runs the band
    val, dt, rows, cores = oracle_sample(w, target_s=min(20.0, 150.0 / max(1, args.steps + args.warmup)))
    for _ in range(max(0, args.warmup - 1)):
        oracle_sample(w, 0, rows_hint=rows[1] - rows[0])
    times = []
    for _ in range(args.steps):
        v, dt, _, _ = oracle_sample(w, 0, rows_hint=rows[1] - rows[0])
        times.append(dt)
    per = sum(times) / len(times)
    value = mdes(w.scene.W, rows[1] - rows[0], w.D, per)
    sample = (f"output rows {rows[0]}..{rows[1] - 1} of the {w.scene.W}x{w.scene.H}x{w.D} frame "
              f"(+{w.agg_r} halo rows of NCC each side), FP64 oracle, OpenMP")
    return {
        "impl": "reference", "metric": METRIC, "value": round(value, 4), "unit": UNIT,
        "n_gpus": ws, "steps": args.steps, "warmup": args.warmup,
        "ms_per_step": round(per * 1e3, 3), "higher_is_better": True, "scaling": "weak",
        "vs_baseline": None, "dtype": "f64", "data": "synthetic (same seeded scene as ours)",
        "config": {"workload": w.name, "W": w.scene.W, "H": w.scene.H, "D": w.D,
                   "ncc_window": 2 * w.ncc_r + 1, "bilateral_window": 2 * w.agg_r + 1},
        "cpu_baseline": {"value": round(value, 4), "unit": UNIT, "cores": cores,
                         "kind": "oracle", "sample": sample},
        "e2e": {"value": round(value, 4), "unit": UNIT, "h2d_bytes_per_step": 0,
                "d2h_bytes_per_step": 0},
        "gpu_launches": 0,
    }


def precision_report(steps: int, warmup: int):
    """Precision form on the 1280x720x64 and 1920x1080x64 workloads: FP32 /
    FP16 / BF16 volumes, each timed (CUDA events, L2 flushed between steps)
    and compared with the full-frame FP64 oracle: integer-disparity mismatch
    rate, subpixel RMS and 3-D point error (mm, f = 700 px, baseline 120 mm)."""
    from paper_1807_07433_gb300 import synth
    return {"report": "precision", "reference": "FP64 oracle, full frame", "steps": steps,
            "warmup": warmup,
            "workloads": [_precision_workload(w, steps, warmup) for w in (synth.C2, synth.C3)]}


def _precision_workload(w, steps: int, warmup: int):
    import numpy as np
    import torch

    import oracle
    from paper_1807_07433_gb300 import sr, synth

    W, H, D = w.scene.W, w.scene.H, w.D
    left, right, _ = synth.make_pair(w.scene)
    oracle.build()
    oracle.set_num_threads(os.cpu_count() or 1)
    p = oracle.Params(W=W, H=H, D=D, ncc_r=w.ncc_r, agg_r=w.agg_r, gamma_d=w.gamma_d,
                      gamma_r=w.gamma_r, lr_thresh=w.lr_thresh, alpha0=w.scene.alpha0,
                      alpha1=w.scene.alpha1, delta=w.delta, f_px=w.f_px, baseline=w.baseline_mm)
    t0 = time.perf_counter()
    o = oracle.match(p, left, right, want=("lbl_l", "gap_l", "dfull", "xyz"))
    t_orc = time.perf_counter() - t0
    dev = torch.device("cuda", 0)
    dl, dr = torch.from_numpy(left).to(dev), torch.from_numpy(right).to(dev)
    flush = torch.empty(L2_FLUSH_BYTES, dtype=torch.uint8, device=dev)
    stream = torch.cuda.current_stream(dev)
    forms = {}
    for name, vt in (("f32", sr.SR_VOL_F32), ("f16", sr.SR_VOL_F16), ("bf16", sr.SR_VOL_BF16)):
        m = sr.Matcher(W, H, D, w.ncc_r, w.agg_r, w.gamma_d, w.gamma_r, w.lr_thresh,
                       vol_dtype=vt, stream=stream)
        m.set_plane(w.scene.alpha0, w.scene.alpha1, w.delta)
        m.set_camera(w.f_px, w.baseline_mm)
        disp = torch.empty((H, W), dtype=torch.float32, device=dev)
        wta = torch.empty((H, W), dtype=torch.int16, device=dev)
        for _ in range(warmup):
            m.match(dl, dr, disp, wta)
        ms = []
        for _ in range(steps):
            flush.zero_()
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            e0.record(stream)
            m.match(dl, dr, disp, wta)
            e1.record(stream)
            e1.synchronize()
            ms.append(e0.elapsed_time(e1))
        xyz = m.reconstruct(disp)
        torch.cuda.synchronize()
        g_d, g_l, g_xyz = disp.cpu().numpy(), wta.cpu().numpy(), xyz.cpu().numpy()
        m.close()
        t = statistics.median(ms) * 1e-3
        diff = g_l != o.lbl_l
        both = np.isfinite(g_d) & np.isfinite(o.dfull) & ~diff
        dd = g_d[both] - o.dfull[both]
        dx = np.linalg.norm(g_xyz[:, both] - o.xyz[:, both], axis=0)
        forms[name] = {
            "mdes": round(mdes(W, H, D, t), 1), "fps": round(1.0 / t, 1),
            "ms_median": round(t * 1e3, 4),
            "label_mismatch_pct": round(100.0 * diff.mean(), 4),
            "label_mismatch_outside_gap_1e-4_pct": round(100.0 * (diff & (o.gap_l >= 1e-4)).mean(), 4),
            "validity_mismatch_pct": round(100.0 * (np.isfinite(g_d) != np.isfinite(o.dfull)).mean(), 4),
            "subpixel_rms_px": float(np.sqrt(np.mean(dd ** 2))),
            "subpixel_max_px": float(np.abs(dd).max()),
            "xyz_rms_mm": float(np.sqrt(np.mean(dx ** 2))),
            "xyz_p99_mm": float(np.quantile(dx, 0.99)),
            "compared_pixels": int(both.sum()),
        }
    return {"workload": w.name, "W": W, "H": H, "D": D, "oracle_s": round(t_orc, 2),
            "forms": forms}




def _gen_pair(scene):
    from paper_1807_07433_gb300 import synth
    left, right, _ = synth.make_pair(scene)
    return left, right


def batch_report(steps: int, warmup: int):
    """Batched form on 64 mixed-size pairs (16 each of 672x376, 1280x720,
    1920x1080, 2208x1242; D = 64, NCC 7x7, bilateral 11x11): one
    sr_match_batch (persistent launches in a CUDA graph, autotuned) with FP32
    and FP16 volumes, against 64 sequential plain FP32 sr_match calls (queued
    back to back, and synchronised after each call)."""
    import multiprocessing as mp

    from paper_1807_07433_gb300 import synth
    ws = synth.batch_workloads()
    with mp.get_context("spawn").Pool(min(16, os.cpu_count() or 1)) as pool:
        data = pool.map(_gen_pair, [w.scene for w in ws])   # before any CUDA call

    import torch
    from paper_1807_07433_gb300 import sr
    w0 = ws[0]
    D = w0.D
    dev = torch.device("cuda", 0)
    stream = torch.cuda.current_stream(dev)
    ins, outs = [], []
    for (left, right) in data:
        H, W = left.shape
        ins.append((torch.from_numpy(left).to(dev), torch.from_numpy(right).to(dev)))
        outs.append(torch.empty((H, W), dtype=torch.float32, device=dev))
    total_de = sum(w.scene.W * w.scene.H * D for w in ws)
    flush = torch.empty(L2_FLUSH_BYTES, dtype=torch.uint8, device=dev)
    res = {}

    def timed(fn):
        for _ in range(warmup):
            fn()
        torch.cuda.synchronize()
        ms = []
        for _ in range(steps):
            flush.zero_()
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            e0.record(stream)
            fn()
            e1.record(stream)
            e1.synchronize()
            ms.append(e0.elapsed_time(e1))
        return statistics.median(ms)

    # 64 sequential plain FP32 calls, one context per image size
    ctxs = {}
    for w in ws:
        key = (w.scene.W, w.scene.H)
        if key not in ctxs:
            ctxs[key] = sr.Matcher(w.scene.W, w.scene.H, D, w.ncc_r, w.agg_r, w.gamma_d,
                                   w.gamma_r, w.lr_thresh, stream=stream)

    def seq(sync):
        for w, (dl, dr), out in zip(ws, ins, outs):
            m = ctxs[(w.scene.W, w.scene.H)]
            m.set_plane(w.scene.alpha0, w.scene.alpha1, w.delta)
            m.match(dl, dr, out)
            if sync:
                torch.cuda.synchronize()
    for name, sync in (("sequential_f32_queued", False), ("sequential_f32_sync_each", True)):
        t = timed(lambda: seq(sync))
        res[name] = {"ms": round(t, 3), "mdes": round(total_de / (t * 1e-3) * 1e-6, 1)}
    for m in ctxs.values():
        m.close()

    for name, vt in (("batched_f32", sr.SR_VOL_F32), ("batched_f16", sr.SR_VOL_F16)):
        m = sr.Matcher(8, 8, D, w0.ncc_r, w0.agg_r, w0.gamma_d, w0.gamma_r, w0.lr_thresh,
                       vol_dtype=vt, stream=stream)
        sr.sr_set_autotune(m.ctx, True)
        descs = [sr.make_pair_desc(dl, dr, out, w.scene.alpha0, w.scene.alpha1, w.delta)
                 for w, (dl, dr), out in zip(ws, ins, outs)]
        sr.sr_match_batch(m.ctx, descs)        # tunes on first use
        torch.cuda.synchronize()
        t = timed(lambda: sr.sr_match_batch(m.ctx, descs))
        res[name] = {"ms": round(t, 3), "mdes": round(total_de / (t * 1e-3) * 1e-6, 1),
                     "schedule": sr.sr_batch_info(m.ctx)}
        m.close()
        torch.cuda.empty_cache()
    return {"report": "batch", "pairs": len(ws), "sizes": [list(s) for s in synth.BATCH_SIZES],
            "D": D, "total_disparity_evaluations": total_de, "steps": steps, "warmup": warmup,
            "l2": "flushed between timed steps", "forms": res}


def adjoint_report(steps: int, warmup: int):
    """Plane refinement on the 1280x720 D64 NCC 7x7 bilateral 11x11 workload:
    time of one sr_grad_plane (L and dL/dalpha, plane hypothesis: every pixel
    at residual delta), then refinement (L-BFGS and Adam, at most 50
    evaluations each) from the true plane perturbed by (U[-1.5, 1.5] px,
    U[-0.01, 0.01] px/row), seed 5, on the scene with potholes and grooves and
    on the same road without them.  Errors are in pixels: alpha0 and the
    alpha1 shift accumulated over the frame, alpha1 (H-1)."""
    import dataclasses

    import numpy as np
    import torch

    from paper_1807_07433_gb300 import refine, sr, synth
    w = synth.C2
    dev = torch.device("cuda", 0)
    stream = torch.cuda.current_stream(dev)
    out = {"report": "adjoint", "workload": w.name, "objective": "sum_p c_agg(p, delta)",
           "steps": steps, "warmup": warmup}
    scenes = {"with_depressions": w.scene,
              "plain_road": dataclasses.replace(w.scene, n_potholes=0, grooves=False)}
    for key, sc in scenes.items():
        left, right, _ = synth.make_pair(sc)
        H, W = left.shape
        with sr.Matcher(W, H, w.D, w.ncc_r, w.agg_r, w.gamma_d, w.gamma_r, stream=stream) as m:
            dl, dr = torch.from_numpy(left).to(dev), torch.from_numpy(right).to(dev)
            dstar = torch.full((H, W), int(w.delta), dtype=torch.int16, device=dev)
            ev = refine.MatcherEvaluator(m, dl, dr, dstar, w.delta)
            ent = {}
            if key == "with_depressions":
                for _ in range(warmup):
                    ev.value_and_grad(sc.alpha0 + 0.3, sc.alpha1)
                ms = []
                for _ in range(steps):
                    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
                    e0.record(stream)
                    m.set_plane(sc.alpha0 + 0.3, sc.alpha1, w.delta)
                    sr.sr_grad_plane(m.ctx, dl, dr, W, dstar)
                    e1.record(stream)
                    e1.synchronize()
                    ms.append(e0.elapsed_time(e1))
                ent["grad_ms_median"] = round(statistics.median(ms), 3)
                gl = torch.empty((H, W), dtype=torch.float32, device=dev)
                gr = torch.empty_like(gl)
                ms = []
                for _ in range(max(3, steps // 4)):
                    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
                    e0.record(stream)
                    sr.sr_grad_plane(m.ctx, dl, dr, W, dstar, gl, gr)
                    e1.record(stream)
                    e1.synchronize()
                    ms.append(e0.elapsed_time(e1))
                ent["grad_with_image_grads_ms_median"] = round(statistics.median(ms), 3)
            rng = np.random.default_rng(5)
            a_init = (sc.alpha0 + rng.uniform(-1.5, 1.5), sc.alpha1 + rng.uniform(-0.01, 0.01))
            L_true = ev.value_and_grad(sc.alpha0, sc.alpha1)[0]
            ent.update({"alpha_true": [sc.alpha0, sc.alpha1], "alpha_init": list(a_init),
                        "err_init_px": [a_init[0] - sc.alpha0,
                                        (a_init[1] - sc.alpha1) * (H - 1)],
                        "L_true_plane": L_true})
            for method in ("lbfgs", "adam"):
                torch.cuda.synchronize()
                t0 = time.perf_counter()
                res = refine.refine_plane(ev, a_init, H, max_evals=50, method=method)
                t_ref = time.perf_counter() - t0
                ent[method] = {
                    "evaluations": len(res.history), "alpha_final": list(res.alpha),
                    "err_final_px": [res.alpha[0] - sc.alpha0,
                                     (res.alpha[1] - sc.alpha1) * (H - 1)],
                    "L_init": res.history[0][2], "L_final": max(h[2] for h in res.history),
                    "wall_s": round(t_ref, 3)}
            out[key] = ent
    return out


def sweep_report(steps: int, warmup: int):
    """Runtime of sr_match at 1280x720, D = 64 for every NCC radius 1..5 and
    bilateral radius 1..7 (the parameters Fig. 4 varies), same scene and
    gamma_d / gamma_r as the benchmark; median over steps CUDA-event timings
    (L2 flushed between steps) plus the per-stage split."""
    import torch

    from paper_1807_07433_gb300 import sr, synth
    w = synth.C2
    left, right, _ = synth.make_pair(w.scene)
    H, W = left.shape
    dev = torch.device("cuda", 0)
    stream = torch.cuda.current_stream(dev)
    dl, dr = torch.from_numpy(left).to(dev), torch.from_numpy(right).to(dev)
    disp = torch.empty((H, W), dtype=torch.float32, device=dev)
    flush = torch.empty(L2_FLUSH_BYTES, dtype=torch.uint8, device=dev)
    rows = []
    for ncc_r in range(1, 6):
        for agg_r in range(1, 8):
            with sr.Matcher(W, H, w.D, ncc_r, agg_r, w.gamma_d, w.gamma_r, w.lr_thresh,
                            stream=stream) as m:
                m.set_plane(w.scene.alpha0, w.scene.alpha1, w.delta)
                for _ in range(warmup):
                    m.match(dl, dr, disp)
                # frame times without the stage events (they would keep the
                # aggregations from overlapping their predecessors), then
                # the stage times in a second pass
                ms, st_rows = [], []
                for _ in range(steps):
                    flush.zero_()
                    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
                    e0.record(stream)
                    m.match(dl, dr, disp)
                    e1.record(stream)
                    ms.append((e0, e1))
                torch.cuda.synchronize()
                ms = [a.elapsed_time(b) for a, b in ms]
                sr.sr_set_profiling(m.ctx, True)
                for _ in range(steps):
                    flush.zero_()
                    m.match(dl, dr, disp)
                    st_rows.append(sr.sr_stage_times(m.ctx))
                sr.sr_set_profiling(m.ctx, False)
                t = statistics.median(ms)
                valid = float(torch.isfinite(disp).float().mean())
            rows.append({"ncc_window": 2 * ncc_r + 1, "bilateral_window": 2 * agg_r + 1,
                         "ms": round(t, 4), "mdes": round(mdes(W, H, w.D, t * 1e-3), 1),
                         "fps": round(1000.0 / t, 1),
                         "ncc_ms": round(statistics.median(r["ncc"] for r in st_rows), 4),
                         "agg_ms": round(statistics.median(r["agg_ref"] + r["agg_tgt"] for r in st_rows), 4),
                         "valid_fraction": round(valid, 4)})
    return {"report": "sweep", "workload": w.name, "W": W, "H": H, "D": w.D, "steps": steps,
            "warmup": warmup, "rows": rows}


def fit_report(steps: int, warmup: int):
    """Sec. II-A plane fitting on the benchmark frame: time of sr_fit_alpha
    (256 RANSAC hypotheses, tau = 0.5 px) and sr_fit_roll (near-field patch
    rows 560-719, columns 320-959) on the disparity map of sr_match, the
    fitted plane against the scene's, and the closed loop match -> fit ->
    match from a perturbed plane."""
    import numpy as np
    import torch

    from paper_1807_07433_gb300 import sr, synth
    w = synth.C2
    left, right, _ = synth.make_pair(w.scene)
    H, W = left.shape
    dev = torch.device("cuda", 0)
    stream = torch.cuda.current_stream(dev)
    dl, dr = torch.from_numpy(left).to(dev), torch.from_numpy(right).to(dev)
    pairs = np.random.default_rng(9).integers(0, H * W, size=(256, 2)).astype(np.int32)
    out = {"report": "fit", "workload": w.name, "hypotheses": 256, "tau_px": 0.5,
           "roll_patch": [320, 560, 960, 720], "steps": steps, "warmup": warmup}
    with sr.Matcher(W, H, w.D, w.ncc_r, w.agg_r, w.gamma_d, w.gamma_r, w.lr_thresh,
                    stream=stream) as m:
        m.set_plane(w.scene.alpha0, w.scene.alpha1, w.delta)
        disp = m.match(dl, dr)

        def timed(fn):
            for _ in range(warmup):
                fn()
            ts = []
            for _ in range(steps):
                torch.cuda.synchronize()
                t0 = time.perf_counter()
                r = fn()
                ts.append(time.perf_counter() - t0)
            return r, statistics.median(ts) * 1e3
        fa, ms_a = timed(lambda: sr.sr_fit_alpha(m.ctx, disp, pairs, 0.5))
        fr, ms_r = timed(lambda: sr.sr_fit_roll(m.ctx, disp, 320, 560, 960, 720))
        out.update({"fit_alpha_ms": round(ms_a, 3), "fit_roll_ms": round(ms_r, 3),
                    "alpha": fa["alpha"].tolist(), "alpha_true": [w.scene.alpha0, w.scene.alpha1],
                    "inliers": fa["n_inliers"], "valid_pixels": int(torch.isfinite(disp).sum()),
                    "gamma": fr[0].tolist(), "roll_rad": fr[1], "roll_pixels": fr[2]})
        loop = []
        a = (w.scene.alpha0 + 1.3, w.scene.alpha1 - 0.004)
        for it in range(3):
            m.set_plane(a[0], a[1], w.delta)
            d = m.match(dl, dr)
            a = tuple(sr.sr_fit_alpha(m.ctx, d, pairs, 0.5)["alpha"])
            loop.append({"iteration": it + 1, "alpha": list(a),
                         "err_px": [a[0] - w.scene.alpha0, (a[1] - w.scene.alpha1) * (H - 1)]})
        out["loop_from_perturbed"] = loop
    return out


def accuracy_report(steps: int, warmup: int):
    """Synthetic analogue of the Sec. III sample-model experiment: on the
    1280x720 scene (f = 700 px, baseline 120 mm), for every pothole clear of
    the other depressions and the frame border, fit the road plane to the
    reconstructed 3-D points of a ring around it (4 to 6 sigma), then take
    the distance to that plane of the reconstructed points near its bottom
    (within sigma / 2) as the measured depth.  The same construction on the
    generator's true disparity gives the true depth.  The error is measured
    minus true depth, in mm."""
    import numpy as np
    import torch

    from paper_1807_07433_gb300 import accuracy, sr, synth
    w = synth.C2
    sc = w.scene
    left, right, d_true = synth.make_pair(sc)
    pots, grooves = synth.features(sc)
    H, W = left.shape
    f, B = w.f_px, w.baseline_mm
    u0, v0 = (W - 1) / 2.0, (H - 1) / 2.0
    dev = torch.device("cuda", 0)
    with sr.Matcher(W, H, w.D, w.ncc_r, w.agg_r, w.gamma_d, w.gamma_r, w.lr_thresh,
                    stream=torch.cuda.current_stream(dev)) as m:
        m.set_plane(sc.alpha0, sc.alpha1, w.delta)
        m.set_camera(f, B, u0, v0)
        disp = m.match(torch.from_numpy(left).to(dev), torch.from_numpy(right).to(dev))
        xyz = m.reconstruct(disp).cpu().numpy().astype(np.float64)
    rows = accuracy.pothole_depths(xyz, d_true, sc, pots, grooves, f, B, u0, v0)
    for r in rows:
        for k in ("true_depth_mm", "measured_depth_mm"):
            r[k] = round(r[k], 2)
        for k in ("error_mm_mean", "error_mm_rms"):
            r[k] = round(r[k], 3)
    allerr = np.array([r["error_mm_mean"] for r in rows])
    return {"report": "accuracy", "workload": w.name, "f_px": f, "baseline_mm": B,
            "potholes_used": len(rows), "potholes_in_scene": len(pots),
            "mean_abs_error_mm": round(float(np.abs(allerr).mean()), 3) if len(rows) else None,
            "max_abs_error_mm": round(float(np.abs(allerr).max()), 3) if len(rows) else None,
            "paper_reported_accuracy_mm": 3.0, "rows": rows}


def restricted_report(steps: int, warmup: int):
    """Restricted search (the paper's Sec. IV plan) on the benchmark frame:
    sr_match against sr_match_restricted with (a) the plane hypothesis (every
    pixel centred at round(delta)) and (b) the previous frame's labels (the
    full search's WTA map) as centres; device time per frame (median, CUDA
    events, L2 flushed), label agreement with the full search, and the FP64
    oracle's restricted search on the full frame for (a)."""
    import numpy as np
    import torch

    import oracle
    from paper_1807_07433_gb300 import sr, synth
    w = synth.C2
    left, right, _ = synth.make_pair(w.scene)
    H, W = left.shape
    dev = torch.device("cuda", 0)
    stream = torch.cuda.current_stream(dev)
    dl, dr = torch.from_numpy(left).to(dev), torch.from_numpy(right).to(dev)
    flush = torch.empty(L2_FLUSH_BYTES, dtype=torch.uint8, device=dev)
    out = {"report": "restricted", "workload": w.name, "steps": steps, "warmup": warmup}
    with sr.Matcher(W, H, w.D, w.ncc_r, w.agg_r, w.gamma_d, w.gamma_r, w.lr_thresh,
                    stream=stream) as m:
        m.set_plane(w.scene.alpha0, w.scene.alpha1, w.delta)
        wta_full = torch.empty((H, W), dtype=torch.int16, device=dev)

        def timed(fn):
            for _ in range(warmup):
                fn()
            ms = []
            for _ in range(steps):
                flush.zero_()
                e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
                e0.record(stream)
                r = fn()
                e1.record(stream)
                e1.synchronize()
                ms.append(e0.elapsed_time(e1))
            return r, statistics.median(ms)
        d_full, t_full = timed(lambda: m.match(dl, dr, wta=wta_full))
        d_full = d_full.cpu().numpy()
        lbl_full = wta_full.cpu().numpy()
        out["full"] = {"ms": round(t_full, 4), "mdes": round(mdes(W, H, w.D, t_full * 1e-3), 1),
                       "valid_fraction": round(float(np.isfinite(d_full).mean()), 4)}
        forms = {"plane_r4": (None, 4), "previous_labels_r3": (wta_full.clone(), 3),
                 "previous_labels_r2": (wta_full.clone(), 2)}
        for name, (centre, r) in forms.items():
            wta = torch.empty((H, W), dtype=torch.int16, device=dev)
            d, t = timed(lambda: m.match_restricted(dl, dr, r, centre=centre, wta=wta))
            d = d.cpu().numpy()
            lbl = wta.cpu().numpy()
            both = np.isfinite(d) & np.isfinite(d_full)
            out[name] = {"ms": round(t, 4),
                         "mdes_equivalent": round(mdes(W, H, w.D, t * 1e-3), 1),
                         "speedup_vs_full": round(t_full / t, 3),
                         "label_agreement_with_full": round(float((lbl == lbl_full).mean()), 5),
                         "valid_fraction": round(float(np.isfinite(d).mean()), 4),
                         "dfull_max_abs_diff_where_both_valid_px":
                             float(np.abs(d[both] - d_full[both]).max())}
            if name == "plane_r4":
                p = oracle.Params(W=W, H=H, D=w.D, ncc_r=w.ncc_r, agg_r=w.agg_r,
                                  gamma_d=w.gamma_d, gamma_r=w.gamma_r, lr_thresh=w.lr_thresh,
                                  alpha0=w.scene.alpha0, alpha1=w.scene.alpha1, delta=w.delta)
                t0 = time.perf_counter()
                o = oracle.match(p, left, right, want=("lbl_l", "gap_l"),
                                 centre=np.full((H, W), int(round(w.delta))), radius=r)
                diff = lbl != o.lbl_l
                out[name]["oracle"] = {
                    "label_mismatch_pct": round(100.0 * diff.mean(), 4),
                    "label_mismatch_outside_gap_1e-4_pct":
                        round(100.0 * (diff & (o.gap_l >= 1e-4)).mean(), 4),
                    "oracle_s": round(time.perf_counter() - t0, 2)}
    return out


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=50)
    ap.add_argument("--warmup", type=int, default=5)
    ap.add_argument("--impl", choices=("ours", "reference"), default="ours")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-forms", action="store_true",
                    help="skip the FP16/BF16 and batched forms of the default line")
    ap.add_argument("--volume", choices=("f32", "f16", "bf16"), default="f32",
                    help="storage type of the cost volumes of the main line (arithmetic stays FP32)")
    ap.add_argument("--form-steps", type=int, default=200,
                    help="timed steps of each extra form (default 200)")
    ap.add_argument("--report", choices=("precision", "batch", "adjoint", "sweep", "fit", "accuracy",
                                                "restricted"), default=None,
                    help="print a report instead of the benchmark line")
    args = ap.parse_args()
    if args.warmup < 3:
        ap.error("--warmup must be >= 3")
    if args.report == "precision":
        print(json.dumps(precision_report(args.steps, args.warmup)), flush=True)
        return
    if args.report == "batch":
        print(json.dumps(batch_report(args.steps, args.warmup)), flush=True)
        return
    if args.report == "adjoint":
        print(json.dumps(adjoint_report(args.steps, args.warmup)), flush=True)
        return
    if args.report == "sweep":
        print(json.dumps(sweep_report(args.steps, args.warmup)), flush=True)
        return
    if args.report == "fit":
        print(json.dumps(fit_report(args.steps, args.warmup)), flush=True)
        return
    if args.report == "accuracy":
        print(json.dumps(accuracy_report(args.steps, args.warmup)), flush=True)
        return
    if args.report == "restricted":
        print(json.dumps(restricted_report(args.steps, args.warmup)), flush=True)
        return
    from paper_1807_07433_gb300 import synth
    w = synth.C2

    if args.impl == "reference":
        line = run_reference(args, w)
        if line is not None:
            print(json.dumps(line), flush=True)
        return

    from paper_1807_07433_gb300 import sr
    if not os.path.exists(sr.LIB_PATH):
        import __graft_entry__
        __graft_entry__.build()
    ws_env, _, _ = _dist()
    batch_data = None
    if ws_env == 1 and not args.no_forms:
        # the 64 pairs of the batched form, rendered before any CUDA call
        batch_data = _gen_pairs_spawn([x.scene for x in synth.batch_workloads()])
    line = run_ours(args, w)
    if line is None:
        return
    ws = line["n_gpus"]
    if ws == 1 and not args.no_forms:
        import torch
        dev = torch.device("cuda", 0)
        with NvmlSampler(0) as clk:
            line["forms_720p"] = forms_720p(w, args.form_steps, 10, dev)
            line["forms_batch"] = forms_batch(args.form_steps, 3, dev, batch_data)
        line["forms_clocks"] = clk.summary()
        line["forms_note"] = (f"{args.form_steps} timed steps per form (median, mean, p10, p90 "
                              "of per-step CUDA-event times, L2 flushed between steps); "
                              "faster_beyond_spread: the form's p90 below the base form's p10")
    if ws == 1 and not args.no_cpu_baseline:
        proto = cpu_baseline_protocol(w)
        c2 = proto["c2_all_cores"]
        line["cpu_baseline"] = {
            "value": c2["value"], "unit": UNIT, "cores": c2["cores"], "kind": "oracle",
            "sample": f"output rows {c2['rows'][0]}..{c2['rows'][1] - 1} of the same frame, "
                      f"repeated for {c2['seconds']:.1f} s, FP64 oracle with OpenMP",
            "protocol": proto}
    print(json.dumps(line), flush=True)


if __name__ == "__main__":
    main()
