"""Stereo-2K frame-rate benchmark of the structured-3DGS frame path on one B300.

Workload: the synthetic city (2M anchors, 6 LOD levels, feature 32, k=10,
hidden 32) along the 300-frame ascending stereo path, 1920x1080 per eye.
A step is one stereo frame (both eyes) through the whole path: culling,
derivation, projection, key generation, two radix sorts, blending.

    python bench.py [--gpus N] [--steps K] [--warmup W] [--form plain|unified]
                    [--impl ours|reference]

Prints one JSON line.  `value` is frames per second over all ranks (frames
are independent; ranks render replicas of the path).  Each frame is timed
with CUDA events on the rendering stream; a >L2 buffer is written between
frames (untimed) so every frame starts with a cold L2.  The reference arm
(--impl reference) times the CPU float64 oracle on a bounded sample.
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

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "stereo-2K FPS & ms/frame at >=40dB PSNR vs FP64 oracle; plain vs cached+BF16"
UNIT = "frames/s"
WORKLOAD = "city 2M anchors, stereo 1920x1080, 300-frame ascending path"


def peaks():
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
            d = json.load(f)
        return {"hbm_gbs": d["hbm_gbs"], "bf16_tflops": d["bf16_tflops"], "src": "measured"}
    except Exception:
        return {"hbm_gbs": 6400.0, "bf16_tflops": 1800.0, "src": "fallback"}


class _CtypesNvml:
    """The few read-only NVML queries the clock sampler makes, through the
    driver's libnvidia-ml (for hosts without the Python NVML binding)."""
    NVML_CLOCK_SM = 1

    def __init__(self):
        import ctypes
        self.C = ctypes
        self.lib = ctypes.CDLL("libnvidia-ml.so.1")

    def _ok(self, r):
        if r != 0:
            raise RuntimeError(f"NVML error {r}")

    def nvmlInit(self):
        self._ok(self.lib.nvmlInit_v2())

    def nvmlDeviceGetHandleByUUID(self, uuid):
        h = self.C.c_void_p()
        self._ok(self.lib.nvmlDeviceGetHandleByUUID(self.C.c_char_p(uuid.encode()), self.C.byref(h)))
        return h

    def nvmlDeviceGetHandleByIndex(self, i):
        h = self.C.c_void_p()
        self._ok(self.lib.nvmlDeviceGetHandleByIndex_v2(self.C.c_uint(i), self.C.byref(h)))
        return h

    def _clock(self, fn, h, kind):
        v = self.C.c_uint()
        self._ok(fn(h, self.C.c_int(kind), self.C.byref(v)))
        return v.value

    def nvmlDeviceGetClockInfo(self, h, kind):
        return self._clock(self.lib.nvmlDeviceGetClockInfo, h, kind)

    def nvmlDeviceGetMaxClockInfo(self, h, kind):
        return self._clock(self.lib.nvmlDeviceGetMaxClockInfo, h, kind)

    def nvmlDeviceGetCurrentClocksEventReasons(self, h):
        v = self.C.c_ulonglong()
        fn = getattr(self.lib, "nvmlDeviceGetCurrentClocksEventReasons", None) or \
            self.lib.nvmlDeviceGetCurrentClocksThrottleReasons
        self._ok(fn(h, self.C.byref(v)))
        return v.value


def _nvml_open(uuid: str, index: int):
    """(nvml module, device handle): the Python NVML binding, else the
    driver's libnvidia-ml through its C API."""
    try:
        import pynvml
    except ImportError:
        pynvml = _CtypesNvml()
    pynvml.nvmlInit()
    try:
        return pynvml, pynvml.nvmlDeviceGetHandleByUUID(uuid)
    except Exception:
        return pynvml, pynvml.nvmlDeviceGetHandleByIndex(index)


def clock_sampler_main(uuid: str, index: int, period_ms: float) -> None:
    """Child process of ClockSampler: prints "ready", then one line per
    sample (SM MHz, max SM MHz, clock-event reason bits) every period_ms
    until its standard input closes.  Reads only; nothing is set."""
    nv, h = _nvml_open(uuid, index)
    mx = float(nv.nvmlDeviceGetMaxClockInfo(h, nv.NVML_CLOCK_SM))
    stop = threading.Event()

    def wait_eof():
        sys.stdin.read()
        stop.set()

    threading.Thread(target=wait_eof, daemon=True).start()
    print("ready", flush=True)
    while True:
        sm = float(nv.nvmlDeviceGetClockInfo(h, nv.NVML_CLOCK_SM))
        bits = int(nv.nvmlDeviceGetCurrentClocksEventReasons(h))
        print(f"{sm} {mx} {bits}", flush=True)
        if stop.wait(period_ms / 1e3):
            break


class ClockSampler:
    """SM clocks and clock-event (throttle) reasons sampled during the timed
    region by a separate process (NVML every 5 ms), so the sampling never
    competes with the timed loop for the interpreter; an nvidia-smi loop if
    NVML is missing.  Reads only; nothing is set.  NVML queries still slow
    the host's CUDA calls (at a 1 ms period the timed loop's host submission
    fell from ~1750 to ~340 frames/s), so the period trades samples against
    the host's pace; the bench reports the loop's wall rate with and without
    the sampler."""
    Q = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
         "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
         "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")
    NVML_BITS = (("hw_slowdown", 0x8), ("hw_thermal_slowdown", 0x40), ("sw_thermal_slowdown", 0x20),
                 ("sw_power_cap", 0x4))

    def __init__(self, device_index: int, period_ms: float = 5.0):
        self.idx = device_index
        self.period_ms = period_ms
        self.proc = None
        self.kind = None
        self.rows = []

    def __enter__(self):
        import torch
        uuid = str(torch.cuda.get_device_properties(self.idx).uuid)
        uuid = uuid if uuid.startswith("GPU-") else "GPU-" + uuid
        try:
            self.proc = subprocess.Popen([sys.executable, os.path.abspath(__file__), "--clock-sampler", uuid,
                                          str(self.idx), str(self.period_ms)],
                                         stdin=subprocess.PIPE, stdout=subprocess.PIPE, stderr=subprocess.DEVNULL,
                                         text=True)
            if self.proc.stdout.readline().strip() == "ready":
                self.kind = "nvml"
                return self
            self.proc.kill()
            self.proc.wait()
        except Exception:
            pass
        try:
            self.proc = subprocess.Popen(["nvidia-smi", f"--id={self.idx}", f"--query-gpu={self.Q}",
                                          "--format=csv,noheader,nounits", "-lms", "100"],
                                         stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
            self.kind = "smi"
        except Exception:
            self.proc = None
        return self

    def __exit__(self, *a):
        if not self.proc:
            return
        try:
            if self.kind == "nvml":
                self.proc.stdin.close()
                out = self.proc.stdout.read()
                self.proc.wait(timeout=10)
                for line in out.splitlines():
                    p = line.split()
                    if len(p) == 3:
                        self.rows.append((float(p[0]), float(p[1]), int(p[2])))
            else:
                self.proc.terminate()
                out = self.proc.stdout.read()
                self.proc.wait(timeout=10)
                self.rows = [[x.strip() for x in line.split(",")] for line in out.splitlines()]
        except Exception:
            self.proc.kill()

    def summary(self):
        if not self.rows:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["unavailable"], "samples": 0}
        if self.kind == "nvml":
            reasons = sorted({n for r in self.rows for n, b in self.NVML_BITS if r[2] & b})
            return {"sm_mhz": statistics.median(r[0] for r in self.rows), "sm_max_mhz": self.rows[0][1],
                    "reasons": reasons, "samples": len(self.rows), "source": "nvml, separate process"}
        sm = [float(r[1]) for r in self.rows if len(r) > 2 and r[1].replace(".", "").isdigit()]
        mx = [float(r[2]) for r in self.rows if len(r) > 2 and r[2].replace(".", "").isdigit()]
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        reasons = set()
        for r in self.rows:
            for i, n in enumerate(names):
                if len(r) > 5 + i and r[5 + i].lower().startswith("active"):
                    reasons.add(n)
        return {"sm_mhz": statistics.median(sm) if sm else None, "sm_max_mhz": max(mx) if mx else None,
                "reasons": sorted(reasons), "samples": len(self.rows), "source": "nvidia-smi"}


def build_workload(n_frames=300):
    import gen
    t0 = time.time()
    model, frames = gen.city_workload(n_frames=n_frames)
    return model, frames, time.time() - t0


# ---------------------------------------------------------------- reference arm (CPU oracle)
def cpu_info() -> dict:
    """The host's CPU model and the cores this process may run on."""
    name = None
    try:
        with open("/proc/cpuinfo") as f:
            for line in f:
                if line.startswith("model name"):
                    name = line.split(":", 1)[1].strip()
                    break
    except OSError:
        pass
    try:
        nproc = len(os.sched_getaffinity(0))
    except AttributeError:
        nproc = os.cpu_count()
    return {"cpu_model": name, "nproc": nproc}


def oracle_frame(model, L, R):
    """One stereo frame through the float64 oracle: filtering, derivation,
    projection and tiled blending of every pixel of both eyes.  Returns
    (seconds, [(rgb, T, margin, contributors) of each eye])."""
    import oracle
    t0 = time.perf_counter()
    outs = [oracle.render_view(model, cam)[0] for cam in (L, R)]
    return time.perf_counter() - t0, outs


def oracle_one_thread(model, L, R) -> float:
    """Seconds of one stereo oracle frame on a single thread."""
    import oracle
    n = oracle.num_threads()
    oracle.set_threads(1)
    try:
        return oracle_frame(model, L, R)[0]
    finally:
        oracle.set_threads(n)


def max_over_ranks(x: float, world: int) -> float:
    """The largest x over all ranks (the slowest rank's time); x itself on one rank."""
    if world <= 1:
        return x
    import torch
    import torch.distributed as dist
    dev = "cuda" if dist.get_backend() == "nccl" else "cpu"
    t = torch.tensor([x], dtype=torch.float64, device=dev)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def job_rate(world: int, steps: int, total_ms: float) -> float:
    """Frames per second of the whole job: every rank renders `steps` frames
    (weak scaling, independent replicas) within the slowest rank's time."""
    return world * steps / (total_ms / 1e3)


def run_reference(args, rank, world):
    """The CPU float64 oracle as it stands on the host's cores: each step is
    one whole stereo frame of the path (every 10th frame: step s renders
    frame 10 s mod 300), warm-up steps the frames halfway between."""
    if rank != 0:
        return
    import oracle
    oracle.build()
    model, frames, _ = build_workload()
    n = len(frames)
    for w in range(args.warmup):
        oracle_frame(model, *frames[(10 * w + 5) % n])
    ts = [oracle_frame(model, *frames[(10 * s) % n])[0] for s in range(args.steps)]
    t1 = oracle_one_thread(model, *frames[150])
    mean = float(np.mean(ts))
    cores = oracle.num_threads()
    info = cpu_info()
    sample = (f"per step one whole stereo frame (both eyes, every pixel) of the path, frames 0, 10, 20, ... in "
              f"float64 on {cores} threads; one frame (150) also on 1 thread")
    line = {"impl": "reference", "metric": METRIC, "value": 1.0 / mean, "unit": UNIT, "n_gpus": world,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": mean * 1e3, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
            "config": {"workload": WORKLOAD, "form": "CPU float64 oracle (plain method)", "l2": "n/a (CPU)",
                       "p99_ms": float(np.percentile(ts, 99)) * 1e3, **info},
            "cpu_baseline": {"value": 1.0 / mean, "unit": UNIT, "cores": cores, "kind": "oracle", "sample": sample,
                             "value_1thread": 1.0 / t1, **info},
            "e2e": {"value": 1.0 / mean, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)


# ---------------------------------------------------------------- our arm
# Forms of the frame path: the plain float32 method and the AI-systems forms.
FORMS = {
    "plain": dict(precision="fp32", stereo_unify=False, reuse="off"),
    "unified": dict(precision="fp32", stereo_unify=True, reuse="off"),
    "bf16": dict(precision="bf16", stereo_unify=False, reuse="off"),
    "cached_bf16": dict(precision="bf16", stereo_unify=False, reuse="depth"),
    "bf16_unified": dict(precision="bf16", stereo_unify=True, reuse="off"),
    "cached_unified": dict(precision="fp32", stereo_unify=True, reuse="depth"),
    "cached_bf16_unified": dict(precision="bf16", stereo_unify=True, reuse="depth"),
    "fp8": dict(precision="fp8", stereo_unify=False, reuse="off"),
    "fp8_unified": dict(precision="fp8", stereo_unify=True, reuse="off"),
    "cached_fp8_unified": dict(precision="fp8", stereo_unify=True, reuse="depth"),
    # exact stereo form: each eye filters its own anchors, the union is derived once
    "exact": dict(precision="fp32", stereo_unify="exact", reuse="off"),
    "bf16_exact": dict(precision="bf16", stereo_unify="exact", reuse="off"),
    "cached_exact": dict(precision="fp32", stereo_unify="exact", reuse="depth"),
    "cached_bf16_exact": dict(precision="bf16", stereo_unify="exact", reuse="depth"),
    "fp8_exact": dict(precision="fp8", stereo_unify="exact", reuse="off"),
    "cached_fp8_exact": dict(precision="fp8", stereo_unify="exact", reuse="depth"),
}
HEADLINE = "cached_bf16_exact"
FP32_LANE_OPS = 148 * 128 * 2.032e9  # SMs x FP32 lanes x max SM clock: FP32 lane operations / s
# Algorithmic work of one (pixel, Gaussian) evaluation of the blend: ~20 FP32
# operations (offset, quadratic form, opacity product and clamp, the two
# thresholds, T update, colour accumulation) and one exponential
OPS_PER_EVAL = 20
# DRAM bytes (read + write) of one launch of a kernel from one ncu capture,
# with the tiling and the frame it was taken on and the SHA-256 prefix of the
# kernel's source file's code at the time (comments left out): reported as
# the roofline's traffic only while that code is unchanged and the timed run
# uses that tiling, else null.
NCU_TRAFFIC = {"k_blend": {"file": "paper_2502_14938_b300/csrc/raster.cu", "sha16": "5eee264595caa890",
                           "tiling": (16, 64, 0), "bytes": 17438208 + 2180096, "frame": 21}}


def _src_sha16(rel: str) -> str:
    """SHA-256 prefix of a source file's code: line comments, trailing blanks
    and empty lines removed, so that an edited comment keeps a capture while
    any change to the code drops it."""
    import hashlib
    with open(os.path.join(ROOT, rel), "rb") as f:
        lines = []
        for line in f.read().decode().splitlines():
            i = line.find("//")
            line = (line[:i] if i >= 0 else line).rstrip()
            if line:
                lines.append(line)
    return hashlib.sha256("\n".join(lines).encode()).hexdigest()[:16]


def ncu_traffic(kernel: str, tiling_key):
    c = NCU_TRAFFIC.get(kernel)
    if not c or c["bytes"] is None or tuple(c["tiling"]) != tuple(tiling_key) or _src_sha16(c["file"]) != c["sha16"]:
        return None, "no capture of the current kernel source at this tiling"
    return c["bytes"], f"ncu dram bytes of one launch, frame {c['frame']}, tiles {tuple(c['tiling'])}"


# The blend's algorithmic work is counted on the paper's rasteriser tiling
# (16x16 tiles, one block per tile), so it does not depend on the tuned shape
WORK_TILING = (16, 16, 0)


def make_renderer(model, form, flags=0, use_graph=True):
    import paper_2502_14938_b300 as pkg
    r = pkg.Renderer(max_views=2, flags=flags, use_graph=use_graph, **FORMS[form])
    mid = r.load_model(model)
    return r, mid


def set_pair(r, mid, L, R):
    import paper_2502_14938_b300 as pkg
    r.set_cameras([pkg.to_camera(L, partner=1, model_id=mid), pkg.to_camera(R, partner=0, model_id=mid)])


# Synthetic ablation in the manner of the paper's Tables 5-6: the headline
# form with one optimisation removed at a time; "w/o fused kernels" runs the
# FP32 decoder as separate operators through device memory (GSC_FLAG_UNFUSED,
# the counterpart of the paper's operator-by-operator pipeline) and compares
# with the fused FP32 row above it.
ABLATION = (("full: cached + BF16 + shared stereo derivation", "cached_bf16_exact", 0),
            ("w/o de-redundancy (per-eye derivation)", "cached_bf16", 0),
            ("w/o reuse", "bf16_exact", 0),
            ("w/o BF16 (FP32 MLPs)", "cached_exact", 0),
            ("w/o fused kernels (FP32 decoder as separate operators)", "cached_exact", 0x20),
            ("none: plain FP32, per eye, no cache", "plain", 0))


def run_ablation(args):
    """AVG and 1%-low FPS, decoding / rasterisation stage times, device
    memory of each ablated form on the timed frames of the path, at one tiling."""
    import torch
    model, frames, t_gen = build_workload()
    flush = torch.empty(256 << 20, dtype=torch.uint8, device="cuda")
    tiling = tuple(args.tile)
    rows = []
    for name, form, flags in ABLATION:
        torch.cuda.synchronize()
        free0, res0 = torch.cuda.mem_get_info()[0], torch.cuda.memory_reserved()
        r, mid, outs, ms, wall = time_form(model, frames, form, args.steps, args.warmup, flush, 1, tiling=tiling,
                                           flags=flags)
        torch.cuda.synchronize()
        lib_bytes = (free0 - torch.cuda.mem_get_info()[0]) - (torch.cuda.memory_reserved() - res0)
        r.close()
        stage, _ = stage_profile(model, frames, form, min(args.steps, len(frames)), flush,
                                 {"tile_w": tiling[0], "tile_h": tiling[1], "blocks_per_sm": tiling[2]}, count=False,
                                 flags=flags)
        dec = stage["cull+plan"] + stage["derive+project"]
        mean, p99 = float(np.mean(ms)), float(np.percentile(ms, 99))
        rows.append({"method": name, "form": form, "unfused": bool(flags & 0x20), "avg_fps": 1e3 / mean, "fps_1pct_low": 1e3 / p99,
                     "ms_mean": mean, "decoding_ms": dec, "rasterization_ms": sum(stage.values()) - dec,
                     "device_gib": lib_bytes / 2 ** 30})
    for row in rows:
        row["speedup_loss"] = rows[0]["avg_fps"] / row["avg_fps"]
    print(json.dumps({"ablation": rows, "workload": "city 2M anchors, stereo 1920x1080, 300-frame ascending path",
                      "steps": args.steps, "warmup": args.warmup, "tiling": list(tiling),
                      "stages": "decoding = culling, cache, tables, derivation and projection; rasterisation = "
                                "sorts, pair offsets, key generation, ranges, blend (eager CUDA events)",
                      "memory": "device memory the library allocated (free-memory drop minus torch's own)"}),
          flush=True)


def run_octree(args):
    """Octree-GS level selection (per-anchor level offsets and the level
    fade) against the plain distance rule on the same city model: frames/s,
    the culling stage and visible anchors, and each form's PSNR against the
    float64 oracle of the octree model (frames rendered in path order)."""
    import torch
    import gen
    import oracle
    model, frames, t_gen = build_workload()
    sigma, beta = 0.5, 0.5
    octree = gen.with_level_offsets(model, sigma=sigma, beta=beta)
    flush = torch.empty(256 << 20, dtype=torch.uint8, device="cuda")
    tiling = tuple(args.tile)
    tl = {"tile_w": tiling[0], "tile_h": tiling[1], "blocks_per_sm": tiling[2]}
    refs = {f: [oracle.render_view(octree, cam)[0][0] for cam in frames[f]] for f in args.psnr_frames}
    rows = []
    for name, m in (("distance LOD (plain rule)", model), ("Octree-GS offsets + fade", octree)):
        for form in (HEADLINE, "plain"):
            r, mid, outs, ms, wall = time_form(m, frames, form, args.steps, args.warmup, flush, 1, tiling=tiling)
            row = {"model": name, "form": form, "fps": 1e3 / float(ms.mean()), "ms_mean": float(ms.mean()),
                   "p99_ms": float(np.percentile(ms, 99))}
            if m is octree:
                row["quality_vs_octree_oracle"], _ = form_quality(r, mid, outs, frames, refs)
            r.close()
            stage, per_frame = stage_profile(m, frames, form, min(args.steps, len(frames)), flush, tl, count=False)
            row["cull+plan_ms"] = stage["cull+plan"]
            row["derive+project_ms"] = stage["derive+project"]
            row["visible_anchors"] = per_frame["visible_anchors"]
            rows.append(row)
    print(json.dumps({"octree": rows, "workload": "city 2M anchors, stereo 1920x1080, 300-frame ascending path",
                      "level_offsets": f"N(0, {sigma}^2) clipped to 3 sigma (synthetic: no trained offsets)",
                      "lod_blend_levels": beta, "steps": args.steps, "warmup": args.warmup, "tiling": list(tiling),
                      "psnr_frames": sorted(refs)}), flush=True)


def run_guides(args):
    """Eq. 4 guiding functions on an accelerating camera: the ascending city
    path with frame k taken at path index k^2 / 30 (speed growing linearly),
    cached BF16 unified form with each guide; per frame the reuse depth
    chosen, the update rate (misses / visible), the device time and the PSNR
    against the same form without the cache."""
    import torch
    import paper_2502_14938_b300 as pkg
    model, frames, _ = build_workload()
    path = [frames[min(len(frames) - 1, k * k // 30)] for k in range(95)]
    W, H = path[0][0].width, path[0][0].height
    ref_r, ref_mid = make_renderer(model, "bf16_unified")
    ref_r.set_tiling(*args.tile)
    ref = [torch.empty((H, W, 3), dtype=torch.float32, device="cuda") for _ in range(2)]
    outs = [torch.empty((H, W, 3), dtype=torch.float32, device="cuda") for _ in range(2)]
    res = {}
    for guide in ("linear", "exp", "staged"):
        r = pkg.Renderer(max_views=2, depth_guide=guide, **FORMS[HEADLINE])
        mid = r.load_model(model)
        r.set_tiling(*args.tile)
        for fr in path:  # grow the buffers, then start from an empty cache
            set_pair(r, mid, *fr)
            r.render_frame(outs)
        r.cache_reset()
        depth, rate, psnr, ms = [], [], [], []
        for fr in path:
            set_pair(r, mid, *fr)
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            e0.record()
            st = r.render_frame(outs)
            e1.record()
            set_pair(ref_r, ref_mid, *fr)
            ref_r.render_frame(ref, stats=False)
            torch.cuda.synchronize()
            ms.append(e0.elapsed_time(e1))
            depth.append(int(st["cache_depth"]))
            rate.append(st["derived_anchors"] / max(1, st["visible_anchors"]))
            mse = max(float(sum(torch.mean((o - q) ** 2) for o, q in zip(outs, ref)) / 2), 1e-10)
            psnr.append(10.0 * np.log10(1.0 / mse))
        r.close()
        res[guide] = {"psnr_db_min": min(psnr), "psnr_db_mean": float(np.mean(psnr)),
                      "update_rate_mean": float(np.mean(rate)), "depth_mean": float(np.mean(depth)),
                      "ms_mean_with_stats": float(np.mean(ms)), "depth": depth,
                      "update_rate": [round(x, 4) for x in rate], "psnr_db": [round(x, 2) for x in psnr]}
    ref_r.close()
    print(json.dumps({"guides": res, "path": "city ascending path, frame k at index k^2/30 (95 frames)",
                      "form": HEADLINE, "tiling": list(args.tile),
                      "psnr": "against the same form without the cache, whole images"}), flush=True)


def run_sched(args):
    """Frames displayed per second by the single-host elastic schedule
    (paper_2502_14938_b300.sched, Alg. 2) with 1-4 fixed workers, each a
    context of its own on its own stream, rendering the city path's stereo
    frames (headline form, device images, one synchronize per frame) from a
    queue that is never empty."""
    import torch
    import paper_2502_14938_b300 as pkg
    from paper_2502_14938_b300.sched import CameraQueue, DisplaySink, ElasticPool
    model, frames, _ = build_workload()
    W, H = frames[0][0].width, frames[0][0].height

    ready = []

    def make(wid):
        r = pkg.Renderer(max_views=2, **FORMS[HEADLINE])
        mid = r.load_model(model)
        r.set_tiling(*args.tile)
        outs = [torch.empty((H, W, 3), dtype=torch.float32, device="cuda") for _ in range(2)]
        for fr in frames[:40]:
            set_pair(r, mid, *fr)
            r.render_frame(outs)
        r.synchronize()
        ready.append(wid)

        def render(fr):
            set_pair(r, mid, *fr)
            r.render_frame(outs, stats=False)
            r.synchronize()
        return render

    res = {}
    n_frames = max(400, 20 * args.steps)
    for n in (1, 2, 3, 4):
        q, sink = CameraQueue(timeout_s=60.0), DisplaySink()
        ready.clear()
        pool = ElasticPool(make, q, sink, min_fps=1, max_fps=1e12, max_workers=n, start_workers=n,
                           window_s=10.0, period_s=1.0)
        while len(ready) < n and pool.failed == 0:  # workers load the model and warm up
            time.sleep(0.01)
        t0 = time.monotonic()
        for k in range(n_frames):
            q.put(frames[k % len(frames)])
        while len(q) > 0 or len(sink.written) + sink.discarded < n_frames:
            time.sleep(0.002)
        dt = time.monotonic() - t0
        pool.close()
        res[str(n)] = {"frames_per_s": len(sink.written) / dt, "discarded": sink.discarded, "failed": pool.failed}
    print(json.dumps({"sched_workers": res, "form": HEADLINE, "tiling": list(args.tile), "frames": n_frames,
                      "note": "device images; the queue is filled at once, so no camera times out"}), flush=True)


def run_profile(args):
    """Minimal run for profilers: W + K frames from --frame, no extras, with
    the tiling of --tile (launches per frame: launches_per_frame_of); with
    --octree the model carries the synthetic Octree-GS level offsets and fade
    of run_octree."""
    import torch
    model, frames, _ = build_workload()
    if args.octree:
        import gen
        model = gen.with_level_offsets(model, sigma=0.5, beta=0.5)
    W, H = frames[0][0].width, frames[0][0].height
    r, mid = make_renderer(model, args.form)
    outs = [torch.empty((H, W, 3), dtype=torch.float32, device="cuda") for _ in range(2)]
    set_pair(r, mid, *frames[args.frame % len(frames)])
    r.set_tiling(*args.tile)
    for s in range(args.warmup + args.steps):
        set_pair(r, mid, *frames[(args.frame + s) % len(frames)])
        st = r.render_frame(outs)
    torch.cuda.synchronize()
    print(json.dumps({"profile_run": True, "form": args.form, "octree": bool(args.octree),
                      "frames": args.warmup + args.steps, "last": st}),
          flush=True)


def time_form(model, frames, form, steps, warmup, flush, world, clk=None, tune=False, tiling=None, flags=0):
    """Per-frame CUDA-event times (ms) of `steps` frames of the path; L2 flushed between frames.
    tune: pick the blend tiling (tile shape, blocks/SM) with the project's autotuner on the
    middle frame of the path first; tiling: a fixed (W, H, blocks/SM) instead."""
    import torch
    W, H = frames[0][0].width, frames[0][0].height
    r, mid = make_renderer(model, form, flags=flags)
    outs = [torch.empty((H, W, 3), dtype=torch.float32, device="cuda") for _ in range(2)]
    for f in range(len(frames)):  # one pass over the path with stats grows buffers to its needs
        set_pair(r, mid, *frames[f])
        r.render_frame(outs)
    r.tiling = {"tile_w": 16, "tile_h": 16, "blocks_per_sm": 0, "source": "default"}
    if tiling is not None:
        r.set_tiling(*tiling)
        r.tiling = {"tile_w": tiling[0], "tile_h": tiling[1], "blocks_per_sm": tiling[2], "source": "fixed"}
        for f in range(len(frames)):  # regrow for the tiling
            set_pair(r, mid, *frames[f])
            r.render_frame(outs)
    elif tune:
        from paper_2502_14938_b300 import autotune
        picks = [frames[i] for i in np.linspace(0, len(frames) - 1, 6).astype(int)]
        setups = [lambda fr=fr: set_pair(r, mid, *fr) for fr in picks]
        best = autotune.tune(r, outs, None, reps=5, setups=setups)
        r.tiling = {k: best[k] for k in ("tile_w", "tile_h", "blocks_per_sm", "source")}
        for f in range(len(frames)):  # regrow for the chosen tiling
            set_pair(r, mid, *frames[f])
            r.render_frame(outs)
    for w in range(warmup):
        set_pair(r, mid, *frames[w % len(frames)])
        r.render_frame(outs, stats=False)
    r.synchronize()
    r.cache_reset()  # reuse forms: the timed run starts at frame 0 with an empty cache
    stream = torch.cuda.current_stream()
    evs = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(steps)]
    if world > 1:
        torch.distributed.barrier()
    torch.cuda.synchronize()
    if clk:
        clk.__enter__()
    wall0 = time.perf_counter()
    for s in range(steps):
        set_pair(r, mid, *frames[s % len(frames)])
        flush.fill_(s & 0xFF)
        evs[s][0].record(stream)
        r.render_frame(outs, stats=False)
        evs[s][1].record(stream)
    torch.cuda.synchronize()
    if world > 1:
        torch.distributed.barrier()
    wall = time.perf_counter() - wall0
    if clk:
        clk.__exit__()
    r.synchronize()  # raises on a deferred capacity / timeout error
    ms = np.array([a.elapsed_time(b) for a, b in evs])
    if clk:  # the same loop again without the clock sampler running (host-side cost of sampling)
        r.cache_reset()
        torch.cuda.synchronize()
        w0 = time.perf_counter()
        for s in range(steps):
            set_pair(r, mid, *frames[s % len(frames)])
            flush.fill_(s & 0xFF)
            r.render_frame(outs, stats=False)
        torch.cuda.synchronize()
        clk.wall_unsampled = time.perf_counter() - w0
        w0 = time.perf_counter()  # and the host's own cost of a step without the device (cameras only)
        for s in range(steps):
            set_pair(r, mid, *frames[s % len(frames)])
        clk.host_set_cameras = time.perf_counter() - w0
        r.synchronize()
    return r, mid, outs, ms, wall


# eager stage events of the library (GSC_FLAG_TIMING)
STAGE_NAMES = ["cull+plan", "derive+project", "sort_depth", "scan+keygen", "sort_tile", "ranges", "blend"]


def stage_profile(model, frames, form, n, flush, tiling=None, count=True, flags=0):
    """Per-stage CUDA-event times on the library's stream (eager launches), with the timed run's tiling."""
    import paper_2502_14938_b300 as pkg
    import torch
    W, H = frames[0][0].width, frames[0][0].height
    rt, mid = make_renderer(model, form, flags=pkg.FLAG_TIMING | flags, use_graph=False)
    set_pair(rt, mid, *frames[0])
    if tiling:
        rt.set_tiling(tiling["tile_w"], tiling["tile_h"], tiling["blocks_per_sm"])
    outs = [torch.empty((H, W, 3), dtype=torch.float32, device="cuda") for _ in range(2)]
    stage = np.zeros(8)
    acc = {"visible_anchors": 0, "derived_anchors": 0, "records": 0, "valid_records": 0, "pairs": 0}
    stage_rows = []
    for s in range(n):
        set_pair(rt, mid, *frames[s % len(frames)])
        flush.fill_(s & 0xFF)
        st = rt.render_frame(outs)
        stage += np.array(st["ms_stage"])
        stage_rows.append([float(x) for x in st["ms_stage"][:7]])
        for k in acc:
            acc[k] += st[k]
    rt.close()
    # the same frames (from an empty cache) through the blend's counting
    # variant: its (pixel, Gaussian) evaluations per frame, on the timed
    # tiling (walk and issued) and on 16x16 tiles (the algorithmic walk)
    acc["blend_walk"] = acc["blend_issued"] = acc["blend_walk16"] = 0
    timed = (tiling["tile_w"], tiling["tile_h"], tiling["blocks_per_sm"]) if tiling else None
    for pass_, t in enumerate((timed, WORK_TILING) if count else ()):
        rw, mid = make_renderer(model, form, flags=pkg.FLAG_BLEND_WORK, use_graph=False)
        if t:
            rw.set_tiling(*t)
        for s in range(n):
            set_pair(rw, mid, *frames[s % len(frames)])
            rw.render_frame(outs, stats=False)
            w, i = rw.debug_blend_work()
            if pass_ == 0:
                acc["blend_walk"] += w
                acc["blend_issued"] += i
            else:
                acc["blend_walk16"] += w
        rw.close()
    names = STAGE_NAMES
    res = {k: v / n for k, v in acc.items()}
    res["stage_rows"] = [dict(zip(names, row)) for row in stage_rows]
    return {nm: float(stage[i] / n) for i, nm in enumerate(names)}, res


def roofline(stage_ms, st, form, W, H, n_anchors, tiling):
    """Dominant stage: algorithmic work per launch / its event time, against a peak."""
    pk = peaks()
    dom = max(stage_ms, key=stage_ms.get)
    P, Rv, R, V = st["pairs"], st["valid_records"], st["records"], st["visible_anchors"]
    pixels = 2 * W * H
    dur = stage_ms[dom] / 1e3
    feat_b = {"fp32": 128, "bf16": 64, "fp8": 32}[FORMS[form]["precision"]]
    if dom == "blend":
        # unit: one (pixel, Gaussian) evaluation of the front-to-back walk
        # over 16x16 tile lists (every Gaussian of the pixel's tile list up
        # to the one it stops at: the paper's rasteriser), counted in the
        # kernel by its counting variant on the same frames; 20 FP32 ops +
        # 1 exp2 each.  On the timed tiling the kernel's own walk and the
        # evaluations it issued (a warp skips records whose box misses its
        # rows) are reported beside it.
        import paper_2502_14938_b300 as pkg
        walk16, walk, ev = st["blend_walk16"], st["blend_walk"], st["blend_issued"]
        ach = walk16 * OPS_PER_EVAL / dur / 1e12
        peak = FP32_LANE_OPS / 1e12
        rates = pkg.native.pipe_rates()
        key = (tiling["tile_w"], tiling["tile_h"], tiling["blocks_per_sm"])
        traffic, traffic_src = ncu_traffic("k_blend", key)
        return {"kernel": "k_blend", "bound": "alu", "achieved": ach, "peak": peak, "unit": "T FP32-op/s",
                "frac": ach / peak,
                "peak_src": "nominal: 148 SMs x 128 FP32 lanes x 2.032 GHz; work = 20 FP32 ops per evaluation "
                            "of the walk over 16x16 tile lists",
                "traffic": traffic, "traffic_src": traffic_src,
                "evals_per_launch": walk16, "walk_evals_timed_tiling": walk, "issued_evals_per_launch": ev,
                "evals_per_s": walk16 / dur, "exp2_frac_of_measured": walk16 / dur / rates["exp2_per_s"],
                "measured_rates": rates, "ms_per_launch": stage_ms[dom],
                "hbm_gbs": (P * 52 + pixels * 12) / dur / 1e9}
    b = stage_bytes(dom, st, form, n_anchors)
    ach = b / dur / 1e9
    return {"kernel": dom, "bound": "hbm", "achieved": ach, "peak": pk["hbm_gbs"], "unit": "GB/s",
            "frac": ach / pk["hbm_gbs"], "peak_src": pk["src"], "traffic": None, "alg_bytes_per_launch": b,
            "ms_per_launch": stage_ms[dom]}


def stage_bytes(stage, st, form, n_anchors):
    """Algorithmic HBM bytes of one frame's stage (each datum read or written once)."""
    P, Rv, R, V = st["pairs"], st["valid_records"], st["records"], st["visible_anchors"]
    feat_b = {"fp32": 128, "bf16": 64, "fp8": 32}[FORMS[form]["precision"]]
    if stage == "sort_tile":      # 2 passes: key + value in and out; tile ranges
        return P * 4 + 2 * P * 16
    if stage == "sort_depth":     # pass 1 reads every record's key, 4 passes move the valid (key, value)
        return R * 8 + Rv * 8 + 3 * Rv * 16
    if stage == "derive+project":  # features + directions + attributes of visible anchors; records out
        return V * (feat_b + 16 + 120) + R * 56
    if stage == "scan+keygen":    # counts and offsets of valid records; pairs out
        return Rv * 16 + P * 8
    if stage == "ranges":
        return P * 4
    if stage == "blend":          # pairs and records of every pair in; the images out
        return P * 52
    return n_anchors * 13 + V * 4  # cull + cache + tables: positions and levels in, visible ids out


def stage_hbm(stage_ms, st, form, W, H, n_anchors):
    """Every stage's algorithmic bytes over its (eagerly timed) duration, against the HBM peak."""
    pk = peaks()
    out = {}
    for s, ms in stage_ms.items():
        b = stage_bytes(s, st, form, n_anchors) + (2 * W * H * 12 if s == "blend" else 0)
        out[s] = {"alg_bytes": b, "gbs": b / (ms / 1e3) / 1e9, "frac": b / (ms / 1e3) / 1e9 / pk["hbm_gbs"]}
    return out


BATCHED_FORM = dict(stereo_unify="exact", precision="bf16", reuse="depth")


def run_batched(args, flush):
    """Batched multi-viewer form: 3 scenes (0.5M / 2M / 4M anchors), 8 viewers,
    13 images (1280x720 mono up to 1920x1080 stereo) rendered as one frame
    (one graph replay), tiling chosen by the autotuner.  Compared with the
    same frame untuned (16x16, one block per tile) and with the 8 viewers
    rendered by 8 separate contexts one after another.  A frame = all 13 images."""
    import torch
    import gen
    import paper_2502_14938_b300 as pkg
    from paper_2502_14938_b300 import autotune
    t0 = time.perf_counter()
    models, viewers, frame_fn = gen.multiviewer_workload()
    t_gen = time.perf_counter() - t0
    n = max(1, min(args.steps, 100))
    frames = [frame_fn(t) for t in range(n)]
    n_img = len(frames[0])
    pixels = sum(c.width * c.height for _, _, c, _ in frames[0])
    outs = [torch.empty((c.height, c.width, 3), dtype=torch.float32, device="cuda") for _, _, c, _ in frames[0]]

    def cams(imgs, mid_of, sel=None):
        """gsc cameras of the images `sel` (all by default); partners renumbered within `sel`."""
        sel = list(range(len(imgs))) if sel is None else sel
        remap = {j: i for i, j in enumerate(sel)}
        return [pkg.to_camera(imgs[j][2], partner=remap.get(imgs[j][3], -1), model_id=mid_of(imgs[j][1]),
                              viewer=imgs[j][0]) for j in sel]

    r = pkg.Renderer(max_views=n_img, **BATCHED_FORM)
    mids = [r.load_model(m) for m in models]
    cam_lists = [cams(f, lambda sc: mids[sc]) for f in frames]

    def timed(setup, render):
        for f in range(n):  # grow buffers (synchronous frames), warm the graph
            setup(f)
            render(True)
        torch.cuda.synchronize()
        for rr in rends:
            rr.cache_reset()
        stream = torch.cuda.current_stream()
        evs = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(n)]
        for f in range(n):
            setup(f)
            flush.fill_(f & 0xFF)
            evs[f][0].record(stream)
            render(False)
            evs[f][1].record(stream)
        torch.cuda.synchronize()
        ms = np.array([a.elapsed_time(b) for a, b in evs])
        return {"fps": 1000.0 / float(ms.mean()), "ms_mean": float(ms.mean()),
                "p99_ms": float(np.percentile(ms, 99)), "images_per_s": n_img * 1000.0 / float(ms.mean()),
                "mpix_per_s": pixels / 1e3 / float(ms.mean())}

    rends = [r]
    r.set_tiling(16, 16, 0)
    untuned = timed(lambda f: r.set_cameras(cam_lists[f]), lambda st: r.render_frame(outs, stats=st))
    r.set_cameras(cam_lists[0])
    t1 = time.perf_counter()
    best = autotune.tune(r, outs, args.tiling_cache, reps=3)
    t_tune = time.perf_counter() - t1
    tuned = timed(lambda f: r.set_cameras(cam_lists[f]), lambda st: r.render_frame(outs, stats=st))
    reuse = []
    for f in range(n):
        r.set_cameras(cam_lists[f])
        st = r.render_frame(outs)
        reuse.append(1.0 - st["derived_anchors"] / max(st["visible_anchors"], 1))

    # the same viewers, one context per viewer, rendered one after another
    sep = []
    for v in range(len(viewers)):
        sel = [i for i, im in enumerate(frames[0]) if im[0] == v]
        rv = pkg.Renderer(max_views=len(sel), **BATCHED_FORM)
        rv.set_tiling(best["tile_w"], best["tile_h"], best["blocks_per_sm"])
        mid = rv.load_model(models[frames[0][sel[0]][1]])
        sep.append((rv, sel, [cams(f, lambda sc, m=mid: m, sel) for f in frames]))
    rends = [x[0] for x in sep]

    def sep_setup(f):
        for rv, sel, cl in sep:
            rv.set_cameras(cl[f])

    def sep_render(st):
        for rv, sel, _ in sep:
            rv.render_frame([outs[i] for i in sel], stats=st)

    separate = timed(sep_setup, sep_render)
    for rv, _, _ in sep:
        rv.close()
    r.close()
    return {"workload": "3 city scenes 0.5M/2M/4M anchors, 8 viewers, 13 images (5 stereo pairs + 3 mono, "
                        "1280x720..1920x1080), BF16 + cache + shared (exact) stereo derivation, one frame = all "
                        "13 images",
            "frames": n, "images": n_img, "pixels_per_frame": pixels, "tuned": tuned,
            "tiling": {k: best[k] for k in ("tile_w", "tile_h", "blocks_per_sm", "ms")},
            "untuned_16x16_per_tile": untuned, "separate_contexts": separate,
            "reuse_frac_mean": float(np.mean(reuse)), "tune_s": t_tune, "gen_s": t_gen}


def _vr3(vr):
    return vr.rec, vr.depth32, vr.gid


def judged_psnr(samples, refs):
    """Per frame of refs: PSNR of both eyes' sampled values against refs[f]."""
    out = []
    for f, (r0, r1) in refs.items():
        got = samples[f].astype(np.float64)
        mse = (np.mean((got[0] - r0) ** 2) + np.mean((got[1] - r1) ** 2)) / 2
        out.append(10 * np.log10(1.0 / max(mse, 1e-10)))
    return out


def run_learned(model, flush, steps):
    """Cache + learned-reuse form on the look-around path (seed 12, 80-95%
    frame-to-frame overlap): 100k labels collected on paths 20-29, GPU
    training, then frame rate (label collection off) and quality of the
    cached BF16 unified form with the depth rule and with the predictor."""
    import torch
    import gen
    import paper_2502_14938_b300 as pkg
    from paper_2502_14938_b300 import reuse
    t0 = time.perf_counter()
    Z, Y, st = reuse.collect(model, [gen.stereo_frames(gen.reuse_path(s)) for s in range(20, 30)], 100_000, seed=1)
    t_collect = time.perf_counter() - t0
    t0 = time.perf_counter()
    theta, losses = reuse.train(Z, Y, gen.reuse_mlp_init(7), epochs=40, batch=4096, lr=2e-3)
    t_train = time.perf_counter() - t0
    path = gen.stereo_frames(gen.reuse_path(12))
    import oracle
    rs = np.random.default_rng(12)
    W, H = path[0][0].width, path[0][0].height
    sample = {f: (rs.integers(0, W, 20000), rs.integers(0, H, 20000)) for f in range(5, len(path), 10)}
    qb = oracle.OrcQuant()
    qb.mode = 1
    refs, plain = {}, {}
    for f, (px, py) in sample.items():
        U = oracle.unified_camera(*path[f])
        refs[f] = [oracle.render(*_vr3(oracle.view_gaussians(model, c, derive_cam=U, quant=qb)), W, H, True, px, py)[0]
                   for c in path[f]]
        plain[f] = [oracle.render(*_vr3(oracle.view_gaussians(model, c)), W, H, True, px, py)[0] for c in path[f]]
    out = {"path": "look-around path seed 12 (120 frames)", "collect_s": t_collect, "train_s": t_train,
           "samples": st["samples"], "positive_frac": st["positive_frac"], "final_loss": float(losses[-1])}
    for name, th in (("depth", None), ("learned", theta)):
        r = pkg.Renderer(max_views=2, precision="bf16", reuse="depth" if th is None else "learned",
                         stereo_unify=True)
        mid = r.load_model(model)
        if th is not None:
            r.reuse_set_weights(th)
        outs = [torch.empty((path[0][0].height, path[0][0].width, 3), dtype=torch.float32, device="cuda")
                for _ in range(2)]
        for L, R in path:
            set_pair(r, mid, L, R)
            r.render_frame(outs)
        r.synchronize()
        r.cache_reset()
        n = min(steps, len(path))
        evs = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(n)]
        stream = torch.cuda.current_stream()
        for f in range(n):
            set_pair(r, mid, *path[f])
            flush.fill_(f & 0xFF)
            evs[f][0].record(stream)
            r.render_frame(outs, stats=False)
            evs[f][1].record(stream)
        torch.cuda.synchronize()
        r.close()
        ms = np.array([a.elapsed_time(b) for a, b in evs])
        ev = reuse.evaluate(model, path, th, sample=sample)
        p_form = judged_psnr(ev["samples"], refs)
        p_plain = judged_psnr(ev["samples"], plain)
        out[name] = {"fps": 1000.0 / float(ms.mean()), "ms_mean": float(ms.mean()),
                     "p99_ms": float(np.percentile(ms, 99)), **{k: ev[k] for k in
                     ("reuse_frac", "wrong_reuse_frac", "psnr_db_min", "psnr_db_mean")},
                     "oracle_psnr_db_min": min(p_form), "oracle_psnr_db_mean": float(np.mean(p_form)),
                     "plain_oracle_psnr_db_min": min(p_plain)}
    out["psnr"] = ("psnr_db_*: whole images against the GPU's same form without the cache; oracle_psnr_db_*: "
                   "20k sampled pixels per eye on every 10th frame against the float64 oracle of the same form "
                   "without the cache (unified camera, bf16-rounded derivation); plain_oracle_psnr_db_min: the "
                   "same pixels against the float64 oracle of the plain per-eye method")
    return out


def form_quality(r, mid, outs, frames, refs):
    """PSNR / max-abs against the oracle images `refs` {frame: [left, right]},
    rendering the path from frame 0 in order (from an empty cache); also the
    reused share of visible anchors per frame."""
    r.cache_reset()
    psnr, maxabs, reuse = [], [], []
    for f in range(max(refs) + 1):
        set_pair(r, mid, *frames[f])
        st = r.render_frame(outs)
        reuse.append(1.0 - st["derived_anchors"] / max(st["visible_anchors"], 1))
        if f not in refs:
            continue
        mse, mx = 0.0, 0.0
        for v in range(2):
            got = outs[v].cpu().numpy().astype(np.float64)
            mse += float(np.mean((got - refs[f][v]) ** 2)) / 2
            mx = max(mx, float(np.abs(got - refs[f][v]).max()))
        psnr.append(10 * np.log10(1.0 / max(mse, 1e-10)))  # identical images count as 100 dB
        maxabs.append(mx)
    return {"psnr_db": psnr, "max_abs": maxabs, "frames": sorted(refs)}, reuse


def quality_pass(model, frames, rends, ref_frames, head):
    """Every form of `rends` ({form: (renderer, model id, outs)}) renders the
    path in order from frame 0 with an empty cache (so reuse is live), with
    frame statistics.  At each frame of `ref_frames` the float64 oracle
    renders both eyes of the plain method (whole images; timed: these are
    the CPU baseline's frames) and every form is compared with it: PSNR
    over all pixels, channels and both eyes; max-abs over all pixels; and,
    for the parity tolerance, max-abs over the decided pixels (no alpha or
    stop decision of the oracle within 1e-4 of its threshold) and the share
    of pixels that are not decided.  Returns (quality per form, per-frame
    rows of the `head` form, oracle seconds per reference frame)."""
    import torch
    for r, _, _ in rends.values():
        r.cache_reset()
    keys = ("psnr_db", "max_abs", "max_abs_decided", "near_threshold_frac")
    q = {form: {"frames": [], **{k: [] for k in keys}} for form in rends}
    rows, cpu_s = [], []
    refs_set = set(ref_frames)
    for f in range(max(ref_frames) + 1):
        st_head = None
        for form, (r, mid, outs) in rends.items():
            set_pair(r, mid, *frames[f])
            st = r.render_frame(outs)
            if form == head:
                st_head = st
        row = {"frame": f, "visible_anchors": int(st_head["visible_anchors"]),
               "derived_anchors": int(st_head["derived_anchors"]), "records": int(st_head["records"]),
               "valid_records": int(st_head["valid_records"]), "pairs": int(st_head["pairs"]),
               "cache_depth": int(st_head["cache_depth"]),
               "update_rate": st_head["derived_anchors"] / max(1, st_head["visible_anchors"])}
        if f in refs_set:
            t, refs = oracle_frame(model, *frames[f])
            cpu_s.append(t)
            dev = [(torch.from_numpy(ref).cuda(), torch.from_numpy(mg).cuda() >= 1e-4) for ref, _, mg, _ in refs]
            for form, (r, mid, outs) in rends.items():
                mse = mx = mxd = nt = 0.0
                for v in range(2):
                    ref, ok = dev[v]
                    err = (outs[v].double() - ref).abs()
                    mse += float((err * err).mean()) / 2
                    mx = max(mx, float(err.max()))
                    e_ok = err.amax(dim=-1)[ok]
                    mxd = max(mxd, float(e_ok.max()) if e_ok.numel() else 0.0)
                    nt += (1.0 - float(ok.double().mean())) / 2
                vals = (10 * np.log10(1.0 / max(mse, 1e-10)), mx, mxd, nt)  # identical images count as 100 dB
                q[form]["frames"].append(f)
                for k, x in zip(keys, vals):
                    q[form][k].append(x)
            row.update({k: q[head][k][-1] for k in keys})
        rows.append(row)
    for form in q:
        if q[form]["psnr_db"]:
            q[form]["psnr_db_min"] = min(q[form]["psnr_db"])
            q[form]["max_abs_decided_max"] = max(q[form]["max_abs_decided"])
            q[form]["near_threshold_frac_max"] = max(q[form]["near_threshold_frac"])
    return q, rows, cpu_s


def per_frame_tile_bits(W, H, tiling):
    tiles = 2 * ((W + tiling["tile_w"] - 1) // tiling["tile_w"]) * ((H + tiling["tile_h"] - 1) // tiling["tile_h"])
    bits = 1
    while (1 << bits) < tiles and bits < 31:
        bits += 1
    return bits


def launches_per_frame_of(form, tile_bits):
    """Library kernels per stereo frame of one model: frame setup, the cull's
    two passes (the second also runs the depth-rule cache probe), plan,
    [cache scan, assign; a learned probe as its own kernel], tables,
    derivation, projection, depth sort (4 launches: three 9-bit passes and
    a fourth that returns at once unless the frame's keys need it), scan,
    key generation, tile sort (one pass per 8 tile-key bits), ranges,
    blend."""
    f = FORMS[form]
    n = 1 + 2 + 1 + 1 + 1 + 1 + 4 + 1 + 1 + (tile_bits + 7) // 8 + 1 + 1
    if f["reuse"] != "off":
        n += 2
    if f["reuse"] == "learned":
        n += 1
    return n


def run_ours(args, rank, world):
    import torch

    dev = int(os.environ.get("LOCAL_RANK", "0"))
    torch.cuda.set_device(dev)
    if args.profile:
        return run_profile(args)
    if args.ablation:
        return run_ablation(args) if rank == 0 else None
    if args.guides:
        return run_guides(args) if rank == 0 else None
    if args.sched:
        return run_sched(args) if rank == 0 else None
    if args.octree:
        return run_octree(args) if rank == 0 else None
    model, frames, t_gen = build_workload()
    W, H = frames[0][0].width, frames[0][0].height
    flush = torch.empty(256 << 20, dtype=torch.uint8, device="cuda")  # > 126 MB L2
    form = args.form
    clk = ClockSampler(dev)
    r, mid, outs, ms, wall = time_form(model, frames, form, args.steps, args.warmup, flush, world, clk,
                                       tune=args.autotune)
    total_ms = max_over_ranks(float(ms.sum()), world)
    others = {}
    rends = {form: (r, mid, outs)}
    for f2 in args.compare:
        if f2 == form:
            continue
        r2, mid2, outs2, ms2, _ = time_form(model, frames, f2, args.steps, args.warmup, flush, 1, tune=args.autotune)
        others[f2] = {"fps": 1000.0 / float(ms2.mean()), "ms_mean": float(ms2.mean()),
                      "p99_ms": float(np.percentile(ms2, 99)), "tiling": r2.tiling}
        rends[f2] = (r2, mid2, outs2)
    if rank != 0:
        return
    mean_ms = total_ms / args.steps
    fps = job_rate(world, args.steps, total_ms)
    stage_ms, per_frame = stage_profile(model, frames, form, min(args.steps, len(frames)), flush, r.tiling)
    stage_rows = per_frame.pop("stage_rows")
    roof = roofline(stage_ms, per_frame, form, W, H, model.n, r.tiling)
    stage_gbs = stage_hbm(stage_ms, per_frame, form, W, H, model.n)

    # ---- quality: every form against the float64 oracle of the plain method
    # on every 10th frame of the path (whole images, both eyes), each form
    # rendered in path order from an empty cache; the oracle's frames are
    # timed as the CPU baseline
    import oracle
    q_all, frame_rows, cpu_s = quality_pass(model, frames, rends, args.psnr_frames, form)
    for f2 in others:
        others[f2]["quality"] = q_all[f2]
        rends[f2][0].close()
    q = q_all[form]
    psnrs = q["psnr_db"]
    reuse_frac = [1.0 - x["update_rate"] for x in frame_rows]
    if args.log:
        with open(args.log, "w") as fl:
            for row in frame_rows:
                f = row["frame"]
                if f < len(ms):
                    row["ms"] = float(ms[f])
                if f < len(stage_rows):
                    row["stage_ms_eager"] = stage_rows[f]
                fl.write(json.dumps(row) + "\n")

    # ---- end to end through the public API with host buffers: the headline
    # form with display images (RGBA8) and pipelined host frames (frame n+1
    # renders while frame n's images are copied to pinned host memory); every
    # step uploads its cameras and reads both images back.  The synchronous
    # float32 variant of the same loop is reported beside it.
    import paper_2502_14938_b300 as pkg
    up = pkg.lib().gsc_debug_frame_upload_bytes()
    n_e2e = min(args.steps, 100)
    host32 = [torch.empty((H, W, 3), dtype=torch.float32, pin_memory=True).numpy() for _ in range(2)]
    t0 = time.perf_counter()
    for s in range(n_e2e):
        set_pair(r, mid, *frames[s % len(frames)])
        r.render_frame_host(host32, stats=False)
    e2e_sync_f32 = {"value": n_e2e / (time.perf_counter() - t0), "unit": UNIT, "h2d_bytes_per_step": up,
                    "d2h_bytes_per_step": 2 * W * H * 3 * 4, "format": "f32", "pipelined": False}
    re = pkg.Renderer(max_views=2, out_format="rgba8", **FORMS[form])
    rmid = re.load_model(model)
    host8 = [[torch.empty((H, W, 4), dtype=torch.uint8, pin_memory=True).numpy() for _ in range(2)] for _ in range(2)]
    for f in range(len(frames)):  # grow the buffers with synchronous frames
        set_pair(re, rmid, *frames[f])
        if f == 0:
            re.set_tiling(r.tiling["tile_w"], r.tiling["tile_h"], r.tiling["blocks_per_sm"])
        re.render_frame_host(host8[0], stats=False)
    re.cache_reset()
    t0 = time.perf_counter()
    for s in range(n_e2e):
        set_pair(re, rmid, *frames[s % len(frames)])
        re.render_frame_host_async(host8[s % 2])
    re.wait_host()
    e2e_s = time.perf_counter() - t0
    re.close()
    e2e = {"value": n_e2e / e2e_s, "unit": UNIT, "h2d_bytes_per_step": up, "d2h_bytes_per_step": 2 * W * H * 4,
           "format": "rgba8", "pipelined": True}

    # ---- CPU baseline: the oracle on a bounded sample
    batched = run_batched(args, flush) if args.batched else None
    learned = run_learned(model, flush, args.steps) if args.learned else None

    cores = oracle.num_threads()
    t1 = oracle_one_thread(model, *frames[150])
    cpu = {"value": len(cpu_s) / float(np.sum(cpu_s)), "unit": UNIT, "cores": cores, "kind": "oracle",
           "sample": f"the {len(cpu_s)} quality reference frames (every 10th frame of the path): whole stereo "
                     f"frames, every pixel of both eyes, float64, {cores} threads; frame 150 also on 1 thread",
           "value_1thread": 1.0 / t1, **cpu_info()}

    launches_per_frame = launches_per_frame_of(form, per_frame_tile_bits(W, H, r.tiling))
    cfg = {"workload": WORKLOAD, "form": form, **FORMS[form], "tiling": r.tiling,
           "l2": "flushed between frames (256 MB write, untimed)",
           "p99_ms": float(np.percentile(ms, 99)), "wall_fps": args.steps / wall,
           "wall_fps_unsampled": args.steps / getattr(clk, "wall_unsampled", float("nan")),
           "host_set_cameras_ms": 1e3 * getattr(clk, "host_set_cameras", float("nan")) / args.steps,
           "psnr_db_min": min(psnrs) if psnrs else None, "psnr_db": psnrs, "max_abs": q["max_abs"],
           "max_abs_decided": q["max_abs_decided"], "near_threshold_frac": q["near_threshold_frac"],
           "psnr_frames": args.psnr_frames,
           "reuse_frac_mean": float(np.mean(reuse_frac)) if reuse_frac else None,
           "e2e_sync_f32": e2e_sync_f32, "compare": others, "batched": batched, "learned_reuse": learned, "stage_ms": stage_ms, "stage_hbm": stage_gbs, "per_frame": per_frame, "gen_s": t_gen}
    line = {"metric": METRIC, "value": fps, "unit": UNIT, "n_gpus": world, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": mean_ms, "higher_is_better": True, "scaling": "weak",
            "vs_baseline": None, "dtype": {"fp32": "f32", "bf16": "bf16+f32", "fp8": "e4m3+f32"}[FORMS[form]["precision"]],
            "data": "synthetic", "config": cfg, "roofline": roof, "cpu_baseline": cpu, "e2e": e2e,
            "clocks": clk.summary(), "gpu_launches": launches_per_frame * args.steps}
    print(json.dumps(line), flush=True)


def main():
    if len(sys.argv) == 5 and sys.argv[1] == "--clock-sampler":
        return clock_sampler_main(sys.argv[2], int(sys.argv[3]), float(sys.argv[4]))
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=300)
    ap.add_argument("--warmup", type=int, default=10)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--form", default=HEADLINE, choices=sorted(FORMS))
    ap.add_argument("--compare", nargs="*", default=["plain", "bf16_exact", "cached_bf16_unified", "fp8_exact",
                                                     "cached_fp8_exact"],
                    help="other forms timed for comparison")
    ap.add_argument("--psnr-frames", type=int, nargs="*", default=list(range(0, 300, 10)),
                    help="path frames compared with the float64 oracle (default: every 10th frame)")
    ap.add_argument("--log", default=None, help="JSON lines file: one line per path frame of the timed form "
                    "(counts, cache depth, update rate, event ms, eager stage ms, PSNR / max-abs at oracle frames)")
    ap.add_argument("--profile", action="store_true", help="minimal run for ncu (no extras)")
    ap.add_argument("--frame", type=int, default=150, help="first path frame of a --profile run")
    ap.add_argument("--tile", type=int, nargs=3, default=[16, 16, 0], metavar=("W", "H", "BPS"),
                    help="blend tiling of a --profile run (tile width, height, blocks per SM)")
    ap.add_argument("--batched", action=argparse.BooleanOptionalAction, default=True,
                    help="also time the batched multi-viewer form (reported under config.batched)")
    ap.add_argument("--tiling-cache", default=None, help="JSON file the autotuner reads / writes")
    ap.add_argument("--autotune", action=argparse.BooleanOptionalAction, default=True,
                    help="tune the headline form's blend tiling before timing it")
    ap.add_argument("--learned", action=argparse.BooleanOptionalAction, default=True,
                    help="also train the reuse predictor and time the learned form (config.learned_reuse)")
    ap.add_argument("--ablation", action="store_true",
                    help="instead of the bench line: the ablation table (one JSON line) at the --tile tiling")
    ap.add_argument("--guides", action="store_true",
                    help="instead of the bench line: Eq. 4 guiding functions on an accelerating path (one JSON line)")
    ap.add_argument("--octree", action="store_true",
                    help="instead of the bench line: Octree-GS level offsets + fade vs the plain LOD rule (one JSON line)")
    ap.add_argument("--sched", action="store_true",
                    help="instead of the bench line: frames/s of the elastic schedule with 1-4 workers (one JSON line)")
    args = ap.parse_args()
    assert args.warmup >= 0 and args.steps >= 1
    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    if world > 1:
        import torch
        import torch.distributed as dist
        backend = "nccl" if args.impl == "ours" and torch.cuda.is_available() else "gloo"
        if backend == "nccl":
            torch.cuda.set_device(int(os.environ.get("LOCAL_RANK", "0")))
        dist.init_process_group(backend)
    if args.impl == "reference":
        run_reference(args, rank, world)
    else:
        run_ours(args, rank, world)
    if world > 1:
        import torch.distributed as dist
        dist.destroy_process_group()


if __name__ == "__main__":
    main()
