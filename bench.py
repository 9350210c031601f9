#!/usr/bin/env python3
"""Benchmark of the light-transport hot path on one B300 (or N, one process each).

Workload: the plenoptic camera of the simulated-plenoptic table (100x100
lenslets x 10x10 pixels, 1000^2 detector and array plane, K = 2x2 pillbox
angular cells) looking at a 128^3 float32 volume of 1 mm voxels holding 20
seeded elongated plumes with lognormal(0, 0.3) turbulence; measurements with
Poisson noise at a peak of 1e4 photons.  One step is one iteration of the
Table V reconstruction: projection A z (slices -> array plane, mask,
microlenses -> detector), residual, back-projection A^T r (both stages), and
the FISTA update with the 26-neighbour quadratic regulariser.

Metric: projector+adjoint ray-samples/s.  A ray-sample is one (beam, slice)
pair (stage 1: array pixel x cell x slice) or one (detector pixel, cell)
pair (stage 2); a step counts the forward and the adjoint once each.

Multi-GPU (torchrun): every rank reconstructs its own independent frame (no
data-path collective), scaling is weak; value = all ranks' ray-samples / the
slowest rank's time.
"""
import argparse
import hashlib
import json
import os
import sys
import threading
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

METRIC = "projector+adjoint ray-samples/s"
UNIT = "ray-samples/s"
WORKLOAD = ("plenoptic camera, 100x100 lenslets x 10x10 px (1000^2 detector), K=2x2 pillbox, "
            "128^3 FP32 plume volume (1 mm voxels), Poisson peak 1e4; one Table V FISTA iteration per step")


def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=1000)
    ap.add_argument("--warmup", type=int, default=5)
    ap.add_argument("--impl", choices=["ours", "reference"], default="ours")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--e2e-steps", type=int, default=200)
    ap.add_argument("--warm-samples", type=int, default=10000,
                    help="training volumes of the warm-start U-Net (the learned-warm-start configuration's 10k; 0 skips)")
    ap.add_argument("--warm-eval", type=int, default=16, help="held-out volumes of the time-to-residual comparison")
    ap.add_argument("--no-autotune", action="store_true",
                    help="pin --forward-variant instead of tuning (fixed launch sequence, e.g. for profiling)")
    ap.add_argument("--forward-variant", type=int, default=5,
                    help="forward kernel variant pinned by --no-autotune (the plan's default is 5)")
    ap.add_argument("--workloads", default="multiview,differentiable",
                    help="further workloads timed after the headline one (comma list; empty: none)")
    ap.add_argument("--workload-steps", type=int, default=10)
    return ap.parse_args()


def max_over_ranks(x, device):
    """The largest x over all ranks (every rank gets it); x itself on one rank."""
    import torch
    import torch.distributed as dist
    t = torch.tensor([float(x)], dtype=torch.float64, device=device)
    if dist.is_available() and dist.is_initialized() and dist.get_world_size() > 1:
        dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def frame_seed(rank):
    """Seed of the frame rank `rank` reconstructs (ranks solve independent
    problems: no data-path collective, weak scaling)."""
    return 2000 + rank


def job_rate(units_per_rank_step, steps, world, t_max):
    """Whole-job throughput: the units every rank processed over the slowest
    rank's time."""
    return world * units_per_rank_step * steps / t_max


def dist_env():
    return (int(os.environ.get("RANK", 0)), int(os.environ.get("WORLD_SIZE", 1)),
            int(os.environ.get("LOCAL_RANK", 0)))


# ---------------------------------------------------------------------------
# clocks during the timed region (NVML reads only)
# ---------------------------------------------------------------------------

class _PyNvml:
    name = "nvml (pynvml)"

    def __init__(self, mod, h):
        self.m, self.h = mod, h

    def sm(self):
        return self.m.nvmlDeviceGetClockInfo(self.h, self.m.NVML_CLOCK_SM)

    def reasons(self):
        return self.m.nvmlDeviceGetCurrentClocksEventReasons(self.h)


class _CtypesNvml:
    """Read-only NVML queries through the driver's libnvidia-ml (clock and
    clock-event reasons of one device); nothing is set."""
    name = "nvml (ctypes)"

    def __init__(self, bus):
        import ctypes
        self.ct = ctypes
        self.lib = ctypes.CDLL("libnvidia-ml.so.1")
        self._ok(self.lib.nvmlInit_v2())
        self.h = ctypes.c_void_p()
        self._ok(self.lib.nvmlDeviceGetHandleByPciBusId_v2(bus.encode(), ctypes.byref(self.h)))

    @staticmethod
    def _ok(rc):
        if rc != 0:
            raise RuntimeError(f"NVML error {rc}")

    def _clock(self, fn):
        v = self.ct.c_uint()
        self._ok(fn(self.h, 1, self.ct.byref(v)))   # NVML_CLOCK_SM = 1
        return int(v.value)

    def max_sm(self):
        return self._clock(self.lib.nvmlDeviceGetMaxClockInfo)

    def sm(self):
        return self._clock(self.lib.nvmlDeviceGetClockInfo)

    def reasons(self):
        v = self.ct.c_ulonglong()
        self._ok(self.lib.nvmlDeviceGetCurrentClocksEventReasons(self.h, self.ct.byref(v)))
        return int(v.value)


class ClockSampler:
    """Samples the SM clock and clock-event reasons of the benchmarked GPU
    while the timed region runs (NVML reads; nvidia-smi as a fallback)."""
    REASONS = {
        "applications_clocks_setting": 0x2, "sw_power_cap": 0x4, "hw_slowdown": 0x8,
        "sync_boost": 0x10, "sw_thermal_slowdown": 0x20, "hw_thermal_slowdown": 0x40,
        "hw_power_brake_slowdown": 0x80,
    }

    def __init__(self, device, period=0.001):
        import torch
        self.period = period
        self.samples = []
        self.reasons = set()
        self.max_mhz = None
        self.errors = []
        self._stop = threading.Event()
        self._t = None
        self._proc = None
        self.nvml = None
        props = torch.cuda.get_device_properties(device)
        self.bus = "%08X:%02X:%02X.0" % (getattr(props, "pci_domain_id", 0), props.pci_bus_id, props.pci_device_id)
        try:
            import pynvml
            pynvml.nvmlInit()
            self.h = pynvml.nvmlDeviceGetHandleByPciBusId(self.bus)
            self.max_mhz = pynvml.nvmlDeviceGetMaxClockInfo(self.h, pynvml.NVML_CLOCK_SM)
            self.nvml = _PyNvml(pynvml, self.h)
        except Exception as e:  # the driver's NVML through ctypes, then nvidia-smi
            self.errors.append("pynvml: " + repr(e)[:200])
            try:
                self.nvml = _CtypesNvml(self.bus)
                self.max_mhz = self.nvml.max_sm()
            except Exception as e2:
                self.nvml = None
                self.errors.append("libnvidia-ml: " + repr(e2)[:200])

    def _run_nvml(self):
        while not self._stop.is_set():
            try:
                self.samples.append(self.nvml.sm())
                mask = self.nvml.reasons()
                for name, bit in self.REASONS.items():
                    if mask & bit:
                        self.reasons.add(name)
            except Exception as e:
                if len(self.errors) < 8:
                    self.errors.append(repr(e)[:200])
            time.sleep(self.period)

    def __enter__(self):
        if self.nvml:
            self._t = threading.Thread(target=self._run_nvml, daemon=True)
            self._t.start()
        else:
            import subprocess
            try:
                self._proc = subprocess.Popen(
                    ["nvidia-smi", "--query-gpu=clocks.sm,clocks.max.sm,clocks_event_reasons.active",
                     "--format=csv,noheader,nounits", "-i", self.bus, "-lms", str(int(self.period * 1000))],
                    stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
            except Exception as e:
                self.errors.append("nvidia-smi: " + repr(e))
        return self

    def __exit__(self, *a):
        self._stop.set()
        if self._t:
            self._t.join()
        if self._proc:
            self._proc.terminate()
            out, _ = self._proc.communicate()
            for line in out.splitlines():
                parts = [p.strip() for p in line.split(",")]
                try:
                    self.samples.append(float(parts[0]))
                    self.max_mhz = float(parts[1])
                    mask = int(parts[2], 16)
                    for name, bit in self.REASONS.items():
                        if mask & bit:
                            self.reasons.add(name)
                except (ValueError, IndexError):
                    pass

    def summary(self):
        out = {"sm_mhz": float(np.median(self.samples)) if self.samples else None,
               "sm_max_mhz": self.max_mhz, "reasons": sorted(self.reasons),
               "samples": len(self.samples), "source": self.nvml.name if self.nvml else "nvidia-smi"}
        if not self.samples:
            out["errors"] = self.errors[:3]
        return out


# ---------------------------------------------------------------------------
# our arm
# ---------------------------------------------------------------------------

KERNEL_SOURCE = {"beam_forward_tma": "lt_beam_tma.cu", "beam_adjoint_tma": "lt_beam_adj.cu"}


def traffic_for(kernel):
    """DRAM bytes per launch of `kernel` from the committed ncu summary, if the
    kernel's source file has not changed since the counters were taken."""
    path = os.path.join(ROOT, "profiles", "ncu_traffic.json")
    src = os.path.join(ROOT, "paper_1812_03358_b300", "csrc", KERNEL_SOURCE.get(kernel, "lt_kernels.cu"))
    try:
        rec = json.load(open(path))
        sha = hashlib.sha1(open(src, "rb").read()).hexdigest()
        ent = rec.get(kernel)
        if ent and ent.get("source_sha1") == sha:
            return ent["dram_bytes_per_launch"]
    except Exception:
        pass
    return None


def hbm_peak():
    """Measured HBM copy bandwidth (GB/s) of the B300s, else the
    fallback figure."""
    try:
        return float(json.load(open(os.path.join(ROOT, "MEASURED_PEAKS.json")))["hbm_gbs"]), "measured"
    except Exception:
        return 6400.0, "fallback"


def measure_peaks(stream, reps=5):
    """Roofline denominators of the on-chip levels, measured here by the
    library's own microbenchmarks (include/lt_peaks.h): shared-memory read
    and L2 read bandwidth (GB/s) and the FP32 FMA rate (TFLOP/s), each the
    best of `reps` CUDA-event-timed launches on the launching stream.  HBM is
    the measured copy bandwidth."""
    import torch
    from paper_1812_03358_b300 import lt
    sms = torch.cuda.get_device_properties(torch.cuda.current_device()).multi_processor_count
    sink = torch.empty(sms * 8 * 256, dtype=torch.float32, device="cuda")
    l2buf = torch.ones(32 * 1024 * 1024 // 4, dtype=torch.float32, device="cuda")   # 32 MB: L2-resident
    h = stream.cuda_stream

    def best(fn):
        fn()
        rate = 0.0
        for _ in range(reps):
            a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            a.record(stream)
            work = fn()
            b.record(stream)
            b.synchronize()
            rate = max(rate, work / (a.elapsed_time(b) * 1e-3))
        return rate

    smem = best(lambda: lt.lt_peak_smem_read(sink.data_ptr(), sms * 4, 4096, h)) / 1e9
    l2 = best(lambda: lt.lt_peak_l2_read(l2buf.data_ptr(), l2buf.numel() // 4, sink.data_ptr(), sms * 8, 256, h)) / 1e9
    fp32 = best(lambda: lt.lt_peak_fp32_fma(sink.data_ptr(), sms * 8, 32768, h)) / 1e12
    hbm, src = hbm_peak()
    return {"smem_GBps": smem, "l2_GBps": l2, "fp32_TFLOPs": fp32, "hbm_GBps": hbm,
            "hbm_source": src + " (MEASURED_PEAKS.json copy bandwidth)" if src == "measured" else src,
            "how": "library microbenchmarks: conflict-free 16 B shared loads (32 KiB per CTA, 4 CTAs/SM), "
                   "L1-bypassing 16 B loads over a 32 MB buffer, 8 independent FMA chains per thread; "
                   "best of 5 CUDA-event-timed launches"}


def level_roofline(ms, dram_b, l2_b, smem_b, flops, peaks):
    """Time bound of every level for one kernel launch (algorithmic bytes or
    flops / that level's measured peak), the level that binds, and the
    memory roofline fraction = the largest memory-level bound / the measured
    time."""
    t = {"dram": dram_b / (peaks["hbm_GBps"] * 1e9), "l2": l2_b / (peaks["l2_GBps"] * 1e9),
         "smem": smem_b / (peaks["smem_GBps"] * 1e9), "fp32": flops / (peaks["fp32_TFLOPs"] * 1e12)}
    mem = max(("dram", "l2", "smem"), key=lambda k: t[k])
    return {"ms": ms, "bytes": {"dram": dram_b, "l2": l2_b, "smem": smem_b}, "flops": flops,
            "bound_us": {k: v * 1e6 for k, v in t.items()}, "binding": max(t, key=t.get),
            "memory_level": mem, "memory_frac": t[mem] / (ms * 1e-3), "fp32_frac": t["fp32"] / (ms * 1e-3)}


def shear_passes(flush, stream, reps=20):
    """The rotation passes of a yawed camera (quarter turn + z shear + x shear,
    and the transposed passes) on a 128^3 volume: CUDA-event time per call, L2
    flushed before each, against the HBM roofline.  Algorithmic bytes per
    pass = 4 (N_in + N_out).  Also timed: a pitched and rolled camera's
    signed permutation and three shear passes (general_*_ms)."""
    import math
    import torch
    from paper_1812_03358_b300 import inputs as I
    from paper_1812_03358_b300 import lt
    yaw = math.radians(30.0)
    vol = I.Volume(128, 128, 128, 1.0, 1.0, 1.0)
    plan = lt.Plan(vol, [I.table_single_lens(64, 0.08, yaw=yaw)])
    (nzr, ny, nxr), _ = plan.camera_grid(0)
    q = math.floor(yaw / (math.pi / 2) + 0.5)
    nxp = vol.nz if q % 2 else vol.nx
    n_in, n_mid, n_out = vol.n, nzr * ny * nxp, nzr * ny * nxr
    nbytes = 4 * (n_in + n_mid) + 4 * (n_mid + n_out)
    g = torch.Generator(device="cuda").manual_seed(5)
    x = torch.rand(1, vol.n, device="cuda", generator=g)
    xc = plan.rotate(0, x)
    xa = plan.rotate_adjoint(0, xc)
    peak, src = hbm_peak()
    out = {"workload": f"128^3 volume (1 mm), yaw 30 deg -> camera grid {nzr}x{ny}x{nxr}",
           "bytes_per_call": nbytes, "peak_GBps": peak, "peak_source": src}
    for name, fn in (("forward", lambda: plan.rotate(0, x, xc)), ("adjoint", lambda: plan.rotate_adjoint(0, xc, xa))):
        ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(reps)]
        for a, b in ev:
            flush.zero_()
            a.record(stream)
            fn()
            b.record(stream)
        torch.cuda.synchronize()
        ms = sum(a.elapsed_time(b) for a, b in ev) / reps
        out[name + "_ms"] = ms
        out[name + "_GBps"] = nbytes / (ms * 1e-3) / 1e9
        out[name + "_frac"] = out[name + "_GBps"] / peak
    plan.close()
    # a pitched and rolled camera: signed permutation + three shear passes
    cam = I.table_single_lens(64, 0.08, yaw=0.5)
    cam.pitch, cam.roll = 0.3, -0.2
    plan = lt.Plan(vol, [cam])
    (gz, gy, gx), _ = plan.camera_grid(0)
    xg = plan.rotate(0, x)
    xga = plan.rotate_adjoint(0, xg)
    out["general_workload"] = f"128^3 volume (1 mm), yaw 0.5, pitch 0.3, roll -0.2 rad -> camera grid {gz}x{gy}x{gx}"
    for name, fn in (("forward", lambda: plan.rotate(0, x, xg)), ("adjoint", lambda: plan.rotate_adjoint(0, xg, xga))):
        ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(reps)]
        for a, b in ev:
            flush.zero_()
            a.record(stream)
            fn()
            b.record(stream)
        torch.cuda.synchronize()
        out["general_" + name + "_ms"] = sum(a.elapsed_time(b) for a, b in ev) / reps
    plan.close()
    return out


def time_to_residual(plan, n_samples, n_plain=200, n_eval=16):
    """Warm start vs plain solver on the bench workload: the U-Net is trained
    here for n_samples volumes made by the projector (seeds 1e6 + i), then both
    arms run on n_eval held-out volumes (seeds 2e6 + j): wall time (CUDA
    events) until the data fit reaches the plain solver's n_plain-iteration
    value, the warm arm including back-projection and U-Net inference (not
    training).  Reported: the median over the held-out volumes of each figure,
    every volume's gain, and the smallest and largest gain."""
    import statistics
    import time as _t
    from paper_1812_03358_b300 import unet, warmstart
    t0 = _t.time()
    ws, losses = warmstart.train(plan, unet.UNet(seed=1), n_samples, lr=1e-3, max_norm=1.0)
    t_train = _t.time() - t0
    rows = []
    for j in range(n_eval):
        x, _, y = warmstart.training_pair(plan, seed=2_000_000 + j)
        rows.append(warmstart.evaluate(plan, ws, y, x, n_plain=n_plain))
    gains = [(r["plain_ms"] / r["warm_ms"]) if r["warm_ms"] else None for r in rows]

    def med(key):
        v = [r[key] for r in rows if r[key] is not None]
        return statistics.median(v) if v else None

    ok = [g for g in gains if g is not None]
    return {"definition": "wall time until the data fit reaches the plain solver's value after n_plain iterations",
            "n_plain": n_plain, "plain_ms": med("plain_ms"), "plain_first_cross_iters": med("plain_first_cross_iters"),
            "warm_ms": med("warm_ms"), "warm_iters": med("warm_iters"), "unet_ms": med("unet_ms"),
            "unet_tflops": med("unet_tflops"), "gain": statistics.median(ok) if ok else None,
            "gain_per_volume": gains, "gain_min": min(ok) if ok else None, "gain_max": max(ok) if ok else None,
            "volume_error_plain": med("err_plain"),
            "volume_error_warm_x0": med("err_x0"), "train_samples": n_samples, "train_s": round(t_train, 1),
            "beta": "1e-3 * mean(D)", "grad_clip_norm": 1.0, "train_reproducible": True, "held_out_seeds": [2_000_000 + j for j in range(n_eval)],
            "statistic": "median over the held-out volumes"}


def timed_steps(fn, steps, warmup, stream):
    """Mean CUDA-event time (ms) of `steps` calls of fn after `warmup` calls;
    the workloads timed this way hold far more than L2 (126 MB) in inputs."""
    import torch
    for _ in range(warmup):
        fn()
    torch.cuda.synchronize()
    a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    a.record(stream)
    for _ in range(steps):
        fn()
    b.record(stream)
    b.synchronize()
    return a.elapsed_time(b) / steps


def workload_multiview(steps, warmup, stream):
    """Batched multi-view reconstruction: four single-lens 2048^2 cameras (2 x 2
    cells) at seeded yaw in [0, 180) degrees and one 200 x 200-lenslet
    plenoptic camera around a 256^3 volume of 0.5 mm voxels, 16 frames of a
    plume field drifting one voxel per frame along +y; one step = one Table V
    iteration of every frame (rotations, projections of every camera and
    frame, back-projections, update), measurements with Poisson noise at a
    peak of 1e4 photons.  Also timed: the forward and adjoint operators alone
    and each yawed camera's rotation passes against the HBM roofline."""
    import torch
    from paper_1812_03358_b300 import inputs as I
    from paper_1812_03358_b300 import lt
    import math
    frames = 16
    vol, cams = I.config_multiview()
    plan = lt.Plan(vol, cams, frames)
    x = torch.stack([I.plume_field_torch(vol, seed=3100, drift_voxels=float(f)) for f in range(frames)]).contiguous()
    y = I.poisson_images_torch(plan.forward(x), 1e4, seed=3200)
    rec = lt.Recon(plan, y, beta=1e-3 * float(plan.adjoint(plan.forward(torch.ones_like(x))).mean()))
    stats = [plan.stats(c) for c in range(len(cams))]
    samples = 2 * frames * sum(st["ray_samples"] for st in stats)
    ms = timed_steps(lambda: rec.iterate(1), steps, warmup, stream)
    ya = plan.new_y()
    xa = plan.new_x()
    fwd_ms = timed_steps(lambda: plan.forward(x, ya), steps, 1, stream)
    adj_ms = timed_steps(lambda: plan.adjoint(y, xa), steps, 1, stream)
    peak, _ = hbm_peak()
    rot = []
    for c, cam in enumerate(cams):
        if cam.yaw == 0.0:
            continue
        (nzr, ny, nxr), _ = plan.camera_grid(c)
        xc = plan.rotate(c, x)
        r_ms = timed_steps(lambda: plan.rotate(c, x, xc), 3, 1, stream)
        # the z pass (quarter turn fused into its gather) reads the volume and
        # writes the z-sheared intermediate, the x pass reads that and writes
        # the camera grid: 4 (N_in + N_mid) + 4 (N_mid + N_out) bytes a frame
        q = math.floor(cam.yaw / (math.pi / 2) + 0.5)
        n_mid = nzr * ny * (vol.nz if q % 2 else vol.nx)
        pass_bytes = 4 * frames * (vol.n + 2 * n_mid + nzr * ny * nxr)
        xr_a = plan.rotate_adjoint(c, xc)
        ra_ms = timed_steps(lambda: plan.rotate_adjoint(c, xc, xr_a), 3, 1, stream)
        rot.append({"camera": c, "yaw_deg": float(np.degrees(cam.yaw)), "grid": [nzr, ny, nxr], "ms": r_ms,
                    "bytes": pass_bytes, "GBps": pass_bytes / (r_ms * 1e-3) / 1e9,
                    "frac": pass_bytes / (r_ms * 1e-3) / 1e9 / peak,
                    "adjoint_ms": ra_ms, "adjoint_GBps": pass_bytes / (ra_ms * 1e-3) / 1e9,
                    "adjoint_frac": pass_bytes / (ra_ms * 1e-3) / 1e9 / peak})
    out = {"workload": workload_multiview.__doc__.split(";")[0].replace("\n", " ").strip(),
           "frames": frames, "cameras": len(cams), "volume": [vol.nx, vol.ny, vol.nz],
           "ray_samples_per_step": samples, "value": samples / (ms * 1e-3), "unit": UNIT, "ms_per_step": ms,
           "steps": steps, "forward_ms": fwd_ms, "adjoint_ms": adj_ms,
           "forward_brick": [st["forward_brick"] for st in stats], "adjoint_box": [st["adjoint_box"] for st in stats],
           "rotations": rot, "peak_GBps": peak}
    rec.close()
    plan.close()
    del x, y, ya, xa
    torch.cuda.empty_cache()
    return out


def workload_differentiable(steps, warmup, stream):
    """TV-regularised non-negative fit: four single-lens 1024^2 cameras (2 x 2
    cells) at yaw 0, 45, 90, 135 degrees around a 256^3 volume of 0.5 mm
    voxels (plume field); one step = one Table V iteration with the
    26-neighbour hyperbola penalty (beta = 1e-3, delta = 1e-3 max x)."""
    import torch
    from paper_1812_03358_b300 import inputs as I
    from paper_1812_03358_b300 import lt
    vol, cams = I.config_differentiable()
    plan = lt.Plan(vol, cams)
    truth = I.plume_field_torch(vol, seed=4100).reshape(1, -1).contiguous()
    y = plan.forward(truth)
    rec = lt.Recon(plan, y, beta=1e-3, psi=1, psi_delta=1e-3 * float(truth.max()))
    stats = [plan.stats(c) for c in range(len(cams))]
    samples = 2 * sum(st["ray_samples"] for st in stats)
    ms = timed_steps(lambda: rec.iterate(1), steps, warmup, stream)
    out = {"workload": workload_differentiable.__doc__.split(";")[0].replace("\n", " ").strip(),
           "cameras": len(cams), "volume": [vol.nx, vol.ny, vol.nz], "ray_samples_per_step": samples,
           "value": samples / (ms * 1e-3), "unit": UNIT, "ms_per_step": ms, "steps": steps}
    rec.close()
    plan.close()
    del truth, y
    torch.cuda.empty_cache()
    return out


def oracle_cell_sample(vol, cam, x):
    """The FP64 oracle, as it stands, on a bounded sample of the headline
    workload: the whole forward and adjoint (both stages, all slices) of one
    of its K angular cells, i.e. 1/K of a step with the same mix of work.
    Returns (seconds, ray-samples of the sample)."""
    from oracle import camera as O
    t0 = time.perf_counter()
    y = O.plenoptic_forward(vol, cam, x, cells=[0])
    O.plenoptic_adjoint(vol, cam, y, cells=[0])
    dt = time.perf_counter() - t0
    n_cells = len(O.lens_cells(cam))
    samples = 2 * (cam.arr_ns * cam.arr_nt * vol.nz + cam.det_ns * cam.det_nt)   # one cell, forward + adjoint
    return dt, samples, n_cells


def blas_threads():
    try:
        from threadpoolctl import threadpool_info
        info = threadpool_info()
        return max(d.get("num_threads", 1) for d in info) if info else 1
    except Exception:
        return os.cpu_count()


def cpu_baseline_sample(vol, cam, x):
    """The oracle on one cell of the workload (oracle_cell_sample): wall-clock
    median of three runs on all host cores (its BLAS threads), and one run on
    one core."""
    import statistics
    runs = [oracle_cell_sample(vol, cam, x) for _ in range(3)]
    t_all = statistics.median(r[0] for r in runs)
    samples = runs[0][1]
    try:
        from threadpoolctl import threadpool_limits
        with threadpool_limits(limits=1):
            t_one = oracle_cell_sample(vol, cam, x)[0]
    except Exception:
        t_one = None
    return {"value": samples / t_all, "unit": UNIT, "cores": blas_threads(), "kind": "oracle",
            "sample": f"FP64 forward + adjoint of one of the workload's {runs[0][2]} angular cells (both stages, "
                      f"all slices; {samples:.3g} ray-samples), wall-clock median of 3 on all cores: "
                      f"{t_all:.2f} s",
            "one_core": ({"value": samples / t_one, "seconds": t_one} if t_one else None)}


def run_ours(args):
    import torch
    import torch.distributed as dist

    from paper_1812_03358_b300 import inputs as I
    from paper_1812_03358_b300 import lt

    rank, world, local = dist_env()
    torch.cuda.set_device(local)
    if world > 1:
        dist.init_process_group("nccl", device_id=torch.device("cuda", local))
    stream = torch.cuda.current_stream()

    vol, cam = I.config_plenoptic()
    x_true = I.plume_field(vol, seed=frame_seed(rank))
    plan = lt.Plan(vol, [cam])
    if args.no_autotune:
        lt.lt_plan_set_forward_variant(plan.handle, args.forward_variant)
        tuned, tune_ms = args.forward_variant, None
        adj_tuned, adj_tune_ms = 1, None
    else:
        tuned, tune_ms = plan.autotune()
        adj_tuned, adj_tune_ms = plan.autotune_adjoint()
    stats = plan.stats(0)
    xt = torch.from_numpy(x_true.reshape(1, -1)).cuda()
    y_clean = plan.forward(xt)
    y_host = I.poisson_images(y_clean.cpu().numpy(), 1e4, seed=2001 + rank)
    y_dev = torch.from_numpy(y_host).cuda()
    ones = torch.ones_like(xt)
    dmean = float(plan.adjoint(plan.forward(ones)).mean())
    beta = 1e-3 * dmean
    rec = lt.Recon(plan, y_dev, beta=beta)
    kpi = rec.kernels_per_iteration()

    flush = torch.empty(512 * 1024 * 1024 // 4, dtype=torch.float32, device="cuda")

    for _ in range(max(args.warmup, 3)):
        flush.zero_()
        rec.iterate(1)
    torch.cuda.synchronize()

    starts = [torch.cuda.Event(enable_timing=True) for _ in range(args.steps)]
    ends = [torch.cuda.Event(enable_timing=True) for _ in range(args.steps)]
    if world > 1:
        dist.barrier()
    torch.cuda.synchronize()
    with ClockSampler(local) as clk:
        w0 = time.perf_counter()
        for s in range(args.steps):
            flush.zero_()                    # L2 flush between timed iterations
            starts[s].record(stream)
            rec.iterate(1)
            ends[s].record(stream)
        torch.cuda.synchronize()
        wall = time.perf_counter() - w0
    if world > 1:
        dist.barrier()
    torch.cuda.synchronize()
    t_dev = sum(a.elapsed_time(b) for a, b in zip(starts, ends)) / 1e3
    t_max = max_over_ranks(t_dev, "cuda")
    samples_step = 2 * stats["ray_samples"]
    value = job_rate(samples_step, args.steps, world, t_max)

    # --- per-stage device times (same stream, CUDA events, L2 flushed) ---
    fa = plan.stage1(0, xt)
    ya = plan.forward(xt)
    ga = plan.stage2_adjoint(0, ya)
    xa = plan.new_x()
    stage_fns = {
        "beam_forward (stage 1, slices->array)": lambda: plan.stage1(0, xt, fa),
        "stage2_forward (array->detector)": lambda: plan.stage2(0, fa, ya),
        "stage2_adjoint (detector->array)": lambda: plan.stage2_adjoint(0, ya, ga),
        "beam_adjoint (stage 1^T, array->voxels)": lambda: plan.stage1_adjoint(0, ga, xa),
    }
    reps = 20
    stage_ms = {}
    for name, fn in stage_fns.items():
        fn()
        ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(reps)]
        for a, b in ev:
            flush.zero_()
            a.record(stream)
            fn()
            b.record(stream)
        torch.cuda.synchronize()
        stage_ms[name] = sum(a.elapsed_time(b) for a, b in ev) / reps
    # --- per-level rooflines of every stage (algorithmic bytes and flops) ---
    peaks = measure_peaks(stream)
    N, Na, K, M = vol.n, cam.arr_ns * cam.arr_nt, stats["n_cells"], cam.m
    b1, b2 = stats["stage1_nnz"], stats["stage2_nnz"]
    tile_b = 4 * stats["stage1_tile_voxels"] + 4 * K * Na
    work = {   # (dram, l2, smem bytes, flops) per launch
        "beam_forward (stage 1, slices->array)": (4 * (N + K * Na + Na), tile_b, 4 * b1, 2 * b1),
        "stage2_forward (array->detector)": (4 * (K * Na + M + Na), 4 * (K * Na + M + Na), 4 * b2, 2 * b2),
        "stage2_adjoint (detector->array)": (4 * (M + K * Na + 2 * Na), 4 * (M + K * Na + 2 * Na), 4 * b2, 2 * b2),
        "beam_adjoint (stage 1^T, array->voxels)": (4 * (K * Na + N), tile_b, 4 * b1, 2 * b1),
    }
    levels = {name: level_roofline(stage_ms[name], *work[name], peaks) for name in stage_ms}
    dom = max(stage_ms, key=stage_ms.get)
    kname = {"beam_forward (stage 1, slices->array)":
             "beam_forward_tma" if stats["forward_brick"] > 0 and tuned == 5 else "beam_forward_batched",
             "stage2_forward (array->detector)": "stage2_lenslet_forward",
             "stage2_adjoint (detector->array)": "stage2_lenslet_adjoint",
             "beam_adjoint (stage 1^T, array->voxels)":
             "beam_adjoint_tma" if stats["adjoint_box"] > 0 and adj_tuned == 1 else "beam_adjoint_batched"}[dom]
    lv = levels[dom]
    mem = lv["memory_level"]
    peak = {"dram": peaks["hbm_GBps"], "l2": peaks["l2_GBps"], "smem": peaks["smem_GBps"]}[mem]
    achieved = lv["bytes"][mem] / (stage_ms[dom] * 1e-3) / 1e9
    roofline = {"bound": {"dram": "hbm"}.get(mem, mem), "kernel": kname, "achieved": achieved, "peak": peak,
                "unit": "GB/s", "frac": achieved / peak, "traffic": traffic_for(kname),
                "work": {"dram": "compulsory: every input read once, every output written once",
                         "l2": "per 32 x 32 target tile, cell and slice the voxel rectangle its footprints "
                               "touch, plus the array plane once",
                         "smem": "4 B of operand per nonzero (pixel, cell, voxel) entry",
                         "fp32": "one FMA per nonzero entry"}[mem],
                "peak_source": "measured by the library's microbenchmark in this run (of measured)",
                "binding_level": lv["binding"], "fp32_frac": lv["fp32_frac"]}

    # --- a2: the rotation passes of a yawed camera (HBM-bound streams) ---
    shear = shear_passes(flush, stream)

    # --- the multi-view and differentiable workloads (rank 0, outside the timed region) ---
    extra = {}
    if rank == 0:
        for name in [w for w in args.workloads.split(",") if w]:
            fn = {"multiview": workload_multiview, "differentiable": workload_differentiable}[name]
            extra[name] = fn(args.workload_steps, 3, stream)

    # --- time-to-residual, warm start vs plain (rank 0 only, outside the timed region) ---
    ttr = time_to_residual(plan, args.warm_samples, n_eval=args.warm_eval) if rank == 0 and args.warm_samples > 0 else None

    # --- end to end through the public API: pinned host y in, volume and data fit out ---
    # Streaming use of the API, NB steps in flight: step i + NB - 1's
    # measurements are copied from pinned host memory on one copy stream
    # while step i iterates (a 4 MB host-to-device copy takes about 0.35 ms
    # on its own, more than one step); after step i the reconstructed volume
    # is copied into a device staging buffer (lt_recon_get, no
    # synchronisation) and from there into pinned host memory on another
    # stream, and the data fit and gains come back asynchronously into
    # pinned memory; the host reads step i's fit and volume NB - 1 steps
    # later.  Every step's copy in and result reads happen inside the timed
    # region.
    NB = 3
    y_pin = torch.from_numpy(y_host.reshape(1, -1)).pin_memory()
    nfr, ncam = plan.frames, len(plan.cams)
    y_stage = [torch.empty_like(y_dev) for _ in range(NB)]
    x_stage = [torch.empty(nfr, plan.nvox, dtype=torch.float32, device="cuda") for _ in range(NB)]
    x_host = [torch.empty(nfr, plan.nvox, dtype=torch.float32).pin_memory() for _ in range(NB)]
    res = [torch.empty(nfr * (ncam + 1), dtype=torch.float64).pin_memory() for _ in range(NB)]
    # one stream per direction, so that measurements come in while volumes
    # go out (the host link is full duplex)
    h2d_stream, d2h_stream = torch.cuda.Stream(), torch.cuda.Stream()
    comp = torch.cuda.current_stream()
    h2d_done = [torch.cuda.Event() for _ in range(NB)]
    consumed = [torch.cuda.Event() for _ in range(NB)]
    step_done = [torch.cuda.Event() for _ in range(NB)]
    x_staged = [torch.cuda.Event() for _ in range(NB)]
    x_home = [torch.cuda.Event() for _ in range(NB)]

    def e2e_run(n):
        fits, vol_sums = [], []

        def fetch(j):   # step j's measurements into y_stage[j % NB]
            b = j % NB
            with torch.cuda.stream(h2d_stream):
                if j >= NB:
                    h2d_stream.wait_event(consumed[b])   # its last reader was step j - NB
                y_stage[b].copy_(y_pin, non_blocking=True)
                h2d_done[b].record(h2d_stream)

        def collect(j):   # step j's results, on the host
            b = j % NB
            step_done[b].synchronize()
            x_home[b].synchronize()
            fits.append(float(res[b][0]))
            vol_sums.append(float(x_host[b][0, :: 4096].sum()))

        for j in range(min(NB - 1, n)):
            fetch(j)
        for i in range(n):
            b = i % NB
            comp.wait_event(h2d_done[b])
            rec.set_data(y_stage[b])
            consumed[b].record(comp)
            if i + NB - 1 < n:
                fetch(i + NB - 1)
            rec.iterate(1)
            if i >= NB:
                comp.wait_event(x_home[b])                 # step i - NB's volume has left x_stage[b]
            rec.copy_x(x_stage[b])
            x_staged[b].record(comp)
            rec.get_async(res[b])
            step_done[b].record(comp)
            with torch.cuda.stream(d2h_stream):
                d2h_stream.wait_event(x_staged[b])
                x_host[b].copy_(x_stage[b], non_blocking=True)
                x_home[b].record(d2h_stream)
            if i >= NB - 1:
                collect(i - (NB - 1))
        for j in range(max(0, n - (NB - 1)), n):
            collect(j)
        return fits, vol_sums

    e2e_run(3)
    torch.cuda.synchronize()
    if world > 1:
        dist.barrier()
    e0 = time.perf_counter()
    fits, vol_sums = e2e_run(args.e2e_steps)
    torch.cuda.synchronize()
    te = time.perf_counter() - e0
    assert len(fits) == args.e2e_steps and all(np.isfinite(fits)) and all(np.isfinite(vol_sums))
    e2e = {"value": job_rate(samples_step, args.e2e_steps, world, max_over_ranks(te, "cuda")), "unit": UNIT,
           "h2d_bytes_per_step": int(y_pin.numel() * 4),
           "d2h_bytes_per_step": int(8 * nfr * (ncam + 1) + 4 * nfr * plan.nvox),
           "steps": args.e2e_steps,
           "path": "pinned host y -> device copy (its own stream, three buffers, issued two steps ahead), "
                   "lt_recon_set_data, lt_recon_iterate(1), lt_recon_get(x) into a device staging buffer, "
                   "volume -> pinned host memory on a second copy stream (the two directions overlap), "
                   "lt_recon_get_async(data fit, gains) into pinned memory; both read on the host two steps later"}

    cpu = None
    if rank == 0 and world == 1 and not args.no_cpu_baseline:
        cpu = cpu_baseline_sample(vol, cam, x_true)

    if rank == 0:
        out = {
            "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": t_max / args.steps * 1e3, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "f32", "data": "synthetic",
            "config": {"workload": WORKLOAD, "volume": [vol.nx, vol.ny, vol.nz], "detector": [cam.det_ns, cam.det_nt],
                       "array_plane": [cam.arr_ns, cam.arr_nt], "cells": stats["n_cells"],
                       "ray_samples_per_step": samples_step, "hit_fraction_stage1": stats["hit_samples"] / stats["stage1_samples"],
                       "beta": beta, "l2": "flushed (512 MB write) between timed iterations",
                       "frames_per_rank": 1, "parallelism": f"replicas x{world}" if world > 1 else "single",
                       "forward_variant": tuned, "autotune_ms": tune_ms,
                       "adjoint_variant": adj_tuned, "adjoint_autotune_ms": adj_tune_ms,
                       "forward_brick": stats["forward_brick"], "adjoint_box": stats["adjoint_box"]},
            "stages_ms": stage_ms,
            "roofline": roofline,
            "peaks": peaks,
            "levels": levels,
            "shear_passes": shear,
            "workloads": extra,
            "time_to_residual": ttr,
            "cpu_baseline": cpu,
            "clocks": clk.summary(),
            "e2e": e2e,
            "gpu_launches": kpi * args.steps,
            "wall_s_timed_region": wall,
        }
        print(json.dumps(out), flush=True)
    if world > 1:
        dist.destroy_process_group()


# ---------------------------------------------------------------------------
# reference arm: the FP64 oracle on the host cores, bounded samples
# ---------------------------------------------------------------------------

def run_reference(args):
    rank, world, _ = dist_env()
    if rank != 0:
        return
    from paper_1812_03358_b300 import inputs as I

    vol, cam = I.config_plenoptic()
    x = I.plume_field(vol, seed=2000)
    for _ in range(args.warmup):
        oracle_cell_sample(vol, cam, x)
    t = 0.0
    for _ in range(args.steps):
        dt, samples, n_cells = oracle_cell_sample(vol, cam, x)
        t += dt
    cores = blas_threads()
    value = samples * args.steps / t
    out = {"impl": "reference", "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world,
           "steps": args.steps, "warmup": args.warmup, "ms_per_step": t / args.steps * 1e3,
           "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
           "data": "synthetic", "config": {"workload": WORKLOAD},
           "cpu_baseline": {"value": value, "unit": UNIT, "cores": cores, "kind": "oracle",
                            "sample": f"per step: FP64 forward + adjoint of one of the workload's {n_cells} angular "
                                      f"cells (both stages, all slices; {samples:.3g} ray-samples)"},
           "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(out), flush=True)


def main():
    args = parse()
    if args.impl == "reference":
        run_reference(args)
    else:
        run_ours(args)


if __name__ == "__main__":
    main()
