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
FP32_PEAK_TFLOPS = 148 * 128 * 2 * 2.032e9 / 1e12   # SMs x FP32 lanes x FMA x max SM clock


def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=1000)
    ap.add_argument("--warmup", type=int, default=5)
    ap.add_argument("--impl", choices=["ours", "reference"], default="ours")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--e2e-steps", type=int, default=200)
    ap.add_argument("--warm-samples", type=int, default=6000,
                    help="training volumes for the warm-start time-to-residual measurement (0: skip)")
    ap.add_argument("--no-autotune", action="store_true",
                    help="pin --forward-variant instead of tuning (fixed launch sequence, e.g. for profiling)")
    ap.add_argument("--forward-variant", type=int, default=2,
                    help="forward kernel variant pinned by --no-autotune (the plan's default is 2)")
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

class ClockSampler:
    """Samples the SM clock and clock-event reasons of the benchmarked GPU
    while the timed region runs (NVML reads; nvidia-smi as a fallback)."""
    REASONS = {
        "applications_clocks_setting": 0x2, "sw_power_cap": 0x4, "hw_slowdown": 0x8,
        "sync_boost": 0x10, "sw_thermal_slowdown": 0x20, "hw_thermal_slowdown": 0x40,
        "hw_power_brake_slowdown": 0x80,
    }

    def __init__(self, device, period=0.02):
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
            self.nvml = pynvml
        except Exception as e:  # fall back to nvidia-smi
            self.errors.append("nvml: " + repr(e))

    def _run_nvml(self):
        nv = self.nvml
        while not self._stop.is_set():
            try:
                self.samples.append(nv.nvmlDeviceGetClockInfo(self.h, nv.NVML_CLOCK_SM))
                mask = nv.nvmlDeviceGetCurrentClocksEventReasons(self.h)
                for name, bit in self.REASONS.items():
                    if mask & bit:
                        self.reasons.add(name)
            except Exception as e:
                self.errors.append(repr(e))
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
               "samples": len(self.samples), "source": "nvml" if self.nvml else "nvidia-smi"}
        if not self.samples:
            out["errors"] = self.errors[:3]
        return out


# ---------------------------------------------------------------------------
# our arm
# ---------------------------------------------------------------------------

def traffic_for(kernel):
    """DRAM bytes per launch of `kernel` from the committed ncu summary, if the
    kernel source has not changed since the counters were taken."""
    path = os.path.join(ROOT, "profiles", "ncu_traffic.json")
    src = os.path.join(ROOT, "paper_1812_03358_b300", "csrc", "lt_kernels.cu")
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


def time_to_residual(plan, n_samples, n_plain=200, n_eval=5):
    """Warm start vs plain solver on the bench workload: the U-Net is trained
    here for n_samples volumes made by the projector (seeds 1e6 + i), then both
    arms run on n_eval held-out volumes (seeds 2e6 + j): wall time (CUDA
    events) until the data fit reaches the plain solver's n_plain-iteration
    value, the warm arm including back-projection and U-Net inference (not
    training).  Reported: the median over the held-out volumes of each figure,
    and every volume's gain."""
    import statistics
    import time as _t
    from paper_1812_03358_b300 import unet, warmstart
    t0 = _t.time()
    ws, losses = warmstart.train(plan, unet.UNet(seed=1), n_samples, lr=1e-3)
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
            "gain_per_volume": gains, "volume_error_plain": med("err_plain"),
            "volume_error_warm_x0": med("err_x0"), "train_samples": n_samples, "train_s": round(t_train, 1),
            "beta": "1e-3 * mean(D)", "held_out_seeds": [2_000_000 + j for j in range(n_eval)],
            "statistic": "median over the held-out volumes"}


def cpu_baseline_sample(vol, cam, x):
    """The FP64 oracle, as it stands, on one projector + adjoint pass of the
    full workload (its BLAS threads on the host cores)."""
    from oracle import camera as O
    try:
        from threadpoolctl import threadpool_info
        cores = max(d.get("num_threads", 1) for d in threadpool_info()) if threadpool_info() else 1
    except Exception:
        cores = os.cpu_count()
    t0 = time.perf_counter()
    y = O.plenoptic_forward(vol, cam, x)
    O.plenoptic_adjoint(vol, cam, y)
    return time.perf_counter() - t0, cores


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
    else:
        tuned, tune_ms = plan.autotune()
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
    nnz = {"beam_forward (stage 1, slices->array)": stats["stage1_nnz"],
           "stage2_forward (array->detector)": stats["stage2_nnz"],
           "stage2_adjoint (detector->array)": stats["stage2_nnz"],
           "beam_adjoint (stage 1^T, array->voxels)": stats["stage1_nnz"]}
    dom = max(stage_ms, key=stage_ms.get)
    achieved = 2.0 * nnz[dom] / (stage_ms[dom] * 1e-3) / 1e12
    kname = {"beam_forward (stage 1, slices->array)": "beam_forward_batched",
             "stage2_forward (array->detector)": "stage2_lenslet_forward",
             "stage2_adjoint (detector->array)": "stage2_lenslet_adjoint",
             "beam_adjoint (stage 1^T, array->voxels)": "beam_adjoint_batched"}[dom]
    roofline = {"bound": "alu", "kernel": kname, "achieved": achieved, "peak": FP32_PEAK_TFLOPS,
                "unit": "TFLOP/s", "frac": achieved / FP32_PEAK_TFLOPS, "traffic": traffic_for(kname),
                "work": "2 flop (one FMA) per nonzero (pixel, cell, voxel) entry evaluated",
                "peak_source": "148 SMs x 128 FP32 lanes x 2 flop x 2.032 GHz (unit counts and max clock)"}

    # --- a2: the rotation passes of a yawed camera (HBM-bound streams) ---
    shear = shear_passes(flush, stream)

    # --- time-to-residual, warm start vs plain (rank 0 only, outside the timed region) ---
    ttr = time_to_residual(plan, args.warm_samples) if rank == 0 and args.warm_samples > 0 else None

    # --- end to end through the public API: pinned host y in, data fit out ---
    # Streaming use of the API: step i + 1's measurements are copied from
    # pinned host memory on a copy stream (double buffer) while step i
    # iterates, and step i's data fit and gains come back asynchronously into
    # pinned memory and are read on the host one step later.  Every step's
    # copy in and result read happen inside the timed region.
    y_pin = torch.from_numpy(y_host.reshape(1, -1)).pin_memory()
    nfr, ncam = plan.frames, len(plan.cams)
    y_stage = [torch.empty_like(y_dev) for _ in range(2)]
    res = [torch.empty(nfr * (ncam + 1), dtype=torch.float64).pin_memory() for _ in range(2)]
    copy_stream = torch.cuda.Stream()
    comp = torch.cuda.current_stream()
    h2d_done = [torch.cuda.Event() for _ in range(2)]
    consumed = [torch.cuda.Event() for _ in range(2)]
    step_done = [torch.cuda.Event() for _ in range(2)]

    def e2e_run(n):
        fits = []
        with torch.cuda.stream(copy_stream):
            y_stage[0].copy_(y_pin, non_blocking=True)
            h2d_done[0].record(copy_stream)
        for i in range(n):
            cur, nxt = i % 2, (i + 1) % 2
            comp.wait_event(h2d_done[cur])
            rec.set_data(y_stage[cur])
            consumed[cur].record(comp)
            if i + 1 < n:
                with torch.cuda.stream(copy_stream):
                    copy_stream.wait_event(consumed[nxt])   # its last reader was step i - 1
                    y_stage[nxt].copy_(y_pin, non_blocking=True)
                    h2d_done[nxt].record(copy_stream)
            rec.iterate(1)
            rec.get_async(res[cur])
            step_done[cur].record(comp)
            if i >= 1:
                step_done[nxt].synchronize()               # step i - 1's result is on the host
                fits.append(float(res[nxt][0]))
        step_done[(n - 1) % 2].synchronize()
        fits.append(float(res[(n - 1) % 2][0]))
        return fits

    e2e_run(3)
    torch.cuda.synchronize()
    if world > 1:
        dist.barrier()
    e0 = time.perf_counter()
    fits = e2e_run(args.e2e_steps)
    torch.cuda.synchronize()
    te = time.perf_counter() - e0
    assert len(fits) == args.e2e_steps and all(np.isfinite(fits))
    e2e = {"value": job_rate(samples_step, args.e2e_steps, world, max_over_ranks(te, "cuda")), "unit": UNIT,
           "h2d_bytes_per_step": int(y_pin.numel() * 4), "d2h_bytes_per_step": int(8 * nfr * (ncam + 1)),
           "steps": args.e2e_steps,
           "path": "pinned host y -> device copy (copy stream, double buffered, overlapping the previous step), "
                   "lt_recon_set_data, lt_recon_iterate(1), lt_recon_get_async(data fit, gains) into pinned "
                   "memory, read on the host one step later"}

    cpu = None
    if rank == 0 and world == 1 and not args.no_cpu_baseline:
        t_cpu, cores = cpu_baseline_sample(vol, cam, x_true)
        cpu = {"value": 2 * stats["ray_samples"] / t_cpu, "unit": UNIT, "cores": cores, "kind": "oracle",
               "sample": f"one FP64 forward + adjoint of the full workload ({t_cpu:.1f} s, numpy/OpenBLAS threads)"}

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
                       "forward_variant": tuned, "autotune_ms": tune_ms},
            "stages_ms": stage_ms,
            "roofline": roofline,
            "shear_passes": shear,
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
    from oracle import camera as O
    from paper_1812_03358_b300 import inputs as I

    vol, cam = I.config_plenoptic()
    x = I.plume_field(vol, seed=2000)
    # sample: stage-1 forward and adjoint of one angular cell over the central
    # 16-slice slab (slices 56..71 keep their true depths: the slab is centred
    # on the volume centre, so d_obj is unchanged)
    slab = I.Volume(vol.nx, vol.ny, 16, vol.dx, vol.dy, vol.dz)
    xs = x.reshape(vol.shape)[56:72]
    cell = O.lens_cells(cam)[0]
    g = np.ones((cam.arr_nt, cam.arr_ns))

    def step():
        O.plenoptic_array_field(slab, cam, xs, cell)
        Ga = g / O.array_basis_volume(cam, cell)
        out = np.zeros(slab.shape)
        for n in range(slab.nz):
            Bs, Bt = O.slice_operators(slab, cam, n, cell, cam.d_lens_mla, cam.arr_ns, cam.arr_nt,
                                       cam.arr_ps, cam.arr_pt)
            out[n] = slab.dz * (Bt.T @ Ga @ Bs)
        return out

    for _ in range(args.warmup):
        step()
    t0 = time.perf_counter()
    for _ in range(args.steps):
        step()
    t = time.perf_counter() - t0
    samples = 2 * cam.arr_ns * cam.arr_nt * 16
    try:
        from threadpoolctl import threadpool_info
        cores = max(d.get("num_threads", 1) for d in threadpool_info())
    except Exception:
        cores = os.cpu_count()
    value = samples * args.steps / t
    out = {"impl": "reference", "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world,
           "steps": args.steps, "warmup": args.warmup, "ms_per_step": t / args.steps * 1e3,
           "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
           "data": "synthetic", "config": {"workload": WORKLOAD},
           "cpu_baseline": {"value": value, "unit": UNIT, "cores": cores, "kind": "oracle",
                            "sample": "per step: FP64 stage-1 forward + adjoint of one angular cell over the central 16 of 128 slices"},
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
