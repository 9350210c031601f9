"""Python binding of the C ABI in include/lt.h (argument marshalling only).

Every function named lt_* here calls the C entry point of the same name in
_lib/liblt.so; device pointers are passed as integers (e.g. tensor.data_ptr()).
The ``Plan`` class is a thin owner of a plan handle that accepts torch CUDA
tensors.  There is no fallback: if the library is missing, loading fails.
"""
from __future__ import annotations

import ctypes
import os
from ctypes import c_float, POINTER, byref, c_char_p, c_double, c_int32, c_int64, c_void_p

import numpy as np

from . import inputs

# The product library; with LT_TEST_HOOKS=1 in the environment the test build
# (the same library plus the fault-injection entry points of
# include/lt_testing.h) is loaded instead.
LIB_PATH = os.path.join(os.path.dirname(os.path.abspath(__file__)), "_lib",
                        "liblt_testhooks.so" if os.environ.get("LT_TEST_HOOKS") == "1" else "liblt.so")

LT_OK, LT_EINVAL, LT_ENOMEM, LT_ECUDA, LT_EUNSUPPORTED, LT_ETIMEOUT = range(6)


class lt_volume_desc(ctypes.Structure):
    _fields_ = [("nx", c_int32), ("ny", c_int32), ("nz", c_int32),
                ("dx", c_double), ("dy", c_double), ("dz", c_double)]


class lt_camera_desc(ctypes.Structure):
    _fields_ = [("kind", c_int32), ("basis", c_int32),
                ("f_main", c_double), ("r_main", c_double), ("d_obj", c_double), ("yaw", c_double),
                ("pitch", c_double), ("roll", c_double),
                ("det_ns", c_int32), ("det_nt", c_int32), ("det_ps", c_double), ("det_pt", c_double),
                ("d_lens_det", c_double), ("ks", c_int32), ("kt", c_int32),
                ("d_lens_mla", c_double), ("d_mla_det", c_double),
                ("mla_ns", c_int32), ("mla_nt", c_int32), ("mla_pitch", c_double),
                ("mla_radius", c_double), ("mla_focal", POINTER(c_double)),
                ("arr_ns", c_int32), ("arr_nt", c_int32), ("arr_ps", c_double), ("arr_pt", c_double),
                ("mla_layout", c_int32), ("arr_mask", POINTER(c_float))]


class lt_recon_params(ctypes.Structure):
    _fields_ = [("beta", c_double), ("nu", c_double), ("psi", c_int32), ("psi_delta", c_double),
                ("reg_scale", c_double), ("estimate_gains", c_int32), ("n_subset", c_int32)]


class lt_camera_stats(ctypes.Structure):
    _fields_ = [("n_cells", c_int64), ("stage1_samples", c_int64), ("stage2_samples", c_int64),
                ("ray_samples", c_int64), ("hit_samples", c_int64), ("stage1_nnz", c_int64),
                ("stage2_nnz", c_int64), ("stage1_tile_voxels", c_int64),
                ("forward_brick", c_int64), ("adjoint_box", c_int64), ("adjoint_chunk", c_int64),
                ("forward_band", c_int64)]


class LtError(RuntimeError):
    def __init__(self, status, msg):
        super().__init__(f"lt status {status}: {msg}")
        self.status = status


_lib = None

_SIGS = {
    "lt_plan_create": (c_int32, [POINTER(lt_volume_desc), POINTER(lt_camera_desc), c_int32, c_int32,
                                 POINTER(c_void_p)]),
    "lt_plan_destroy": (c_int32, [c_void_p]),
    "lt_plan_sizes": (c_int32, [c_void_p, POINTER(c_int64), POINTER(c_int64)]),
    "lt_forward": (c_int32, [c_void_p, c_void_p, c_void_p, c_void_p]),
    "lt_adjoint": (c_int32, [c_void_p, c_void_p, c_void_p, c_void_p]),
    "lt_forward_camera": (c_int32, [c_void_p, c_int32, c_void_p, c_void_p, c_void_p]),
    "lt_adjoint_camera": (c_int32, [c_void_p, c_int32, c_void_p, c_void_p, c_int32, c_void_p]),
    "lt_forward_camera_noalloc": (c_int32, [c_void_p, c_int32, c_void_p, c_void_p, c_void_p]),
    "lt_camera_cells": (c_int32, [c_void_p, c_int32, POINTER(c_int32)]),
    "lt_camera_grid": (c_int32, [c_void_p, c_int32, POINTER(lt_volume_desc)]),
    "lt_forward_subset": (c_int32, [c_void_p, c_void_p, c_void_p, c_int32, c_int32, c_void_p]),
    "lt_adjoint_subset": (c_int32, [c_void_p, c_void_p, c_void_p, c_int32, c_int32, c_void_p]),
    "lt_rotate_volume": (c_int32, [c_void_p, c_int32, c_void_p, c_void_p, c_void_p]),
    "lt_rotate_volume_adjoint": (c_int32, [c_void_p, c_int32, c_void_p, c_void_p, c_int32, c_void_p]),
    "lt_plenoptic_stage1": (c_int32, [c_void_p, c_int32, c_void_p, c_void_p, c_void_p]),
    "lt_plenoptic_stage1_adjoint": (c_int32, [c_void_p, c_int32, c_void_p, c_void_p, c_int32, c_void_p]),
    "lt_plenoptic_stage2": (c_int32, [c_void_p, c_int32, c_void_p, c_void_p, c_void_p]),
    "lt_plenoptic_stage2_adjoint": (c_int32, [c_void_p, c_int32, c_void_p, c_void_p, c_void_p]),
    "lt_recon_create": (c_int32, [c_void_p, c_void_p, c_void_p, POINTER(lt_recon_params), c_void_p,
                                  c_void_p, POINTER(c_void_p)]),
    "lt_recon_iterate": (c_int32, [c_void_p, c_int32, c_void_p]),
    "lt_recon_get": (c_int32, [c_void_p, c_void_p, POINTER(c_double), POINTER(c_double), c_void_p]),
    "lt_recon_get_async": (c_int32, [c_void_p, c_void_p, c_void_p]),
    "lt_recon_iterations": (c_int32, [c_void_p, POINTER(c_int64)]),
    "lt_recon_state_size": (c_int32, [c_void_p, POINTER(c_int64)]),
    "lt_recon_get_state": (c_int32, [c_void_p, c_void_p]),
    "lt_recon_set_state": (c_int32, [c_void_p, c_void_p]),
    "lt_recon_destroy": (c_int32, [c_void_p]),
    "lt_camera_stats_get": (c_int32, [c_void_p, c_int32, POINTER(lt_camera_stats)]),
    "lt_recon_set_data": (c_int32, [c_void_p, c_void_p, c_void_p, c_void_p]),
    "lt_recon_kernels_per_iteration": (c_int32, [c_void_p, POINTER(c_int32)]),
    "lt_autotune_variants": (c_int32, []),
    "lt_plan_autotune": (c_int32, [c_void_p, c_void_p, POINTER(c_double), POINTER(c_int32)]),
    "lt_plan_set_forward_variant": (c_int32, [c_void_p, c_int32]),
    "lt_projector_status": (c_int32, [POINTER(c_int32), c_int32]),
    "lt_plan_set_adjoint_variant": (c_int32, [c_void_p, c_int32]),
    "lt_plan_autotune_adjoint": (c_int32, [c_void_p, c_void_p, POINTER(c_double), POINTER(c_int32)]),
    "lt_last_error": (c_char_p, []),
    "lt_peak_smem_read": (c_int32, [c_void_p, c_int32, c_int32, c_void_p, POINTER(c_double)]),
    "lt_peak_l2_read": (c_int32, [c_void_p, c_int64, c_void_p, c_int32, c_int32, c_void_p, POINTER(c_double)]),
    "lt_peak_fp32_fma": (c_int32, [c_void_p, c_int32, c_int32, c_void_p, POINTER(c_double)]),
}


def lib():
    """Load liblt.so (built in-tree); raises if it has not been built."""
    global _lib
    if _lib is None:
        if not os.path.exists(LIB_PATH):
            raise RuntimeError(f"{LIB_PATH} is missing: build it with "
                               "`python -m paper_1812_03358_b300.build` (no CPU fallback exists)")
        L = ctypes.CDLL(LIB_PATH)
        for name, (res, args) in _SIGS.items():
            fn = getattr(L, name)
            fn.restype = res
            fn.argtypes = args
        if hasattr(L, "lt_test_fail_allocation_after"):   # the test build
            L.lt_test_fail_allocation_after.restype = None
            L.lt_test_fail_allocation_after.argtypes = [c_int32]
        _lib = L
    return _lib


def _check(status):
    if status != LT_OK:
        raise LtError(status, lib().lt_last_error().decode())


def lt_last_error() -> str:
    return lib().lt_last_error().decode()


def volume_desc(vol: inputs.Volume) -> lt_volume_desc:
    return lt_volume_desc(vol.nx, vol.ny, vol.nz, vol.dx, vol.dy, vol.dz)


def camera_desc(cam: inputs.Camera, keep: list) -> lt_camera_desc:
    d = lt_camera_desc()
    for name, _ in lt_camera_desc._fields_:
        if name in ("mla_focal", "arr_mask"):
            continue
        setattr(d, name, getattr(cam, name))
    if cam.mla_focal is not None:
        arr = np.ascontiguousarray(cam.mla_focal, dtype=np.float64)
        keep.append(arr)
        d.mla_focal = arr.ctypes.data_as(POINTER(c_double))
    if getattr(cam, "arr_mask", None) is not None:
        m = np.ascontiguousarray(cam.arr_mask, dtype=np.float32).reshape(-1)
        keep.append(m)
        d.arr_mask = m.ctypes.data_as(POINTER(c_float))
    return d


def lt_plan_create(vol: inputs.Volume, cams, n_frames: int = 1) -> c_void_p:
    keep = []
    cams = list(cams)
    arr = (lt_camera_desc * len(cams))(*[camera_desc(c, keep) for c in cams])
    v = volume_desc(vol)
    h = c_void_p()
    _check(lib().lt_plan_create(byref(v), arr, len(cams), n_frames, byref(h)))
    return h


def lt_plan_destroy(plan) -> None:
    _check(lib().lt_plan_destroy(plan))


def lt_plan_sizes(plan, n_cams: int):
    nv = c_int64()
    offs = (c_int64 * (n_cams + 1))()
    _check(lib().lt_plan_sizes(plan, byref(nv), offs))
    return nv.value, list(offs)


def lt_forward(plan, x_ptr: int, y_ptr: int, stream: int = 0) -> None:
    _check(lib().lt_forward(plan, x_ptr, y_ptr, stream))


def lt_adjoint(plan, y_ptr: int, x_ptr: int, stream: int = 0) -> None:
    _check(lib().lt_adjoint(plan, y_ptr, x_ptr, stream))


def lt_forward_camera(plan, cam: int, x_ptr: int, y_ptr: int, stream: int = 0) -> None:
    _check(lib().lt_forward_camera(plan, cam, x_ptr, y_ptr, stream))


def lt_adjoint_camera(plan, cam: int, y_ptr: int, x_ptr: int, accumulate: int = 0, stream: int = 0) -> None:
    _check(lib().lt_adjoint_camera(plan, cam, y_ptr, x_ptr, accumulate, stream))


def lt_forward_camera_noalloc(plan, cam: int, x_ptr: int, y_ptr: int, stream: int = 0) -> None:
    _check(lib().lt_forward_camera_noalloc(plan, cam, x_ptr, y_ptr, stream))


def lt_camera_cells(plan, cam: int) -> int:
    k = c_int32()
    _check(lib().lt_camera_cells(plan, cam, byref(k)))
    return k.value


def lt_forward_subset(plan, x_ptr, y_ptr, n_subset, subset, stream=0):
    _check(lib().lt_forward_subset(plan, x_ptr, y_ptr, n_subset, subset, stream))


def lt_adjoint_subset(plan, y_ptr, x_ptr, n_subset, subset, stream=0):
    _check(lib().lt_adjoint_subset(plan, y_ptr, x_ptr, n_subset, subset, stream))


def lt_camera_grid(plan, cam: int) -> lt_volume_desc:
    g = lt_volume_desc()
    _check(lib().lt_camera_grid(plan, cam, byref(g)))
    return g


def lt_rotate_volume(plan, cam, x_ptr, xc_ptr, stream=0):
    _check(lib().lt_rotate_volume(plan, cam, x_ptr, xc_ptr, stream))


def lt_rotate_volume_adjoint(plan, cam, xc_ptr, x_ptr, accumulate=0, stream=0):
    _check(lib().lt_rotate_volume_adjoint(plan, cam, xc_ptr, x_ptr, accumulate, stream))


def lt_plenoptic_stage1(plan, cam, x_ptr, fa_ptr, stream=0):
    _check(lib().lt_plenoptic_stage1(plan, cam, x_ptr, fa_ptr, stream))


def lt_plenoptic_stage1_adjoint(plan, cam, fa_ptr, x_ptr, accumulate=0, stream=0):
    _check(lib().lt_plenoptic_stage1_adjoint(plan, cam, fa_ptr, x_ptr, accumulate, stream))


def lt_plenoptic_stage2(plan, cam, fa_ptr, y_ptr, stream=0):
    _check(lib().lt_plenoptic_stage2(plan, cam, fa_ptr, y_ptr, stream))


def lt_plenoptic_stage2_adjoint(plan, cam, y_ptr, fa_ptr, stream=0):
    _check(lib().lt_plenoptic_stage2_adjoint(plan, cam, y_ptr, fa_ptr, stream))


def lt_plan_autotune(plan, stream: int = 0):
    n = lib().lt_autotune_variants()
    times = (c_double * n)()
    chosen = c_int32()
    _check(lib().lt_plan_autotune(plan, stream, times, byref(chosen)))
    return chosen.value, list(times)


def lt_test_fail_allocation_after(n: int) -> None:
    """Fault injection (test build only, LT_TEST_HOOKS=1): the n-th device
    allocation from now on fails (LT_ENOMEM); n <= 0 turns it off."""
    lib().lt_test_fail_allocation_after(int(n))


def lt_projector_status(clear: bool = False) -> int:
    """Device status word of the projector kernels (0 after correct runs);
    synchronises the device."""
    f = c_int32()
    _check(lib().lt_projector_status(byref(f), int(clear)))
    return f.value


def lt_plan_autotune_adjoint(plan, stream: int = 0):
    """Times both adjoint kernel choices and keeps the faster; returns
    (chosen, [direct ms, box-staged ms])."""
    times = (c_double * 2)()
    chosen = c_int32(0)
    _check(lib().lt_plan_autotune_adjoint(plan, stream, times, byref(chosen)))
    return chosen.value, list(times)


def lt_plan_set_adjoint_variant(plan, variant: int) -> None:
    """1: box-staged adjoint where the camera fits it (default); 0: direct."""
    _check(lib().lt_plan_set_adjoint_variant(plan, variant))


def lt_plan_set_forward_variant(plan, variant: int) -> None:
    _check(lib().lt_plan_set_forward_variant(plan, variant))


def lt_camera_stats_get(plan, cam: int) -> dict:
    st = lt_camera_stats()
    _check(lib().lt_camera_stats_get(plan, cam, byref(st)))
    return {name: getattr(st, name) for name, _ in lt_camera_stats._fields_}


def lt_recon_set_data(rec, y_ptr: int, w_ptr: int = 0, stream: int = 0) -> None:
    _check(lib().lt_recon_set_data(rec, y_ptr, w_ptr or None, stream))


def lt_recon_kernels_per_iteration(rec) -> int:
    n = c_int32()
    _check(lib().lt_recon_kernels_per_iteration(rec, byref(n)))
    return n.value


def lt_recon_create(plan, y_ptr: int, w_ptr: int, params: lt_recon_params, x0_ptr: int = 0,
                    stream: int = 0) -> c_void_p:
    h = c_void_p()
    _check(lib().lt_recon_create(plan, y_ptr, w_ptr or None, byref(params), x0_ptr or None, stream, byref(h)))
    return h


def lt_recon_iterate(rec, n_iter: int, stream: int = 0) -> None:
    _check(lib().lt_recon_iterate(rec, n_iter, stream))


def lt_recon_get(rec, x_ptr: int, n_frames: int, n_cams: int, stream: int = 0):
    gains = (c_double * (n_frames * n_cams))()
    fit = (c_double * n_frames)()
    _check(lib().lt_recon_get(rec, x_ptr or None, gains, fit, stream))
    return np.array(gains).reshape(n_frames, n_cams), np.array(fit)


def lt_recon_get_x(rec, x_ptr: int, stream: int = 0) -> None:
    """Enqueues a device-to-device copy of x into x_ptr (lt_recon_get with
    NULL gains and data fit: no synchronisation)."""
    _check(lib().lt_recon_get(rec, x_ptr, None, None, stream))


def lt_recon_get_async(rec, host_ptr: int, stream: int = 0) -> None:
    """Enqueues the data fit [F] and gains [F][n_cams] into the (page-locked)
    host buffer at host_ptr; valid once the stream has passed this point."""
    _check(lib().lt_recon_get_async(rec, host_ptr, stream))


def lt_recon_iterations(rec) -> int:
    n = c_int64()
    _check(lib().lt_recon_iterations(rec, byref(n)))
    return n.value


def lt_recon_get_state(rec) -> bytes:
    n = c_int64()
    _check(lib().lt_recon_state_size(rec, byref(n)))
    buf = ctypes.create_string_buffer(n.value)
    _check(lib().lt_recon_get_state(rec, buf))
    return buf.raw


def lt_recon_set_state(rec, state: bytes) -> None:
    buf = ctypes.create_string_buffer(state, len(state))
    _check(lib().lt_recon_set_state(rec, buf))


def lt_recon_destroy(rec) -> None:
    _check(lib().lt_recon_destroy(rec))


def lt_peak_smem_read(sink_ptr: int, ctas: int, reps: int, stream: int = 0) -> float:
    """Launches the shared-memory read microbenchmark (include/lt_peaks.h);
    returns the bytes it reads."""
    b = c_double()
    _check(lib().lt_peak_smem_read(sink_ptr, ctas, reps, stream, byref(b)))
    return b.value


def lt_peak_l2_read(buf_ptr: int, n16: int, sink_ptr: int, ctas: int, reps: int, stream: int = 0) -> float:
    """Launches the L2 read microbenchmark over buf[n16] 16-byte words;
    returns the bytes it reads."""
    b = c_double()
    _check(lib().lt_peak_l2_read(buf_ptr, n16, sink_ptr, ctas, reps, stream, byref(b)))
    return b.value


def lt_peak_fp32_fma(sink_ptr: int, ctas: int, reps: int, stream: int = 0) -> float:
    """Launches the FP32 FMA microbenchmark; returns its flops."""
    f = c_double()
    _check(lib().lt_peak_fp32_fma(sink_ptr, ctas, reps, stream, byref(f)))
    return f.value


# ---------------------------------------------------------------------------
# torch convenience wrapper (plumbing: allocation and the current stream)
# ---------------------------------------------------------------------------

def _stream():
    import torch
    return torch.cuda.current_stream().cuda_stream


def _dev_f32(t, numel, what):
    import torch
    if not (isinstance(t, torch.Tensor) and t.is_cuda and t.dtype == torch.float32 and t.is_contiguous()):
        raise TypeError(f"{what} must be a contiguous float32 CUDA tensor")
    if t.numel() != numel:
        raise ValueError(f"{what} has {t.numel()} elements, expected {numel}")
    return t.data_ptr()


class Plan:
    """Owner of an lt_plan handle for a volume and a list of cameras."""

    def __init__(self, vol: inputs.Volume, cams, frames: int = 1):
        self.vol = vol
        self.cams = list(cams)
        self.frames = frames
        self.handle = lt_plan_create(vol, self.cams, frames)
        self.nvox, self.offsets = lt_plan_sizes(self.handle, len(self.cams))
        self.m_total = self.offsets[-1]
        self.cells = [lt_camera_cells(self.handle, c) for c in range(len(self.cams))]

    def close(self):
        if self.handle is not None:
            lt_plan_destroy(self.handle)
            self.handle = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def new_x(self):
        import torch
        return torch.empty(self.frames, self.nvox, device="cuda", dtype=torch.float32)

    def new_y(self):
        import torch
        return torch.empty(self.frames, self.m_total, device="cuda", dtype=torch.float32)

    def forward(self, x, y=None):
        y = self.new_y() if y is None else y
        lt_forward(self.handle, _dev_f32(x, self.frames * self.nvox, "x"),
                   _dev_f32(y, self.frames * self.m_total, "y"), _stream())
        return y

    def adjoint(self, y, x=None):
        x = self.new_x() if x is None else x
        lt_adjoint(self.handle, _dev_f32(y, self.frames * self.m_total, "y"),
                   _dev_f32(x, self.frames * self.nvox, "x"), _stream())
        return x

    def forward_subset(self, x, n_subset, subset, y=None):
        """sum over the cells k % n_subset == subset of every camera (Sec. V)."""
        y = self.new_y() if y is None else y
        lt_forward_subset(self.handle, _dev_f32(x, self.frames * self.nvox, "x"),
                          _dev_f32(y, self.frames * self.m_total, "y"), n_subset, subset, _stream())
        return y

    def adjoint_subset(self, y, n_subset, subset, x=None):
        x = self.new_x() if x is None else x
        lt_adjoint_subset(self.handle, _dev_f32(y, self.frames * self.m_total, "y"),
                          _dev_f32(x, self.frames * self.nvox, "x"), n_subset, subset, _stream())
        return x

    def forward_camera(self, cam, x, y=None):
        import torch
        m = self.offsets[cam + 1] - self.offsets[cam]
        y = torch.empty(self.frames, m, device="cuda", dtype=torch.float32) if y is None else y
        lt_forward_camera(self.handle, cam, _dev_f32(x, self.frames * self.nvox, "x"),
                          _dev_f32(y, self.frames * m, "y"), _stream())
        return y

    def adjoint_camera(self, cam, y, x=None, accumulate=False):
        m = self.offsets[cam + 1] - self.offsets[cam]
        x = self.new_x() if x is None else x
        lt_adjoint_camera(self.handle, cam, _dev_f32(y, self.frames * m, "y"),
                          _dev_f32(x, self.frames * self.nvox, "x"), int(accumulate), _stream())
        return x

    def autotune(self):
        """Times the forward kernel variants on this plan and keeps the fastest."""
        return lt_plan_autotune(self.handle, _stream())

    def autotune_adjoint(self):
        """Times the adjoint kernel choices on this plan and keeps the faster."""
        return lt_plan_autotune_adjoint(self.handle, _stream())

    def stats(self, cam):
        return lt_camera_stats_get(self.handle, cam)

    def camera_grid(self, cam):
        """(nz, ny, nx) and (dz, dy, dx) of camera cam's rotated grid."""
        g = lt_camera_grid(self.handle, cam)
        return (g.nz, g.ny, g.nx), (g.dz, g.dy, g.dx)

    def rotate(self, cam, x, xc=None):
        """x_c = E^x E^z P x on camera cam's grid (Sec. III-A)."""
        import torch
        shp, _ = self.camera_grid(cam)
        n = int(np.prod(shp))
        xc = torch.empty(self.frames, n, device="cuda", dtype=torch.float32) if xc is None else xc
        lt_rotate_volume(self.handle, cam, _dev_f32(x, self.frames * self.nvox, "x"),
                         _dev_f32(xc, self.frames * n, "xc"), _stream())
        return xc

    def rotate_adjoint(self, cam, xc, x=None, accumulate=False):
        shp, _ = self.camera_grid(cam)
        n = int(np.prod(shp))
        x = self.new_x() if x is None else x
        lt_rotate_volume_adjoint(self.handle, cam, _dev_f32(xc, self.frames * n, "xc"),
                                 _dev_f32(x, self.frames * self.nvox, "x"), int(accumulate), _stream())
        return x

    def array_shape(self, cam):
        c = self.cams[cam]
        return (self.frames, self.cells[cam], c.arr_nt, c.arr_ns)

    def stage1(self, cam, x, fa=None):
        import torch
        shp = self.array_shape(cam)
        fa = torch.empty(shp, device="cuda", dtype=torch.float32) if fa is None else fa
        lt_plenoptic_stage1(self.handle, cam, _dev_f32(x, self.frames * self.nvox, "x"),
                            _dev_f32(fa, int(np.prod(shp)), "fa"), _stream())
        return fa

    def stage1_adjoint(self, cam, fa, x=None, accumulate=False):
        shp = self.array_shape(cam)
        x = self.new_x() if x is None else x
        lt_plenoptic_stage1_adjoint(self.handle, cam, _dev_f32(fa, int(np.prod(shp)), "fa"),
                                    _dev_f32(x, self.frames * self.nvox, "x"), int(accumulate), _stream())
        return x

    def stage2(self, cam, fa, y=None):
        import torch
        shp = self.array_shape(cam)
        m = self.offsets[cam + 1] - self.offsets[cam]
        y = torch.empty(self.frames, m, device="cuda", dtype=torch.float32) if y is None else y
        lt_plenoptic_stage2(self.handle, cam, _dev_f32(fa, int(np.prod(shp)), "fa"),
                            _dev_f32(y, self.frames * m, "y"), _stream())
        return y

    def stage2_adjoint(self, cam, y, fa=None):
        import torch
        shp = self.array_shape(cam)
        m = self.offsets[cam + 1] - self.offsets[cam]
        fa = torch.empty(shp, device="cuda", dtype=torch.float32) if fa is None else fa
        lt_plenoptic_stage2_adjoint(self.handle, cam, _dev_f32(y, self.frames * m, "y"),
                                    _dev_f32(fa, int(np.prod(shp)), "fa"), _stream())
        return fa


class Recon:
    """Owner of an lt_recon handle (Table V solver) for a Plan and measurements y."""

    def __init__(self, plan: Plan, y, w=None, beta=0.0, nu=0.0, psi=0, psi_delta=1.0,
                 reg_scale=26.0, estimate_gains=True, x0=None, n_subset=1):
        self.plan = plan
        n = plan.frames * plan.m_total
        prm = lt_recon_params(float(beta), float(nu), int(psi), float(psi_delta), float(reg_scale),
                              int(bool(estimate_gains)), int(n_subset))
        self.handle = lt_recon_create(plan.handle, _dev_f32(y, n, "y"),
                                      _dev_f32(w, n, "w") if w is not None else 0, prm,
                                      _dev_f32(x0, plan.frames * plan.nvox, "x0") if x0 is not None else 0,
                                      _stream())

    def iterate(self, n_iter: int):
        lt_recon_iterate(self.handle, n_iter, _stream())

    def set_data(self, y, w=None):
        n = self.plan.frames * self.plan.m_total
        lt_recon_set_data(self.handle, _dev_f32(y, n, "y"), _dev_f32(w, n, "w") if w is not None else 0,
                          _stream())

    def kernels_per_iteration(self) -> int:
        return lt_recon_kernels_per_iteration(self.handle)

    def get(self, x=None):
        x = self.plan.new_x() if x is None else x
        gains, fit = lt_recon_get(self.handle, _dev_f32(x, self.plan.frames * self.plan.nvox, "x"),
                                  self.plan.frames, len(self.plan.cams), _stream())
        return x, gains, fit

    def copy_x(self, x):
        """Enqueues a copy of the current x into the device tensor x on the
        current stream (no synchronisation)."""
        lt_recon_get_x(self.handle, _dev_f32(x, self.plan.frames * self.plan.nvox, "x"), _stream())

    def get_async(self, out):
        """Enqueues [data_fit[F], gains[F][n_cams]] into `out`, a page-locked
        float64 host tensor of F * (n_cams + 1) values, on the current stream
        (read it after an event or a synchronise)."""
        import torch
        n = self.plan.frames * (len(self.plan.cams) + 1)
        if out.device.type != "cpu" or out.dtype != torch.float64 or out.numel() < n or not out.is_pinned():
            raise ValueError(f"get_async needs a pinned float64 host tensor of {n} values")
        lt_recon_get_async(self.handle, out.data_ptr(), _stream())

    @property
    def iterations(self):
        return lt_recon_iterations(self.handle)

    def state(self) -> bytes:
        return lt_recon_get_state(self.handle)

    def load_state(self, state: bytes):
        lt_recon_set_state(self.handle, state)

    def close(self):
        if self.handle is not None:
            lt_recon_destroy(self.handle)
            self.handle = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass
