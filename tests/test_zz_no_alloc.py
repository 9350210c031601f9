"""The allocation-free plenoptic forward (lt_forward_camera_noalloc), called
through the C ABI, against the regular lt_forward_camera.

It serves callers that cannot allocate device memory where they project
(memory-pool-managed frameworks that forbid raw cudaMalloc, real-time loops
that must not allocate or synchronise); its array-plane intermediate lives
in a static device array that every call shares.  Checked here: two calls
in a row match the regular forward; once the first call on the device has
loaded the array, further calls leave the device's free memory unchanged;
a call on a smaller plan right after a larger plan filled the array with
other data is unaffected by those stale contents; a rotated plenoptic camera
is served; oversize requests and single-lens cameras are refused.  This file
is collected last on purpose."""
import math

import numpy as np
import pytest

torch = pytest.importorskip("torch")

from paper_1812_03358_b300 import build, inputs as I, lt

pytestmark = pytest.mark.gpu

TOL = 1e-5


def rel_l2(a, b):
    return float(np.linalg.norm(a.ravel() - b.ravel()) / np.linalg.norm(b.ravel()))


def _both(plan, cam, x, stream):
    """(allocation-free result, regular result) of camera 0 of `plan`."""
    y_ref = torch.empty(plan.frames, cam.m, device="cuda")
    y_na = torch.full((plan.frames, cam.m), float("nan"), device="cuda")
    lt.lt_forward_camera(plan.handle, 0, x.data_ptr(), y_ref.data_ptr(), stream)
    lt.lt_forward_camera_noalloc(plan.handle, 0, x.data_ptr(), y_na.data_ptr(), stream)
    torch.cuda.synchronize()
    return y_na.cpu().numpy().astype(np.float64), y_ref.cpu().numpy().astype(np.float64)


def test_noalloc_forward_matches_regular_forward_twice():
    build.build()
    vol, cam = I.config_plenoptic()
    plan = lt.Plan(vol, [cam])
    stream = torch.cuda.current_stream().cuda_stream
    for seed in (2000, 2003):   # two calls in a row, different inputs
        x = torch.from_numpy(I.plume_field(vol, seed=seed).reshape(1, -1)).cuda()
        a, b = _both(plan, cam, x, stream)
        assert np.all(np.isfinite(a))
        assert rel_l2(a, b) < TOL
    plan.close()


def test_noalloc_reserves_nothing_after_its_first_call():
    build.build()
    vol, cam = I.config_plenoptic()
    plan = lt.Plan(vol, [cam])
    stream = torch.cuda.current_stream().cuda_stream
    x = torch.from_numpy(I.plume_field(vol, seed=2001).reshape(1, -1)).cuda()
    y = torch.empty(1, cam.m, device="cuda")
    lt.lt_forward_camera_noalloc(plan.handle, 0, x.data_ptr(), y.data_ptr(), stream)   # loads the array
    torch.cuda.synchronize()
    free0, _ = torch.cuda.mem_get_info()
    for _ in range(3):
        lt.lt_forward_camera_noalloc(plan.handle, 0, x.data_ptr(), y.data_ptr(), stream)
    torch.cuda.synchronize()
    free1, _ = torch.cuda.mem_get_info()
    assert free1 == free0
    plan.close()


def test_noalloc_ignores_stale_contents_of_a_larger_plan():
    build.build()
    stream = torch.cuda.current_stream().cuda_stream
    # the full-size plan fills the whole array (4 cells x 10^6 array pixels) with its plane
    vol, cam = I.config_plenoptic()
    big = lt.Plan(vol, [cam])
    xb = torch.from_numpy(I.plume_field(vol, seed=2002).reshape(1, -1)).cuda() * 7.0
    yb = torch.empty(1, cam.m, device="cuda")
    lt.lt_forward_camera_noalloc(big.handle, 0, xb.data_ptr(), yb.data_ptr(), stream)
    torch.cuda.synchronize()
    # then a smaller plenoptic camera (60 x 60 lenslets of 8 x 8 px, 3 x 3 cells),
    # yawed, over a 64^3 volume, which reads a prefix of the array in another layout
    v2 = I.Volume(64, 64, 64, 2.0, 2.0, 2.0)
    c2 = I.plenoptic_camera(n_lenslets=60, px_per_lenslet=8, pitch_px=0.025, ks=3, kt=3)
    c2.yaw = math.radians(20.0)
    small = lt.Plan(v2, [c2])
    x2 = torch.from_numpy(I.plume_field(v2, seed=2004).reshape(1, -1)).cuda()
    a, b = _both(small, c2, x2, stream)
    assert np.all(np.isfinite(a)) and np.abs(b).max() > 0
    assert rel_l2(a, b) < TOL
    assert np.abs(a - b).max() <= TOL * np.abs(b).max()
    big.close()
    small.close()


def test_noalloc_rejects_oversize_and_single_lens():
    build.build()
    vol, cam = I.config_plenoptic()
    plan2 = lt.Plan(vol, [cam], frames=2)          # 2 x 4 x 10^6 floats > 4 Mi
    x = torch.zeros(2, vol.n, device="cuda")
    y = torch.zeros(2, cam.m, device="cuda")
    with pytest.raises(lt.LtError) as e:
        lt.lt_forward_camera_noalloc(plan2.handle, 0, x.data_ptr(), y.data_ptr(), 0)
    assert e.value.status == lt.LT_EINVAL and "exceeds the static scratch" in str(e.value)
    v1, c1 = I.config_single_small()
    p1 = lt.Plan(v1, [c1])
    x1 = torch.zeros(1, v1.n, device="cuda")
    y1 = torch.zeros(1, c1.m, device="cuda")
    with pytest.raises(lt.LtError) as e:
        lt.lt_forward_camera_noalloc(p1.handle, 0, x1.data_ptr(), y1.data_ptr(), 0)
    assert e.value.status == lt.LT_EINVAL
    plan2.close()
    p1.close()
