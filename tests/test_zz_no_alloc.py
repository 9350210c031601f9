"""The allocation-free plenoptic forward (lt_forward_camera_noalloc), called
through the C ABI, matches the regular lt_forward_camera on two calls in a
row.  It serves callers that cannot allocate device memory where they
project; its intermediate lives in a static array shared by all calls.
This file is collected last on purpose."""
import numpy as np
import pytest

torch = pytest.importorskip("torch")

from paper_1812_03358_b300 import build, inputs as I, lt

pytestmark = pytest.mark.gpu

TOL = 1e-5


def rel_l2(a, b):
    return float(np.linalg.norm(a.ravel() - b.ravel()) / np.linalg.norm(b.ravel()))


def test_noalloc_forward_matches_regular_forward_twice():
    build.build()
    vol, cam = I.config_plenoptic()
    plan = lt.Plan(vol, [cam])
    stream = torch.cuda.current_stream().cuda_stream
    for seed in (2000, 2003):   # two calls in a row, different inputs
        x = torch.from_numpy(I.plume_field(vol, seed=seed).reshape(1, -1)).cuda()
        y_ref = torch.empty(1, cam.m, device="cuda")
        y_na = torch.full((1, cam.m), float("nan"), device="cuda")
        lt.lt_forward_camera(plan.handle, 0, x.data_ptr(), y_ref.data_ptr(), stream)
        lt.lt_forward_camera_noalloc(plan.handle, 0, x.data_ptr(), y_na.data_ptr(), stream)
        torch.cuda.synchronize()
        a, b = y_na.cpu().numpy().astype(np.float64), y_ref.cpu().numpy().astype(np.float64)
        assert np.all(np.isfinite(a))
        assert rel_l2(a, b) < TOL


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
