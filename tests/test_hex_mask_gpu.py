"""GPU parity of hexagonal three-focal microlens arrays and coded masks
(Sec. II-D, eq. occlusion) against the FP64 oracle: tiny and 400^2-pixel
hexagonal cameras, a square camera with a random coded mask, and mask
superposition on the GPU path."""
import numpy as np
import pytest

torch = pytest.importorskip("torch")

from oracle import camera as O
from paper_1812_03358_b300 import build, inputs as I, lt

pytestmark = pytest.mark.gpu

TOL = 1e-5


def rel_l2(a, b):
    return float(np.linalg.norm(np.ravel(a) - np.ravel(b)) / np.linalg.norm(np.ravel(b)))


@pytest.fixture(scope="module", autouse=True)
def _lib():
    build.build()
    lt.lib()


def dev(a):
    return torch.from_numpy(np.ascontiguousarray(a, dtype=np.float32)).cuda()


def host(t):
    torch.cuda.synchronize()
    return t.detach().cpu().numpy().astype(np.float64)


def check(vol, cam, seed):
    x = I.gaussian_blobs(vol, seed=seed)
    y = I.uniform_random(cam.m, seed=seed + 1)
    plan = lt.Plan(vol, [cam])
    yg = host(plan.forward(dev(x).reshape(1, -1)))
    xg = host(plan.adjoint(dev(y).reshape(1, -1)))
    assert rel_l2(yg, O.forward(vol, cam, x)) < TOL, rel_l2(yg, O.forward(vol, cam, x))
    assert rel_l2(xg, O.adjoint(vol, cam, y)) < TOL, rel_l2(xg, O.adjoint(vol, cam, y))
    return plan, x, y


def test_tiny_hexagonal_camera_matches_oracle():
    vol, cam = I.tiny_hex_plenoptic()
    check(vol, cam, 1100)


def test_hexagonal_camera_400px_matches_oracle():
    cam = I.hex_plenoptic_camera(n_cols=40, n_rows=46, n_px=400)
    vol = I.Volume(48, 48, 16, 2.5, 2.5, 8.0)
    check(vol, cam, 1102)


def test_coded_mask_matches_oracle_and_superposes():
    vol, cam = I.tiny_plenoptic()
    rng = np.random.default_rng(7)
    m = (rng.random((cam.arr_nt, cam.arr_ns)) < 0.6).astype(np.float32)
    cam.arr_mask = m
    plan_a, x, y = check(vol, cam, 1104)
    cam.arr_mask = 1.0 - m
    plan_b, _, _ = check(vol, cam, 1104)
    cam.arr_mask = None
    plan_c = lt.Plan(vol, [cam])
    xs, ys = dev(x).reshape(1, -1), dev(y).reshape(1, -1)
    sum_f = host(plan_a.forward(xs)) + host(plan_b.forward(xs))
    sum_a = host(plan_a.adjoint(ys)) + host(plan_b.adjoint(ys))
    assert rel_l2(sum_f, host(plan_c.forward(xs))) < 1e-6
    assert rel_l2(sum_a, host(plan_c.adjoint(ys))) < 1e-6
    # a fractional (grey) mask on the hexagonal camera
    hvol, hcam = I.tiny_hex_plenoptic()
    hcam.arr_mask = rng.random((hcam.arr_nt, hcam.arr_ns)).astype(np.float32)
    check(hvol, hcam, 1106)
