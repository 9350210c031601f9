"""GPU parity of rotated cameras (Sec. III-A: quarter turns + z/x shear
re-projections, then the aligned camera) against the FP64 oracle, forward and
adjoint, single-lens and plenoptic, and inside the reconstruction."""
import math

import numpy as np
import pytest

torch = pytest.importorskip("torch")

from oracle import camera as O
from oracle import recon as OR
from paper_1812_03358_b300 import build, inputs as I, lt

pytestmark = pytest.mark.gpu

TOL = 1e-5


def rel_l2(a, b):
    return float(np.linalg.norm(np.ravel(a) - np.ravel(b)) / np.linalg.norm(np.ravel(b)))


@pytest.fixture(scope="module", autouse=True)
def _lib():
    build.build()


def dev(a):
    return torch.from_numpy(np.ascontiguousarray(a, dtype=np.float32)).cuda()


def host(t):
    torch.cuda.synchronize()
    return t.detach().cpu().numpy().astype(np.float64)


@pytest.mark.parametrize("yaw", [0.3, -0.7, math.pi / 4, 1.9, math.pi / 2, 3.0, -2.2])
def test_rotated_single_lens_matches_oracle(yaw):
    vol = I.Volume(12, 9, 10, 4.0, 4.5, 5.0)
    cam = I.table_single_lens(28, 0.3, yaw=yaw, ks=2, kt=2)
    x = I.gaussian_blobs(vol, seed=1010)
    y = I.uniform_random(cam.m, seed=31)
    plan = lt.Plan(vol, [cam])
    yg = host(plan.forward(dev(x).reshape(1, -1)))
    xg = host(plan.adjoint(dev(y).reshape(1, -1)))
    yo = O.forward(vol, cam, x).ravel()
    xo = O.adjoint(vol, cam, y).ravel()
    assert rel_l2(yg, yo) < TOL, rel_l2(yg, yo)
    assert rel_l2(xg, xo) < TOL, rel_l2(xg, xo)


def test_rotated_plenoptic_matches_oracle():
    vol, cam = I.tiny_plenoptic()
    cam.yaw = 0.4
    x = I.gaussian_blobs(vol, seed=1011)
    y = I.uniform_random(cam.m, seed=32)
    plan = lt.Plan(vol, [cam])
    assert rel_l2(host(plan.forward(dev(x).reshape(1, -1))), O.forward(vol, cam, x)) < TOL
    assert rel_l2(host(plan.adjoint(dev(y).reshape(1, -1))), O.adjoint(vol, cam, y)) < TOL


def test_multiview_dot_product_identity():
    vol = I.Volume(64, 64, 64, 1.6, 1.6, 1.6)
    cams = [I.table_single_lens(128, 0.01, yaw=y, ks=2, kt=2) for y in (0.0, 0.5, 2.1, -1.2)]
    plan = lt.Plan(vol, cams)
    rng = np.random.default_rng(0)
    x = rng.random(vol.n).astype(np.float32)
    y = rng.random(plan.m_total).astype(np.float32)
    ax = host(plan.forward(dev(x).reshape(1, -1)))
    aty = host(plan.adjoint(dev(y).reshape(1, -1)))
    lhs = float(np.dot(ax.ravel(), y.astype(np.float64)))
    rhs = float(np.dot(x.astype(np.float64), aty.ravel()))
    assert abs(lhs - rhs) <= 1e-5 * abs(lhs)


def test_multiview_reconstruction_iterations_match_oracle():
    vol = I.Volume(12, 10, 12, 5.0, 5.0, 5.0)
    cams = [I.table_single_lens(24, 0.35, yaw=y) for y in (0.0, 0.9, -1.8)]
    x_true = I.gaussian_blobs(vol, seed=1012)
    ys = [O.forward(vol, c, x_true).ravel() for c in cams]
    ys[2] = ys[2] / 1.7
    plan = lt.Plan(vol, cams)
    rec = lt.Recon(plan, dev(np.concatenate(ys)).reshape(1, -1), beta=1e-4)
    rec.iterate(20)
    xg = host(rec.get()[0])
    ops = [(lambda v, c=c: O.forward(vol, c, v).ravel(), lambda r, c=c: O.adjoint(vol, c, r).ravel()) for c in cams]
    ref = OR.fista(ops, ys, [None] * 3, vol.shape, 20, beta=1e-4)
    assert rel_l2(xg, ref["x"]) < 1e-4


@pytest.mark.parametrize("yaw", [0.0, 0.3, -0.7, math.pi / 4, -math.pi / 4, 1.9, math.pi / 2, 3.0, -2.2])
def test_rotate_volume_and_adjoint_match_oracle(yaw):
    """The rotation passes alone (lt_rotate_volume / _adjoint) against the
    oracle's x^r = E^x E^z P x and its transpose, elementwise, on a ragged
    non-cubic grid; the camera grid equals the oracle's rotated grid."""
    check_rotation(I.Volume(13, 9, 11, 4.0, 4.5, 5.0), yaw)


@pytest.mark.parametrize("yaw", [2.1, -1.2])
def test_quarter_turn_passes_span_several_tiles(yaw):
    """One and three quarter turns take the transposed z adjoint (tiles of 32
    columns by 64 sources).  A 70 x 5 x 45 grid gives two column tiles (the
    second ragged) and two tiles along the sheared axis (the second ragged),
    checked elementwise against the oracle with the forward passes."""
    check_rotation(I.Volume(70, 5, 45, 4.0, 4.5, 5.0), yaw)


def check_rotation(vol, yaw):
    from oracle import rotation as OR_
    cam = I.table_single_lens(28, 0.3, yaw=yaw)
    plan = lt.Plan(vol, [cam])
    x = I.gaussian_blobs(vol, seed=1012).reshape(vol.shape) + 0.1 * I.uniform_random(vol.shape, seed=33)
    shp, sizes = plan.camera_grid(0)
    if yaw == 0.0:
        ref, (sx, sy, sz) = np.asarray(x, dtype=np.float64), (vol.dx, vol.dy, vol.dz)
    else:
        ref, (sx, sy, sz) = OR_.rotate(x, (vol.dx, vol.dy, vol.dz), yaw)
        oshape, osz, _ = OR_.rotated_grid(vol.shape, (vol.dx, vol.dy, vol.dz), yaw)
        assert tuple(shp) == tuple(oshape)
    assert tuple(shp) == ref.shape
    assert np.allclose(sizes, (sz, sy, sx), rtol=1e-12)
    xc = host(plan.rotate(0, dev(x).reshape(1, -1))).reshape(shp)
    assert np.abs(xc - ref).max() <= 1e-5 * np.abs(ref).max(), np.abs(xc - ref).max()
    g = I.uniform_random(int(np.prod(shp)), seed=34).reshape(shp)
    gref = np.asarray(g, dtype=np.float64) if yaw == 0.0 else \
        OR_.rotate_adjoint(g, vol.shape, (vol.dx, vol.dy, vol.dz), yaw)
    xa = host(plan.rotate_adjoint(0, dev(g).reshape(1, -1))).reshape(vol.shape)
    assert np.abs(xa - gref).max() <= 1e-5 * np.abs(gref).max()
    # accumulate adds onto what is there
    base = dev(x).reshape(1, -1)
    acc = host(plan.rotate_adjoint(0, dev(g).reshape(1, -1), x=base, accumulate=True)).reshape(vol.shape)
    assert np.abs(acc - (gref + x)).max() <= 1e-5 * np.abs(gref + x).max()
    # adjoint identity <R x, g> = <x, R^T g>
    lhs, rhs = float(np.vdot(xc, g)), float(np.vdot(x, xa))
    assert abs(lhs - rhs) <= 1e-5 * abs(lhs)


GENERAL = [(0.0, 0.35, 0.0), (0.0, 0.0, -0.5), (0.4, -0.3, 0.2), (2.5, 0.6, -1.1), (0.0, math.pi / 2, 0.0),
           (1.0, 0.0, math.pi / 2)]


@pytest.mark.parametrize("angles", GENERAL)
def test_general_rotation_matches_oracle(angles):
    """Pitch and roll (signed permutation + three shear passes) against the
    oracle's rotate_general and its transpose, elementwise, ragged grid."""
    from oracle import rotation as OR_
    vol = I.Volume(9, 7, 8, 4.0, 4.5, 5.0)
    cam = I.table_single_lens(28, 0.3, yaw=angles[0])
    cam.pitch, cam.roll = angles[1], angles[2]
    plan = lt.Plan(vol, [cam])
    x = I.gaussian_blobs(vol, seed=1013).reshape(vol.shape) + 0.1 * I.uniform_random(vol.shape, seed=35)
    T = OR_.camera_rotation(*angles)
    ref, (sx, sy, sz) = OR_.rotate_general(x, (vol.dx, vol.dy, vol.dz), T)
    shp, sizes = plan.camera_grid(0)
    assert tuple(shp) == ref.shape
    assert np.allclose(sizes, (sz, sy, sx), rtol=1e-12)
    xc = host(plan.rotate(0, dev(x).reshape(1, -1))).reshape(shp)
    assert np.abs(xc - ref).max() <= 1e-5 * np.abs(ref).max(), np.abs(xc - ref).max()
    g = I.uniform_random(int(np.prod(shp)), seed=36).reshape(shp)
    gref = OR_.rotate_general_adjoint(g, vol.shape, (vol.dx, vol.dy, vol.dz), T)
    xa = host(plan.rotate_adjoint(0, dev(g).reshape(1, -1))).reshape(vol.shape)
    assert np.abs(xa - gref).max() <= 1e-5 * np.abs(gref).max()


def test_pitched_and_rolled_cameras_match_oracle():
    vol = I.Volume(10, 9, 8, 4.0, 4.5, 5.0)
    cam = I.table_single_lens(28, 0.3, yaw=0.3, ks=2, kt=2)
    cam.pitch, cam.roll = 0.25, -0.35
    x = I.gaussian_blobs(vol, seed=1014)
    y = I.uniform_random(cam.m, seed=37)
    plan = lt.Plan(vol, [cam])
    assert rel_l2(host(plan.forward(dev(x).reshape(1, -1))), O.forward(vol, cam, x)) < TOL
    assert rel_l2(host(plan.adjoint(dev(y).reshape(1, -1))), O.adjoint(vol, cam, y)) < TOL
    pvol, pcam = I.tiny_plenoptic()
    pcam.pitch, pcam.roll = -0.2, 0.3
    px = I.gaussian_blobs(pvol, seed=1015)
    py = I.uniform_random(pcam.m, seed=38)
    pplan = lt.Plan(pvol, [pcam])
    assert rel_l2(host(pplan.forward(dev(px).reshape(1, -1))), O.forward(pvol, pcam, px)) < TOL
    assert rel_l2(host(pplan.adjoint(dev(py).reshape(1, -1))), O.adjoint(pvol, pcam, py)) < TOL
