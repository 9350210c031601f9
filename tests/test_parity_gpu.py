"""GPU parity: the CUDA projector / adjoint (through the C ABI) against the
FP64 oracle, element by element, on the same seeded inputs.

Tolerance: 1e-5 relative L2 for forward and adjoint (float32 accumulation
along beams against float64), per the stated target; elementwise checks use
|gpu - oracle| <= 1e-5 * max|oracle| + 1e-6 * |oracle|.
"""
import numpy as np
import pytest

torch = pytest.importorskip("torch")

from oracle import camera as O
from paper_1812_03358_b300 import build, inputs as I, lt

pytestmark = pytest.mark.gpu

TOL = 1e-5


def rel_l2(a, b):
    return float(np.linalg.norm(np.ravel(a) - np.ravel(b)) / np.linalg.norm(np.ravel(b)))


def close_elementwise(a, b, tol=TOL):
    a = np.ravel(a).astype(np.float64)
    b = np.ravel(b).astype(np.float64)
    return bool(np.all(np.abs(a - b) <= tol * np.abs(b).max() + 1e-6 * np.abs(b)))


@pytest.fixture(scope="module", autouse=True)
def _lib():
    build.build()
    lt.lib()
    assert torch.cuda.is_available()


def dev(a):
    return torch.from_numpy(np.ascontiguousarray(a, dtype=np.float32)).cuda()


def host(t):
    torch.cuda.synchronize()
    return t.detach().cpu().numpy().astype(np.float64)


def gpu_fwd_adj(vol, cam, x, y, frames=1):
    plan = lt.Plan(vol, [cam], frames)
    yg = host(plan.forward(dev(x).reshape(frames, -1)))
    xg = host(plan.adjoint(dev(y).reshape(frames, -1)))
    return plan, yg, xg


def _single_cases():
    vol1, cam1 = I.config_single_small()
    yield "32^3->64^2 K=1", vol1, cam1
    yield "ragged 13x11x7 -> 37x23 K=2x2", I.Volume(13, 11, 7, 4.0, 4.5, 6.0), \
        I.Camera(kind=0, det_ns=37, det_nt=23, det_ps=0.31, det_pt=0.27, ks=2, kt=2)
    c = I.table_single_lens(48, 0.12, ks=3, kt=2)
    c.basis = I.BASIS_DIRAC
    yield "dirac 3x2", I.Volume(20, 17, 9, 3.0, 3.0, 5.0), c
    c = I.table_single_lens(40, 0.2, ks=4, kt=4)
    yield "4x4 cells (corners cut by the aperture)", I.Volume(16, 16, 12, 4.0, 4.0, 4.0), c


@pytest.mark.parametrize("case", list(_single_cases()), ids=lambda c: c[0])
def test_single_lens_forward_adjoint_match_oracle(case):
    _, vol, cam = case
    x = I.gaussian_blobs(vol, seed=1000)
    y = I.uniform_random(cam.m, seed=17)
    _, yg, xg = gpu_fwd_adj(vol, cam, x, y)
    yo = O.single_forward(vol, cam, x).ravel()
    xo = O.single_adjoint(vol, cam, y).ravel()
    assert rel_l2(yg, yo) < TOL, rel_l2(yg, yo)
    assert rel_l2(xg, xo) < TOL, rel_l2(xg, xo)
    assert close_elementwise(yg, yo) and close_elementwise(xg, xo)


def test_single_lens_multiframe_and_multicamera():
    vol = I.Volume(12, 10, 8, 4.0, 4.0, 5.0)
    cams = [I.table_single_lens(30, 0.25), I.table_single_lens(20, 0.4, ks=2, kt=2)]
    frames = 3
    xs = np.stack([I.gaussian_blobs(vol, seed=1000 + f).ravel() for f in range(frames)])
    plan = lt.Plan(vol, cams, frames)
    yg = host(plan.forward(dev(xs)))
    ys = np.stack([I.uniform_random(plan.m_total, seed=50 + f) for f in range(frames)])
    xg = host(plan.adjoint(dev(ys)))
    for f in range(frames):
        for c, cam in enumerate(cams):
            a, b = plan.offsets[c], plan.offsets[c + 1]
            assert rel_l2(yg[f, a:b], O.single_forward(vol, cam, xs[f]).ravel()) < TOL
        xo = sum(O.single_adjoint(vol, cam, ys[f, plan.offsets[c]:plan.offsets[c + 1]]).ravel()
                 for c, cam in enumerate(cams))
        assert rel_l2(xg[f], xo) < TOL


def test_tiny_plenoptic_stages_and_operator():
    vol, cam = I.tiny_plenoptic()
    x = I.gaussian_blobs(vol, seed=1001)
    y = I.uniform_random(cam.m, seed=23)
    plan = lt.Plan(vol, [cam])
    fa_g = host(plan.stage1(0, dev(x).reshape(1, -1)))[0]
    fa_o = np.stack([O.plenoptic_array_field(vol, cam, x, cell) for cell in O.lens_cells(cam)])
    assert rel_l2(fa_g, fa_o) < TOL
    # stage 2 on identical inputs
    y2 = host(plan.stage2(0, dev(fa_g[None])))
    assert rel_l2(y2, O.plenoptic_stage2(cam, fa_g)) < TOL
    g_g = host(plan.stage2_adjoint(0, dev(y).reshape(1, -1)))[0]
    assert rel_l2(g_g, O.plenoptic_stage2_adjoint(cam, y)) < TOL
    x1 = host(plan.stage1_adjoint(0, dev(g_g[None])))
    assert rel_l2(x1, O.plenoptic_stage1_adjoint(vol, cam, g_g)) < TOL
    _, yg, xg = gpu_fwd_adj(vol, cam, x, y)
    assert rel_l2(yg, O.plenoptic_forward(vol, cam, x)) < TOL
    assert rel_l2(xg, O.plenoptic_adjoint(vol, cam, y)) < TOL


def test_explicit_matrix_columns_tiny():
    # A e_j for every voxel against the oracle's explicit matrix, and A^T e_i.
    vol = I.Volume(4, 3, 3, 5.0, 5.0, 6.0)
    cam = I.table_single_lens(10, 0.5, ks=2, kt=2)
    A = O.single_matrix(vol, cam)
    plan = lt.Plan(vol, [cam], frames=vol.n)
    E = np.eye(vol.n, dtype=np.float32)
    cols = host(plan.forward(dev(E)))           # frame j = A e_j
    assert np.abs(cols.T - A).max() <= TOL * np.abs(A).max()
    plan2 = lt.Plan(vol, [cam], frames=cam.m)
    rows = host(plan2.adjoint(dev(np.eye(cam.m, dtype=np.float32))))
    assert np.abs(rows - A).max() <= TOL * np.abs(A).max()


@pytest.fixture(scope="module")
def plenoptic_full():
    vol, cam = I.config_plenoptic()
    x = I.plume_field(vol, seed=2000)
    plan = lt.Plan(vol, [cam])
    return vol, cam, x, plan


def test_plenoptic_full_size_stage1_elementwise(plenoptic_full):
    vol, cam, x, plan = plenoptic_full
    fa_g = host(plan.stage1(0, dev(x).reshape(1, -1)))[0]
    for ci, cell in enumerate(O.lens_cells(cam)):
        fa_o = O.plenoptic_array_field(vol, cam, x, cell)
        assert rel_l2(fa_g[ci], fa_o) < TOL
        assert close_elementwise(fa_g[ci], fa_o)


def test_plenoptic_full_size_forward_adjoint(plenoptic_full):
    vol, cam, x, plan = plenoptic_full
    yg = host(plan.forward(dev(x).reshape(1, -1)))
    yo = O.plenoptic_forward(vol, cam, x)
    assert rel_l2(yg, yo) < TOL and close_elementwise(yg, yo)
    y = I.poisson_images(yo, 1e4, seed=5)
    xg = host(plan.adjoint(dev(y).reshape(1, -1)))
    xo = O.plenoptic_adjoint(vol, cam, y)
    assert rel_l2(xg, xo) < TOL and close_elementwise(xg, xo)


def test_dot_product_identity_full_size(plenoptic_full):
    vol, cam, x, plan = plenoptic_full
    rng = np.random.default_rng(0)
    xr = rng.random(vol.n).astype(np.float32)
    yr = rng.random(cam.m).astype(np.float32)
    ax = host(plan.forward(dev(xr).reshape(1, -1)))
    aty = host(plan.adjoint(dev(yr).reshape(1, -1)))
    lhs = float(np.dot(ax.ravel(), yr.astype(np.float64)))
    rhs = float(np.dot(xr.astype(np.float64), aty.ravel()))
    assert abs(lhs - rhs) <= 1e-6 * abs(lhs)


def test_forward_is_deterministic(plenoptic_full):
    vol, cam, x, plan = plenoptic_full
    a = host(plan.forward(dev(x).reshape(1, -1)))
    b = host(plan.forward(dev(x).reshape(1, -1)))
    assert np.array_equal(a, b)
