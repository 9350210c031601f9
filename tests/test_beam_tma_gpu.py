"""The brick-staged forward (volume bricks brought to shared memory by TMA
by a producer warp, contracted by four consumer warps) against the FP64 oracle and against the direct beam
kernel, through the C ABI.

Plans use the brick-staged kernel by default (forward variant 5) wherever
the planner could size its bricks and the source rows are a multiple of 4
floats; lt_camera_stats reports the brick size (0 = direct kernel).  The
projector's device status word must stay 0 (no brick or band overflow, no
TMA wait that gave up)."""
import numpy as np
import pytest

torch = pytest.importorskip("torch")

from oracle import camera as O
from paper_1812_03358_b300 import build, inputs as I, lt

pytestmark = pytest.mark.gpu

TOL = 1e-5
TMA, DIRECT = 5, 2


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
    lt.lt_projector_status(clear=True)
    yield
    assert lt.lt_projector_status() == 0


def dev(a):
    return torch.from_numpy(np.ascontiguousarray(a, dtype=np.float32)).cuda()


def host(t):
    torch.cuda.synchronize()
    return t.detach().cpu().numpy().astype(np.float64)


def _cases():
    vol, cam = I.config_single_small()
    yield "32^3 -> 64^2, one cell", vol, cam, True
    yield "40x36x12 -> ragged 45x37, 2x2 cells", I.Volume(40, 36, 12, 3.0, 3.2, 5.0), \
        I.Camera(kind=0, det_ns=45, det_nt=37, det_ps=0.09, det_pt=0.08, ks=2, kt=2), True
    c = I.table_single_lens(44, 0.1, ks=3, kt=3)
    yield "coarse pixels (wide band), 3x3 cells", I.Volume(16, 20, 10, 4.0, 4.0, 4.0), c, True
    c = I.table_single_lens(36, 0.09, ks=8, kt=8)
    yield "8x8 cell grid (more cells than lanes)", I.Volume(20, 16, 10, 4.0, 4.0, 5.0), c, True
    c = I.table_single_lens(40, 0.08, ks=2, kt=1)
    c.basis = I.BASIS_DIRAC
    yield "Dirac cells", I.Volume(24, 16, 9, 3.0, 3.0, 5.0), c, True
    yield "odd row length keeps the direct kernel", I.Volume(13, 11, 7, 4.0, 4.5, 6.0), \
        I.Camera(kind=0, det_ns=37, det_nt=23, det_ps=0.31, det_pt=0.27, ks=2, kt=2), False


@pytest.mark.parametrize("case", list(_cases()), ids=lambda c: c[0])
def test_brick_forward_matches_oracle(case):
    _, vol, cam, staged = case
    plan = lt.Plan(vol, [cam])
    assert (plan.stats(0)["forward_brick"] > 0) == staged
    x = I.gaussian_blobs(vol, seed=1000)
    yo = O.single_forward(vol, cam, x).ravel()
    for variant in (TMA, DIRECT):
        lt.lt_plan_set_forward_variant(plan.handle, variant)
        yg = host(plan.forward(dev(x).reshape(1, -1)))
        assert rel_l2(yg, yo) < TOL, (variant, rel_l2(yg, yo))
        assert close_elementwise(yg, yo), variant
    plan.close()


def test_both_t_contraction_forms_match_oracle():
    """Two-tap footprints take the per-row t-contraction, three-tap ones the
    band form (four pixel rows per lane over shared band rows); both against
    the oracle elementwise."""
    forms = set()
    # coarse voxels: two taps; 0.5 mm voxels 128 mm deep before a 5 um
    # detector (the multi-view cameras' geometry, small): defocus gives three
    # taps while four pixel rows still step through two voxel rows
    for vol, cam in ((I.Volume(24, 20, 10, 3.0, 3.0, 4.0), I.table_single_lens(48, 0.07, ks=2, kt=2)),
                     (I.Volume(16, 16, 8, 0.5, 0.5, 16.0), I.table_single_lens(64, 0.005, ks=2, kt=2))):
        plan = lt.Plan(vol, [cam])
        st = plan.stats(0)
        assert st["forward_brick"] > 0
        forms.add(st["forward_band"])
        x = I.gaussian_blobs(vol, seed=1005)
        yo = O.single_forward(vol, cam, x).ravel()
        yg = host(plan.forward(dev(x).reshape(1, -1)))
        assert rel_l2(yg, yo) < TOL and close_elementwise(yg, yo), st
        plan.close()
    assert forms == {0, 1}, forms


def test_brick_forward_frames_are_independent():
    vol = I.Volume(20, 16, 12, 4.0, 4.0, 5.0)
    cams = [I.table_single_lens(36, 0.09), I.table_single_lens(28, 0.11, ks=2, kt=2)]
    frames = 3
    xs = np.stack([I.gaussian_blobs(vol, seed=1200 + f).ravel() for f in range(frames)])
    plan = lt.Plan(vol, cams, frames)
    assert all(plan.stats(c)["forward_brick"] > 0 for c in range(len(cams)))
    yg = host(plan.forward(dev(xs)))
    for f in range(frames):
        for c, cam in enumerate(cams):
            a, b = plan.offsets[c], plan.offsets[c + 1]
            yo = O.single_forward(vol, cam, xs[f]).ravel()
            assert rel_l2(yg[f, a:b], yo) < TOL and close_elementwise(yg[f, a:b], yo)
    plan.close()


def test_brick_forward_tiny_plenoptic_array_plane():
    vol, cam = I.tiny_plenoptic()
    plan = lt.Plan(vol, [cam])
    assert plan.stats(0)["forward_brick"] > 0
    x = I.gaussian_blobs(vol, seed=1001)
    fa_g = host(plan.stage1(0, dev(x).reshape(1, -1)))[0]
    fa_o = np.stack([O.plenoptic_array_field(vol, cam, x, cell) for cell in O.lens_cells(cam)])
    assert rel_l2(fa_g, fa_o) < TOL and close_elementwise(fa_g, fa_o)
    plan.close()


def test_brick_forward_full_size_plenoptic_equals_direct_kernel():
    vol, cam = I.config_plenoptic()
    plan = lt.Plan(vol, [cam])
    assert plan.stats(0)["forward_brick"] > 0
    x = dev(I.plume_field(vol, seed=2000).reshape(1, -1))
    out = {}
    for variant in (TMA, DIRECT):
        lt.lt_plan_set_forward_variant(plan.handle, variant)
        out[variant] = host(plan.stage1(0, x))
    # the same entries summed in another order
    assert rel_l2(out[TMA], out[DIRECT]) < 1e-6
    assert close_elementwise(out[TMA], out[DIRECT], 1e-6)
    # pixels no footprint reaches are exact zeros in both
    assert np.array_equal(out[TMA] == 0, out[DIRECT] == 0)
    plan.close()


def test_brick_forward_is_deterministic_and_status_clean():
    vol, cam = I.config_plenoptic()
    plan = lt.Plan(vol, [cam])
    x = dev(I.plume_field(vol, seed=2001).reshape(1, -1))
    a = host(plan.forward(x))
    b = host(plan.forward(x))
    assert np.array_equal(a, b)
    assert lt.lt_projector_status() == 0
    plan.close()


# ---------------------------------------------------------------------------
# the box-staged adjoint (image boxes brought to shared memory by TMA once per
# voxel tile, cell and chunk of slices)
# ---------------------------------------------------------------------------

@pytest.mark.parametrize("case", list(_cases()), ids=lambda c: c[0])
def test_box_adjoint_matches_oracle(case):
    _, vol, cam, staged = case
    plan = lt.Plan(vol, [cam])
    # the adjoint stages image boxes: its rows must be a multiple of 4 floats too
    assert (plan.stats(0)["adjoint_box"] > 0) == (staged and cam.det_ns % 4 == 0)
    y = I.uniform_random(cam.m, seed=29)
    xo = O.single_adjoint(vol, cam, y).ravel()
    for variant in (1, 0):
        lt.lt_plan_set_adjoint_variant(plan.handle, variant)
        xg = host(plan.adjoint(dev(y).reshape(1, -1)))
        assert rel_l2(xg, xo) < TOL, (variant, rel_l2(xg, xo))
        assert close_elementwise(xg, xo), variant
    plan.close()


def test_box_adjoint_frames_cameras_and_accumulation():
    vol = I.Volume(20, 16, 12, 4.0, 4.0, 5.0)
    cams = [I.table_single_lens(36, 0.09), I.table_single_lens(28, 0.11, ks=2, kt=2)]
    frames = 3
    plan = lt.Plan(vol, cams, frames)
    assert all(plan.stats(c)["adjoint_box"] > 0 for c in range(len(cams)))
    ys = np.stack([I.uniform_random(plan.m_total, seed=70 + f) for f in range(frames)])
    xg = host(plan.adjoint(dev(ys)))
    for f in range(frames):
        xo = sum(O.single_adjoint(vol, cam, ys[f, plan.offsets[c]:plan.offsets[c + 1]]).ravel()
                 for c, cam in enumerate(cams))
        assert rel_l2(xg[f], xo) < TOL and close_elementwise(xg[f], xo)
    plan.close()


def test_box_adjoint_full_size_plenoptic_equals_direct_kernel():
    vol, cam = I.config_plenoptic()
    plan = lt.Plan(vol, [cam])
    assert plan.stats(0)["adjoint_box"] > 0
    ga = dev(np.random.default_rng(3).random((1, plan.cells[0], cam.arr_nt, cam.arr_ns)))
    out = {}
    for variant in (1, 0):
        lt.lt_plan_set_adjoint_variant(plan.handle, variant)
        out[variant] = host(plan.stage1_adjoint(0, ga))
    assert rel_l2(out[1], out[0]) < 1e-6
    assert close_elementwise(out[1], out[0], 1e-6)
    y = dev(I.uniform_random(cam.m, seed=31).reshape(1, -1))
    a = host(plan.adjoint(y))
    b = host(plan.adjoint(y))
    assert np.array_equal(a, b)
    assert lt.lt_projector_status() == 0
    plan.close()
