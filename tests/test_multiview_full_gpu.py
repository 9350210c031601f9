"""The batched multi-view workload at full size: four single-lens 2048 x 2048
cameras (2 x 2 cells) at seeded yaw in [0, 180) degrees and one 200 x 200
lenslet plenoptic camera around a 256^3 volume (0.5 mm voxels), 16 frames of
a drifting plume field, every camera x frame in one persistent launch.
Checked at this size: the batched launch equals per-camera launches bit for
bit; the adjoint identity <A x, y> = <x, A^T y>; every rotation conserves the
voxel sum; sampled rotated voxels of the first and last frames equal the
oracle's; a yawed camera's image equals the unrotated camera's image of the
rotated volume; sampled blocks of the plenoptic camera's array plane (every cell,
first and last frames) equal the oracle's; a CUDA graph of the autotuned
plan replays the eager result; the yawed cameras' box-staged adjoint (boxes
of four slices: their footprints drift too far over eight) equals the direct
gather adjoint."""
import numpy as np
import pytest

torch = pytest.importorskip("torch")

from oracle import camera as O
from oracle import rotation as OR_
from paper_1812_03358_b300 import build, inputs as I, lt

pytestmark = pytest.mark.gpu

FRAMES = 16


@pytest.fixture(scope="module")
def multiview():
    build.build()
    vol, cams = I.config_multiview()
    plan = lt.Plan(vol, cams, FRAMES)
    x = torch.stack([I.plume_field_torch(vol, seed=3100, drift_voxels=float(f)) for f in range(FRAMES)])
    yield vol, cams, plan, x.contiguous()
    plan.close()


def test_batched_forward_equals_per_camera(multiview):
    vol, cams, plan, x = multiview
    yb = plan.forward(x)
    for c in range(len(cams)):
        yc = plan.forward_camera(c, x)
        ys = yb[:, plan.offsets[c]:plan.offsets[c + 1]]
        assert torch.equal(ys, yc), f"camera {c}: max |diff| {float((ys - yc).abs().max())}"
    assert torch.isfinite(yb).all() and float(yb.abs().max()) > 0


def test_adjoint_identity(multiview):
    vol, cams, plan, x = multiview
    g = torch.Generator(device="cuda").manual_seed(17)
    xr = torch.rand(FRAMES, plan.nvox, device="cuda", generator=g)
    yr = torch.rand(FRAMES, plan.m_total, device="cuda", generator=g)
    lhs = float((plan.forward(xr).double() * yr.double()).sum())
    rhs = float((xr.double() * plan.adjoint(yr).double()).sum())
    assert abs(lhs - rhs) <= 1e-5 * abs(lhs)


def test_rotations_conserve_sum_and_match_oracle_samples(multiview):
    vol, cams, plan, x = multiview
    sizes = (vol.dx, vol.dy, vol.dz)
    rng = np.random.default_rng(23)
    for c, cam in enumerate(cams):
        if cam.kind != I.CAM_SINGLE:
            continue
        shp, _ = plan.camera_grid(c)
        assert shp == OR_.rotated_grid(vol.shape, sizes, cam.yaw)[0]
        xc = plan.rotate(c, x)
        s_in = x.double().sum(dim=1)
        s_out = xc.double().sum(dim=1)
        assert float(((s_out - s_in).abs() / s_in).max()) <= 1e-5
        idx = [(int(rng.integers(shp[0] // 4, 3 * shp[0] // 4)), int(rng.integers(0, shp[1])),
                int(rng.integers(shp[2] // 4, 3 * shp[2] // 4))) for _ in range(24)]
        flat = [(i * shp[1] + j) * shp[2] + k for i, j, k in idx]
        for f in (0, FRAMES - 1):
            xf = x[f].cpu().numpy().reshape(vol.shape)
            ref = OR_.rotate_voxels(xf, sizes, cam.yaw, idx)
            got = xc[f, flat].cpu().numpy().astype(np.float64)
            scale = float(np.abs(xf).max())
            assert np.all(np.abs(got - ref) <= 1e-5 * scale + 1e-6 * np.abs(ref))
        del xc


def test_rotated_camera_is_unrotated_camera_on_rotated_grid(multiview):
    """A yawed camera's image equals the image of the same camera at yaw 0
    looking at the rotated volume on the camera grid (the projection of
    an unrotated camera being pinned against the oracle elementwise)."""
    import dataclasses
    vol, cams, plan, x = multiview
    for c in (0, 2):
        (nz, ny, nx), (dz, dy, dx) = plan.camera_grid(c)
        plan_r = lt.Plan(I.Volume(nx, ny, nz, dx, dy, dz), [dataclasses.replace(cams[c], yaw=0.0)], FRAMES)
        xr = plan.rotate(c, x)
        y_r = plan_r.forward(xr)
        y_c = plan.forward_camera(c, x)
        scale = float(y_c.abs().max())
        assert scale > 0
        assert float((y_r - y_c).abs().max()) <= 1e-6 * scale
        plan_r.close()
        del xr, y_r, y_c


def test_plenoptic_array_blocks_match_oracle(multiview):
    vol, cams, plan, x = multiview
    c = next(i for i, cam in enumerate(cams) if cam.kind == I.CAM_PLENOPTIC)
    cam = cams[c]
    fa = plan.stage1(c, x)   # [frames][cells][arr_nt][arr_ns]
    rng = np.random.default_rng(29)
    for f in (0, FRAMES - 1):
        xf = x[f].cpu().numpy().reshape(vol.shape)
        for ci, cell in enumerate(O.lens_cells(cam)):
            rows = np.sort(rng.choice(np.arange(cam.arr_nt // 4, 3 * cam.arr_nt // 4), 3, replace=False))
            cols = np.sort(rng.choice(np.arange(cam.arr_ns // 4, 3 * cam.arr_ns // 4), 48, replace=False))
            ref = O.plenoptic_array_block(vol, cam, xf, cell, rows, cols)
            r_t = torch.as_tensor(rows, device="cuda")
            c_t = torch.as_tensor(cols, device="cuda")
            got = fa[f, ci].index_select(0, r_t).index_select(1, c_t).cpu().numpy().astype(np.float64)
            scale = float(np.abs(ref).max())
            assert scale > 0
            assert np.all(np.abs(got - ref) <= 1e-5 * scale + 1e-6 * np.abs(ref))


def test_graph_replay_of_autotuned_plan(multiview):
    vol, cams, plan, x = multiview
    chosen, times = plan.autotune()
    assert 0 <= chosen < len(times)
    y_eager = plan.forward(x)
    x_eager = plan.adjoint(y_eager)
    yo = torch.empty_like(y_eager)
    xo = torch.empty_like(x_eager)
    s = torch.cuda.Stream()
    s.wait_stream(torch.cuda.current_stream())
    with torch.cuda.stream(s):
        plan.forward(x, yo)
        plan.adjoint(yo, xo)
    torch.cuda.synchronize()
    gr = torch.cuda.CUDAGraph()
    with torch.cuda.graph(gr, stream=s):
        plan.forward(x, yo)
        plan.adjoint(yo, xo)
    yo.zero_()
    xo.zero_()
    gr.replay()
    torch.cuda.synchronize()
    assert torch.equal(yo, y_eager) and torch.equal(xo, x_eager)


def test_yawed_box_adjoint_equals_direct_gather(multiview):
    vol, cams, plan, x = multiview
    for c, cam in enumerate(cams):
        if cam.yaw == 0.0:
            continue
        st = plan.stats(c)
        assert st["adjoint_box"] > 0 and st["adjoint_chunk"] in (4, 8)
    yf = plan.forward(x)
    out = {}
    for variant in (1, 0):
        lt.lt_plan_set_adjoint_variant(plan.handle, variant)
        out[variant] = plan.adjoint(yf).double()
    lt.lt_plan_set_adjoint_variant(plan.handle, 1)
    a, b = out[1], out[0]
    assert float((a - b).norm() / b.norm()) < 1e-6
    assert bool(torch.all((a - b).abs() <= 1e-6 * b.abs().max() + 1e-6 * b.abs()))
    assert lt.lt_projector_status() == 0
