"""Degenerate sizes and limits of the projector: a single voxel seen by a
single pixel (one and four angular cells, pillbox and Dirac), a one-voxel
column seen by a one-pixel-high detector row, zero inputs giving exact zeros,
and the plan refusing cameras whose windows exceed the kernels' limits (a
host-side check, before any launch)."""
import numpy as np
import pytest

torch = pytest.importorskip("torch")

from oracle import camera as O
from paper_1812_03358_b300 import build, inputs as I, lt

pytestmark = pytest.mark.gpu

TOL = 1e-5


def host(t):
    torch.cuda.synchronize()
    return t.detach().cpu().numpy().astype(np.float64)


def dev(a):
    return torch.from_numpy(np.ascontiguousarray(a, dtype=np.float32)).cuda()


def _cases():
    yield "1 voxel, 1 pixel, K=1", I.Volume(1, 1, 1, 5.0, 5.0, 5.0), I.table_single_lens(1, 0.3)
    yield "1 voxel, 1 pixel, K=2x2", I.Volume(1, 1, 1, 5.0, 5.0, 5.0), I.table_single_lens(1, 0.3, ks=2, kt=2)
    c = I.table_single_lens(3, 0.2, ks=2, kt=1)
    c.basis = I.BASIS_DIRAC
    yield "1 voxel, 3x3 pixels, Dirac 2x1", I.Volume(1, 1, 1, 4.0, 4.0, 4.0), c
    c = I.Camera(kind=I.CAM_SINGLE, det_ns=37, det_nt=1, det_ps=0.05, det_pt=0.2, ks=2, kt=2)
    yield "1x1x9 column, 37x1 row", I.Volume(1, 1, 9, 3.0, 3.0, 3.0), c
    c = I.Camera(kind=I.CAM_SINGLE, det_ns=1, det_nt=29, det_ps=0.2, det_pt=0.05)
    yield "5x1x1 row, 1x29 column", I.Volume(5, 1, 1, 3.0, 3.0, 3.0), c


@pytest.mark.parametrize("case", list(_cases()), ids=lambda c: c[0])
def test_degenerate_sizes_match_oracle(case):
    build.build()
    _, vol, cam = case
    plan = lt.Plan(vol, [cam])
    x = I.uniform_random(vol.n, seed=5, lo=0.5, hi=1.0)
    y = I.uniform_random(cam.m, seed=6)
    yg = host(plan.forward(dev(x).reshape(1, -1))).ravel()
    xg = host(plan.adjoint(dev(y).reshape(1, -1))).ravel()
    yo = O.single_forward(vol, cam, x).ravel()
    xo = O.single_adjoint(vol, cam, y).ravel()
    assert np.abs(yo).max() > 0 and np.abs(xo).max() > 0   # the camera sees the volume
    assert np.all(np.abs(yg - yo) <= TOL * np.abs(yo).max() + 1e-6 * np.abs(yo))
    assert np.all(np.abs(xg - xo) <= TOL * np.abs(xo).max() + 1e-6 * np.abs(xo))
    plan.close()


def test_zero_inputs_give_exact_zeros():
    build.build()
    vol, cam = I.tiny_plenoptic()
    plan = lt.Plan(vol, [cam], 3)
    y = plan.forward(torch.zeros(3, plan.nvox, device="cuda"))
    x = plan.adjoint(torch.zeros(3, plan.m_total, device="cuda"))
    assert not bool(y.any()) and not bool(x.any())
    plan.close()


def test_windows_beyond_the_kernel_limits_are_refused():
    build.build()
    vol = I.Volume(16, 16, 16, 1.0, 1.0, 1.0)
    with pytest.raises(lt.LtError) as e:   # one pixel spans ~115 voxels: forward window
        lt.Plan(vol, [I.table_single_lens(8, 5.0)])
    assert "pixel footprint spans" in str(e.value)
    vol = I.Volume(8, 8, 8, 10.0, 10.0, 10.0)
    with pytest.raises(lt.LtError) as e:   # one voxel covers ~860 pixels: adjoint window
        lt.Plan(vol, [I.table_single_lens(64, 0.0005)])
    assert "covered by" in str(e.value)
