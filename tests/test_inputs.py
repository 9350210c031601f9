"""The seeded workload generators: the full-size configurations have the
sizes they are named for, and the torch plume generator (used for GPU-side
inputs) evaluates the same plumes as the numpy recipe (with turbulence off,
so that only the shared PCG64 parameter draws matter), drift included."""
import math

import numpy as np
import pytest

torch = pytest.importorskip("torch")

from paper_1812_03358_b300 import inputs as I


def test_multiview_configuration():
    vol, cams = I.config_multiview()
    assert (vol.nx, vol.ny, vol.nz, vol.dx) == (256, 256, 256, 0.5)
    single = [c for c in cams if c.kind == I.CAM_SINGLE]
    plen = [c for c in cams if c.kind == I.CAM_PLENOPTIC]
    assert len(single) == 4 and len(plen) == 1
    assert all(c.det_ns == c.det_nt == 2048 and 0.0 <= c.yaw < math.pi for c in single)
    assert (plen[0].mla_ns, plen[0].mla_nt) == (200, 200)
    assert len({c.yaw for c in single}) == 4
    again = I.config_multiview()[1]
    assert [c.yaw for c in again] == [c.yaw for c in cams]


def test_differentiable_configuration():
    vol, cams = I.config_differentiable()
    assert (vol.nx, vol.ny, vol.nz) == (256, 256, 256)
    assert len(cams) == 4 and all(c.det_ns == c.det_nt == 1024 for c in cams)
    assert np.allclose([c.yaw for c in cams], np.deg2rad([0, 45, 90, 135]))


@pytest.mark.parametrize("drift", [0.0, 3.0])
def test_torch_plumes_match_numpy_recipe(drift):
    vol = I.Volume(24, 20, 16, 1.0, 1.0, 1.0)
    a = I.plume_field(vol, seed=77, turbulence=0.0, drift_voxels=drift).ravel().astype(np.float64)
    b = I.plume_field_torch(vol, seed=77, turbulence=0.0, device="cpu",
                            drift_voxels=drift).numpy().astype(np.float64)
    assert np.abs(a).max() > 0
    assert np.abs(a - b).max() <= 1e-5 * np.abs(a).max()
