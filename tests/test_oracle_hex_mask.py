"""Hexagonal multi-focus microlens arrays and coded masks (Sec. II-D, eq.
occlusion; the simulated camera's hexagonal pattern) in the oracle, pinned by
the lattice geometry, a brute-force ownership search, the focal-length
colouring, the explicit system matrix, and superposition of complementary
masks."""
import numpy as np

from oracle import camera as O
from paper_1812_03358_b300 import inputs as I


def test_hex_lattice_neighbours_are_one_pitch_apart():
    cam = I.hex_plenoptic_camera(n_cols=9, n_rows=9)
    S, T = O.lenslet_centres_2d(cam)
    P = np.stack([S, T], 1)
    d = np.sqrt(((P[:, None, :] - P[None, :, :]) ** 2).sum(-1))
    mu = 4 * 9 + 4                       # an interior lenslet
    nn = np.sort(d[mu])[1:8]
    assert np.allclose(nn[:6], cam.mla_pitch, rtol=1e-12) and nn[6] > 1.5 * cam.mla_pitch
    assert abs(S.mean()) < 0.2 * cam.mla_pitch and abs(T.mean()) < 1e-12


def test_neighbouring_lenslets_have_different_focal_lengths():
    cam = I.hex_plenoptic_camera(n_cols=12, n_rows=11)
    S, T = O.lenslet_centres_2d(cam)
    f = cam.mla_focal.ravel()
    P = np.stack([S, T], 1)
    d = np.sqrt(((P[:, None, :] - P[None, :, :]) ** 2).sum(-1))
    i, j = np.nonzero(np.isclose(d, cam.mla_pitch, rtol=1e-9))
    assert len(i) > 0 and np.all(f[i] != f[j])


def test_hex_ownership_matches_brute_force():
    _, cam = I.tiny_hex_plenoptic()
    own = O.lenslet_owner(cam)
    S, T = O.lenslet_centres_2d(cam)
    s = O.centers(cam.arr_ns, cam.arr_ps)
    t = O.centers(cam.arr_nt, cam.arr_pt)
    for jt in range(cam.arr_nt):
        for js in range(cam.arr_ns):
            d2 = (s[js] - S) ** 2 + (t[jt] - T) ** 2
            inside = np.nonzero(d2 < cam.mla_radius ** 2)[0]
            assert len(inside) <= 1
            assert own[jt, js] == (inside[0] if len(inside) else -1)
    assert (own >= 0).mean() > 0.5


def test_hex_matrix_free_equals_explicit_matrix_and_transpose():
    vol, cam = I.tiny_hex_plenoptic()
    A = O.plenoptic_matrix(vol, cam)
    x = I.gaussian_blobs(vol, seed=21).ravel()
    y = I.uniform_random(cam.m, seed=22)
    assert np.allclose(np.ravel(O.plenoptic_forward(vol, cam, x)), A @ x, rtol=1e-11, atol=1e-13)
    assert np.allclose(np.ravel(O.plenoptic_adjoint(vol, cam, y)), A.T @ y, rtol=1e-11, atol=1e-13)
    assert np.abs(A).max() > 0


def test_complementary_coded_masks_superpose():
    """M enters linearly: masks m and 1 - m add up to the unmasked camera, on
    the square and the hexagonal array; a half-transmitting mask halves it."""
    for vol, cam in (I.tiny_plenoptic(), I.tiny_hex_plenoptic()):
        x = I.gaussian_blobs(vol, seed=23).ravel()
        y = I.uniform_random(cam.m, seed=24)
        full_f = np.ravel(O.forward(vol, cam, x))
        full_a = np.ravel(O.adjoint(vol, cam, y))
        rng = np.random.default_rng(25)
        m = (rng.random((cam.arr_nt, cam.arr_ns)) < 0.5).astype(np.float64)
        parts_f, parts_a = 0.0, 0.0
        for mm in (m, 1.0 - m):
            cam.arr_mask = mm
            parts_f = parts_f + np.ravel(O.forward(vol, cam, x))
            parts_a = parts_a + np.ravel(O.adjoint(vol, cam, y))
        assert np.allclose(parts_f, full_f, rtol=1e-12, atol=1e-14 * np.abs(full_f).max())
        assert np.allclose(parts_a, full_a, rtol=1e-12, atol=1e-14 * np.abs(full_a).max())
        cam.arr_mask = np.full((cam.arr_nt, cam.arr_ns), 0.5)
        assert np.allclose(np.ravel(O.forward(vol, cam, x)), 0.5 * full_f, rtol=1e-12)
        cam.arr_mask = m
        # a mask that blocks everything blocks everything
        cam.arr_mask = np.zeros((cam.arr_nt, cam.arr_ns))
        assert np.abs(np.ravel(O.forward(vol, cam, x))).max() == 0.0
        cam.arr_mask = None
