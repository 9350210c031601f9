"""Pins of the oracle's camera operators (Sec. II-E/F, Sec. III, Sec. IV-A).

Values fixed independently of the oracle's own assembly: the pinhole-limit
closed form, the total-flux (etendue) closed form, a Monte Carlo ray trace
through the thin lens, the lattice count of the microlens mask, the stage-two
column sums, and the explicit-matrix / matrix-free / transpose identities.
"""
import numpy as np
import pytest

from oracle import camera, optics
from paper_1812_03358_b300 import inputs as I


def _small_single(ks=1, kt=1, det=24, pitch=0.3):
    vol = I.Volume(7, 6, 5, 4.0, 4.0, 6.0)
    cam = I.table_single_lens(det, pitch, ks=ks, kt=kt)
    return vol, cam


def test_explicit_matrix_equals_matrix_free_single():
    rng = np.random.default_rng(0)
    for ks in (1, 2):
        vol, cam = _small_single(ks, ks)
        A = camera.single_matrix(vol, cam)
        x = rng.random(vol.n)
        y = rng.random(cam.m)
        assert np.allclose(A @ x, camera.single_forward(vol, cam, x).ravel(), rtol=1e-13, atol=1e-18)
        assert np.allclose(A.T @ y, camera.single_adjoint(vol, cam, y).ravel(), rtol=1e-13, atol=1e-18)


def test_explicit_matrix_equals_matrix_free_plenoptic():
    rng = np.random.default_rng(1)
    vol, cam = I.tiny_plenoptic()
    A = camera.plenoptic_matrix(vol, cam)
    x = rng.random(vol.n)
    y = rng.random(cam.m)
    scale = np.abs(A).sum(axis=1).max()
    assert np.abs(A @ x - camera.plenoptic_forward(vol, cam, x).ravel()).max() < 1e-13 * scale
    assert np.abs(A.T @ y - camera.plenoptic_adjoint(vol, cam, y).ravel()).max() < 1e-13 * np.abs(A).sum(axis=0).max()
    assert np.count_nonzero(A) > 0


def test_dot_product_adjoint_identity():
    rng = np.random.default_rng(2)
    vol, cam = I.config_single_small()
    x = rng.random(vol.n)
    y = rng.random(cam.m)
    lhs = np.vdot(camera.single_forward(vol, cam, x).ravel(), y)
    rhs = np.vdot(x, camera.single_adjoint(vol, cam, y).ravel())
    assert abs(lhs - rhs) < 1e-13 * abs(lhs)
    vol, cam = I.tiny_plenoptic()
    x = rng.random(vol.n)
    y = rng.random(cam.m)
    lhs = np.vdot(camera.plenoptic_forward(vol, cam, x).ravel(), y)
    rhs = np.vdot(x, camera.plenoptic_adjoint(vol, cam, y).ravel())
    assert abs(lhs - rhs) < 1e-13 * abs(lhs)


@pytest.mark.parametrize("ks", [1, 2])
def test_pinhole_limit_closed_form(ks):
    # A uniform box of density rho projects, on a pixel whose footprint lies
    # inside the box on every slice, to rho * L_z * Dp_s Dp_t * sum_k D0_s D0_t / D^2
    # (the chord length through the box times the pixel's etendue).
    vol, cam = I.config_single_small()
    cam.ks = cam.kt = ks
    rho = 0.7
    x = np.full(vol.n, rho)
    y = camera.single_forward(vol, cam, x)
    cells = camera.lens_cells(cam)
    expect = rho * vol.nz * vol.dz * cam.det_ps * cam.det_pt * sum(c[2] * c[3] for c in cells) / cam.d_lens_det ** 2
    c = cam.det_ns // 2
    for i, j in [(c, c), (c - 5, c + 3), (c + 10, c - 10)]:
        assert abs(y[i, j] - expect) < 1e-12 * expect
    # a pixel whose beams miss the box entirely sees nothing
    assert y[0, 0] == 0.0


def test_total_flux_closed_form():
    # With a detector that catches every ray, the total signal of voxel j is
    # dz * sum_k (dx D0_s / d_n) (dy D0_t / d_n): the flux through each lens
    # cell of the collapsed slice (Sec. III), independent of the optics behind
    # the lens.
    vol = I.Volume(5, 4, 6, 2.0, 2.0, 5.0)
    cam = I.table_single_lens(60, 0.05, ks=2, kt=2)
    rng = np.random.default_rng(4)
    x = rng.random(vol.n)
    y = camera.single_forward(vol, cam, x)
    d = camera.slice_distances(vol, cam)
    cells = camera.lens_cells(cam)
    X = x.reshape(vol.shape)
    expect = sum(vol.dz * X[n].sum() * sum(vol.dx * c[2] * vol.dy * c[3] for c in cells) / d[n] ** 2
                 for n in range(vol.nz))
    assert abs(y.sum() - expect) < 1e-12 * expect


def test_monte_carlo_ray_trace_single_lens():
    # Rays from points uniform on a voxel's face (the collapsed slice) through
    # points uniform in a lens cell, traced through the thin lens to the
    # detector.  B = (dx D0 / d) * P(ray lands in pixel) per axis.
    vol = I.Volume(3, 3, 3, 3.0, 3.0, 5.0)
    cam = I.table_single_lens(16, 0.2, ks=2, kt=2)
    jx, jy, jz = 2, 1, 0
    e = np.zeros(vol.shape)
    e[jz, jy, jx] = 1.0
    model = camera.single_forward(vol, cam, e.ravel())
    rng = np.random.default_rng(5)
    n = 400000
    d = camera.slice_distances(vol, cam)[jz]
    hist = np.zeros_like(model)
    X = optics.compose(optics.propagate(cam.d_lens_det), optics.refract(cam.f_main), optics.propagate(d))
    xs = camera.centers(vol.nx, vol.dx)[jx]
    ys = camera.centers(vol.ny, vol.dy)[jy]
    for (sk, tk, d0s, d0t) in camera.lens_cells(cam):
        s = xs + vol.dx * (rng.random(n) - 0.5)
        t = ys + vol.dy * (rng.random(n) - 0.5)
        ls = sk + d0s * (rng.random(n) - 0.5)
        lt = tk + d0t * (rng.random(n) - 0.5)
        ps, _ = optics.apply(X, s, (ls - s) / d)
        pt, _ = optics.apply(X, t, (lt - t) / d)
        i_s = np.floor(ps / cam.det_ps + cam.det_ns / 2).astype(int)
        i_t = np.floor(pt / cam.det_pt + cam.det_nt / 2).astype(int)
        ok = (i_s >= 0) & (i_s < cam.det_ns) & (i_t >= 0) & (i_t < cam.det_nt)
        w = vol.dz * (vol.dx * d0s / d) * (vol.dy * d0t / d) / n
        np.add.at(hist, (i_t[ok], i_s[ok]), w)
    tot = model.sum()
    assert abs(hist.sum() - tot) < 3e-3 * tot
    # per-pixel agreement within Monte Carlo noise
    err = np.abs(hist - model)
    sigma = np.sqrt(np.maximum(model, 1e-30) * (tot / n) * 4)
    assert np.all(err <= 6 * sigma + 1e-6 * tot)


def test_zero_outside_footprints():
    vol = I.Volume(48, 48, 8, 3.125, 3.125, 3.125)   # 150 mm wide, FOV ~118 mm
    _, cam = I.config_single_small()
    g = camera.single_adjoint(vol, cam, np.ones(cam.m)).reshape(vol.shape)
    assert np.all(g[:, :, 0] == 0.0) and np.all(g[:, 0, :] == 0.0)
    assert np.all(g[:, 24, 24] > 0.0)


def test_microlens_mask_lattice_count():
    # 10x10 array pixels under a lenslet of radius 5 pixel pitches: the pixel
    # centres are the half-integer points (a, b); those with a^2 + b^2 < 25 are
    # 20 per quadrant, 80 per lenslet.
    cam = I.plenoptic_camera(n_lenslets=7)
    owner = camera.lenslet_owner(cam)
    counts = np.bincount(owner[owner >= 0], minlength=49)
    assert np.all(counts == 80)
    # each lenslet owns pixels only inside its own 10x10 block
    jt, js = np.nonzero(owner >= 0)
    mu = owner[jt, js]
    assert np.all(js // 10 == mu % 7) and np.all(jt // 10 == mu // 7)


def test_stage_two_column_sums_equal_array_basis_volume():
    # Summed over every detector pixel, the array -> detector transport of an
    # array pixel carries its whole basis measure D_a D0 / D_mum per axis.
    cam = I.plenoptic_camera(n_lenslets=5)
    cell = camera.lens_cells(cam)[1]
    sk, tk, d0s, d0t = cell
    cs, _ = camera.lenslet_centers(cam)
    Xd, X0 = camera.lenslet_maps(cam, cam.mla_focal[2, 2], cs[2])
    det = camera.centers(cam.det_ns, cam.det_ps)
    src = camera.centers(cam.arr_ns, cam.arr_ps)[20:30]
    B = camera.matrix_1d(cam, Xd, X0, det, cam.det_ps, sk, d0s, src, cam.arr_ps)
    assert np.allclose(B.sum(axis=0), cam.arr_ps * d0s / cam.d_lens_mla, rtol=1e-12)


def test_plenoptic_total_flux_equals_masked_array_flux():
    # Everything that passes the mask reaches the detector: the plenoptic
    # image's total equals the total, over unmasked array pixels, of the image
    # formed on the array plane by the main lens alone.
    rng = np.random.default_rng(6)
    vol, cam = I.tiny_plenoptic()
    x = rng.random(vol.n)
    y = camera.plenoptic_forward(vol, cam, x)
    single = I.Camera(kind=0, f_main=cam.f_main, r_main=cam.r_main, d_obj=cam.d_obj,
                      det_ns=cam.arr_ns, det_nt=cam.arr_nt, det_ps=cam.arr_ps, det_pt=cam.arr_pt,
                      d_lens_det=cam.d_lens_mla, ks=cam.ks, kt=cam.kt)
    img = camera.single_forward(vol, single, x)
    expect = img[camera.lenslet_owner(cam) >= 0].sum()
    assert abs(y.sum() - expect) < 1e-12 * expect


def test_array_block_equals_whole_array_field():
    vol, cam = I.tiny_plenoptic()
    x = I.gaussian_blobs(vol, seed=1300)
    rng = np.random.default_rng(3)
    for cell in camera.lens_cells(cam):
        full = camera.plenoptic_array_field(vol, cam, x, cell)
        rows = np.sort(rng.choice(cam.arr_nt, size=5, replace=False))
        cols = np.sort(rng.choice(cam.arr_ns, size=7, replace=False))
        blk = camera.plenoptic_array_block(vol, cam, x, cell, rows, cols)
        assert np.abs(blk - full[np.ix_(rows, cols)]).max() <= 1e-13 * np.abs(full).max()
        allb = camera.plenoptic_array_block(vol, cam, x, cell, np.arange(cam.arr_nt), np.arange(cam.arr_ns))
        assert np.abs(allb - full).max() <= 1e-13 * np.abs(full).max()
