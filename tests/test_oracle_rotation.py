"""Pins of the oracle's rotated perspectives (Sec. III-A): the shear
decomposition reproduces the rotation matrix, zero angle is the identity,
quarter turns equal numpy's rot90, every shear conserves mass, the shear
entries equal an independent closed form (average of the box-overlap hat over
the sheared cell), a smooth blob rotates into the analytically rotated
blob up to resampling error, and the per-voxel spot check equals the whole
rotation at every voxel."""
import math

import numpy as np
import pytest

from oracle import rotation as R


@pytest.mark.parametrize("theta", [-0.7, -0.3, 0.0, 0.2, 0.785])
def test_decomposition_reproduces_rotation(theta):
    Dg, a, b = R.shear_factors(theta)
    Sx = np.array([[1, 0, a], [0, 1, 0], [0, 0, 1.0]])
    Sz = np.array([[1, 0, 0], [0, 1, 0], [b, 0, 1.0]])
    assert np.allclose(np.diag(Dg) @ Sz @ Sx, R.yaw_matrix(theta), atol=1e-14)


def test_split_angle_range():
    for th in np.linspace(-7, 7, 101):
        n, r = R.split_angle(th)
        assert abs(r) <= math.pi / 4 + 1e-12
        assert abs(R.yaw_matrix(th) - R.yaw_matrix(n * math.pi / 2) @ R.yaw_matrix(r)).max() < 1e-12


def test_zero_angle_is_identity():
    rng = np.random.default_rng(0)
    X = rng.random((5, 4, 6))
    Rv, sizes = R.rotate(X, (1.0, 1.0, 1.5), 0.0)
    # padding of one voxel on each side in z and x, identity inside
    assert Rv.shape == (7, 4, 8)
    assert np.allclose(Rv[1:-1, :, 1:-1], X, atol=1e-15) and abs(Rv.sum() - X.sum()) < 1e-12


@pytest.mark.parametrize("n", [1, 2, 3])
def test_quarter_turns_sample_the_rotated_function(n):
    # f^P(p) = f(Theta_90^n p): sampling an analytic f on the original grid and
    # quarter-turning must equal sampling f at the rotated centres of the new grid.
    nz, ny, nx = 5, 3, 4
    sizes = (1.0, 2.0, 3.0)
    f = lambda x, y, z: np.sin(0.3 * x + 0.1) + 0.5 * y * y + np.cos(0.2 * z) * x + 0.01 * z ** 3
    cen = lambda m, d: (np.arange(m) - (m - 1) / 2) * d
    Z, Y, X = np.meshgrid(cen(nz, sizes[2]), cen(ny, sizes[1]), cen(nx, sizes[0]), indexing="ij")
    P, sp = R.quarter_turn(f(X, Y, Z), n, sizes)
    T = np.rint(R.yaw_matrix(n * math.pi / 2)).astype(int)
    Zp, Yp, Xp = np.meshgrid(cen(P.shape[0], sp[2]), cen(P.shape[1], sp[1]), cen(P.shape[2], sp[0]), indexing="ij")
    ox = T[0, 0] * Xp + T[0, 2] * Zp
    oz = T[2, 0] * Xp + T[2, 2] * Zp
    assert np.allclose(P, f(ox, Yp, oz), atol=1e-12)
    assert sp == ((3.0, 2.0, 1.0) if n % 2 else (1.0, 2.0, 3.0))


@pytest.mark.parametrize("theta", [0.3, -0.6, 0.78])
def test_shears_conserve_mass(theta):
    rng = np.random.default_rng(1)
    X = rng.random((6, 3, 7))
    Dg, a, b = R.shear_factors(theta)
    sizes = (1.0 / Dg[0], 1.0, 1.3 / Dg[2])
    Z, _ = R.shear_z(X, sizes, b)
    assert abs(Z.sum() - X.sum()) < 1e-12 * X.sum()
    XX, _ = R.shear_x(Z, sizes, a)
    assert abs(XX.sum() - X.sum()) < 1e-12 * X.sum()


def _hat_avg(u, beta):
    def H(t):
        t = np.clip(t, -1.0, 1.0)
        return np.where(t < 0, t + t * t / 2, t - t * t / 2)
    if beta == 0:
        return max(0.0, 1 - abs(u))
    return float((H(u + beta / 2) - H(u - beta / 2)) / beta)


def test_shear_entries_closed_form():
    rng = np.random.default_rng(2)
    for _ in range(300):
        dz, dx = rng.uniform(0.5, 2.0), rng.uniform(0.5, 2.0)
        b = rng.uniform(-1.2, 1.2)
        xc = rng.uniform(-10, 10)
        zi, zj = rng.uniform(-5, 5), rng.uniform(-5, 5)
        e = R.shear_entry(zi, zj, dz, xc, dx, b)
        u = (zi - zj + b * xc) / dz
        assert abs(e - _hat_avg(u, abs(b) * dx / dz)) < 1e-12


def test_rotated_blob_matches_analytic_rotation():
    n = 32
    d = 1.0
    c = (np.arange(n) - (n - 1) / 2) * d
    Z, Y, X = np.meshgrid(c, c, c, indexing="ij")
    sig = np.array([4.0, 3.0, 6.0])
    mu = np.array([2.0, -1.0, 3.0])
    f = lambda x, y, z: np.exp(-0.5 * (((x - mu[0]) / sig[0]) ** 2 + ((y - mu[1]) / sig[1]) ** 2 + ((z - mu[2]) / sig[2]) ** 2))
    vol = f(X, Y, Z)
    theta = 0.5
    Rv, sr = R.rotate(vol, (d, d, d), theta)
    nz, ny, nx = Rv.shape
    zr = (np.arange(nz) - (nz - 1) / 2) * sr[2]
    yr = (np.arange(ny) - (ny - 1) / 2) * sr[1]
    xr = (np.arange(nx) - (nx - 1) / 2) * sr[0]
    Zr, Yr, Xr = np.meshgrid(zr, yr, xr, indexing="ij")
    T = R.yaw_matrix(theta)
    px = T[0, 0] * Xr + T[0, 2] * Zr
    pz = T[2, 0] * Xr + T[2, 2] * Zr
    ref = f(px, Yr, pz)
    err = np.linalg.norm(Rv - ref) / np.linalg.norm(ref)
    # box-basis resampling blur is a few percent at sigma = 3-6 voxels; the
    # opposite rotation (a sign error) would be far off
    wrong = f(T[0, 0] * Xr - T[0, 2] * Zr, Yr, -T[2, 0] * Xr + T[2, 2] * Zr)
    err_wrong = np.linalg.norm(Rv - wrong) / np.linalg.norm(wrong)
    assert err < 0.05 and err_wrong > 5 * err, (err, err_wrong)


@pytest.mark.parametrize("theta", [0.3, -0.7, 0.785, 1.9, 3.0, -2.2])
def test_rotate_voxels_equals_rotate_everywhere(theta):
    rng = np.random.default_rng(7)
    X = rng.random((5, 3, 6))
    sizes = (1.0, 1.2, 0.8)
    full, _ = R.rotate(X, sizes, theta)
    idx = [(i, j, k) for i in range(full.shape[0]) for j in range(full.shape[1])
           for k in range(full.shape[2])]
    got = R.rotate_voxels(X, sizes, theta, idx)
    assert np.abs(got - full.ravel()).max() <= 1e-13 * np.abs(full).max()
