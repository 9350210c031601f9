"""General camera orientations (yaw, pitch, roll; Sec. III-A, eq. rot,decomp
with all three shears) in the oracle, pinned by:
* the factorisation Theta = P D S_z S_x S_y (matrix identity) and the choice
  of P (a proper signed permutation leaving the smallest residual rotation);
* the shear entry against dense quadrature and, with one shear coefficient
  zero, against the polygon-clipping entry of the yaw passes;
* mass conservation of every pass (partition of unity of the hat);
* reduction to the yaw-only rotation (already pinned) when pitch = roll = 0;
* an anisotropic Gaussian sampled on the rotated grid (analytic rotation),
  against the wrong rotation as a control;
* exact quarter turns about x and z, and the adjoint identity."""
import math

import numpy as np
import pytest

from oracle import rotation as R


def rng(seed):
    return np.random.default_rng(seed)


def test_factorisation_reproduces_the_rotation():
    g = rng(0)
    for _ in range(20):
        T = R.camera_rotation(*g.uniform(-math.pi, math.pi, 3))
        P, Tr = R.split_rotation(T)
        assert np.allclose(P @ Tr, T, atol=1e-14)
        assert round(np.linalg.det(P)) == 1 and np.allclose(np.abs(P).sum(0), 1)
        Dg, co = R.factor_rotation(Tr)
        Sz, Sx, Sy = R.shear_matrices(co)
        assert np.allclose(np.diag(Dg) @ Sz @ Sx @ Sy, Tr, atol=1e-13)
        assert np.all(Dg > 0)
        # the residual is the smallest rotation among all 24 choices
        ang = lambda M: math.acos(max(-1.0, min(1.0, (np.trace(M) - 1) / 2)))
        assert all(ang(Tr) <= ang(Q.T @ T) + 1e-12 for Q in R._PERMS)


def test_hat_average_against_quadrature_and_polygon_entry():
    g = rng(1)
    n = 1200
    for _ in range(12):
        c, al, be = g.uniform(-2.5, 2.5), g.uniform(0, 1.5), g.uniform(0, 1.2)
        u = (np.arange(n) + 0.5) / n - 0.5
        U1, U2 = np.meshgrid(u * al, u * be)
        q = np.maximum(0.0, 1.0 - np.abs(c + U1 + U2)).mean()
        assert abs(R.hat_avg2(c, al, be) - q) < 2e-5
    # one coefficient zero: the yaw passes' polygon-clipping entry
    for _ in range(12):
        zo, zs, x, b = g.uniform(-3, 3), g.uniform(-3, 3), g.uniform(-4, 4), g.uniform(-0.6, 0.6)
        dz, dx = 1.3, 0.9
        ref = R.shear_entry(zo, zs, dz, x, dx, b)
        got = R.hat_avg2((zo - zs + b * x) / dz, abs(b) * dx / dz, 0.0)
        assert abs(got - ref) < 1e-12


@pytest.mark.parametrize("axis", [0, 1, 2])
def test_every_pass_conserves_mass(axis):
    X = rng(2).random((5, 6, 7))
    Y, pad = R.shear_pass(X, (1.0, 1.2, 0.8), axis, 0.31, -0.44)
    assert abs(Y.sum() - X.sum()) < 1e-11 * X.sum()
    assert pad >= 1


@pytest.mark.parametrize("yaw", [0.3, -0.7, 1.9, 3.0, -2.2])
def test_pure_yaw_reduces_to_the_yaw_rotation(yaw):
    X = rng(3).random((5, 4, 6))
    sizes = (4.0, 4.5, 5.0)
    a, sa = R.rotate(X, sizes, yaw)
    b, sb = R.rotate_general(X, sizes, R.camera_rotation(yaw, 0.0, 0.0))
    assert a.shape == b.shape
    assert np.allclose(sa, sb, rtol=1e-12)
    assert np.abs(a - b).max() <= 1e-12 * np.abs(a).max()


def _blob(p):
    c = np.array([1.0, -1.0, 0.5])
    sig = np.array([2.5, 3.5, 2.0])
    return np.exp(-0.5 * (((p - c) / sig) ** 2).sum(-1))


def _sample(shape, sizes, M):
    nz, ny, nx = shape
    zc = (np.arange(nz) - (nz - 1) / 2) * sizes[2]
    yc = (np.arange(ny) - (ny - 1) / 2) * sizes[1]
    xc = (np.arange(nx) - (nx - 1) / 2) * sizes[0]
    Z, Y, X = np.meshgrid(zc, yc, xc, indexing="ij")
    return _blob(np.stack([X, Y, Z], -1) @ M.T)


@pytest.mark.parametrize("angles", [(0.0, 0.35, 0.0), (0.0, 0.0, -0.25), (0.5, 0.35, -0.25)])
def test_anisotropic_blob_matches_its_analytic_rotation(angles):
    """Box-basis resampling blurs a blob of sigma 2-3.5 voxels by a few per
    cent; the inverse rotation (a sign or order error) is far off."""
    sizes, shape = (1.0, 1.0, 1.0), (18, 18, 18)
    X = _sample(shape, sizes, np.eye(3))
    T = R.camera_rotation(*angles)
    Xr, sr = R.rotate_general(X, sizes, T)
    ref = _sample(Xr.shape, sr, T)
    wrong = _sample(Xr.shape, sr, T.T)
    err = np.linalg.norm(Xr - ref) / np.linalg.norm(ref)
    err_w = np.linalg.norm(Xr - wrong) / np.linalg.norm(wrong)
    assert err < 0.06, err
    assert err_w > 4 * err, (err, err_w)


@pytest.mark.parametrize("angles", [(0.0, math.pi / 2, 0.0), (0.0, 0.0, math.pi / 2), (math.pi / 2, math.pi, 0.0)])
def test_quarter_turns_are_exact_relabellings(angles):
    X = rng(4).random((3, 4, 5))
    T = R.camera_rotation(*angles)
    Xr, sr = R.rotate_general(X, (1.0, 2.0, 3.0), T)
    # no shear: the result is X relabelled, padded by zeros
    assert np.isclose(Xr.sum(), X.sum())
    assert sorted(np.round(Xr[Xr != 0], 12)) == sorted(np.round(X.ravel(), 12))
    assert sorted(sr) == [1.0, 2.0, 3.0]


def test_adjoint_identity():
    g = rng(5)
    shape, sizes = (4, 5, 6), (1.1, 0.9, 1.3)
    T = R.camera_rotation(0.4, -0.3, 0.2)
    X = g.random(shape)
    Xr, _ = R.rotate_general(X, sizes, T)
    G = g.random(Xr.shape)
    lhs = float(np.vdot(Xr, G))
    rhs = float(np.vdot(X, R.rotate_general_adjoint(G, shape, sizes, T)))
    assert abs(lhs - rhs) <= 1e-12 * abs(lhs)


def test_camera_with_pitch_and_roll_is_adjoint_consistent():
    """The camera model through a general orientation: <A x, y> = <x, A^T y>."""
    from oracle import camera as O
    from paper_1812_03358_b300 import inputs as I
    vol = I.Volume(6, 5, 4, 4.0, 4.5, 5.0)
    cam = I.table_single_lens(14, 0.5, yaw=0.3, ks=2, kt=1)
    cam.pitch, cam.roll = 0.25, -0.4
    x = rng(6).random(vol.n)
    y = rng(7).random(cam.m)
    lhs = float(np.vdot(np.ravel(O.forward(vol, cam, x)), y))
    rhs = float(np.vdot(x, np.ravel(O.adjoint(vol, cam, y))))
    assert abs(lhs - rhs) <= 1e-11 * abs(lhs)
