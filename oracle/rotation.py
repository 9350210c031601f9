"""Rotated perspectives by shears (Sec. III-A) - oracle, test infrastructure.

A camera turned by a yaw theta about the volume's y axis sees the object in
rotated coordinates p^r with p = Theta p^r,
    Theta = [[cos, 0, sin], [0, 1, 0], [-sin, 0, cos]].
Following Sec. III-A, theta is split into n quarter turns (an exact
permutation of the voxel grid) and a residual |theta_r| <= 45 degrees, and the
residual rotation is decomposed as Theta_r = D S_z S_x (eq. rot,decomp with
S_y = I for a rotation about y):
    D = diag(cos, 1, 1/cos),  S_x: x -> x + tan(theta) z,  S_z: z -> z - sin cos x.
D only rescales the voxel sizes to (dx/cos, dy, dz cos).  Each shear is a
least-squares re-projection of the box basis (eq. rot,toeplitz): the entry
between output voxel i and source voxel j of the same column is the overlap
area of output cell i with the sheared source cell j, divided by the cell
area.  This oracle computes those overlaps by exact polygon clipping.

Output grids (reading: the paper does not fix them): after the z shear the
z axis is padded symmetrically by Pz = ceil(|b| nx dx'/2 / dz') + 1 voxels so
that every sheared cell lies inside; the x shear pads x likewise with
Px = ceil(|a| nz' dz'/2 / dx') + 1.  The rotated volume is [nz'][ny][nx'].
"""
import math

import numpy as np

from . import transport


def yaw_matrix(theta):
    c, s = math.cos(theta), math.sin(theta)
    return np.array([[c, 0.0, s], [0.0, 1.0, 0.0], [-s, 0.0, c]])


def split_angle(theta):
    """theta = n * 90 deg + residual, |residual| <= 45 deg, n in {0,1,2,3}.
    Sec. III-A takes residuals below 45 degrees; at exactly 45 degrees the
    quarter-turn count is rounded half up: n = floor(theta / 90 deg + 1/2)."""
    n = int(math.floor(theta / (math.pi / 2) + 0.5))
    return n % 4, theta - n * (math.pi / 2)


def shear_factors(theta_r):
    """D diagonal, a (S_x: x += a z) and b (S_z: z += b x) of Theta_r = D S_z S_x."""
    c, s = math.cos(theta_r), math.sin(theta_r)
    return np.array([c, 1.0, 1.0 / c]), s / c, -s * c


def quarter_turn(X, n, sizes):
    """f^P(p) = f(Theta_90^n p) sampled on the permuted grid: an exact
    relabelling of voxels.  X is [nz][ny][nx]; sizes (dx, dy, dz)."""
    dx, dy, dz = sizes
    nz, ny, nx = X.shape
    iz, iy, ix = np.meshgrid(np.arange(nz), np.arange(ny), np.arange(nx), indexing="ij")
    if n == 0:
        return X.copy(), (dx, dy, dz)
    if n == 1:     # f^P(x, y, z) = f(z, y, -x): new x <- old -z, new z <- old x
        out = np.empty((nx, ny, nz))
        out[ix, iy, nz - 1 - iz] = X
        return out, (dz, dy, dx)
    if n == 2:     # f(-x, y, -z)
        out = np.empty((nz, ny, nx))
        out[nz - 1 - iz, iy, nx - 1 - ix] = X
        return out, (dx, dy, dz)
    out = np.empty((nx, ny, nz))   # n == 3: f(-z, y, x): new x <- old z, new z <- old -x
    out[nx - 1 - ix, iy, iz] = X
    return out, (dz, dy, dx)


def shear_entry(center_out, center_src, d_shear, pos_other, d_other, slope):
    """(1/(d_shear d_other)) * area of {(o, v): |o - pos_other| <= d_other/2,
    |v - center_out| <= d_shear/2, |v + slope o - center_src| <= d_shear/2}:
    the LS coefficient of output cell (center_out) for the sheared source cell
    (center_src) in the column/row at pos_other (polygon clipping)."""
    o0, o1 = pos_other - d_other / 2, pos_other + d_other / 2
    v0, v1 = center_out - d_shear / 2, center_out + d_shear / 2
    poly = [(o0, v0), (o1, v0), (o1, v1), (o0, v1)]
    for cs, cu, c0 in [(slope, 1.0, -(center_src - d_shear / 2)), (-slope, -1.0, center_src + d_shear / 2)]:
        poly = transport._clip(poly, cs, cu, c0)
        if not poly:
            return 0.0
    return transport._area(poly) / (d_shear * d_other)


def _centres(n, d):
    return (np.arange(n) - (n - 1) / 2.0) * d


def shear_z(X, sizes, b):
    """E^z: g1(q) = g0(q_x, q_y, q_z + b q_x) projected on a z-padded grid."""
    dx, dy, dz = sizes
    nz, ny, nx = X.shape
    pz = int(math.ceil(abs(b) * nx * dx / 2 / dz)) + 1
    nzo = nz + 2 * pz
    zs, zo, xs = _centres(nz, dz), _centres(nzo, dz), _centres(nx, dx)
    out = np.zeros((nzo, ny, nx))
    for ix in range(nx):
        E = np.zeros((nzo, nz))
        for i in range(nzo):
            for j in range(nz):
                # candidate pairs only: the sheared cell j spans z_j - b x over the column
                if abs(zo[i] - (zs[j] - b * xs[ix])) < dz + abs(b) * dx / 2 + 1e-12:
                    E[i, j] = shear_entry(zo[i], zs[j], dz, xs[ix], dx, b)
        out[:, :, ix] = E @ X[:, :, ix]
    return out, pz


def shear_x(X, sizes, a):
    """E^x: g2(q) = g1(q_x + a q_z, q_y, q_z) projected on an x-padded grid."""
    dx, dy, dz = sizes
    nz, ny, nx = X.shape
    px = int(math.ceil(abs(a) * nz * dz / 2 / dx)) + 1
    nxo = nx + 2 * px
    xs, xo, zs = _centres(nx, dx), _centres(nxo, dx), _centres(nz, dz)
    out = np.zeros((nz, ny, nxo))
    for iz in range(nz):
        E = np.zeros((nxo, nx))
        for i in range(nxo):
            for j in range(nx):
                if abs(xo[i] - (xs[j] - a * zs[iz])) < dx + abs(a) * dz / 2 + 1e-12:
                    E[i, j] = shear_entry(xo[i], xs[j], dx, zs[iz], dz, a)
        out[iz] = X[iz] @ E.T
    return out, px


def rotated_grid(shape, sizes, theta):
    """Shape [nz', ny, nx'], voxel sizes and quarter turns of the rotated volume."""
    n, tr = split_angle(theta)
    nz, ny, nx = shape
    if n % 2 == 1:
        nz, nx = nx, nz
        sizes = (sizes[2], sizes[1], sizes[0])
    Dg, a, b = shear_factors(tr)
    sz = (sizes[0] / Dg[0], sizes[1], sizes[2] / Dg[2])
    pz = int(math.ceil(abs(b) * nx * sz[0] / 2 / sz[2])) + 1
    nzo = nz + 2 * pz
    px = int(math.ceil(abs(a) * nzo * sz[2] / 2 / sz[0])) + 1
    return (nzo, ny, nx + 2 * px), sz, n


def rotate(X, sizes, theta):
    """x^r = E^x E^z P x (Sec. III-A) and the rotated voxel sizes."""
    n, tr = split_angle(theta)
    Xp, sp = quarter_turn(np.asarray(X, dtype=np.float64), n, sizes)
    Dg, a, b = shear_factors(tr)
    sr = (sp[0] / Dg[0], sp[1], sp[2] / Dg[2])
    Z, _ = shear_z(Xp, sr, b)
    R, _ = shear_x(Z, sr, a)
    return R, sr


def rotation_matrix(shape, sizes, theta):
    """Explicit matrix of `rotate` (columns = rotated unit voxels), tiny grids."""
    N = int(np.prod(shape))
    cols = []
    for j in range(N):
        e = np.zeros(N)
        e[j] = 1.0
        R, _ = rotate(e.reshape(shape), sizes, theta)
        cols.append(R.ravel())
    return np.stack(cols, axis=1)


def shear_z_adjoint(G, sizes, b, nz):
    """(E^z)^T: from the padded grid [nz'][ny][nx] back to [nz][ny][nx]."""
    dx, dy, dz = sizes
    nzo, ny, nx = G.shape
    zs, zo, xs = _centres(nz, dz), _centres(nzo, dz), _centres(nx, dx)
    out = np.zeros((nz, ny, nx))
    for ix in range(nx):
        E = np.zeros((nzo, nz))
        for i in range(nzo):
            for j in range(nz):
                if abs(zo[i] - (zs[j] - b * xs[ix])) < dz + abs(b) * dx / 2 + 1e-12:
                    E[i, j] = shear_entry(zo[i], zs[j], dz, xs[ix], dx, b)
        out[:, :, ix] = E.T @ G[:, :, ix]
    return out


def shear_x_adjoint(G, sizes, a, nx):
    """(E^x)^T: from [nz][ny][nx'] back to [nz][ny][nx]."""
    dx, dy, dz = sizes
    nz, ny, nxo = G.shape
    xs, xo, zs = _centres(nx, dx), _centres(nxo, dx), _centres(nz, dz)
    out = np.zeros((nz, ny, nx))
    for iz in range(nz):
        E = np.zeros((nxo, nx))
        for i in range(nxo):
            for j in range(nx):
                if abs(xo[i] - (xs[j] - a * zs[iz])) < dx + abs(a) * dz / 2 + 1e-12:
                    E[i, j] = shear_entry(xo[i], xs[j], dx, zs[iz], dz, a)
        out[iz] = G[iz] @ E
    return out


def quarter_turn_adjoint(P, n, shape):
    """Inverse (= transpose) of the quarter-turn permutation, back to shape."""
    nz, ny, nx = shape
    iz, iy, ix = np.meshgrid(np.arange(nz), np.arange(ny), np.arange(nx), indexing="ij")
    if n == 0:
        return P.copy()
    if n == 1:
        return P[ix, iy, nz - 1 - iz]
    if n == 2:
        return P[nz - 1 - iz, iy, nx - 1 - ix]
    return P[nx - 1 - ix, iy, iz]


def rotate_adjoint(G, shape, sizes, theta):
    """P^T (E^z)^T (E^x)^T applied to a rotated-grid array G."""
    n, tr = split_angle(theta)
    nz, ny, nx = shape
    nzp, nxp = (nx, nz) if n % 2 else (nz, nx)
    sp = (sizes[2], sizes[1], sizes[0]) if n % 2 else sizes
    Dg, a, b = shear_factors(tr)
    sr = (sp[0] / Dg[0], sp[1], sp[2] / Dg[2])
    Z = shear_x_adjoint(np.asarray(G, dtype=np.float64), sr, a, nxp)
    Xp = shear_z_adjoint(Z, sr, b, nzp)
    return quarter_turn_adjoint(Xp, n, shape)
