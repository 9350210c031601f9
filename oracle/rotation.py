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


def rotate_voxels(X, sizes, theta, idx):
    """Values of rotate(X, sizes, theta) at the output voxels idx (rows
    (izr, iy, ixr)), each formed from its own entries: the x shear's entries
    of row izr times the z-sheared values of that row, each of those the z
    shear's entries of its column times the quarter-turned volume.  The same
    shear_entry terms as shear_z and shear_x, for spot checks of volumes too
    large for `rotate`."""
    n, tr = split_angle(theta)
    Xp, sp = quarter_turn(np.asarray(X, dtype=np.float64), n, sizes)
    Dg, a, b = shear_factors(tr)
    dx, dy, dz = sp[0] / Dg[0], sp[1], sp[2] / Dg[2]
    nz, ny, nx = Xp.shape
    pz = int(math.ceil(abs(b) * nx * dx / 2 / dz)) + 1
    nzo = nz + 2 * pz
    px = int(math.ceil(abs(a) * nzo * dz / 2 / dx)) + 1
    zs, zo = _centres(nz, dz), _centres(nzo, dz)
    xs, xo = _centres(nx, dx), _centres(nx + 2 * px, dx)
    out = np.zeros(len(idx))
    for m, (iz, iy, ix) in enumerate(idx):
        for j in range(nx):   # source column j of the z-sheared row iz
            if not abs(xo[ix] - (xs[j] - a * zo[iz])) < dx + abs(a) * dz / 2 + 1e-12:
                continue
            ex = shear_entry(xo[ix], xs[j], dx, zo[iz], dz, a)
            if ex == 0.0:
                continue
            zval = 0.0
            for k in range(nz):
                if abs(zo[iz] - (zs[k] - b * xs[j])) < dz + abs(b) * dx / 2 + 1e-12:
                    zval += shear_entry(zo[iz], zs[k], dz, xs[j], dx, b) * Xp[k, iy, j]
            out[m] += ex * zval
    return out


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


# ---------------------------------------------------------------------------
# General orientations: yaw, pitch and roll (Sec. III-A, eq. rot,decomp with
# all three shears).  Theta = R_y(yaw) R_x(pitch) R_z(roll), p = Theta p^r.
# Theta = P Theta_r with P a proper signed permutation (quarter turns, an
# exact relabelling of voxels) chosen to maximise trace(P^T Theta), and
# Theta_r = D S_z S_x S_y with
#     S_z: z += a x + b y,   S_x: x += c y + d z,   S_y: y += e x + f z,
# applied left to right: D rescales the voxel sizes, then one least-squares
# re-projection pass per shear (eq. rot,toeplitz).  The entry between output
# cell i and source cell j of a column is the unit hat of the cell overlap
# averaged over the column's cell: with the shift s1 u + s2 v varying over
# the (u, v) cell, the average of hat(c + U1 + U2) for U1, U2 uniform of
# widths |s1| du / dt and |s2| dv / dt.
# Output grids: each pass pads its axis symmetrically by
#     P = ceil((|s1| n_u du + |s2| n_v dv) / 2 / dt) + 1,
# and a pass whose two coefficients are zero is the identity (no padding).
# ---------------------------------------------------------------------------

def rot_x(phi):
    c, s = math.cos(phi), math.sin(phi)
    return np.array([[1.0, 0.0, 0.0], [0.0, c, -s], [0.0, s, c]])


def rot_z(psi):
    c, s = math.cos(psi), math.sin(psi)
    return np.array([[c, -s, 0.0], [s, c, 0.0], [0.0, 0.0, 1.0]])


def camera_rotation(yaw, pitch=0.0, roll=0.0):
    """Theta of a camera turned by yaw (about y), pitch (about x) and roll
    (about z, the optical axis): R_y(yaw) R_x(pitch) R_z(roll)."""
    return yaw_matrix(yaw) @ rot_x(pitch) @ rot_z(roll)


def _proper_signed_permutations():
    out = []
    for perm in [(0, 1, 2), (0, 2, 1), (1, 0, 2), (1, 2, 0), (2, 0, 1), (2, 1, 0)]:
        for signs in [(sx, sy, sz) for sx in (1, -1) for sy in (1, -1) for sz in (1, -1)]:
            P = np.zeros((3, 3))
            for m in range(3):
                P[m, perm[m]] = signs[m]
            if round(np.linalg.det(P)) == 1:
                out.append(P)
    return out


_PERMS = _proper_signed_permutations()


def split_rotation(Theta):
    """Theta = P Theta_r: P the proper signed permutation (one of 24) with the
    largest trace(P^T Theta), the first of the fixed enumeration on ties."""
    best, best_tr = None, -np.inf
    for P in _PERMS:
        tr = float(np.trace(P.T @ Theta))
        if tr > best_tr + 1e-12:
            best, best_tr = P, tr
    Tr = best.T @ Theta
    Tr[np.abs(Tr) < 1e-12] = 0.0     # rounding residue of exact quarter turns
    return best, Tr


def factor_rotation(Tr):
    """D (diagonal, as a 3-vector) and (a, b, c, d, e, f) of
    Tr = D S_z S_x S_y (elimination, row by row)."""
    Dy = Tr[1, 1]
    e, f = Tr[1, 0] / Dy, Tr[1, 2] / Dy
    Dx = Tr[0, 0] - Tr[0, 1] * e
    c = Tr[0, 1] / Dx
    d = Tr[0, 2] / Dx - c * f
    u = Tr[2, 0] - Tr[2, 1] * e
    v = Tr[2, 1] - u * c
    Dz = Tr[2, 2] - u * (d + c * f) - v * f
    return np.array([Dx, Dy, Dz]), (u / Dz, v / Dz, c, d, e, f)


def shear_matrices(coeffs):
    a, b, c, d, e, f = coeffs
    Sz = np.array([[1.0, 0.0, 0.0], [0.0, 1.0, 0.0], [a, b, 1.0]])
    Sx = np.array([[1.0, c, d], [0.0, 1.0, 0.0], [0.0, 0.0, 1.0]])
    Sy = np.array([[1.0, 0.0, 0.0], [e, 1.0, f], [0.0, 0.0, 1.0]])
    return Sz, Sx, Sy


def permute_volume(X, P, sizes):
    """f^P(p) = f(P p) on the permuted grid (exact relabelling).  X [nz][ny][nx],
    sizes (dx, dy, dz); returns the permuted array and its voxel sizes."""
    X = np.asarray(X, dtype=np.float64)
    n_src = (X.shape[2], X.shape[1], X.shape[0])        # (nx, ny, nz)
    km = [int(np.nonzero(P[m])[0][0]) for m in range(3)]  # source axis m <- permuted axis km[m]
    n_new = [0, 0, 0]
    s_new = [0.0, 0.0, 0.0]
    for m in range(3):
        n_new[km[m]] = n_src[m]
        s_new[km[m]] = sizes[m]
    iz, iy, ix = np.meshgrid(np.arange(n_new[2]), np.arange(n_new[1]), np.arange(n_new[0]), indexing="ij")
    inew = (ix, iy, iz)
    src = []
    for m in range(3):
        i = inew[km[m]]
        src.append(i if P[m, km[m]] > 0 else n_src[m] - 1 - i)
    return X[src[2], src[1], src[0]], tuple(s_new)


def permute_volume_adjoint(Y, P, shape):
    """Transpose of permute_volume (a permutation: its inverse) back to shape."""
    X = np.zeros(shape)
    n_src = (shape[2], shape[1], shape[0])
    km = [int(np.nonzero(P[m])[0][0]) for m in range(3)]
    iz, iy, ix = np.meshgrid(np.arange(Y.shape[0]), np.arange(Y.shape[1]), np.arange(Y.shape[2]), indexing="ij")
    inew = (ix, iy, iz)
    src = []
    for m in range(3):
        i = inew[km[m]]
        src.append(i if P[m, km[m]] > 0 else n_src[m] - 1 - i)
    X[src[2], src[1], src[0]] = Y
    return X


def _hat(t):
    return max(0.0, 1.0 - abs(t))


def _gl2(fn, lo, hi):
    """Two-point Gauss-Legendre on [lo, hi]: exact for cubics."""
    m, r = 0.5 * (lo + hi), 0.5 * (hi - lo) / math.sqrt(3.0)
    return 0.5 * (hi - lo) * (fn(m - r) + fn(m + r))


def hat_avg2(c, alpha, beta):
    """E[hat(c + U1 + U2)], U1 ~ U(-alpha/2, alpha/2), U2 ~ U(-beta/2, beta/2)
    (widths >= 0), integrated exactly: the density of U1 + U2 is a trapezoid,
    the integrand is piecewise quadratic between the merged kinks."""
    alpha, beta = abs(alpha), abs(beta)
    if alpha < beta:
        alpha, beta = beta, alpha
    if alpha == 0.0:
        return _hat(c)
    h = 0.5 * (alpha + beta)            # support [-h, h]
    g = 0.5 * (alpha - beta)            # plateau [-g, g], height 1/alpha

    def pdf(s):
        a = abs(s)
        if a >= h:
            return 0.0
        if a <= g or beta == 0.0:
            return 1.0 / alpha
        return (h - a) / (alpha * beta)

    knots = sorted({-h, -g, g, h, -c - 1.0, -c, -c + 1.0})
    knots = [k for k in knots if -h <= k <= h]
    total = 0.0
    for lo, hi in zip(knots[:-1], knots[1:]):
        if hi > lo:
            total += _gl2(lambda s: _hat(c + s) * pdf(s), lo, hi)
    return total


def shear_pass(X, sizes, axis, s1, s2):
    """One least-squares shear pass along `axis` (0 = x, 1 = y, 2 = z) of a
    [nz][ny][nx] array: output cell i of the column at (u, v) (the other two
    axes in increasing order) takes source cell j with weight
    hat_avg2((t_i - t_j + s1 u + s2 v) / dt, |s1| du / dt, |s2| dv / dt).
    Returns the padded array and the padding."""
    X = np.asarray(X, dtype=np.float64)
    if s1 == 0.0 and s2 == 0.0:                  # no shear: the identity, no padding
        return X.copy(), 0
    A = np.moveaxis(X, 2 - axis, -1)             # [..., n_axis], other axes in array order
    others = [k for k in (0, 1, 2) if k != axis]  # coordinate axes u (first), v (second)
    n_all = (X.shape[2], X.shape[1], X.shape[0])
    n, dt = n_all[axis], sizes[axis]
    nu, du = n_all[others[0]], sizes[others[0]]
    nv, dv = n_all[others[1]], sizes[others[1]]
    pad = int(math.ceil((abs(s1) * nu * du + abs(s2) * nv * dv) / 2.0 / dt)) + 1
    no = n + 2 * pad
    ts, to = _centres(n, dt), _centres(no, dt)
    us, vs = _centres(nu, du), _centres(nv, dv)
    al, be = abs(s1) * du / dt, abs(s2) * dv / dt
    out_shape = list(A.shape[:-1]) + [no]
    out = np.zeros(out_shape)
    # array axes of A[..., n]: the remaining two array axes are (2 - others[1], 2 - others[0])
    # in array order (higher coordinate axis first)
    for iv in range(nv):
        for iu in range(nu):
            sh = s1 * us[iu] + s2 * vs[iv]
            E = np.zeros((no, n))
            for i in range(no):
                for j in range(n):
                    cc = (to[i] - ts[j] + sh) / dt
                    if abs(cc) < 1.0 + 0.5 * (al + be) + 1e-12:
                        E[i, j] = hat_avg2(cc, al, be)
            col = A[iv, iu, :]
            out[iv, iu, :] = E @ col
    return np.moveaxis(out, -1, 2 - axis), pad


def shear_pass_adjoint(G, sizes, axis, s1, s2, n):
    """Transpose of shear_pass back to length n along `axis`."""
    G = np.asarray(G, dtype=np.float64)
    if s1 == 0.0 and s2 == 0.0:
        return G.copy()
    A = np.moveaxis(G, 2 - axis, -1)
    others = [k for k in (0, 1, 2) if k != axis]
    n_all = (G.shape[2], G.shape[1], G.shape[0])
    no, dt = n_all[axis], sizes[axis]
    nu, du = n_all[others[0]], sizes[others[0]]
    nv, dv = n_all[others[1]], sizes[others[1]]
    ts, to = _centres(n, dt), _centres(no, dt)
    us, vs = _centres(nu, du), _centres(nv, dv)
    al, be = abs(s1) * du / dt, abs(s2) * dv / dt
    out = np.zeros(list(A.shape[:-1]) + [n])
    for iv in range(nv):
        for iu in range(nu):
            sh = s1 * us[iu] + s2 * vs[iv]
            E = np.zeros((no, n))
            for i in range(no):
                for j in range(n):
                    cc = (to[i] - ts[j] + sh) / dt
                    if abs(cc) < 1.0 + 0.5 * (al + be) + 1e-12:
                        E[i, j] = hat_avg2(cc, al, be)
            out[iv, iu, :] = E.T @ A[iv, iu, :]
    return np.moveaxis(out, -1, 2 - axis)


def general_plan(shape, sizes, Theta):
    """(P, voxel sizes after D, coefficients, permuted shape) of a rotation."""
    P, Tr = split_rotation(Theta)
    Dg, coeffs = factor_rotation(Tr)
    nz, ny, nx = shape
    n_src = (nx, ny, nz)
    km = [int(np.nonzero(P[m])[0][0]) for m in range(3)]
    n_new, s_new = [0, 0, 0], [0.0, 0.0, 0.0]
    for m in range(3):
        n_new[km[m]] = n_src[m]
        s_new[km[m]] = sizes[m]
    sr = tuple(s_new[k] / Dg[k] for k in range(3))
    return P, sr, coeffs, (n_new[2], n_new[1], n_new[0])


def rotate_general(X, sizes, Theta):
    """x^r = E^y E^x E^z P x for a general orientation; returns the rotated
    array [nz'][ny'][nx'] and its voxel sizes (dx', dy', dz')."""
    P, sr, (a, b, c, d, e, f), _ = general_plan(np.shape(X), sizes, Theta)
    Xp, _ = permute_volume(X, P, sizes)
    Z, _ = shear_pass(Xp, sr, 2, a, b)
    Y, _ = shear_pass(Z, sr, 0, c, d)
    R, _ = shear_pass(Y, sr, 1, e, f)
    return R, sr


def rotate_general_adjoint(G, shape, sizes, Theta):
    P, sr, (a, b, c, d, e, f), pshape = general_plan(shape, sizes, Theta)
    nzp, nyp, nxp = pshape
    Y = shear_pass_adjoint(G, sr, 1, e, f, nyp)
    Z = shear_pass_adjoint(Y, sr, 0, c, d, nxp)
    Xp = shear_pass_adjoint(Z, sr, 2, a, b, nzp)
    return permute_volume_adjoint(Xp, P, shape)
