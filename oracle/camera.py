"""Camera system models (Sec. II-C..F and Sec. III) - oracle, test infrastructure.

Conventions (shared with the descriptors in the inputs module, not with any
CUDA code):
  * the camera's optical axis passes through the volume centre, the main lens
    is d_obj in front of it; slice n sits at object distance
    d_n = d_obj + (n - (nz-1)/2) dz and has its s and t axes along the
    volume's x and y axes (Sec. III: camera and object axes aligned);
  * pixel / voxel / lenslet centres are (index - (count-1)/2) * pitch;
  * the angular plane is the main lens (Sec. II-F); the lens is divided into
    ks x kt cells of width 2 r / ks tiling [-r, r]^2, and cells whose centre is
    strictly inside the aperture disc are kept (reading of Sec. II-B for a
    round lens), ordered with the s cell index fastest;
  * images are [nt][ns] with s fastest (Sec. IV, column-major views).

Scale factors.  The paper's detector model writes sqrt(V^d) sum_k f^d_k and the
plenoptic model sqrt(V^mu) B^{d mu}; with the un-normalised indicator bases of
eq. lf,disc the detector integral of basis element (k, i) is exactly
B^{ds}_k applied to the source coefficients, so (reading of Sec. II-E/F):
      single lens :  y = sum_k sum_n B^{dn}_k w^n,            w^n = dz x^n
      plenoptic   :  y = sum_k sum_mu B^{d mu}_k M_mu (1/V^a) sum_n B^{an}_k w^n
with V^a = (Da_s D0_s / D_mum) (Da_t D0_t / D_mum) the array-plane basis
volume.  The slice collapse w^n = dz x^n follows Sec. III (small angle, no
obliquity factor).  The mask M is binary: an array pixel belongs to lenslet mu
when its centre lies strictly inside mu's disc, and B^{d mu} acts only on mu's
own pixels.
"""
import numpy as np

from . import optics, transport


# ---------------------------------------------------------------------------
# grids and cells
# ---------------------------------------------------------------------------

def centers(n, pitch):
    return (np.arange(n, dtype=np.float64) - (n - 1) / 2.0) * pitch


def lens_cells(cam):
    """Angular cells on the main lens: list of (s_k, t_k, D0_s, D0_t)."""
    r = cam.r_main
    d0s = 2.0 * r / cam.ks
    d0t = 2.0 * r / cam.kt
    cells = []
    for kt in range(cam.kt):
        for ks in range(cam.ks):
            sk = -r + (ks + 0.5) * d0s
            tk = -r + (kt + 0.5) * d0t
            if sk * sk + tk * tk < r * r:
                cells.append((sk, tk, d0s, d0t))
    return cells


def _active(ci, cells):
    """Cell ci takes part (all cells when `cells` is None): the angular-plane
    subsets of the view-subset approximation (Sec. V, eq. subset)."""
    return cells is None or ci in cells


def slice_distances(vol, cam):
    return cam.d_obj + centers(vol.nz, vol.dz)


def _entry(cam):
    return transport.dirac_entry if cam.basis == 1 else transport.pillbox_entry


def matrix_1d(cam, Xpq, X0q, tgt, dp, s_k, d0, src, dsrc):
    """Dense 1-D transport matrix [len(tgt), len(src)] for one angular cell."""
    tgt = np.asarray(tgt, dtype=np.float64)[:, None]
    src = np.asarray(src, dtype=np.float64)[None, :]
    return _entry(cam)(optics.s_row(Xpq), optics.s_row(X0q), tgt, dp, s_k, d0,
                       src - dsrc / 2.0, src + dsrc / 2.0)


def slice_maps(cam, d, d_img):
    """Maps from a slice at object distance d: to the angular plane (the
    main lens, T_d) and through the main lens to an image plane d_img behind
    it (T_{d_img} o R_f o T_d)."""
    X0q = optics.propagate(d)
    Xpq = optics.compose(optics.propagate(d_img), optics.refract(cam.f_main),
                         optics.propagate(d))
    return Xpq, X0q


def slice_operators(vol, cam, n, cell, d_img, tgt_ns, tgt_nt, tgt_ps, tgt_pt):
    """(Bs, Bt) of the transport from slice n to an image plane (eq. xport,sep)."""
    sk, tk, d0s, d0t = cell
    d = slice_distances(vol, cam)[n]
    Xpq, X0q = slice_maps(cam, d, d_img)
    Bs = matrix_1d(cam, Xpq, X0q, centers(tgt_ns, tgt_ps), tgt_ps, sk, d0s,
                   centers(vol.nx, vol.dx), vol.dx)
    Bt = matrix_1d(cam, Xpq, X0q, centers(tgt_nt, tgt_pt), tgt_pt, tk, d0t,
                   centers(vol.ny, vol.dy), vol.dy)
    return Bs, Bt


# ---------------------------------------------------------------------------
# single-lens camera (Sec. II-F1, Sec. III)
# ---------------------------------------------------------------------------

def single_forward(vol, cam, x, cells=None):
    """y = sum_k sum_n B^{dn}_k (dz x^n), image [nt][ns] (k over `cells`)."""
    X = np.asarray(x, dtype=np.float64).reshape(vol.shape)
    y = np.zeros((cam.det_nt, cam.det_ns))
    for ci, cell in enumerate(lens_cells(cam)):
        if not _active(ci, cells):
            continue
        for n in range(vol.nz):
            Bs, Bt = slice_operators(vol, cam, n, cell, cam.d_lens_det,
                                     cam.det_ns, cam.det_nt, cam.det_ps, cam.det_pt)
            y += vol.dz * (Bt @ X[n] @ Bs.T)
    return y


def single_adjoint(vol, cam, y, cells=None):
    """x = A^T y = sum_k sum_n dz (B^{dn}_k)^T y  (Sec. IV-A: B^{pq} = (B^{qp})^T)."""
    Y = np.asarray(y, dtype=np.float64).reshape(cam.det_nt, cam.det_ns)
    x = np.zeros(vol.shape)
    for ci, cell in enumerate(lens_cells(cam)):
        if not _active(ci, cells):
            continue
        for n in range(vol.nz):
            Bs, Bt = slice_operators(vol, cam, n, cell, cam.d_lens_det,
                                     cam.det_ns, cam.det_nt, cam.det_ps, cam.det_pt)
            x[n] += vol.dz * (Bt.T @ Y @ Bs)
    return x


def single_matrix(vol, cam):
    """Explicit A (M x N) for tiny cameras: column blocks dz kron(Bt, Bs)."""
    M, N = cam.det_ns * cam.det_nt, vol.n
    A = np.zeros((M, N))
    blk = vol.nx * vol.ny
    for cell in lens_cells(cam):
        for n in range(vol.nz):
            Bs, Bt = slice_operators(vol, cam, n, cell, cam.d_lens_det,
                                     cam.det_ns, cam.det_nt, cam.det_ps, cam.det_pt)
            A[:, n * blk:(n + 1) * blk] += vol.dz * np.kron(Bt, Bs)
    return A


# ---------------------------------------------------------------------------
# plenoptic camera (Sec. II-F2, eq. plenoptic,factor)
# ---------------------------------------------------------------------------

def array_basis_volume(cam, cell):
    """V^a of the array-plane basis; X^{0a}: array plane back to the lens."""
    _, _, d0s, d0t = cell
    su = optics.s_row(optics.propagate(-cam.d_lens_mla))[1]
    return (transport.basis_volume(su, cam.arr_ps, d0s) *
            transport.basis_volume(su, cam.arr_pt, d0t))


def lenslet_centers(cam):
    return centers(cam.mla_ns, cam.mla_pitch), centers(cam.mla_nt, cam.mla_pitch)


def lenslet_centres_2d(cam):
    """Centres (s_mu, t_mu), mu = mt * mla_ns + ms: the square grid, or the
    hexagonal lattice (rows mla_pitch * sqrt(3)/2 apart, odd rows shifted by
    half a pitch, the lattice centred on the axis: column offset -1/4 pitch)."""
    ms = np.arange(cam.mla_ns)
    mt = np.arange(cam.mla_nt)
    if getattr(cam, "mla_layout", 0) == 1:
        t = (mt - (cam.mla_nt - 1) / 2.0) * cam.mla_pitch * np.sqrt(3.0) / 2.0
        S = (ms[None, :] - (cam.mla_ns - 1) / 2.0 + 0.5 * (mt[:, None] % 2) - 0.25) * cam.mla_pitch
        T = np.broadcast_to(t[:, None], S.shape)
    else:
        cs, ct = lenslet_centers(cam)
        S = np.broadcast_to(cs[None, :], (cam.mla_nt, cam.mla_ns))
        T = np.broadcast_to(ct[:, None], (cam.mla_nt, cam.mla_ns))
    return np.array(S, dtype=np.float64).ravel(), np.array(T, dtype=np.float64).ravel()


def transmission(cam):
    """The diagonal of the occlusion mask M (Sec. II-D, eq. occlusion) on the
    array grid: the microlens apertures (pixels owned by a lenslet) times an
    optional coded-mask transmission in [0, 1]."""
    m = (lenslet_owner(cam) >= 0).astype(np.float64)
    if getattr(cam, "arr_mask", None) is not None:
        m = m * np.asarray(cam.arr_mask, dtype=np.float64).reshape(cam.arr_nt, cam.arr_ns)
    return m


def lenslet_owner(cam):
    """owner[jt, js] = mt * mla_ns + ms of the lenslet whose disc strictly
    contains the array-pixel centre, -1 where the mask M blocks (Sec. II-D)."""
    if getattr(cam, "mla_layout", 0) == 1:
        return _hex_owner(cam)
    s = centers(cam.arr_ns, cam.arr_ps)
    t = centers(cam.arr_nt, cam.arr_pt)
    cs, ct = lenslet_centers(cam)
    ms = np.rint(s / cam.mla_pitch + (cam.mla_ns - 1) / 2.0).astype(np.int64)
    mt = np.rint(t / cam.mla_pitch + (cam.mla_nt - 1) / 2.0).astype(np.int64)
    oks = (ms >= 0) & (ms < cam.mla_ns)
    okt = (mt >= 0) & (mt < cam.mla_nt)
    msc = np.clip(ms, 0, cam.mla_ns - 1)
    mtc = np.clip(mt, 0, cam.mla_nt - 1)
    ds = s - cs[msc]
    dt = t - ct[mtc]
    inside = (ds[None, :] ** 2 + dt[:, None] ** 2 < cam.mla_radius ** 2)
    inside &= oks[None, :] & okt[:, None]
    return np.where(inside, mtc[:, None] * cam.mla_ns + msc[None, :], -1)


def _hex_owner(cam):
    """Hexagonal lattice: the nearest centre among the lenslets of the three
    nearest rows, kept when its disc strictly contains the pixel centre."""
    s = centers(cam.arr_ns, cam.arr_ps)[None, :]
    t = centers(cam.arr_nt, cam.arr_pt)[:, None]
    S, T = lenslet_centres_2d(cam)
    S = S.reshape(cam.mla_nt, cam.mla_ns)
    T = T.reshape(cam.mla_nt, cam.mla_ns)
    rowh = cam.mla_pitch * np.sqrt(3.0) / 2.0
    owner = np.full((cam.arr_nt, cam.arr_ns), -1, dtype=np.int64)
    mt0 = np.rint(t / rowh + (cam.mla_nt - 1) / 2.0).astype(np.int64)
    for dm in (-1, 0, 1):
        mt = mt0 + dm
        okt = (mt >= 0) & (mt < cam.mla_nt)
        mtc = np.clip(mt, 0, cam.mla_nt - 1)
        ms = np.rint(s / cam.mla_pitch + (cam.mla_ns - 1) / 2.0 - 0.5 * (mtc % 2) + 0.25).astype(np.int64)
        oks = (ms >= 0) & (ms < cam.mla_ns)
        msc = np.clip(ms, 0, cam.mla_ns - 1)
        d2 = (s - S[mtc, msc]) ** 2 + (t - T[mtc, msc]) ** 2
        inside = okt & oks & (d2 < cam.mla_radius ** 2)
        owner = np.where(inside, mtc * cam.mla_ns + msc, owner)
    return owner


def lenslet_maps(cam, f_mu, c_mu):
    """Array plane -> detector through lenslet mu (T_{D_mud} o R_{f_mu, c_mu})
    and array plane -> main lens (propagation back by D_mum)."""
    Xdq = optics.compose(optics.propagate(cam.d_mla_det), optics.refract(f_mu, c_mu))
    X0q = optics.propagate(-cam.d_lens_mla)
    return Xdq, X0q


class _StageTwo:
    """Per-lenslet 1-D matrices of the array -> detector transport over the
    lenslet's block (the bounding rows / columns of the pixels it owns),
    memoised by (axis, centre, focal length, block, cell)."""

    def __init__(self, cam):
        self.cam = cam
        self.owner = lenslet_owner(cam)
        self.trans = transmission(cam)
        self.S, self.T = lenslet_centres_2d(cam)
        self.arr_s = centers(cam.arr_ns, cam.arr_ps)
        self.arr_t = centers(cam.arr_nt, cam.arr_pt)
        self.det_s = centers(cam.det_ns, cam.det_ps)
        self.det_t = centers(cam.det_nt, cam.det_pt)
        self.cache = {}
        nmu = cam.mla_ns * cam.mla_nt
        jt, js = np.nonzero(self.owner >= 0)
        mu = self.owner[jt, js]
        lo_c = np.full(nmu, cam.arr_ns); hi_c = np.full(nmu, -1)
        lo_r = np.full(nmu, cam.arr_nt); hi_r = np.full(nmu, -1)
        np.minimum.at(lo_c, mu, js); np.maximum.at(hi_c, mu, js)
        np.minimum.at(lo_r, mu, jt); np.maximum.at(hi_r, mu, jt)
        self.cols = [np.arange(lo_c[m], hi_c[m] + 1) for m in range(nmu)]
        self.rows = [np.arange(lo_r[m], hi_r[m] + 1) for m in range(nmu)]

    def mat(self, axis, mu, f_mu, cell_idx, cell):
        cam = self.cam
        sk, tk, d0s, d0t = cell
        if axis == 0:
            key = (0, float(self.S[mu]), float(f_mu), int(self.cols[mu][0]) if len(self.cols[mu]) else -1,
                   len(self.cols[mu]), cell_idx)
        else:
            key = (1, float(self.T[mu]), float(f_mu), int(self.rows[mu][0]) if len(self.rows[mu]) else -1,
                   len(self.rows[mu]), cell_idx)
        if key not in self.cache:
            if axis == 0:
                Xdq, X0q = lenslet_maps(cam, f_mu, self.S[mu])
                B = matrix_1d(cam, Xdq, X0q, self.det_s, cam.det_ps, sk, d0s,
                              self.arr_s[self.cols[mu]], cam.arr_ps)
            else:
                Xdq, X0q = lenslet_maps(cam, f_mu, self.T[mu])
                B = matrix_1d(cam, Xdq, X0q, self.det_t, cam.det_pt, tk, d0t,
                              self.arr_t[self.rows[mu]], cam.arr_pt)
            nz = np.nonzero(np.any(B != 0.0, axis=1))[0]
            self.cache[key] = (nz, B[nz])
        return self.cache[key]


def plenoptic_array_field(vol, cam, x, cell):
    """Masked array-plane coefficients M (1/V^a) sum_n B^{an}_k (dz x^n)."""
    X = np.asarray(x, dtype=np.float64).reshape(vol.shape)
    Fa = np.zeros((cam.arr_nt, cam.arr_ns))
    for n in range(vol.nz):
        Bs, Bt = slice_operators(vol, cam, n, cell, cam.d_lens_mla,
                                 cam.arr_ns, cam.arr_nt, cam.arr_ps, cam.arr_pt)
        Fa += vol.dz * (Bt @ X[n] @ Bs.T)
    Fa /= array_basis_volume(cam, cell)
    return transmission(cam) * Fa


def plenoptic_array_block(vol, cam, x, cell, rows, cols):
    """Entries [rows][cols] of plenoptic_array_field: the same sum with each
    axis' transport matrix restricted to those array rows and columns (spot
    checks of planes too large for the whole field)."""
    X = np.asarray(x, dtype=np.float64).reshape(vol.shape)
    rows, cols = np.asarray(rows), np.asarray(cols)
    sk, tk, d0s, d0t = cell
    ts = centers(cam.arr_ns, cam.arr_ps)[cols]
    tt = centers(cam.arr_nt, cam.arr_pt)[rows]
    Fa = np.zeros((len(rows), len(cols)))
    for n in range(vol.nz):
        Xpq, X0q = slice_maps(cam, slice_distances(vol, cam)[n], cam.d_lens_mla)
        Bs = matrix_1d(cam, Xpq, X0q, ts, cam.arr_ps, sk, d0s, centers(vol.nx, vol.dx), vol.dx)
        Bt = matrix_1d(cam, Xpq, X0q, tt, cam.arr_pt, tk, d0t, centers(vol.ny, vol.dy), vol.dy)
        Fa += vol.dz * (Bt @ X[n] @ Bs.T)
    Fa /= array_basis_volume(cam, cell)
    return transmission(cam)[np.ix_(rows, cols)] * Fa


def plenoptic_stage2(cam, fields, st=None, cells=None):
    """y = sum_k sum_mu B^{d mu}_k fa_k for given (masked) array-plane fields
    [K][arr_nt][arr_ns] (k over `cells`)."""
    st = _StageTwo(cam) if st is None else st
    y = np.zeros((cam.det_nt, cam.det_ns))
    for ci, cell in enumerate(lens_cells(cam)):
        if not _active(ci, cells):
            continue
        Fa = np.asarray(fields[ci], dtype=np.float64)
        for mt in range(cam.mla_nt):
            for ms in range(cam.mla_ns):
                mu = mt * cam.mla_ns + ms
                rows, cols = st.rows[mu], st.cols[mu]
                if len(rows) == 0 or len(cols) == 0:
                    continue
                f_mu = cam.mla_focal[mt, ms]
                rs, Bs = st.mat(0, mu, f_mu, ci, cell)
                rt, Bt = st.mat(1, mu, f_mu, ci, cell)
                if len(rs) == 0 or len(rt) == 0:
                    continue
                sub = Fa[np.ix_(rows, cols)] * (st.owner[np.ix_(rows, cols)] == mu)
                y[np.ix_(rt, rs)] += Bt @ sub @ Bs.T
    return y


def plenoptic_stage2_adjoint(cam, y, st=None, cells=None):
    """M sum_mu (B^{d mu}_k)^T y for every cell: fields [K][arr_nt][arr_ns]
    (zero for cells outside `cells`)."""
    st = _StageTwo(cam) if st is None else st
    Y = np.asarray(y, dtype=np.float64).reshape(cam.det_nt, cam.det_ns)
    out = []
    for ci, cell in enumerate(lens_cells(cam)):
        Ga = np.zeros((cam.arr_nt, cam.arr_ns))
        if not _active(ci, cells):
            out.append(Ga)
            continue
        for mt in range(cam.mla_nt):
            for ms in range(cam.mla_ns):
                mu = mt * cam.mla_ns + ms
                rows, cols = st.rows[mu], st.cols[mu]
                if len(rows) == 0 or len(cols) == 0:
                    continue
                f_mu = cam.mla_focal[mt, ms]
                rs, Bs = st.mat(0, mu, f_mu, ci, cell)
                rt, Bt = st.mat(1, mu, f_mu, ci, cell)
                if len(rs) == 0 or len(rt) == 0:
                    continue
                g = Bt.T @ Y[np.ix_(rt, rs)] @ Bs
                own = st.owner[np.ix_(rows, cols)] == mu
                Ga[np.ix_(rows, cols)] += np.where(own, g * st.trans[np.ix_(rows, cols)], 0.0)
        out.append(Ga)
    return np.stack(out)


def plenoptic_stage1_adjoint(vol, cam, fields, cells=None):
    """sum_k sum_n dz (B^{an}_k)^T (1/V^a) g_k for given fields g."""
    x = np.zeros(vol.shape)
    for ci, cell in enumerate(lens_cells(cam)):
        if not _active(ci, cells):
            continue
        Ga = np.asarray(fields[ci], dtype=np.float64) / array_basis_volume(cam, cell)
        for n in range(vol.nz):
            Bs, Bt = slice_operators(vol, cam, n, cell, cam.d_lens_mla,
                                     cam.arr_ns, cam.arr_nt, cam.arr_ps, cam.arr_pt)
            x[n] += vol.dz * (Bt.T @ Ga @ Bs)
    return x


def plenoptic_forward(vol, cam, x, return_array=False, cells=None):
    """y = sum_k sum_mu B^{d mu}_k M_mu (1/V^a) sum_n B^{an}_k w^n."""
    fields = np.stack([plenoptic_array_field(vol, cam, x, cell) if _active(ci, cells)
                       else np.zeros((cam.arr_nt, cam.arr_ns)) for ci, cell in enumerate(lens_cells(cam))])
    y = plenoptic_stage2(cam, fields, cells=cells)
    if return_array:
        return y, fields
    return y


def plenoptic_adjoint(vol, cam, y, return_array=False, cells=None):
    """x = sum_k sum_n dz (B^{an}_k)^T (1/V^a) M sum_mu (B^{d mu}_k)^T y."""
    fields = plenoptic_stage2_adjoint(cam, y, cells=cells)
    x = plenoptic_stage1_adjoint(vol, cam, fields, cells=cells)
    if return_array:
        return x, fields
    return x


def plenoptic_matrix(vol, cam):
    """Explicit A for tiny plenoptic cameras, built term by term from the
    factorised model (eq. plenoptic,factor)."""
    owner = lenslet_owner(cam)
    S_mu, T_mu = lenslet_centres_2d(cam)
    arr_s = centers(cam.arr_ns, cam.arr_ps)
    arr_t = centers(cam.arr_nt, cam.arr_pt)
    det_s = centers(cam.det_ns, cam.det_ps)
    det_t = centers(cam.det_nt, cam.det_pt)
    Na = cam.arr_ns * cam.arr_nt
    blk = vol.nx * vol.ny
    A = np.zeros((cam.det_ns * cam.det_nt, vol.n))
    for cell in lens_cells(cam):
        sk, tk, d0s, d0t = cell
        S1 = np.zeros((Na, vol.n))
        for n in range(vol.nz):
            Bs, Bt = slice_operators(vol, cam, n, cell, cam.d_lens_mla,
                                     cam.arr_ns, cam.arr_nt, cam.arr_ps, cam.arr_pt)
            S1[:, n * blk:(n + 1) * blk] = vol.dz * np.kron(Bt, Bs)
        S2 = np.zeros((cam.det_ns * cam.det_nt, Na))
        for mt in range(cam.mla_nt):
            for ms in range(cam.mla_ns):
                mu = mt * cam.mla_ns + ms
                f_mu = cam.mla_focal[mt, ms]
                Xs, X0 = lenslet_maps(cam, f_mu, S_mu[mu])
                Xt, _ = lenslet_maps(cam, f_mu, T_mu[mu])
                Bs = matrix_1d(cam, Xs, X0, det_s, cam.det_ps, sk, d0s, arr_s, cam.arr_ps)
                Bt = matrix_1d(cam, Xt, X0, det_t, cam.det_pt, tk, d0t, arr_t, cam.arr_pt)
                own = (owner.reshape(-1) == mu).astype(np.float64)
                S2 += np.kron(Bt, Bs) * own[None, :]
        mask = transmission(cam).reshape(-1)
        A += S2 @ (mask[:, None] * S1) / array_basis_volume(cam, cell)
    return A


# ---------------------------------------------------------------------------
# rotated cameras (Sec. III-A: A_c = C_c o rotation) and dispatch
# ---------------------------------------------------------------------------

class Grid:
    """Plain voxel-grid description (duck-types the volume descriptor)."""

    def __init__(self, nx, ny, nz, dx, dy, dz):
        self.nx, self.ny, self.nz, self.dx, self.dy, self.dz = nx, ny, nz, dx, dy, dz

    @property
    def n(self):
        return self.nx * self.ny * self.nz

    @property
    def shape(self):
        return (self.nz, self.ny, self.nx)


class _Aligned:
    """The camera descriptor with the yaw removed (it sees the rotated grid)."""

    def __init__(self, cam):
        self.__dict__.update(cam.__dict__)
        self.yaw = 0.0
        self.pitch = 0.0
        self.roll = 0.0

    @property
    def m(self):
        return self.det_ns * self.det_nt


def _general(cam):
    """The camera has a pitch or roll: the three-shear rotation applies."""
    return getattr(cam, "pitch", 0.0) != 0.0 or getattr(cam, "roll", 0.0) != 0.0


def _rotated(cam):
    return cam.yaw != 0.0 or _general(cam)


def rotated_volume(vol, cam, x):
    from . import rotation
    X = np.asarray(x, dtype=np.float64).reshape(vol.shape)
    sizes = (vol.dx, vol.dy, vol.dz)
    if _general(cam):
        Xr, sr = rotation.rotate_general(X, sizes, rotation.camera_rotation(cam.yaw, cam.pitch, cam.roll))
    else:
        Xr, sr = rotation.rotate(X, sizes, cam.yaw)
    g = Grid(Xr.shape[2], Xr.shape[1], Xr.shape[0], sr[0], sr[1], sr[2])
    return g, Xr


def _aligned_forward(vol, cam, x, cells=None):
    if cam.kind == 1:
        return plenoptic_forward(vol, cam, x, cells=cells)
    return single_forward(vol, cam, x, cells=cells)


def _aligned_adjoint(vol, cam, y, cells=None):
    if cam.kind == 1:
        return plenoptic_adjoint(vol, cam, y, cells=cells)
    return single_adjoint(vol, cam, y, cells=cells)


def forward(vol, cam, x, cells=None):
    """A x, or sum_{k in cells} A_k x (angular-plane subset, Sec. V)."""
    if _rotated(cam):
        g, Xr = rotated_volume(vol, cam, x)
        return _aligned_forward(g, _Aligned(cam), Xr, cells)
    return _aligned_forward(vol, cam, x, cells)


def adjoint(vol, cam, y, cells=None):
    if _rotated(cam):
        from . import rotation
        sizes = (vol.dx, vol.dy, vol.dz)
        if _general(cam):
            T = rotation.camera_rotation(cam.yaw, cam.pitch, cam.roll)
            Xr, sr = rotation.rotate_general(np.zeros(vol.shape), sizes, T)   # grid only
            shape_r = Xr.shape
        else:
            shape_r, sr, _ = rotation.rotated_grid(vol.shape, sizes, cam.yaw)
        g = Grid(shape_r[2], shape_r[1], shape_r[0], sr[0], sr[1], sr[2])
        Gr = _aligned_adjoint(g, _Aligned(cam), y, cells)
        if _general(cam):
            return rotation.rotate_general_adjoint(Gr, vol.shape, sizes, T)
        return rotation.rotate_adjoint(Gr, vol.shape, sizes, cam.yaw)
    return _aligned_adjoint(vol, cam, y, cells)


def system_matrix(vol, cam):
    if cam.kind == 1:
        return plenoptic_matrix(vol, cam)
    return single_matrix(vol, cam)
