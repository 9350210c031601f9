"""Reconstruction algorithm of Table V (Sec. V) - oracle, test infrastructure.

Penalised weighted non-negative least squares with unknown camera gains
(eq. pls):

  Psi(x, {g_c}) = 1/2 ||A_1 x - y_1||^2_{W_1} + sum_{c>1} 1/2 ||A_c x - g_c y_c||^2_{W_c}
                  + nu ||x||_1 + R(x),
  R(x) = beta/2 sum_j sum_{l in N26(j)} psi(x_j - x_l)                 (eq. reg)

solved by the preconditioned FISTA iteration of Table V with the diagonal
majoriser D = diag(sum_c A_c^T W_c A_c 1) (Appendix A).

Readings:
  * the t update of Table V is t^{(n+1)};
  * gains are computed from the projection of the momentum point z^{(n)};
  * where D_j + 26 beta = 0 (a voxel no camera sees, beta = 0) w_j = 0;
  * psi is the quadratic t^2/2 (the paper's experiments) or the hyperbola
    delta^2 (sqrt(1 + (t/delta)^2) - 1) (even, convex, curvature <= 1);
  * the regulariser curvature bound is 26 beta as printed; ``reg_scale``
    lets a caller use the exact 36 beta bound of the 26-neighbour Laplacian.
"""
import itertools

import numpy as np

OFFSETS = [o for o in itertools.product((-1, 0, 1), repeat=3) if o != (0, 0, 0)]


def psi_prime(t, psi, delta):
    if psi == 0:
        return t
    return t / np.sqrt(1.0 + (t / delta) ** 2)


def grad_R(z, shape, beta, psi=0, delta=1.0):
    """dR/dx_j = beta sum_{l in N26(j)} psi'(x_j - x_l); neighbours outside
    the volume do not exist."""
    Z = np.asarray(z, dtype=np.float64).reshape(shape)
    g = np.zeros(shape)
    nz, ny, nx = shape
    for oz, oy, ox in OFFSETS:
        # neighbour l = j + o exists where 0 <= index + o < n on every axis
        sz = slice(max(0, -oz), nz - max(0, oz))
        sy = slice(max(0, -oy), ny - max(0, oy))
        sx = slice(max(0, -ox), nx - max(0, ox))
        tz = slice(max(0, oz), nz - max(0, -oz))
        ty = slice(max(0, oy), ny - max(0, -oy))
        tx = slice(max(0, ox), nx - max(0, -ox))
        g[sz, sy, sx] += psi_prime(Z[sz, sy, sx] - Z[tz, ty, tx], psi, delta)
    return beta * g.reshape(-1)


def R_value(x, shape, beta, psi=0, delta=1.0):
    X = np.asarray(x, dtype=np.float64).reshape(shape)
    nz, ny, nx = shape
    acc = 0.0
    for oz, oy, ox in OFFSETS:
        sz = slice(max(0, -oz), nz - max(0, oz))
        sy = slice(max(0, -oy), ny - max(0, oy))
        sx = slice(max(0, -ox), nx - max(0, ox))
        tz = slice(max(0, oz), nz - max(0, -oz))
        ty = slice(max(0, oy), ny - max(0, -oy))
        tx = slice(max(0, ox), nx - max(0, -ox))
        d = X[sz, sy, sx] - X[tz, ty, tx]
        acc += np.sum(0.5 * d * d if psi == 0 else delta ** 2 * (np.sqrt(1 + (d / delta) ** 2) - 1))
    return 0.5 * beta * acc


def optimal_gain(y, p, w):
    """gamma_c = y^T W p / y^T W y (Table V step 1b; eq. optimal,gain)."""
    den = float(np.sum(w * y * y))
    return float(np.sum(w * y * p)) / den if den > 0 else 0.0


def majorizer(ops, weights, n):
    """D = diag(sum_c A_c^T W_c A_c 1) (Table V initialisation)."""
    ones = np.ones(n)
    D = np.zeros(n)
    for (A, At), w in zip(ops, weights):
        D += At(w * A(ones))
    return D


def objective(ops, ys, weights, gains, x, shape, beta, nu, psi=0, delta=1.0):
    val = 0.0
    for (A, _), y, w, g in zip(ops, ys, weights, gains):
        r = A(x) - g * y
        val += 0.5 * float(np.sum(w * r * r))
    return val + nu * float(np.sum(np.abs(x))) + R_value(x, shape, beta, psi, delta)


def subset_cells(n_cells, n_subset, it):
    """Cells of the angular-plane subset used at iteration `it` (0-based):
    every n_subset-th cell in lexicographic order, k = it mod n_subset,
    it mod n_subset + n_subset, ... (Sec. V, view-subset acceleration)."""
    return [k for k in range(n_cells) if k % n_subset == it % n_subset]


def fista(ops, ys, weights, shape, n_iter, beta=0.0, nu=0.0, psi=0, delta=1.0,
          reg_scale=26.0, x0=None, estimate_gains=True, history=False, n_subset=1, n_cells=None):
    """Table V.  ops: list of (A_c, A_c^T) callables on flat float64 vectors;
    ys / weights: flat measurement and weight vectors.  Returns a dict with
    x, z, gains, t, D (and the per-iteration data-fit at z if history).

    With n_subset > 1 (eq. subset) the callables also take cells=[k, ...] and
    n_cells[c] gives camera c's K; iteration `it` uses S = subset_cells(K,
    n_subset, it) and a = K / |S|: p = a sum_{k in S} A_ck z, the gain from p,
    r = p - gamma y and g_c = a sum_{k in S} A_ck^T W r.  A camera whose subset
    is empty contributes no gradient (a = 0).  The majoriser D stays the full
    one (all cells)."""
    n = int(np.prod(shape))
    ys = [np.asarray(y, dtype=np.float64).reshape(-1) for y in ys]
    weights = [np.ones_like(y) if w is None else np.asarray(w, dtype=np.float64).reshape(-1)
               for y, w in zip(ys, weights)]
    D = majorizer(ops, weights, n)
    x = np.zeros(n) if x0 is None else np.asarray(x0, dtype=np.float64).reshape(-1).copy()
    z = x.copy()
    t = 1.0
    gains = [1.0] + [0.0 if estimate_gains else 1.0] * (len(ops) - 1)
    denom = D + reg_scale * beta
    fits = []
    for _ in range(n_iter):
        g = np.zeros(n)
        fit = 0.0
        for c, ((A, At), y, w) in enumerate(zip(ops, ys, weights)):
            if n_subset > 1:
                S = subset_cells(n_cells[c], n_subset, len(fits))
                a = n_cells[c] / len(S) if S else 0.0
                p = a * A(z, cells=S) if S else np.zeros_like(y)
            else:
                p = A(z)
            if c > 0 and estimate_gains:
                gains[c] = optimal_gain(y, p, w)
            r = p - gains[c] * y
            fit += 0.5 * float(np.sum(w * r * r))
            if n_subset > 1:
                if S:
                    g += a * At(w * r, cells=S)
            else:
                g += At(w * r)
        fits.append(fit)
        t_new = (1.0 + np.sqrt(1.0 + 4.0 * t * t)) / 2.0
        step = g + grad_R(z, shape, beta, psi, delta)
        safe = np.where(denom > 0, denom, 1.0)
        wv = np.where(denom > 0, np.maximum(z - step / safe, 0.0), 0.0)
        x_new = np.maximum(wv - nu, 0.0)
        z = x_new + ((t - 1.0) / t_new) * (x_new - x)
        x = x_new
        t = t_new
    out = dict(x=x, z=z, gains=gains, t=t, D=D)
    if history:
        out["fits"] = fits
    return out
