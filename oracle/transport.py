"""One-dimensional light-transport entries (Sec. II-C) - oracle, test infrastructure.

The entry [B^{pq}_k]_{ij} of the least-squares transport (eq. xport) factors
into an s integral and a t integral (eq. xport,int / xport,sep).  Each factor
is the (s, u) inner product of eq. xport,ip:

    B = area{ (s, u) on plane q :  s in source cell j,
                                   X^{0q}_s(s, u) in angular cell k,
                                   X^{pq}_s(s, u) in target pixel i }

for the pillbox angular basis (a = rect, and a^2 = a), and the length of the
line X^{0q}_s = s_k inside the other two sets times Delta^0/|X^{0q}_su| for
the Dirac basis.

Three independent evaluations are provided:
  pillbox_entry   -- Table III closed form: trapezoid blur kernel g with the
                     four breakpoints tau (all four +/- combinations, sorted),
                     height min(|D0/X0q_su|, |Dp/Xpq_su|), magnification 1/alpha,
                     integrated exactly over the source cell.
  dirac_entry     -- Table II closed form (box kernel).
  polygon_entry   -- direct geometry: Sutherland-Hodgman clipping of the
                     source-cell rectangle in (s, u) against the angular-cell
                     strip and the target-pixel strip, area by the shoelace
                     formula.  Shares no algebra with the tables.
Readings of garbled/ambiguous table entries:
  * tau-hat is written with a linked "+/- ... -/+"; a trapezoid has four
    breakpoints, so all four sign combinations are used.
  * the blur height's "X^{pqk}_su" is read as X^{pq}_su.
  * Table II's blur kernel is written in w; it is read as s.
"""
import numpy as np


def _rows(Xpq, X0q):
    Pss, Psu, Pb = Xpq
    Lss, Lsu, Lb = X0q
    return Pss, Psu, Pb, Lss, Lsu, Lb


def _clip_interval(lo, hi, a, b):
    L = np.maximum(lo, a)
    H = np.minimum(hi, b)
    return L, H, H > L


def trapezoid_integral(t1, t2, t3, t4, a, b):
    """Exact integral over [a, b] of the unit-height trapezoid g of Table III:
    (s - t1)/(t2 - t1) on [t1, t2), 1 on [t2, t3), 1 - (s - t3)/(t4 - t3) on
    [t3, t4), 0 elsewhere.  Zero-width ramps contribute nothing."""
    t1, t2, t3, t4, a, b = np.broadcast_arrays(*(np.asarray(v, dtype=np.float64)
                                                 for v in (t1, t2, t3, t4, a, b)))
    out = np.zeros(t1.shape)
    L, H, ok = _clip_interval(t1, t2, a, b)
    w = t2 - t1
    ok = ok & (w > 0)
    ws = np.where(ok, w, 1.0)
    out += np.where(ok, ((H - t1) ** 2 - (L - t1) ** 2) / (2.0 * ws), 0.0)
    L, H, ok = _clip_interval(t2, t3, a, b)
    out += np.where(ok, H - L, 0.0)
    L, H, ok = _clip_interval(t3, t4, a, b)
    w = t4 - t3
    ok = ok & (w > 0)
    ws = np.where(ok, w, 1.0)
    out += np.where(ok, ((t4 - L) ** 2 - (t4 - H) ** 2) / (2.0 * ws), 0.0)
    return out


def pillbox_params(Xpq, X0q, dp, s_k, d0):
    """Table III blur parameters: sorted breakpoints tau (relative to the
    magnified pixel centre s_i/alpha), height h and magnification 1/alpha."""
    Pss, Psu, Pb, Lss, Lsu, Lb = _rows(Xpq, X0q)
    alpha = Pss - Psu * Lss / Lsu
    beta = Psu / Lsu
    gamma = Pb - Psu * Lb / Lsu
    tau_hat = [(sp * dp / 2.0 - beta * (s_k + sk * d0 / 2.0) - gamma) / alpha
               for sp in (1.0, -1.0) for sk in (1.0, -1.0)]
    tau = np.sort(np.array(tau_hat))
    h_lens = abs(d0 / Lsu)
    h_pix = abs(dp / Psu) if Psu != 0.0 else np.inf
    h = min(h_lens, h_pix)
    return tau, h, 1.0 / alpha


def pillbox_entry(Xpq, X0q, s_i, dp, s_k, d0, a, b):
    """[B^{pq}_k]_{ij} (one axis) for the pillbox angular basis, Table III.

    Xpq, X0q: position rows (X_ss, X_su, Xbar_s) of the maps from the source
    plane q to the target plane p and to the angular plane.  s_i, dp: target
    pixel centre and width; s_k, d0: angular cell centre and width; [a, b]:
    source cell.  Arrays broadcast."""
    tau, h, mag = pillbox_params(Xpq, X0q, dp, s_k, d0)
    shift = mag * np.asarray(s_i, dtype=np.float64)
    return h * trapezoid_integral(shift + tau[0], shift + tau[1],
                                  shift + tau[2], shift + tau[3], a, b)


def dirac_params(Xpq, X0q, dp, s_k, d0):
    """Table II blur parameters (box kernel)."""
    Pss, Psu, Pb, Lss, Lsu, Lb = _rows(Xpq, X0q)
    alpha = Pss - Lss * Psu / Lsu
    beta = Pb + Psu * (s_k - Lb) / Lsu
    tau = np.sort(np.array([(dp / 2.0 - beta) / alpha, (-dp / 2.0 - beta) / alpha]))
    h = d0 / abs(Lsu)
    return tau, h, 1.0 / alpha


def dirac_entry(Xpq, X0q, s_i, dp, s_k, d0, a, b):
    """[B^{pq}_k]_{ij} (one axis) for the Dirac angular basis, Table II."""
    tau, h, mag = dirac_params(Xpq, X0q, dp, s_k, d0)
    shift = mag * np.asarray(s_i, dtype=np.float64)
    L, H, ok = _clip_interval(shift + tau[0], shift + tau[1], np.asarray(a, float), np.asarray(b, float))
    return h * np.where(ok, H - L, 0.0)


def basis_volume(X0p_su, dp, d0):
    """One-axis factor of the basis-element volume V^p = Dp * |D0 / X0p_su|
    (Table II; also used for the pillbox basis - the exact measure of the
    set {s in pixel, X0p_s in cell} does not depend on the angular basis)."""
    return dp * abs(d0 / X0p_su)


# ---------------------------------------------------------------------------
# Independent geometric evaluation (no Table II/III algebra)
# ---------------------------------------------------------------------------

def _clip(poly, cs, cu, c0):
    """Sutherland-Hodgman: keep the part of a convex polygon with
    cs*s + cu*u + c0 >= 0."""
    out = []
    n = len(poly)
    for i in range(n):
        P = poly[i]
        Q = poly[(i + 1) % n]
        fp = cs * P[0] + cu * P[1] + c0
        fq = cs * Q[0] + cu * Q[1] + c0
        if fp >= 0:
            out.append(P)
        if (fp >= 0) != (fq >= 0):
            t = fp / (fp - fq)
            out.append((P[0] + t * (Q[0] - P[0]), P[1] + t * (Q[1] - P[1])))
    return out


def _area(poly):
    if len(poly) < 3:
        return 0.0
    s0, u0 = poly[0]
    acc = 0.0
    for i in range(1, len(poly) - 1):
        s1, u1 = poly[i][0] - s0, poly[i][1] - u0
        s2, u2 = poly[i + 1][0] - s0, poly[i + 1][1] - u0
        acc += s1 * u2 - s2 * u1
    return abs(acc) / 2.0


def polygon_entry(Xpq, X0q, s_i, dp, s_k, d0, a, b):
    """Area of {s in [a,b], X0q_s in cell k, Xpq_s in pixel i} in (s, u)
    by polygon clipping (scalar arguments)."""
    Pss, Psu, Pb, Lss, Lsu, Lb = _rows(Xpq, X0q)
    us = [(s_k + e * d0 / 2.0 - Lb - Lss * s) / Lsu for s in (a, b) for e in (-1.0, 1.0)]
    umin, umax = min(us), max(us)
    poly = [(a, umin), (b, umin), (b, umax), (a, umax)]
    strips = [(Lss, Lsu, Lb - (s_k - d0 / 2.0)), (-Lss, -Lsu, (s_k + d0 / 2.0) - Lb),
              (Pss, Psu, Pb - (s_i - dp / 2.0)), (-Pss, -Psu, (s_i + dp / 2.0) - Pb)]
    for cs, cu, c0 in strips:
        poly = _clip(poly, cs, cu, c0)
        if not poly:
            return 0.0
    return _area(poly)
