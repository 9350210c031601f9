"""Pins of the oracle's 1-D transport entries (Sec. II-C, Tables II and III).

Each entry is fixed by something other than the table formulas themselves:
an independent polygon-clipping area, brute-force quadrature, closed-form
row/column sums (phase-space measure) and special cases.
"""
import numpy as np
import pytest

from oracle import optics, transport


def _geometries(seed=0, n=40):
    """(Xpq, X0q, label) position rows for the three kinds of transport the
    cameras use: slice -> detector through the main lens, slice -> array plane,
    array plane -> detector through an off-axis microlens."""
    rng = np.random.default_rng(seed)
    out = []
    for i in range(n):
        kind = i % 3
        if kind == 0:
            f = rng.uniform(20, 120)
            D = f * rng.uniform(1.01, 1.4)
            d = rng.uniform(100, 2500)
            Xpq = optics.compose(optics.propagate(D), optics.refract(f), optics.propagate(d))
            X0q = optics.propagate(d)
        elif kind == 1:
            f = rng.uniform(50, 120)
            D = f * rng.uniform(1.02, 1.1)
            d0 = 1.0 / (1.0 / f - 1.0 / D)
            d = d0 + rng.uniform(-60, 60)
            Xpq = optics.compose(optics.propagate(D), optics.refract(f), optics.propagate(d))
            X0q = optics.propagate(d)
        else:
            fm = rng.uniform(2.5, 3.5)
            c = rng.uniform(-10, 10)
            Xpq = optics.compose(optics.propagate(rng.uniform(1.5, 3.0)), optics.refract(fm, c))
            X0q = optics.propagate(-rng.uniform(80, 150))
        out.append((optics.s_row(Xpq), optics.s_row(X0q), kind))
    return out


def _jacobian(Xpq, X0q):
    return X0q[0] * Xpq[1] - X0q[1] * Xpq[0]


def test_table3_equals_polygon_clipping():
    rng = np.random.default_rng(11)
    worst = 0.0
    for Xpq, X0q, kind in _geometries(1, 60):
        dp = rng.uniform(0.005, 0.1)
        d0 = rng.uniform(0.3, 9.0)
        sk = rng.uniform(-4, 4)
        si = rng.uniform(-8, 8)
        tau, h, mag = transport.pillbox_params(Xpq, X0q, dp, sk, d0)
        lo, hi = si * mag + tau[0], si * mag + tau[3]
        w = hi - lo
        scale = d0 * dp / abs(_jacobian(Xpq, X0q))
        for _ in range(6):
            a = lo + w * rng.uniform(-0.5, 1.1)
            b = a + w * rng.uniform(0.05, 1.5)
            e1 = float(transport.pillbox_entry(Xpq, X0q, si, dp, sk, d0, a, b))
            e2 = transport.polygon_entry(Xpq, X0q, si, dp, sk, d0, a, b)
            worst = max(worst, abs(e1 - e2) / scale)
    assert worst < 1e-11, worst


def test_in_focus_entry_is_a_box():
    # X^{pq}_su = 0: the target position does not depend on u, so the entry is
    # Delta0/|X0q_su| times the length of {s in [a,b]: Pss s + Pb in pixel}.
    Xpq = (-0.0667, 0.0, 0.013)
    X0q = (1.0, 1680.0, 0.0)
    dp, d0, sk, si = 0.02, 4.5, 2.25, 0.37
    lo = (si - dp / 2 - Xpq[2]) / Xpq[0]
    hi = (si + dp / 2 - Xpq[2]) / Xpq[0]
    lo, hi = min(lo, hi), max(lo, hi)
    for a, b in [(lo - 1, lo + 0.1), (lo + 0.05, hi - 0.05), (hi - 0.1, hi + 3), (hi + 0.1, hi + 1)]:
        expect = d0 / 1680.0 * max(0.0, min(b, hi) - max(a, lo))
        got = float(transport.pillbox_entry(Xpq, X0q, si, dp, sk, d0, a, b))
        assert abs(got - expect) <= 1e-15 + 1e-12 * expect
        assert abs(transport.polygon_entry(Xpq, X0q, si, dp, sk, d0, a, b) - expect) <= 1e-15 + 1e-11 * expect


def test_pillbox_bruteforce_quadrature():
    # 2-D midpoint rule over (s, u) with the ray maps applied directly.
    for Xpq, X0q, kind in _geometries(5, 6):
        Mp = (np.array([[Xpq[0], Xpq[1]], [0, 1]]), np.array([Xpq[2], 0]))
        M0 = (np.array([[X0q[0], X0q[1]], [0, 1]]), np.array([X0q[2], 0]))
        dp, d0, sk, si = 0.05, 3.0, 0.7, 0.2
        tau, h, mag = transport.pillbox_params(Xpq, X0q, dp, sk, d0)
        lo, hi = si * mag + tau[0], si * mag + tau[3]
        a, b = lo + 0.3 * (hi - lo), hi + 0.2 * (hi - lo)
        us = [(sk + e * d0 / 2 - X0q[2] - X0q[0] * s) / X0q[1] for s in (a, b) for e in (-1, 1)]
        umin, umax = min(us), max(us)
        n = 1200
        s = a + (np.arange(n) + 0.5) * (b - a) / n
        u = umin + (np.arange(n) + 0.5) * (umax - umin) / n
        S, U = np.meshgrid(s, u, indexing="ij")
        lens, _ = optics.apply(M0, S, U)
        pos, _ = optics.apply(Mp, S, U)
        inside = (np.abs(lens - sk) <= d0 / 2) & (np.abs(pos - si) <= dp / 2)
        quad = inside.sum() * (b - a) * (umax - umin) / n / n
        exact = float(transport.pillbox_entry(Xpq, X0q, si, dp, sk, d0, a, b))
        assert abs(quad - exact) <= 6e-3 * exact


def test_row_and_column_sums_are_phase_space_measures():
    # Summed over a partition of the source plane, the entries give the
    # measure of {X0q in cell, Xpq in pixel} = D0 Dp / |J|; summed over a
    # partition of the target plane, the measure of {s in cell j, X0q in cell}
    # = Dq D0 / |X0q_su|.
    rng = np.random.default_rng(3)
    for Xpq, X0q, kind in _geometries(7, 30):
        dp = rng.uniform(0.005, 0.05)
        d0 = rng.uniform(0.5, 5.0)
        sk = rng.uniform(-2, 2)
        si = rng.uniform(-3, 3)
        tau, h, mag = transport.pillbox_params(Xpq, X0q, dp, sk, d0)
        lo, hi = si * mag + tau[0], si * mag + tau[3]
        dq = (hi - lo) / rng.uniform(0.3, 5.0)
        edges = lo - dq * rng.uniform(0.1, 0.9) + dq * np.arange(0, int((hi - lo) / dq) + 3)
        row = transport.pillbox_entry(Xpq, X0q, si, dp, sk, d0, edges[:-1], edges[1:]).sum()
        assert abs(row - d0 * dp / abs(_jacobian(Xpq, X0q))) < 1e-12 * row
        # column: source cell [a, b], targets tile the image of the cell
        a, b = lo, lo + dq
        tgt = np.concatenate([[si], si + dp * np.arange(1, 4000)])
        tgt = np.concatenate([tgt, si - dp * np.arange(1, 4000)])
        col = transport.pillbox_entry(Xpq, X0q, tgt, dp, sk, d0, a, b).sum()
        assert abs(col - dq * d0 / abs(X0q[1])) < 1e-10 * col


def test_dirac_bruteforce_and_pillbox_limit():
    rng = np.random.default_rng(9)
    for Xpq, X0q, kind in _geometries(13, 12):
        dp, d0, sk, si = 0.03, 2.0, rng.uniform(-1, 1), rng.uniform(-1, 1)
        tau, h, mag = transport.dirac_params(Xpq, X0q, dp, sk, d0)
        lo, hi = si * mag + tau[0], si * mag + tau[1]
        a, b = lo - 0.4 * (hi - lo), hi - 0.3 * (hi - lo)
        exact = float(transport.dirac_entry(Xpq, X0q, si, dp, sk, d0, a, b))
        # brute force: rays from s in [a, b] through the lens point s_k
        n = 200000
        s = a + (np.arange(n) + 0.5) * (b - a) / n
        u = (sk - X0q[2] - X0q[0] * s) / X0q[1]
        pos = Xpq[0] * s + Xpq[1] * u + Xpq[2]
        quad = d0 / abs(X0q[1]) * np.count_nonzero(np.abs(pos - si) <= dp / 2) * (b - a) / n
        assert abs(quad - exact) <= 2 * d0 / abs(X0q[1]) * (b - a) / n + 1e-15
        # thin pillbox cells converge to the Dirac entry at rate O(eps)
        errs = []
        for eps in (1e-2, 1e-3):
            thin = float(transport.pillbox_entry(Xpq, X0q, si, dp, sk, eps, a, b)) * d0 / eps
            errs.append(abs(thin - exact))
        assert errs[1] <= max(0.2 * errs[0], 1e-9 * exact + 1e-18)


def test_basis_volume_matches_polygon():
    # V^p (one axis) = measure of {s in pixel, X0p_s in cell}: a polygon
    # whose target strip is made wide enough to never clip.
    for d in (112.0, 31.3, 2.2):
        X0p = optics.s_row(optics.propagate(-d))
        dp, d0 = 0.02, 4.5
        area = transport.polygon_entry((0.0, 0.0, 0.0), X0p, 0.0, 1e9, 0.3, d0, -dp / 2, dp / 2)
        assert abs(area - transport.basis_volume(X0p[1], dp, d0)) < 1e-12 * area
