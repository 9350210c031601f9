"""Ray maps of geometric optics (Sec. II-A, Table I) - oracle, test infrastructure.

A ray crossing a plane normal to the optical axis is theta = (s, u, t, v):
position (s, t) and slope (u, v) = (ds/dz, dt/dz), with z increasing from the
scene towards the detector.  Every map used by the paper is affine and
separable into an (s, u) block and a (t, v) block (Sec. II-A, the separable
form of X).  This module handles one axis: a map is a pair (M, b) with M a
2x2 float64 matrix and b a 2-vector, acting as theta' = M theta + b.
"""
import numpy as np


def identity():
    return np.eye(2), np.zeros(2)


def propagate(d):
    """Free-space propagation by d (Table I, T_d): s' = s + d u, u' = u."""
    return np.array([[1.0, d], [0.0, 1.0]]), np.zeros(2)


def refract(f, s0=0.0):
    """Thin-lens refraction, focal length f, centre s0 (Table I, R_f):
    s' = s, u' = u - s/f + s0/f."""
    return np.array([[1.0, 0.0], [-1.0 / f, 1.0]]), np.array([0.0, s0 / f])


def compose(*maps):
    """compose(A, B, C) = A o B o C (C applied first)."""
    M, b = identity()
    for Mi, bi in reversed(maps):
        M, b = Mi @ M, Mi @ b + bi
    return M, b


def apply(X, s, u):
    M, b = X
    return M[0, 0] * s + M[0, 1] * u + b[0], M[1, 0] * s + M[1, 1] * u + b[1]


def s_row(X):
    """(X_ss, X_su, Xbar_s): the position row of a map (Sec. II-A notation)."""
    M, b = X
    return float(M[0, 0]), float(M[0, 1]), float(b[0])
