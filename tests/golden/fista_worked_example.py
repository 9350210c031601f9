"""Worked example of the Table V iteration (Sec. V) in exact arithmetic.

Writes fista_worked_example.json: three iterations of preconditioned FISTA on
a problem small enough to follow by hand, every intermediate quantity of
every step recorded, so that each line can be checked against Table V with a
calculator.  The arithmetic is exact (rationals and nested square roots,
sympy as the calculator) and only rounded to 17 significant digits when
written.  Nothing here imports the oracle or the CUDA library: the values
pin the oracle's iteration, they do not come from it.

Problem (three voxels on a line along x, shape (1, 1, 3), so voxel j's
26-neighbourhood inside the volume is j - 1 and j + 1):

  camera 1: A_1 = [[2,1,0],[1,3,1],[0,1,2]], y_1 = [3, 4, -1], W_1 = I
  camera 2: A_2 = [[1,0,1],[1,1,0]],         y_2 = [1, 2],     W_2 = diag(2, 1)

Table V, as read here: x^0 = z^0 = 0, t^0 = 1, gamma_1 = 1 and gamma_2 = 0
(recomputed from p_2 before use when gains are estimated, else 1);
D = diag(sum_c A_c^T W_c A_c 1) = [11, 21, 11] + [6, 2, 4] = [17, 23, 15];
per iteration n:
  p_c = A_c z^n;  gamma_c = y_c^T W_c p_c / y_c^T W_c y_c  (c > 1);
  r_c = p_c - gamma_c y_c;  g = sum_c A_c^T W_c r_c;
  grad R(z)_j = beta sum_{l in N(j)} (z_j - z_l)   (quadratic psi);
  t^{n+1} = (1 + sqrt(1 + 4 (t^n)^2)) / 2;
  w = [z^n - (g + grad R(z^n)) / (D + 26 beta)]_+;
  x^{n+1} = [w - nu]_+;
  z^{n+1} = x^{n+1} + ((t^n - 1) / t^{n+1}) (x^{n+1} - x^n).
The data fit recorded for iteration n is 1/2 sum_c ||r_c||^2_{W_c}.

Two cases: "l1" (beta = 0, nu = 1/10, gains estimated), where the w clamp
and the nu threshold zero voxel 2 from the second iteration on, and
"quadratic" (beta = 1/4, nu = 0, gains estimated), where the w clamp
zeroes voxel 2 in the third iteration.

    python tests/golden/fista_worked_example.py
"""
import json
import os

import sympy as sp

HERE = os.path.dirname(os.path.abspath(__file__))

A1 = sp.Matrix([[2, 1, 0], [1, 3, 1], [0, 1, 2]])
Y1 = sp.Matrix([3, 4, -1])
W1 = sp.Matrix([1, 1, 1])
A2 = sp.Matrix([[1, 0, 1], [1, 1, 0]])
Y2 = sp.Matrix([1, 2])
W2 = sp.Matrix([2, 1])
CASES = {
    "l1": dict(beta=sp.Integer(0), nu=sp.Rational(1, 10), estimate_gains=True),
    "quadratic": dict(beta=sp.Rational(1, 4), nu=sp.Integer(0), estimate_gains=True),
}
N_ITER = 3


def had(a, b):
    return sp.Matrix([a[i] * b[i] for i in range(a.shape[0])])


def num(v):
    return float(sp.N(v, 30))


def vec(v):
    return [num(e) for e in v]


def line_grad_R(z, beta):
    n = z.shape[0]
    return sp.Matrix([beta * sum(z[j] - z[l] for l in (j - 1, j + 1) if 0 <= l < n) for j in range(n)])


def derive(beta, nu, estimate_gains):
    n = A1.shape[1]
    ones = sp.ones(n, 1)
    D = A1.T * had(W1, A1 * ones) + A2.T * had(W2, A2 * ones)
    x = sp.zeros(n, 1)
    z = sp.zeros(n, 1)
    t = sp.Integer(1)
    gamma2 = sp.Integer(0) if estimate_gains else sp.Integer(1)
    steps = []
    for it in range(N_ITER):
        p1, p2 = A1 * z, A2 * z
        if estimate_gains:
            gamma2 = (Y2.T * had(W2, p2))[0] / (Y2.T * had(W2, Y2))[0]
        r1, r2 = p1 - Y1, p2 - gamma2 * Y2
        g = A1.T * had(W1, r1) + A2.T * had(W2, r2)
        fit = sp.Rational(1, 2) * ((r1.T * had(W1, r1))[0] + (r2.T * had(W2, r2))[0])
        gR = line_grad_R(z, beta)
        t_new = (1 + sp.sqrt(1 + 4 * t * t)) / 2
        pre = sp.Matrix([z[j] - (g[j] + gR[j]) / (D[j] + 26 * beta) for j in range(n)])
        w = sp.Matrix([sp.Max(v, 0) for v in pre])
        x_new = sp.Matrix([sp.Max(w[j] - nu, 0) for j in range(n)])
        z_new = x_new + ((t - 1) / t_new) * (x_new - x)
        steps.append({"iteration": it + 1, "p1": vec(p1), "p2": vec(p2), "gamma2": num(gamma2),
                      "r1": vec(r1), "r2": vec(r2), "g": vec(g), "grad_R": vec(gR), "data_fit": num(fit),
                      "w_before_clamp": vec(pre), "w": vec(w), "x": vec(x_new), "t": num(t_new), "z": vec(z_new)})
        x, z, t = x_new, z_new, t_new
    return {"D": vec(D), "steps": steps}


def main():
    out = {"source": "Table V (Sec. V), derived in exact arithmetic by tests/golden/fista_worked_example.py",
           "A1": [[int(v) for v in A1.row(i)] for i in range(A1.rows)], "y1": [int(v) for v in Y1],
           "w1": [int(v) for v in W1],
           "A2": [[int(v) for v in A2.row(i)] for i in range(A2.rows)], "y2": [int(v) for v in Y2],
           "w2": [int(v) for v in W2], "shape": [1, 1, 3], "reg_scale": 26, "cases": {}}
    for name, c in CASES.items():
        out["cases"][name] = {"beta": num(c["beta"]), "nu": num(c["nu"]), "estimate_gains": c["estimate_gains"],
                              **derive(**c)}
    with open(os.path.join(HERE, "fista_worked_example.json"), "w") as f:
        json.dump(out, f, indent=1)


if __name__ == "__main__":
    main()
