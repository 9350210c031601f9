"""Step-by-step pin of the oracle's Table V iteration (Sec. V).

The limit pins (scipy NNLS, L-BFGS-B) hold for any convergent variant of the
iteration; the GPU solver, however, is compared with the oracle after a
fixed number of iterations, so the oracle's sequence itself must be the one
Table V prints.  tests/golden/fista_worked_example.json records three
iterations of a three-voxel, two-camera problem derived in exact arithmetic
(every intermediate quantity listed), and the oracle must reproduce x, z,
t, the estimated gain and the data fit of every iteration.

The second test plants plausible mistakes in a copy of the oracle's
iteration (momentum coefficient, order of the t update, the nu threshold,
the point the gain is estimated at, the point the regulariser gradient is
taken at, the majoriser's regulariser term, the gradient step's base point,
the weights in the gradient) and checks that the worked example rejects
each of them.
"""
import inspect
import json
import os
import textwrap

import numpy as np
import pytest

from oracle import recon

GOLDEN = json.load(open(os.path.join(os.path.dirname(__file__), "golden", "fista_worked_example.json")))


def _problem():
    A1 = np.array(GOLDEN["A1"], dtype=np.float64)
    A2 = np.array(GOLDEN["A2"], dtype=np.float64)
    ops = [(lambda v, A=A1: A @ v, lambda r, A=A1: A.T @ r), (lambda v, A=A2: A @ v, lambda r, A=A2: A.T @ r)]
    ys = [np.array(GOLDEN["y1"], float), np.array(GOLDEN["y2"], float)]
    ws = [np.array(GOLDEN["w1"], float), np.array(GOLDEN["w2"], float)]
    return ops, ys, ws


def _mismatches(fista, case):
    """Quantities of the worked example that `fista` does not reproduce."""
    ops, ys, ws = _problem()
    c = GOLDEN["cases"][case]
    bad = []
    for step in c["steps"]:
        n = step["iteration"]
        out = fista(ops, ys, ws, tuple(GOLDEN["shape"]), n_iter=n, beta=c["beta"], nu=c["nu"],
                    reg_scale=GOLDEN["reg_scale"], estimate_gains=c["estimate_gains"], history=True)
        checks = {"D": (out["D"], c["D"]), "x": (out["x"], step["x"]), "z": (out["z"], step["z"]),
                  "t": (out["t"], step["t"]), "gamma2": (out["gains"][1], step["gamma2"]),
                  "data_fit": (out["fits"][-1], step["data_fit"])}
        for name, (got, want) in checks.items():
            got, want = np.atleast_1d(np.asarray(got, float)), np.atleast_1d(np.asarray(want, float))
            if not np.allclose(got, want, rtol=1e-12, atol=1e-14):
                bad.append((n, name, got.tolist(), want.tolist()))
    return bad


@pytest.mark.parametrize("case", sorted(GOLDEN["cases"]))
def test_oracle_reproduces_worked_example(case):
    assert _mismatches(recon.fista, case) == []


def test_worked_example_exercises_the_clamps():
    # the example is only a pin of the clamps if they act in it
    l1 = GOLDEN["cases"]["l1"]["steps"]
    assert l1[1]["w_before_clamp"][2] < 0.0 and l1[1]["x"][2] == 0.0
    nu = GOLDEN["cases"]["l1"]["nu"]
    assert l1[0]["w"][2] > nu and abs(l1[0]["x"][2] - (l1[0]["w"][2] - nu)) < 1e-15   # nu shrinks a positive w
    q = GOLDEN["cases"]["quadratic"]["steps"]
    assert q[2]["w_before_clamp"][2] < 0.0 and q[2]["x"][2] == 0.0
    assert any(v < 0 for s in q for v in s["z"])   # momentum leaves the non-negative orthant


# (name, text in the oracle's fista, planted replacement)
PLANTS = [
    ("momentum coefficient (t_new - 1) / t_new", "((t - 1.0) / t_new)", "((t_new - 1.0) / t_new)"),
    ("t advanced before its first use", "    t = 1.0\n", "    t = (1.0 + np.sqrt(5.0)) / 2.0\n"),
    ("nu threshold divided by D", "np.maximum(wv - nu, 0.0)", "np.maximum(wv - nu / safe, 0.0)"),
    ("gain estimated at x instead of z", "gains[c] = optimal_gain(y, p, w)", "gains[c] = optimal_gain(y, A(x), w)"),
    ("regulariser gradient at x instead of z", "grad_R(z, shape", "grad_R(x, shape"),
    ("majoriser without the regulariser's scale", "D + reg_scale * beta", "D + beta"),
    ("gradient step from x instead of z", "np.maximum(z - step / safe", "np.maximum(x - step / safe"),
    ("weights dropped from the gradient", "g += At(w * r)", "g += At(r)"),
]


@pytest.mark.parametrize("name,old,new", PLANTS, ids=[p[0] for p in PLANTS])
def test_worked_example_rejects_planted_mistake(name, old, new):
    src = textwrap.dedent(inspect.getsource(recon.fista))
    assert src.count(old) == 1, f"the oracle no longer contains {old!r}; update the plant"
    ns = dict(vars(recon))
    exec(compile(src.replace(old, new), "<planted fista>", "exec"), ns)
    planted = ns["fista"]
    assert any(_mismatches(planted, case) for case in GOLDEN["cases"]), name
