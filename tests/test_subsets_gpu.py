"""GPU parity of view-subset acceleration (Sec. V, eq. subset) against the
FP64 oracle: the subset operators (lt_forward_subset / lt_adjoint_subset) for
single-lens, rotated and plenoptic cameras, their partition identity, and the
subset reconstruction after a fixed number of iterations (with gain
estimation across cameras of different K)."""
import numpy as np
import pytest

torch = pytest.importorskip("torch")

from oracle import camera as O
from oracle import recon as OR
from paper_1812_03358_b300 import build, inputs as I, lt

pytestmark = pytest.mark.gpu

TOL = 1e-5


def rel_l2(a, b):
    return float(np.linalg.norm(np.ravel(a) - np.ravel(b)) / np.linalg.norm(np.ravel(b)))


@pytest.fixture(scope="module", autouse=True)
def _lib():
    build.build()
    lt.lib()


def dev(a):
    return torch.from_numpy(np.ascontiguousarray(a, dtype=np.float32)).cuda()


def host(t):
    torch.cuda.synchronize()
    return t.detach().cpu().numpy().astype(np.float64)


def cases():
    vol = I.Volume(12, 9, 10, 4.0, 4.5, 5.0)
    tv, tc = I.tiny_plenoptic()
    return {
        "single": (vol, I.table_single_lens(28, 0.3, ks=2, kt=2)),
        "rotated": (vol, I.table_single_lens(28, 0.3, yaw=0.7, ks=3, kt=2)),
        "plenoptic": (tv, tc),
    }


@pytest.mark.parametrize("which", ["single", "rotated", "plenoptic"])
def test_subset_operators_match_oracle(which):
    vol, cam = cases()[which]
    plan = lt.Plan(vol, [cam])
    K = plan.cells[0]
    x = I.gaussian_blobs(vol, seed=1020).ravel()
    y = I.uniform_random(plan.m_total, seed=40)
    full_y = host(plan.forward(dev(x).reshape(1, -1)))[0]
    full_x = host(plan.adjoint(dev(y).reshape(1, -1)))[0]
    for N in (2, 3):
        sum_y, sum_x = 0.0, 0.0
        for s in range(N):
            S = OR.subset_cells(K, N, s)
            yg = host(plan.forward_subset(dev(x).reshape(1, -1), N, s))[0]
            xg = host(plan.adjoint_subset(dev(y).reshape(1, -1), N, s))[0]
            yo = np.ravel(O.forward(vol, cam, x, cells=S))
            xo = np.ravel(O.adjoint(vol, cam, y, cells=S))
            assert rel_l2(yg, yo) < TOL, (N, s, rel_l2(yg, yo))
            assert rel_l2(xg, xo) < TOL, (N, s, rel_l2(xg, xo))
            sum_y, sum_x = sum_y + yg, sum_x + xg
        assert rel_l2(sum_y, full_y) < 1e-6
        assert rel_l2(sum_x, full_x) < 1e-6


def test_subset_reconstruction_matches_oracle():
    vol = I.Volume(16, 16, 16, 5.0, 5.0, 5.0)
    cams = [I.table_single_lens(36, 0.25, ks=2, kt=2), I.table_single_lens(30, 0.3, yaw=1.1, ks=3, kt=1)]
    x_true = I.gaussian_blobs(vol, seed=1005)
    ys = [np.ravel(O.forward(vol, c, x_true)) for c in cams]
    ys[1] = ys[1] / 1.7
    plan = lt.Plan(vol, cams)
    rec = lt.Recon(plan, dev(np.concatenate(ys)).reshape(1, -1), beta=1e-4, n_subset=2)
    rec.iterate(12)
    xg, gains, _ = rec.get()
    ops = [(lambda v, cells=None, c=c: np.ravel(O.forward(vol, c, v, cells=cells)),
            lambda r, cells=None, c=c: np.ravel(O.adjoint(vol, c, r, cells=cells))) for c in cams]
    ref = OR.fista(ops, ys, [None, None], vol.shape, 12, beta=1e-4, n_subset=2, n_cells=[4, 3])
    assert rel_l2(host(xg)[0], ref["x"]) < 1e-4, rel_l2(host(xg)[0], ref["x"])
    assert abs(gains[0][1] - ref["gains"][1]) < 1e-4 * abs(ref["gains"][1])
    # the subset iterates are not the full iterates here (out of focus)
    full = OR.fista([(lambda v, c=c: np.ravel(O.forward(vol, c, v)), lambda r, c=c: np.ravel(O.adjoint(vol, c, r)))
                     for c in cams], ys, [None, None], vol.shape, 12, beta=1e-4)
    assert rel_l2(ref["x"], full["x"]) > 1e-4


def test_subset_reconstruction_resumes_on_the_right_subset():
    vol = I.Volume(16, 16, 16, 5.0, 5.0, 5.0)
    cams = [I.table_single_lens(36, 0.25, ks=2, kt=2)]
    x_true = I.gaussian_blobs(vol, seed=1006)
    y = dev(np.ravel(O.forward(vol, cams[0], x_true))).reshape(1, -1)
    plan = lt.Plan(vol, cams)
    a = lt.Recon(plan, y, n_subset=4)
    a.iterate(7)
    state = a.state()
    a.iterate(5)
    b = lt.Recon(plan, y, n_subset=4)
    b.load_state(state)
    b.iterate(5)
    assert np.array_equal(host(a.get()[0]), host(b.get()[0]))
