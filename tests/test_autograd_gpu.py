"""The projector as a torch.autograd.Function: gradients of objectives built
on it against FP64 finite differences of the oracle's objective, and the
Jacobians of project / backproject against the oracle's explicit A and A^T
(16^3 volume, one 32x32 single-lens camera)."""
import numpy as np
import pytest

torch = pytest.importorskip("torch")

from oracle import camera as O
from oracle import recon as OR
from paper_1812_03358_b300 import autograd as AG
from paper_1812_03358_b300 import build, inputs as I, lt

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def setup():
    build.build()
    vol = I.Volume(16, 16, 16, 6.25, 6.25, 6.25)
    cam = I.table_single_lens(32, 0.16)
    plan = lt.Plan(vol, [cam])
    return vol, cam, plan


def tv26(x, shape, beta, delta):
    """beta/2 sum_j sum_{l in N26(j)} delta^2 (sqrt(1 + ((x_j - x_l)/delta)^2) - 1), in torch."""
    X = x.reshape(shape)
    nz, ny, nx = shape
    acc = x.new_zeros(())
    for oz in (-1, 0, 1):
        for oy in (-1, 0, 1):
            for ox in (-1, 0, 1):
                if (oz, oy, ox) == (0, 0, 0):
                    continue
                a = X[max(0, -oz):nz - max(0, oz), max(0, -oy):ny - max(0, oy), max(0, -ox):nx - max(0, ox)]
                b = X[max(0, oz):nz - max(0, -oz), max(0, oy):ny - max(0, -oy), max(0, ox):nx - max(0, -ox)]
                d = a - b
                acc = acc + (delta ** 2 * (torch.sqrt(1 + (d / delta) ** 2) - 1)).sum()
    return 0.5 * beta * acc


def test_tv_objective_gradient_matches_oracle_finite_differences(setup):
    vol, cam, plan = setup
    x0 = I.gaussian_blobs(vol, seed=1000).astype(np.float64).ravel()
    y = O.single_forward(vol, cam, I.gaussian_blobs(vol, seed=1001)).ravel()
    beta, delta = 1e-3, 0.05

    def f_oracle(x):
        r = O.single_forward(vol, cam, x).ravel() - y
        return 0.5 * np.dot(r, r) + OR.R_value(x, vol.shape, beta, psi=1, delta=delta)

    xt = torch.tensor(x0, dtype=torch.float32, device="cuda", requires_grad=True)
    yt = torch.tensor(y, dtype=torch.float32, device="cuda")
    loss = 0.5 * ((AG.project(plan, xt) - yt) ** 2).sum() + tv26(xt, vol.shape, beta, delta)
    loss.backward()
    g = xt.grad.detach().cpu().numpy().astype(np.float64)
    rng = np.random.default_rng(0)
    # sample voxels where the data term is active and a few elsewhere
    idx = np.concatenate([np.argsort(-np.abs(g))[:10], rng.choice(vol.n, 10, replace=False)])
    h = 1e-4
    scale = np.abs(g).max()
    for j in idx:
        e = np.zeros(vol.n)
        e[j] = h
        fd = (f_oracle(x0 + e) - f_oracle(x0 - e)) / (2 * h)
        assert abs(fd - g[j]) <= 1e-4 * scale, (j, fd, g[j])


def test_projector_jacobian_is_explicit_matrix(setup):
    vol, cam, plan = setup
    A = O.single_matrix(vol, cam)
    x = torch.zeros(vol.n, device="cuda")
    J = torch.autograd.functional.jacobian(lambda v: AG.project(plan, v), x)   # rows via backward = A^T
    J = J.cpu().numpy().astype(np.float64)
    assert np.abs(J - A).max() <= 1e-5 * np.abs(A).max()


def test_backprojector_jacobian_is_transpose(setup):
    vol, cam, plan = setup
    A = O.single_matrix(vol, cam)
    y = torch.zeros(cam.m, device="cuda")
    J = torch.autograd.functional.jacobian(lambda v: AG.backproject(plan, v), y)   # rows via backward = A
    J = J.cpu().numpy().astype(np.float64)
    assert np.abs(J - A.T).max() <= 1e-5 * np.abs(A).max()


def test_tv_regularised_nonnegative_fit_decreases_objective(setup):
    vol, cam, plan = setup
    x_true = torch.from_numpy(I.gaussian_blobs(vol, seed=1002).ravel()).cuda()
    y = AG.project(plan, x_true).detach()
    x = torch.zeros(vol.n, device="cuda", requires_grad=True)
    opt = torch.optim.Adam([x], lr=0.02)
    losses = []
    for _ in range(60):
        opt.zero_grad()
        loss = 0.5 * ((AG.project(plan, x) - y) ** 2).sum() + tv26(x, vol.shape, 1e-4, 0.05)
        loss.backward()
        opt.step()
        with torch.no_grad():
            x.clamp_(min=0.0)
        losses.append(float(loss.detach()))
    assert losses[-1] < 0.2 * losses[0]
