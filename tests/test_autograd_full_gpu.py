"""The differentiable reconstruction at full size: four single-lens 1024 x
1024 cameras (2 x 2 cells) at yaw 0, 45, 90, 135 degrees around a 256^3
volume, the projector as a torch.autograd.Function inside a TV-regularised
(26-neighbour hyperbola, beta 1e-3) nonnegative least-squares fit.  Checked
at this size: autograd's gradient of the data term is exactly the adjoint of
the residual; the TV gradient at sampled voxels matches central differences
of the oracle's regulariser (evaluated on the 3 x 3 x 3 neighbourhood, which
holds every term that involves the voxel); projected gradient descent
lowers the objective at every step and keeps x >= 0."""
import numpy as np
import pytest

torch = pytest.importorskip("torch")

from oracle import recon as OR
from paper_1812_03358_b300 import autograd as AG
from paper_1812_03358_b300 import build, inputs as I, lt

pytestmark = pytest.mark.gpu

BETA, DELTA = 1e-3, 0.05


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


@pytest.fixture(scope="module")
def fit():
    build.build()
    vol, cams = I.config_differentiable()
    plan = lt.Plan(vol, cams)
    truth = I.plume_field_torch(vol, seed=4100).reshape(1, -1)
    y = plan.forward(truth)
    yield vol, plan, truth, y
    plan.close()


def test_data_gradient_is_adjoint_of_residual(fit):
    vol, plan, truth, y = fit
    x = (0.5 * truth).requires_grad_(True)
    loss = 0.5 * ((AG.project(plan, x) - y) ** 2).sum()
    loss.backward()
    with torch.no_grad():
        ref = plan.adjoint(plan.forward(x) - y)
    assert torch.equal(x.grad, ref)


def test_tv_gradient_matches_oracle_central_differences(fit):
    vol, plan, truth, y = fit
    x = truth.clone().requires_grad_(True)
    tv26(x, vol.shape, BETA, DELTA).backward()
    g = x.grad.reshape(vol.shape).cpu().numpy().astype(np.float64)
    X = truth.reshape(vol.shape).cpu().numpy().astype(np.float64)
    rng = np.random.default_rng(31)
    h = 1e-4
    for _ in range(24):
        k, j, i = (int(v) for v in rng.integers(1, 255, size=3))
        crop = X[k - 1:k + 2, j - 1:j + 2, i - 1:i + 2].copy()
        lo, hi = crop.copy(), crop.copy()
        lo[1, 1, 1] -= h
        hi[1, 1, 1] += h
        fd = (OR.R_value(hi, (3, 3, 3), BETA, psi=1, delta=DELTA) -
              OR.R_value(lo, (3, 3, 3), BETA, psi=1, delta=DELTA)) / (2 * h)
        assert abs(g[k, j, i] - fd) <= 1e-3 * abs(fd) + 1e-7


def test_projected_tv_fit_lowers_objective(fit):
    """Projected gradient descent with step 1/L on the measurement-normalised
    objective 0.5 ||A x / s - y / s||^2 + TV(x), s = max y, L = ||A||^2 / s^2
    (power iteration) + 52 beta (the TV Hessian bound: 26 neighbours, each
    pair term's second derivative at most beta / 2, each pair counted twice):
    a descent method for a convex L-smooth objective, so every step lowers it."""
    vol, plan, truth, y = fit
    s = float(y.abs().max())
    g = torch.Generator(device="cuda").manual_seed(41)
    v = torch.rand(truth.shape, device="cuda", generator=g)
    lam = 0.0
    for _ in range(8):
        with torch.no_grad():
            w = plan.adjoint(plan.forward(v)) / (s * s)
            lam = float(w.norm() / v.norm())
            v = w / w.norm()
    step = 1.0 / (1.05 * lam + 52 * BETA)
    x = torch.zeros_like(truth).requires_grad_(True)
    opt = torch.optim.SGD([x], lr=step)
    losses = []
    for _ in range(12):
        opt.zero_grad()
        loss = 0.5 * ((AG.project(plan, x) / s - y / s) ** 2).sum() + tv26(x, vol.shape, BETA, DELTA)
        loss.backward()
        opt.step()
        with torch.no_grad():
            x.clamp_(min=0.0)
        losses.append(float(loss.detach()))
    assert all(b <= a * (1 + 1e-6) for a, b in zip(losses, losses[1:]))
    assert losses[-1] < 0.7 * losses[0]
    assert float(x.detach().min()) >= 0.0 and bool(torch.isfinite(x.detach()).all())
