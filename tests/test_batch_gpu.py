"""Batched launches: one persistent forward launch over cameras of uneven
detector sizes (single-lens, rotated, plenoptic) x frames equals per-camera
launches; the multi-camera gather adjoint equals the sum of per-camera
adjoints; every autotuner variant agrees, and the adjoint autotuner keeps
the faster of the two adjoint kernels; a CUDA graph of forward + adjoint
replays the eager result."""
import numpy as np
import pytest

torch = pytest.importorskip("torch")

from oracle import camera as O
from paper_1812_03358_b300 import build, inputs as I, lt

pytestmark = pytest.mark.gpu


def host(t):
    torch.cuda.synchronize()
    return t.detach().cpu().numpy().astype(np.float64)


@pytest.fixture(scope="module")
def mixed():
    build.build()
    vol = I.Volume(24, 20, 22, 3.0, 3.0, 3.0)
    _, pc = I.tiny_plenoptic()
    cams = [I.table_single_lens(40, 0.12), I.table_single_lens(33, 0.17, yaw=0.6, ks=2, kt=2),
            I.table_single_lens(57, 0.09, yaw=-2.0, ks=3, kt=2), pc,
            I.table_single_lens(21, 0.25, ks=2, kt=2)]
    frames = 2
    plan = lt.Plan(vol, cams, frames)
    xs = np.stack([I.gaussian_blobs(vol, seed=1100 + f).ravel() for f in range(frames)])
    ys = np.stack([I.uniform_random(plan.m_total, seed=1200 + f) for f in range(frames)])
    return vol, cams, plan, torch.from_numpy(xs).cuda(), torch.from_numpy(ys).cuda()


def test_batched_forward_equals_per_camera(mixed):
    vol, cams, plan, x, y = mixed
    yb = host(plan.forward(x))
    for c in range(len(cams)):
        yc = host(plan.forward_camera(c, x))
        assert np.array_equal(yb[:, plan.offsets[c]:plan.offsets[c + 1]], yc)


def test_batched_adjoint_equals_sum_of_per_camera(mixed):
    vol, cams, plan, x, y = mixed
    xb = host(plan.adjoint(y))
    acc = None
    for c in range(len(cams)):
        yc = y[:, plan.offsets[c]:plan.offsets[c + 1]].contiguous()
        acc = plan.adjoint_camera(c, yc, acc, accumulate=acc is not None)
    xs = host(acc)
    assert np.abs(xb - xs).max() <= 1e-6 * np.abs(xs).max()


def test_batched_operator_matches_oracle(mixed):
    vol, cams, plan, x, y = mixed
    yb = host(plan.forward(x))
    xh = x.cpu().numpy().astype(np.float64)
    for f in range(2):
        for c, cam in enumerate(cams):
            ref = O.forward(vol, cam, xh[f]).ravel()
            got = yb[f, plan.offsets[c]:plan.offsets[c + 1]]
            assert np.linalg.norm(got - ref) <= 1e-5 * np.linalg.norm(ref)


def test_every_autotune_variant_agrees(mixed):
    vol, cams, plan, x, y = mixed
    chosen, times = plan.autotune()
    assert 0 <= chosen < len(times) and all(t > 0 for t in times)
    outs = []
    for v in range(len(times)):
        lt.lt_plan_set_forward_variant(plan.handle, v)
        outs.append(host(plan.forward(x)))
    lt.lt_plan_set_forward_variant(plan.handle, chosen)
    for o in outs[1:]:
        assert np.abs(o - outs[0]).max() <= 1e-6 * np.abs(outs[0]).max()
    with pytest.raises(lt.LtError):
        lt.lt_plan_set_forward_variant(plan.handle, len(times))


def test_adjoint_autotune_keeps_the_faster_of_two_equal_operators(mixed):
    vol, cams, plan, x, y = mixed
    chosen, times = plan.autotune_adjoint()
    assert chosen in (0, 1) and all(t > 0 for t in times)
    assert times[chosen] == min(times)
    outs = {}
    for v in (0, 1):
        lt.lt_plan_set_adjoint_variant(plan.handle, v)
        outs[v] = host(plan.adjoint(y))
    lt.lt_plan_set_adjoint_variant(plan.handle, chosen)
    assert np.abs(outs[1] - outs[0]).max() <= 1e-6 * np.abs(outs[0]).max()


def test_graph_capture_replays_forward_and_adjoint(mixed):
    vol, cams, plan, x, y = mixed
    y_eager = host(plan.forward(x))
    x_eager = host(plan.adjoint(y))
    yo = torch.empty_like(y)
    xo = torch.empty_like(x)
    s = torch.cuda.Stream()
    with torch.cuda.stream(s):
        plan.forward(x, yo)   # warm-up on the capture stream
        plan.adjoint(y, xo)
    torch.cuda.synchronize()
    g = torch.cuda.CUDAGraph()
    with torch.cuda.graph(g, stream=s):
        plan.forward(x, yo)
        plan.adjoint(y, xo)
    yo.zero_()
    xo.zero_()
    g.replay()
    torch.cuda.synchronize()
    assert np.array_equal(host(yo), y_eager)
    assert np.array_equal(host(xo), x_eager)
