"""The learned warm start: the U-Net, trained briefly on plume volumes and the
images the forward model makes of them, gives an initial volume closer to the
truth than the plain solver reaches in its iterations, and the warm-started
solver reaches the plain solver's data fit (64^3 volume at 2 mm, the 1000^2
plenoptic camera, held-out seeds)."""
import pytest

torch = pytest.importorskip("torch")

from paper_1812_03358_b300 import build, inputs as I, lt

pytestmark = pytest.mark.gpu


def test_trained_network_beats_plain_solver_on_volume_error():
    build.build()
    from paper_1812_03358_b300 import unet, warmstart as WS
    plan = lt.Plan(I.Volume(64, 64, 64, 2.0, 2.0, 2.0), [I.plenoptic_camera()])
    ws, losses = WS.train(plan, unet.UNet(seed=1), n_samples=800, lr=1e-3, log_every=40)
    late = [l for s, l, _ in losses if s >= 400]
    assert sum(late) / len(late) < 0.8 * losses[0][1], losses
    x, bp, y = WS.training_pair(plan, seed=2_000_000)
    x0 = ws.infer(bp)
    assert torch.isfinite(x0).all() and (x0 >= 0).all()
    res = WS.evaluate(plan, ws, y, x, n_plain=60)
    assert res["err_x0"] < res["err_plain"], res
    assert res["warm_iters"] is not None and res["warm_iters"] <= 60, res
    assert res["warm_ms"] > res["unet_ms"] > 0, res


def test_warm_start_reaches_the_plain_fit_sooner_at_full_size():
    """The bench camera at 128^3 x 1 mm: trained on 6000 generated volumes
    (a fixed budget of about a minute), the warm start reaches the plain
    solver's 200-iteration data fit in less wall time than the plain solver,
    median over eight held-out volumes (time includes the back-projection and
    the U-Net inference, not the training)."""
    import statistics
    build.build()
    from paper_1812_03358_b300 import unet, warmstart as WS
    vol, cam = I.config_plenoptic()
    plan = lt.Plan(vol, [cam])
    ws, _ = WS.train(plan, unet.UNet(seed=1), n_samples=6000, lr=1e-3)
    gains = []
    for j in range(8):
        x, _, y = WS.training_pair(plan, seed=2_000_000 + j)
        r = WS.evaluate(plan, ws, y, x, n_plain=200)
        assert r["warm_ms"] is not None, r
        gains.append(r["plain_ms"] / r["warm_ms"])
    assert statistics.median(gains) > 1.0, gains
    plan.close()
