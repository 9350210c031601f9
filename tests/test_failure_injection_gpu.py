"""Failure detection with faults made on the host: an injected allocation
failure comes back as LT_ENOMEM from plan and solver creation and leaves the
library usable; a tensor-core kernel whose MMAs are withheld (so its bounded
mbarrier wait has nothing to wait for) reports LT_ETIMEOUT, writes nothing and
leaves the context usable.  Nothing here faults or hangs the GPU."""
import numpy as np
import pytest
import torch

from oracle import camera as O
from paper_1812_03358_b300 import build, inputs as I, lt
from paper_1812_03358_b300 import unet as U

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _lib():
    build.build()
    lt.lib()


def test_allocation_failures_are_reported_and_recovered():
    vol, cam = I.config_single_small()
    failed = 0
    for n in range(1, 64):
        lt.lt_test_fail_allocation_after(n)
        try:
            plan = lt.Plan(vol, [cam])
        except lt.LtError as e:
            assert e.status == lt.LT_ENOMEM, str(e)
            failed += 1
            continue
        finally:
            lt.lt_test_fail_allocation_after(0)
        # n is past the plan's allocations: the plan works; now fail the solver's
        y = plan.forward(torch.zeros(1, plan.nvox, device="cuda"))
        for m in range(1, 32):
            lt.lt_test_fail_allocation_after(m)
            try:
                rec = lt.Recon(plan, y)
            except lt.LtError as e:
                assert e.status == lt.LT_ENOMEM, str(e)
                continue
            finally:
                lt.lt_test_fail_allocation_after(0)
            rec.close()
            break
        plan.close()
        break
    assert failed >= 3
    # the library is intact: a fresh plan matches the oracle
    x = I.gaussian_blobs(vol, seed=1000)
    plan = lt.Plan(vol, [cam])
    yg = plan.forward(torch.from_numpy(x.reshape(1, -1)).cuda()).cpu().numpy().ravel()
    yo = O.forward(vol, cam, x).ravel()
    assert np.linalg.norm(yg - yo) <= 1e-5 * np.linalg.norm(yo)
    plan.close()


@pytest.mark.parametrize("path", [U.CONV_TCGEN05_CHUNKED, U.CONV_TCGEN05_ZWALK], ids=["chunked", "z-walking"])
def test_tensor_core_wait_that_runs_out_is_reported(path):
    D, H, W, Ci, Co = 2, 4, 128, 16, 16
    V = D * H * W
    x = torch.randn(V * Ci, device="cuda").to(torch.bfloat16)
    w = (0.1 * torch.randn(Co * 27 * Ci, device="cuda")).to(torch.bfloat16)
    out = torch.full((V * Co,), 7.0, device="cuda")
    U.device_status()                                       # clean start
    U._call("lt_nn_test_stall_tensor_core", 1, U._s())
    try:
        U.conv3d(x, w, None, None, out, Ci=Ci, Co=Co, dims=(D, H, W), relu=False, path=path)
        with pytest.raises(lt.LtError) as e:
            U.device_status()
        assert e.value.status == lt.LT_ETIMEOUT
        assert torch.all(out == 7.0)                        # no output written
    finally:
        U._call("lt_nn_test_stall_tensor_core", 0, U._s())
    U.device_status()                                       # cleared
    U.conv3d(x, w, None, None, out, Ci=Ci, Co=Co, dims=(D, H, W), relu=False, path=path)
    ref = torch.empty_like(out)
    U.conv3d(x, w, None, None, ref, Ci=Ci, Co=Co, dims=(D, H, W), relu=False, path=U.CONV_WARP_MMA)
    U.device_status()
    assert float((out - ref).norm() / ref.norm()) < 1e-5
