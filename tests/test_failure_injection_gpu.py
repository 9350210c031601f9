"""Failure detection with faults made on the host: an injected allocation
failure comes back as LT_ENOMEM from plan and solver creation and leaves the
library usable; a tensor-core kernel whose MMAs are withheld (so its bounded
mbarrier wait has nothing to wait for) reports LT_ETIMEOUT, writes nothing and
leaves the context usable.  Nothing here faults or hangs the GPU.

The injection entry points exist only in the test build of the library
(include/lt_testing.h), so each check runs in a child process started with
LT_TEST_HOOKS=1, which makes the binding load that build."""
import os
import subprocess
import sys

import numpy as np
import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))

pytestmark = pytest.mark.gpu


def _in_test_build(check):
    from paper_1812_03358_b300 import build
    build.build()
    env = {**os.environ, "LT_TEST_HOOKS": "1", "PYTHONPATH": ROOT + os.pathsep + os.environ.get("PYTHONPATH", "")}
    out = subprocess.run([sys.executable, os.path.abspath(__file__), check], cwd=ROOT, env=env,
                         capture_output=True, text=True, timeout=600)
    assert out.returncode == 0, out.stdout[-3000:] + out.stderr[-3000:]
    assert "CHECK OK" in out.stdout


def test_allocation_failures_are_reported_and_recovered():
    _in_test_build("alloc")


@pytest.mark.parametrize("path", ["chunked", "zwalk"])
def test_tensor_core_wait_that_runs_out_is_reported(path):
    _in_test_build("stall-" + path)


# ---------------------------------------------------------------------------
# the checks, run in the child process against the test build
# ---------------------------------------------------------------------------

def check_allocation_failures():
    import torch
    from oracle import camera as O
    from paper_1812_03358_b300 import inputs as I, lt
    assert lt.LIB_PATH.endswith("liblt_testhooks.so")
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


def check_tensor_core_stall(path):
    import torch
    from paper_1812_03358_b300 import lt
    from paper_1812_03358_b300 import unet as U
    path = {"chunked": U.CONV_TCGEN05_CHUNKED, "zwalk": U.CONV_TCGEN05_ZWALK}[path]
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


if __name__ == "__main__":
    which = sys.argv[1]
    if which == "alloc":
        check_allocation_failures()
    else:
        check_tensor_core_stall(which.split("-", 1)[1])
    print("CHECK OK")
