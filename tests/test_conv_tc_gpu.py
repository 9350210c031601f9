"""tcgen05 convolution (operands in shared memory, accumulators in tensor
memory) against a float64 PyTorch convolution of the same bfloat16 operands
on the host, and against the warp-level MMA kernel.

The reference is the plain definition of the layer: a 3x3x3 cross-correlation
with zero padding 1, out[v][co] = b[co] + sum_{tap, ci} w[co][tap][ci]
in[v + tap][ci], tap = (dz+1)*9 + (dy+1)*3 + (dx+1).  bfloat16 products are
exact in float32, so the only difference is the float32 summation order of
27 Ci terms: relative L2 error below 1e-5 on the float32 output, and the
bfloat16 output within one bfloat16 rounding (2^-8 relative) of it.
"""
import numpy as np
import pytest
import torch

from paper_1812_03358_b300 import lt
from paper_1812_03358_b300 import unet as U

pytestmark = pytest.mark.gpu


def _operands(D, H, W, Ci, Co, seed):
    g = torch.Generator().manual_seed(seed)
    x = torch.randn(D * H * W * Ci, generator=g).to(torch.bfloat16)
    w = (0.1 * torch.randn(Co * 27 * Ci, generator=g)).to(torch.bfloat16)
    b = 0.1 * torch.randn(Co, generator=g)
    return x, w, b


def _reference(x, w, b, D, H, W, Ci, Co, relu):
    xt = x.double().reshape(1, D, H, W, Ci).permute(0, 4, 1, 2, 3)
    wt = w.double().reshape(Co, 3, 3, 3, Ci).permute(0, 4, 1, 2, 3)
    y = torch.nn.functional.conv3d(xt, wt, b.double(), padding=1)
    if relu:
        y = torch.relu(y)
    return y.permute(0, 2, 3, 4, 1).reshape(D * H * W, Co)


def _run(path, x, w, b, D, H, W, Ci, Co, relu, o_stride=None, o_off=0):
    V = D * H * W
    os_ = o_stride or Co
    out_f = torch.full((V * os_,), 7.0, device="cuda")
    out_b = torch.full((V * os_,), 7.0, device="cuda", dtype=torch.bfloat16)
    U.conv3d(x.cuda(), w.cuda(), b.cuda(), out_b, out_f, Ci=Ci, Co=Co, dims=(D, H, W), o_stride=o_stride,
             o_off=o_off, relu=relu, path=path)
    U.device_status()
    return out_f.reshape(V, os_).cpu(), out_b.reshape(V, os_).float().cpu()


CASES = [  # (D, H, W, Ci, Co, relu)
    (2, 2, 128, 16, 16, False),
    (4, 6, 128, 32, 16, True),
    (2, 4, 256, 16, 32, False),
    (6, 2, 128, 48, 64, True),
    (2, 2, 128, 16, 48, False),
    (4, 2, 128, 32, 96, True),
    (2, 2, 64, 16, 16, False),      # 64-voxel x runs: half of every MMA's rows unused
    (4, 2, 64, 32, 32, True),
    (2, 4, 192, 96, 32, False),
    (2, 2, 64, 16, 48, True),
    (10, 4, 128, 16, 16, True),     # 16 input channels, H % 4 == 0: the z-walking kernel (ragged last z block)
    (3, 8, 64, 16, 32, False),
    (16, 4, 128, 16, 32, False),
]


def _kernels(D, H, Ci, Co):
    """The tcgen05 kernels that tile this shape."""
    out = []
    if H % 2 == 0 and D % 2 == 0:
        out.append(U.CONV_TCGEN05_CHUNKED)
    if Ci == 16 and H % 4 == 0 and Co % 48:
        out.append(U.CONV_TCGEN05_ZWALK)
    return out


@pytest.mark.parametrize("case", CASES, ids=lambda c: "x".join(map(str, c[:5])) + ("-relu" if c[5] else ""))
def test_tcgen05_conv_matches_reference(case):
    D, H, W, Ci, Co, relu = case
    x, w, b = _operands(D, H, W, Ci, Co, seed=D * 100 + Ci)
    ref = _reference(x, w, b, D, H, W, Ci, Co, relu)
    kernels = _kernels(D, H, Ci, Co)
    assert kernels
    for path in kernels + [U.CONV_TCGEN05]:
        yf, yb = _run(path, x, w, b, D, H, W, Ci, Co, relu)
        err = float((yf.double() - ref).norm() / ref.norm())
        assert err < 1e-5, (path, err)
        assert torch.all((yb.double() - yf.double()).abs() <= 2.0 ** -8 * yf.double().abs() + 1e-30)


@pytest.mark.parametrize("path", [U.CONV_TCGEN05_CHUNKED, U.CONV_TCGEN05_ZWALK], ids=["chunked", "z-walking"])
def test_tcgen05_conv_writes_only_its_channel_slice(path):
    D, H, W, Ci, Co = 2, 4, 128, 16, 16
    x, w, b = _operands(D, H, W, Ci, Co, seed=5)
    ref = _reference(x, w, b, D, H, W, Ci, Co, True)
    yf, yb = _run(path, x, w, b, D, H, W, Ci, Co, True, o_stride=48, o_off=16)
    assert torch.all(yf[:, :16] == 7.0) and torch.all(yf[:, 32:] == 7.0)
    assert torch.all(yb[:, :16] == 7.0) and torch.all(yb[:, 32:] == 7.0)
    assert float((yf[:, 16:32].double() - ref).norm() / ref.norm()) < 1e-5


def test_tcgen05_and_warp_mma_kernels_agree():
    D, H, W, Ci, Co = 2, 4, 128, 32, 32
    x, w, b = _operands(D, H, W, Ci, Co, seed=9)
    a, _ = _run(U.CONV_TCGEN05, x, w, b, D, H, W, Ci, Co, True)
    c, _ = _run(U.CONV_WARP_MMA, x, w, b, D, H, W, Ci, Co, True)
    assert float((a - c).norm() / c.norm()) < 1e-5


def test_tcgen05_conv_rejects_shapes_it_cannot_tile():
    for D, H, W in ((2, 2, 32), (3, 2, 64), (2, 2, 96), (3, 6, 64)):
        x, w, b = _operands(D, H, W, 16, 16, seed=3)
        with pytest.raises(lt.LtError):
            _run(U.CONV_TCGEN05, x, w, b, D, H, W, 16, 16, False)
    x, w, b = _operands(3, 4, 64, 16, 16, seed=4)      # odd D: the chunked kernel alone cannot
    with pytest.raises(lt.LtError):
        _run(U.CONV_TCGEN05_CHUNKED, x, w, b, 3, 4, 64, 16, 16, False)
    x, w, b = _operands(2, 2, 64, 32, 16, seed=4)      # 32 input channels: not the z-walking kernel
    with pytest.raises(lt.LtError):
        _run(U.CONV_TCGEN05_ZWALK, x, w, b, 2, 2, 64, 32, 16, False)


def test_unet_at_full_resolution_is_unchanged_by_the_tcgen05_layers(monkeypatch):
    """The whole network at 128^3 (where the full-resolution layers take the
    tcgen05 kernel by default) against the same network with every layer
    forced onto the warp-level MMA kernel: forward output and input gradient."""
    n = 128
    net = U.UNet(seed=3)
    g = torch.Generator().manual_seed(11)
    x = torch.zeros(n, n, n, 16)
    x[..., 0] = torch.rand(n, n, n, generator=g)
    xb = x.bfloat16().cuda()
    gout = (0.01 * torch.randn(n, n, n, 16, generator=g)).cuda()   # float32, as backward expects

    def run():
        out = net.forward(xb, keep=True).float().clone()
        gin = net.backward(gout).float().clone()
        torch.cuda.synchronize()
        return out, gin

    out_tc, gin_tc = run()
    U.device_status()
    calls = U._call

    def warp_only(name, *args):
        if name == "lt_nn_conv3d_ex":
            args = list(args)
            args[-2] = U.CONV_WARP_MMA
        return calls(name, *args)

    monkeypatch.setattr(U, "_call", warp_only)
    out_w, gin_w = run()
    assert float((out_tc - out_w).norm() / out_w.norm()) < 1e-5
    assert float((gin_tc - gin_w).norm() / gin_w.norm()) < 1e-5


@pytest.mark.parametrize("path", [U.CONV_TCGEN05_CHUNKED, U.CONV_TCGEN05_ZWALK, U.CONV_WARP_MMA],
                         ids=["chunked", "z-walking", "warp-mma"])
def test_batched_frames_are_independent(path):
    """Two frames in one call (the ABI's batch argument): each equals the
    reference convolution of its own frame."""
    D, H, W, Ci, Co = 2, 4, 128, 16, 16
    xs, refs = [], []
    w = b = None
    for f in range(2):
        x, w_, b_ = _operands(D, H, W, Ci, Co, seed=40)
        x = (x.float() * (1.0 + f)).to(torch.bfloat16)         # a different frame, same weights
        w, b = w_, b_
        xs.append(x)
        refs.append(_reference(x, w, b, D, H, W, Ci, Co, True))
    V = D * H * W
    xin, wd, bd = torch.cat(xs).cuda(), w.cuda(), b.cuda()   # alive until the kernel has run
    out_f = torch.full((2 * V * Co,), 7.0, device="cuda")
    U._call("lt_nn_conv3d_ex", xin.data_ptr(), wd.data_ptr(), bd.data_ptr(), None, out_f.data_ptr(),
            2, D, H, W, Ci, Co, Co, 0, 1, path, U._s())
    U.device_status()
    y = out_f.reshape(2, V, Co).cpu().double()
    for f in range(2):
        assert float((y[f] - refs[f]).norm() / refs[f].norm()) < 1e-5, f
