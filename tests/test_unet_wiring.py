"""The U-Net's forward/backward wiring (shapes of every layer call) runs end
to end with the kernels replaced by a no-op recorder, on the CPU: every
buffer handed to a kernel has exactly the size that kernel will touch."""
import pytest
import torch

from paper_1812_03358_b300 import unet


def test_forward_backward_shapes(monkeypatch):
    calls = []
    monkeypatch.setattr(unet, "DEVICE", "cpu")
    monkeypatch.setattr(unet, "_call", lambda name, *a: calls.append(name))
    monkeypatch.setattr(unet, "_s", lambda: 0)
    net = unet.UNet(seed=0)
    x = torch.zeros(16, 16, 16, 16, dtype=torch.bfloat16)
    out = net.forward(x, keep=True)
    assert out.shape == (16, 16, 16, 16)
    gi = net.backward(torch.zeros_like(out))
    assert gi.shape == (16, 16, 16, 16)
    # one forward conv per layer, one weight gradient and one data gradient each
    assert calls.count("lt_nn_conv3d_ex") == 2 * 15 and calls.count("lt_nn_conv3d_wgrad") == 15
    with pytest.raises(ValueError):
        unet.conv3d(torch.zeros(10, dtype=torch.bfloat16), net.head.wb, None, torch.zeros(10, dtype=torch.bfloat16),
                    Ci=16, Co=16, dims=(2, 2, 2))
