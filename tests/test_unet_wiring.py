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


def test_layer_calls_reject_wrong_element_types(monkeypatch):
    """A tensor of the wrong element type would make a kernel read or write
    past its buffer (a bfloat16 gradient read as float32 is twice as long):
    the binding refuses it before anything is launched."""
    calls = []
    monkeypatch.setattr(unet, "DEVICE", "cpu")
    monkeypatch.setattr(unet, "_call", lambda name, *a: calls.append(name))
    monkeypatch.setattr(unet, "_s", lambda: 0)
    net = unet.UNet(seed=0)
    x = torch.zeros(16, 16, 16, 16, dtype=torch.bfloat16)
    out = net.forward(x, keep=True)
    n = len(calls)
    with pytest.raises(TypeError):
        net.backward(torch.zeros_like(out).bfloat16())
    with pytest.raises(TypeError):
        net.backward(torch.zeros(8, 8, 8, 16))              # wrong shape
    with pytest.raises(TypeError):
        unet.conv3d(torch.zeros(2 * 2 * 2 * 16), net.head.wb, None, torch.zeros(2 * 2 * 2 * 16, dtype=torch.bfloat16),
                    Ci=16, Co=16, dims=(2, 2, 2))            # float32 input where bfloat16 is read
    with pytest.raises(TypeError):
        unet.conv3d(torch.zeros(8 * 16, dtype=torch.bfloat16), net.head.wb, None, None,
                    torch.zeros(8 * 16, dtype=torch.bfloat16), Ci=16, Co=16, dims=(2, 2, 2))   # bf16 out_f
    assert len(calls) == n                                   # nothing reached the library
