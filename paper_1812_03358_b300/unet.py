"""Learned warm start: a 3D U-Net over the lt_nn_* kernels (marshalling only).

The network maps a normalised back-projection to an initial volume for the
Table V reconstruction (which then refines it; the plain solver stays the
fallback and the reference the result is measured against).  Four levels, 16-128 channels, 3x3x3
convolutions with ReLU, 2x2x2 average pooling, nearest upsampling and
channel-concatenated skips; bfloat16 activations and weights, float32
accumulation, float32 master weights updated by Adam.  Every layer runs in the
library's CUDA kernels; torch only allocates memory.

Input/output convention (scale-equivariant): with D = A^T A 1 the diagonal of
the majoriser, u = (A^T y / D) / m where m = max(A^T y / D); the network
predicts x / m, so x0 = m * net(u).
"""
from __future__ import annotations

import ctypes
from ctypes import c_float, c_int32, c_int64, c_void_p

import numpy as np
import torch

from . import lt

_SIGS = {
    "lt_nn_conv3d": [c_void_p, c_void_p, c_void_p, c_void_p, c_void_p, c_int32, c_int32, c_int32, c_int32, c_int32,
                     c_int32, c_int32, c_int32, c_int32, c_void_p],
    "lt_nn_conv3d_ex": [c_void_p, c_void_p, c_void_p, c_void_p, c_void_p, c_int32, c_int32, c_int32, c_int32,
                        c_int32, c_int32, c_int32, c_int32, c_int32, c_int32, c_void_p],
    "lt_nn_device_status": [c_void_p],
    "lt_nn_conv3d_wgrad": [c_void_p, c_void_p, c_void_p, c_void_p, c_void_p, c_int64, c_int32, c_int32, c_int32,
                           c_int32, c_int32, c_int32, c_void_p],
    "lt_nn_conv3d_wgrad_workspace": [c_int32, c_int32, c_int32, c_int32, c_int32, c_int32, c_void_p],
    "lt_nn_grad_norm_clip": [c_void_p, c_int64, c_float, c_void_p, c_void_p, c_void_p],
    "lt_nn_conv3d_flip": [c_void_p, c_void_p, c_int32, c_int32, c_void_p],
    "lt_nn_f32_to_bf16": [c_void_p, c_void_p, c_int64, c_void_p],
    "lt_nn_bf16_to_f32": [c_void_p, c_void_p, c_int64, c_void_p],
    "lt_nn_relu_backward": [c_void_p, c_void_p, c_int64, c_void_p],
    "lt_nn_avgpool2": [c_void_p, c_void_p, c_int32, c_int32, c_int32, c_int32, c_int32, c_int32, c_int32, c_void_p],
    "lt_nn_avgpool2_backward": [c_void_p, c_void_p, c_int32, c_int32, c_int32, c_int32, c_int32, c_int32, c_int32,
                                c_void_p],
    "lt_nn_upsample2": [c_void_p, c_void_p, c_int32, c_int32, c_int32, c_int32, c_int32, c_int32, c_int32, c_void_p],
    "lt_nn_upsample2_backward": [c_void_p, c_void_p, c_int32, c_int32, c_int32, c_int32, c_int32, c_int32, c_int32,
                                 c_void_p],
    "lt_nn_copy_channels": [c_void_p, c_void_p, c_int64, c_int32, c_int32, c_int32, c_int32, c_int32, c_void_p],
    "lt_nn_add": [c_void_p, c_void_p, c_void_p, c_int64, c_void_p],
    "lt_nn_prepare_input": [c_void_p, c_void_p, c_void_p, c_void_p, c_void_p, c_int64, c_void_p],
    "lt_nn_unpack_output": [c_void_p, c_void_p, c_void_p, c_int64, c_void_p],
    "lt_nn_mse": [c_void_p, c_void_p, c_void_p, c_void_p, c_void_p, c_int64, c_void_p],
    "lt_nn_adam": [c_void_p, c_void_p, c_void_p, c_void_p, c_void_p, c_void_p, c_int64, c_float, c_float, c_float,
                   c_float, c_int32, c_void_p],
}
_bound = False


def nn():
    global _bound
    L = lt.lib()
    if not _bound:
        for name, args in _SIGS.items():
            fn = getattr(L, name)
            fn.restype = c_int32
            fn.argtypes = args
        if hasattr(L, "lt_nn_test_stall_tensor_core"):   # the test build
            L.lt_nn_test_stall_tensor_core.restype = c_int32
            L.lt_nn_test_stall_tensor_core.argtypes = [c_int32, c_void_p]
        _bound = True
    return L


def _call(name, *args):
    lt._check(getattr(nn(), name)(*args))


def pool(s, p, d, C):
    _need(s, int(np.prod(d)) * C, "avgpool input")
    if p.numel() != int(np.prod(d)) * C // 8:
        raise ValueError("avgpool output shape")
    _call("lt_nn_avgpool2", _pb(s), _pb(p), 1, *d, C, C, 0, _s())


def pool_back(g, gs, d, C):
    if g.numel() != int(np.prod(d)) * C // 8 or gs.numel() != int(np.prod(d)) * C:
        raise ValueError("avgpool backward shapes")
    _call("lt_nn_avgpool2_backward", _pb(g), _pb(gs), 1, *d, C, C, 0, _s())


def upsample(x, cat, dsmall, cx, ctot):
    if x.numel() != int(np.prod(dsmall)) * cx or cat.numel() != 8 * int(np.prod(dsmall)) * ctot:
        raise ValueError("upsample shapes")
    _call("lt_nn_upsample2", _pb(x), _pb(cat), 1, *dsmall, cx, ctot, 0, _s())


def upsample_back(g, gx, dsmall, cx, ctot):
    if gx.numel() != int(np.prod(dsmall)) * cx or g.numel() != 8 * int(np.prod(dsmall)) * ctot:
        raise ValueError("upsample backward shapes")
    _call("lt_nn_upsample2_backward", _pb(g), _pb(gx), 1, *dsmall, cx, ctot, 0, _s())


def copy_channels(src, dst, voxels, C, s_stride, s_off, d_stride, d_off):
    if src.numel() != voxels * s_stride or dst.numel() != voxels * d_stride:
        raise ValueError("copy_channels shapes")
    _call("lt_nn_copy_channels", _pb(src), _pb(dst), voxels, C, s_stride, s_off, d_stride, d_off, _s())


def _p(t):
    return t.data_ptr() if t is not None else None


def _ptr(t, dtype, what):
    """Device pointer of a contiguous tensor of the element type the kernel
    reads or writes (a tensor of another type would make it run past the
    buffer); None passes through."""
    if t is None:
        return None
    if t.dtype != dtype:
        raise TypeError(f"{what}: expected {dtype}, got {t.dtype}")
    if not t.is_contiguous():
        raise ValueError(f"{what}: the tensor must be contiguous")
    if t.device.type != torch.device(DEVICE).type:
        raise ValueError(f"{what}: expected a {DEVICE} tensor, got {t.device}")
    return t.data_ptr()


def _pb(t, what="bfloat16 operand"):
    return _ptr(t, torch.bfloat16, what)


def _pf(t, what="float32 operand"):
    return _ptr(t, torch.float32, what)


def _s():
    return lt._stream()


DEVICE = "cuda"
NORM_WORK = 256          # LT_NN_NORM_WORK: scratch floats of lt_nn_grad_norm_clip


def bf16(*shape):
    return torch.empty(*shape, dtype=torch.bfloat16, device=DEVICE)


# ---- layer calls (names follow the C ABI) ---------------------------------

def _need(t, n, what):
    if t is not None and t.numel() < n:
        raise ValueError(f"{what}: {t.numel()} elements, the layer needs {n}")


def _need_at_least(t, n, what):
    if t.numel() < n:
        raise ValueError(f"{what}: {t.numel()} elements, the call needs {n}")


# lt_nn_conv3d_ex kernel choice
CONV_AUTO, CONV_WARP_MMA, CONV_TCGEN05, CONV_TCGEN05_CHUNKED, CONV_TCGEN05_ZWALK = 0, 1, 2, 3, 4


def device_status():
    """Raises LtError if a tcgen05 kernel gave up waiting for the tensor core
    (synchronises the stream; clears the status)."""
    _call("lt_nn_device_status", _s())


def conv3d(inp, w, b, out_bf=None, out_f=None, *, Ci, Co, dims, o_stride=None, o_off=0, relu=True,
           path=CONV_AUTO):
    D, H, W = dims
    V = D * H * W
    _need(inp, V * Ci, "conv3d input")
    _need(w, 27 * Ci * Co, "conv3d weights")
    _need(b, Co, "conv3d bias")
    _need(out_bf, V * (o_stride or Co), "conv3d output")
    _need(out_f, V * (o_stride or Co), "conv3d output")
    if inp.numel() != V * Ci:
        raise ValueError("conv3d input shape does not match dims x Ci")
    _call("lt_nn_conv3d_ex", _pb(inp, "conv3d input"), _pb(w, "conv3d weights"), _pf(b, "conv3d bias"),
          _pb(out_bf, "conv3d output"), _pf(out_f, "conv3d output"), 1, D, H, W, Ci, Co,
          o_stride or Co, o_off, int(relu), int(path), _s())


def wgrad_workspace_floats(*, Ci, Co, dims):
    """Floats of device workspace lt_nn_conv3d_wgrad needs for this shape."""
    n = c_int64(0)
    _call("lt_nn_conv3d_wgrad_workspace", 1, *dims, Ci, Co, ctypes.byref(n))
    return int(n.value)


def conv3d_wgrad(inp, g, dw, db, *, Ci, Co, dims, work=None):
    """dw += weight gradient, db += bias gradient (deterministic).  `work`: a
    float32 device workspace of at least wgrad_workspace_floats() elements
    (allocated here when None)."""
    D, H, W = dims
    V = D * H * W
    if inp.numel() != V * Ci or g.numel() != V * Co:
        raise ValueError("conv3d_wgrad: input / gradient shapes do not match dims")
    _need(dw, 27 * Ci * Co, "conv3d_wgrad dw")
    _need(db, Co, "conv3d_wgrad db")
    need = wgrad_workspace_floats(Ci=Ci, Co=Co, dims=dims)
    if work is None:
        work = torch.empty(max(need, 1), device=DEVICE)
    _need_at_least(work, need, "conv3d_wgrad workspace")
    _call("lt_nn_conv3d_wgrad", _pb(inp, "wgrad input"), _pb(g, "wgrad gradient"), _pf(dw, "wgrad dw"),
          _pf(db, "wgrad db"), _pf(work, "wgrad workspace"), work.numel(), 1, D, H, W, Ci, Co, _s())


class Conv:
    """One 3x3x3 convolution's parameters: float32 master weights [Co][27][Ci]
    and bias, the weights' bfloat16 copy and the gradients.  The network moves
    them into its flat parameter buffers (Adam and the gradient norm run once
    over all of them); these attributes are then views into those buffers."""

    def __init__(self, ci, co, gen):
        self.ci, self.co = ci, co
        std = (2.0 / (27 * ci)) ** 0.5
        self.w = (torch.randn(co, 27, ci, generator=gen, dtype=torch.float32) * std).to(DEVICE)
        self.b = torch.zeros(co, device=DEVICE)
        self.wb = bf16(co, 27, ci)
        self.wt = bf16(ci, 27, co)
        self.gw = torch.zeros_like(self.w)
        self.gb = torch.zeros_like(self.b)
        self.sync_bf16()

    def sync_bf16(self):
        _call("lt_nn_f32_to_bf16", _pf(self.w), _pb(self.wb), self.w.numel(), _s())

    def flip(self):
        _call("lt_nn_conv3d_flip", _pb(self.wb), _pb(self.wt), self.ci, self.co, _s())


class UNet:
    """4-level 3D U-Net, channels (16, 32, 64, 128); spatial size divisible by 8."""

    CH = (16, 32, 64, 128)

    def __init__(self, seed=0):
        gen = torch.Generator().manual_seed(seed)
        c1, c2, c3, c4 = self.CH
        self.enc = [(Conv(16, c1, gen), Conv(c1, c1, gen)), (Conv(c1, c2, gen), Conv(c2, c2, gen)),
                    (Conv(c2, c3, gen), Conv(c3, c3, gen))]
        self.bott = (Conv(c3, c4, gen), Conv(c4, c4, gen))
        self.dec = [(Conv(c4 + c3, c3, gen), Conv(c3, c3, gen)), (Conv(c3 + c2, c2, gen), Conv(c2, c2, gen)),
                    (Conv(c2 + c1, c1, gen), Conv(c1, c1, gen))]
        self.head = Conv(c1, 16, gen)
        self.step = 0
        self._flatten()
        self.clip = torch.zeros(2, device=DEVICE)                 # {scale, gradient norm} of the last step
        self._norm_work = torch.empty(NORM_WORK, device=DEVICE)
        self._wg_work = torch.empty(0, device=DEVICE)

    def _flatten(self):
        """Parameters, gradients and Adam moments of every layer in four flat
        float32 buffers (and the bfloat16 weights in a fifth); each weight and
        bias block starts at a multiple of 64 elements."""
        segs, off = [], 0
        for c in self.convs():
            for name in ("w", "b"):
                n = getattr(c, name).numel()
                segs.append((c, name, off, n))
                off += -(-n // 64) * 64
        self.n_params = off
        self.P = torch.zeros(off, device=DEVICE)
        self.G = torch.zeros(off, device=DEVICE)
        self.M = torch.zeros(off, device=DEVICE)
        self.V = torch.zeros(off, device=DEVICE)
        self.PB = bf16(off)
        for c, name, o, n in segs:
            t = getattr(c, name)
            self.P[o:o + n].copy_(t.reshape(-1))
            setattr(c, name, self.P[o:o + n].view(t.shape))
            if name == "w":
                c.gw = self.G[o:o + n].view(t.shape)
                c.wb = self.PB[o:o + n].view(t.shape)
            else:
                c.gb = self.G[o:o + n].view(t.shape)
        _call("lt_nn_f32_to_bf16", _pf(self.P), _pb(self.PB), off, _s())

    def _workspace(self, floats):
        if self._wg_work.numel() < floats:
            self._wg_work = torch.empty(floats, device=DEVICE)
        return self._wg_work

    def flops(self, dims):
        """Multiply-add flops (2 per MAC) of one forward pass on a D x H x W
        input: 2 * voxels * 27 * Ci * Co per convolution."""
        D, H, W = dims
        total = 0
        for l, (ca, cb) in enumerate(self.enc):
            v = (D >> l) * (H >> l) * (W >> l)
            total += 2 * v * 27 * (ca.ci * ca.co + cb.ci * cb.co)
        v = (D >> 3) * (H >> 3) * (W >> 3)
        total += 2 * v * 27 * sum(c.ci * c.co for c in self.bott)
        for i, (ca, cb) in enumerate(self.dec):
            l = 2 - i
            v = (D >> l) * (H >> l) * (W >> l)
            total += 2 * v * 27 * (ca.ci * ca.co + cb.ci * cb.co)
        return total + 2 * D * H * W * 27 * self.head.ci * self.head.co

    def convs(self):
        out = []
        for a, b in self.enc:
            out += [a, b]
        out += list(self.bott)
        for a, b in self.dec:
            out += [a, b]
        return out + [self.head]

    # -- forward -------------------------------------------------------------
    def forward(self, u, keep=False):
        """u: bfloat16 [D][H][W][16] (channel 0 = input).  Returns the float32
        output [D][H][W][16] (channel 0 = prediction)."""
        D, H, W, _ = u.shape
        c1, c2, c3, c4 = self.CH
        dims = [(D >> l, H >> l, W >> l) for l in range(4)]
        acts = {}
        x = u
        skips = []
        for l, (ca, cb) in enumerate(self.enc):
            d = dims[l]
            a = bf16(*d, ca.co)
            conv3d(x, ca.wb, ca.b, a, Ci=ca.ci, Co=ca.co, dims=d)
            s = bf16(*d, cb.co)
            conv3d(a, cb.wb, cb.b, s, Ci=cb.ci, Co=cb.co, dims=d)
            acts[("enc", l)] = (x, a, s)
            skips.append(s)
            p = bf16(*dims[l + 1], cb.co)
            pool(s, p, d, cb.co)
            x = p
        d = dims[3]
        ca, cb = self.bott
        a = bf16(*d, ca.co)
        conv3d(x, ca.wb, ca.b, a, Ci=ca.ci, Co=ca.co, dims=d)
        bo = bf16(*d, cb.co)
        conv3d(a, cb.wb, cb.b, bo, Ci=cb.ci, Co=cb.co, dims=d)
        acts["bott"] = (x, a, bo)
        x, cx = bo, c4
        for i, (ca, cb) in enumerate(self.dec):
            l = 2 - i
            d = dims[l]
            skip = skips[l]
            cs = skip.shape[-1]
            cat = bf16(*d, cx + cs)
            upsample(x, cat, dims[l + 1], cx, cx + cs)
            copy_channels(skip, cat, int(np.prod(d)), cs, cs, 0, cx + cs, cx)
            a = bf16(*d, ca.co)
            conv3d(cat, ca.wb, ca.b, a, Ci=ca.ci, Co=ca.co, dims=d)
            o = bf16(*d, cb.co)
            conv3d(a, cb.wb, cb.b, o, Ci=cb.ci, Co=cb.co, dims=d)
            acts[("dec", i)] = (cat, a, o, cx)
            x, cx = o, cb.co
        out = torch.empty(*dims[0], 16, device=DEVICE, dtype=torch.float32)
        hb = bf16(*dims[0], 16)
        conv3d(x, self.head.wb, self.head.b, hb, out, Ci=self.head.ci, Co=16, dims=dims[0], relu=False)
        acts["head"] = (x,)
        if keep:
            self._acts, self._dims = acts, dims
        return out

    # -- backward ------------------------------------------------------------
    def _conv_back(self, conv, inp, out_act, g, dims, relu=True):
        """g: bfloat16 gradient w.r.t. conv output (Co channels).  Returns the
        gradient w.r.t. its input (Ci channels)."""
        if relu:
            if out_act.numel() != g.numel():
                raise ValueError("relu backward shapes")
            _call("lt_nn_relu_backward", _pb(out_act), _pb(g), g.numel(), _s())
        work = self._workspace(max(1, wgrad_workspace_floats(Ci=conv.ci, Co=conv.co, dims=dims)))
        conv3d_wgrad(inp, g, conv.gw, conv.gb, Ci=conv.ci, Co=conv.co, dims=dims, work=work)
        conv.flip()
        gi = bf16(*dims, conv.ci)
        conv3d(g, conv.wt, None, gi, Ci=conv.co, Co=conv.ci, dims=dims, relu=False)
        return gi

    def backward(self, g_out):
        """g_out: float32 gradient w.r.t. the output [D][H][W][16]."""
        acts, dims = self._acts, self._dims
        if g_out.dtype != torch.float32 or tuple(g_out.shape) != (*dims[0], 16):
            raise TypeError(f"backward: expected a float32 {(*dims[0], 16)} gradient, got {g_out.dtype} "
                            f"{tuple(g_out.shape)}")
        self.G.zero_()
        g = bf16(*g_out.shape)
        _call("lt_nn_f32_to_bf16", _pf(g_out, "output gradient (float32)"), _pb(g), g_out.numel(), _s())
        (x,) = acts["head"]
        g = self._conv_back(self.head, x, None, g, dims[0], relu=False)
        skip_grads = [None, None, None]
        for i in reversed(range(3)):          # finest decoder level first
            ca, cb = self.dec[i]
            l = 2 - i
            cat, a, o, cx = acts[("dec", i)]
            d = dims[l]
            g = self._conv_back(cb, a, o, g, d)
            g = self._conv_back(ca, cat, a, g, d)           # gradient w.r.t. the concatenation
            cs = cat.shape[-1] - cx
            gs = bf16(*d, cs)
            copy_channels(g, gs, int(np.prod(d)), cs, cx + cs, cx, cs, 0)
            skip_grads[l] = gs
            gx = bf16(*dims[l + 1], cx)
            upsample_back(g, gx, dims[l + 1], cx, cx + cs)
            g = gx
        x, a, bo = acts["bott"]
        g = self._conv_back(self.bott[1], a, bo, g, dims[3])
        g = self._conv_back(self.bott[0], x, a, g, dims[3])
        for l in reversed(range(3)):
            ca, cb = self.enc[l]
            x, a, s = acts[("enc", l)]
            d = dims[l]
            gs = bf16(*d, cb.co)
            pool_back(g, gs, d, cb.co)
            if skip_grads[l].numel() != gs.numel():
                raise ValueError("skip gradient shape")
            _call("lt_nn_add", _pb(gs), _pb(skip_grads[l]), _pb(gs), gs.numel(), _s())
            g = self._conv_back(cb, a, s, gs, d)
            g = self._conv_back(ca, x, a, g, d)
        return g

    def adam_step(self, lr, max_norm=0.0):
        """One Adam step over every parameter, the gradient first scaled to a
        global norm of at most max_norm (no clipping when max_norm <= 0; a
        non-finite gradient is dropped).  self.clip holds {scale, norm} on the
        device afterwards."""
        self.step += 1
        _call("lt_nn_grad_norm_clip", _pf(self.G), self.n_params, float(max_norm), _pf(self._norm_work),
              _pf(self.clip), _s())
        _call("lt_nn_adam", _pf(self.P), _pb(self.PB), _pf(self.G), _pf(self.clip), _pf(self.M), _pf(self.V),
              self.n_params, lr, 0.9, 0.999, 1e-8, self.step, _s())


class WarmStart:
    """Network input preparation, inference and training on (x_true, A^T y)
    pairs, all in the library's kernels."""

    def __init__(self, plan, net: UNet):
        self.plan = plan
        self.net = net
        n = plan.nvox
        ones = torch.ones(1, n, device="cuda")
        self.D = plan.adjoint(plan.forward(ones)).reshape(-1).contiguous()
        self.r = torch.empty(n, device="cuda")
        self.m = torch.zeros(1, device="cuda")
        self.loss = torch.zeros(1, device="cuda")
        v = plan.vol
        self.dims = (v.nz, v.ny, v.nx)
        self.u = bf16(*self.dims, 16)

    def prepare(self, bp):
        _call("lt_nn_prepare_input", _pf(bp, "back-projection"), _pf(self.D), _pf(self.r), _pf(self.m), _pb(self.u),
              self.r.numel(), _s())
        return self.u

    def infer(self, bp):
        """x0 (float32 [n_vox]) from a back-projection A^T y."""
        out = self.net.forward(self.prepare(bp))
        x0 = torch.empty(self.r.numel(), device="cuda")
        _call("lt_nn_unpack_output", _pf(out), _pf(self.m), _pf(x0), x0.numel(), _s())
        return x0

    def train_step(self, bp, x_true, lr, max_norm=0.0):
        out = self.net.forward(self.prepare(bp), keep=True)
        g = torch.empty_like(out)
        self.loss.zero_()
        _call("lt_nn_mse", _pf(out), _pf(x_true, "target volume"), _pf(self.m), _pf(g), _pf(self.loss), x_true.numel(),
              _s())
        self.net.backward(g)
        self.net.adam_step(lr, max_norm)
        return self.loss
