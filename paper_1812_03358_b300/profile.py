"""Run one stage of the benchmark workloads on its own, for timing and for
profilers (ncu captures a named kernel of a short, fixed launch sequence).

    python -m paper_1812_03358_b300.profile --op beam_forward --reps 3
    python -m paper_1812_03358_b300.profile --op conv --conv 16,16,128 --reps 3

Workload "plenoptic128": the plenoptic camera (100 x 100 lenslets of 10 x 10
pixels, 2 x 2 cells) over a 128^3 plume volume of 1 mm voxels, as in the
benchmark.  Ops: beam_forward / beam_adjoint (stage one and its adjoint),
stage2_forward / stage2_adjoint (microlenses), forward / adjoint (the whole
camera), recon_step (one Table V iteration), multiview_step (one Table V
iteration of the batched multi-view workload: four yawed 2048^2 cameras and a
200 x 200-lenslet plenoptic camera around 256^3 voxels, 16 frames, or
--frames), multiview_forward / multiview_adjoint (that workload's whole
projector or back-projector), conv (one
U-Net convolution
layer: input channels, output channels, grid size; tcgen05 kernel where the
shape allows it).  Each op runs once to warm up, then `reps` times, each
timed with CUDA events on the current stream after an L2 flush (a 512 MB
write); the mean and minimum are printed.
"""
import argparse
import os
import sys

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)


def _plenoptic_ops(variant):
    import torch
    from paper_1812_03358_b300 import inputs as I
    from paper_1812_03358_b300 import lt
    vol, cam = I.config_plenoptic()
    plan = lt.Plan(vol, [cam])
    if variant is not None:
        lt.lt_plan_set_forward_variant(plan.handle, variant)
    x = torch.from_numpy(I.plume_field(vol, seed=2000).reshape(1, -1)).cuda()
    fa = plan.stage1(0, x)
    y = plan.forward(x)
    ga = plan.stage2_adjoint(0, y)
    xa = plan.new_x()
    rec = lt.Recon(plan, y, beta=1e-3)
    ops = {
        "beam_forward": lambda: plan.stage1(0, x, fa),
        "stage2_forward": lambda: plan.stage2(0, fa, y),
        "stage2_adjoint": lambda: plan.stage2_adjoint(0, y, ga),
        "beam_adjoint": lambda: plan.stage1_adjoint(0, ga, xa),
        "forward": lambda: plan.forward(x, y),
        "adjoint": lambda: plan.adjoint(y, xa),
        "recon_step": lambda: rec.iterate(1),
    }
    return ops, (plan, rec)


def _multiview_op(op, frames):
    import torch
    from paper_1812_03358_b300 import inputs as I
    from paper_1812_03358_b300 import lt
    vol, cams = I.config_multiview()
    plan = lt.Plan(vol, cams, frames)
    x = torch.stack([I.plume_field_torch(vol, seed=3100, drift_voxels=float(f)) for f in range(frames)]).contiguous()
    y = I.poisson_images_torch(plan.forward(x), 1e4, seed=3200)
    if op == "multiview_forward":
        return (lambda: plan.forward(x, y)), (plan, x, y)
    if op == "multiview_adjoint":
        xa = plan.new_x()
        return (lambda: plan.adjoint(y, xa)), (plan, xa, y)
    rec = lt.Recon(plan, y, beta=1e-3)
    del x
    return (lambda: rec.iterate(1)), (plan, rec, y)


def _conv_op(ci, co, n, path):
    import torch
    from paper_1812_03358_b300 import unet
    layer = unet.Conv(ci, co, torch.Generator().manual_seed(3))
    g = torch.Generator(device="cuda").manual_seed(4)
    xin = torch.randn(n, n, n, ci, device="cuda", generator=g).to(torch.bfloat16)
    out = torch.empty(n, n, n, co, device="cuda", dtype=torch.bfloat16)
    return (lambda: unet.conv3d(xin, layer.wb, layer.b, out, Ci=ci, Co=co, dims=(n, n, n), path=path)), \
        (layer, xin, out)


def main(argv=None):
    import torch
    ap = argparse.ArgumentParser(description=__doc__.split("\n\n")[0])
    ap.add_argument("--op", default="beam_forward")
    ap.add_argument("--reps", type=int, default=3)
    ap.add_argument("--variant", type=int, default=None, help="forward kernel variant (default: the plan's)")
    ap.add_argument("--frames", type=int, default=16, help="multi-view ops: frames of the workload")
    ap.add_argument("--conv", default="16,16,128", help="conv: input channels, output channels, grid size")
    ap.add_argument("--conv-path", type=int, default=0,
                    help="conv kernel: 0 automatic, 1 warp MMA, 2 tcgen05, 3 tcgen05 chunked, 4 tcgen05 z-walking")
    a = ap.parse_args(argv)
    from paper_1812_03358_b300 import build
    build.build()
    torch.cuda.set_device(0)
    if a.op == "conv":
        ci, co, n = (int(v) for v in a.conv.split(","))
        fn, keep = _conv_op(ci, co, n, a.conv_path)
    elif a.op.startswith("multiview_"):
        fn, keep = _multiview_op(a.op, a.frames)
    else:
        ops, keep = _plenoptic_ops(a.variant)
        fn = ops[a.op]
    flush = torch.empty(512 * 1024 * 1024 // 4, dtype=torch.float32, device="cuda")
    stream = torch.cuda.current_stream()
    fn()
    torch.cuda.synchronize()
    times = []
    torch.cuda.nvtx.range_push("timed")   # ncu --nvtx --nvtx-include "timed/" selects the timed launches
    for _ in range(a.reps):
        flush.zero_()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        fn()
        e1.record(stream)
        e1.synchronize()
        times.append(e0.elapsed_time(e1))
    torch.cuda.nvtx.range_pop()
    print(f"{a.op}: mean {sum(times) / len(times):.4f} ms, min {min(times):.4f} ms over {a.reps} runs")
    del keep


if __name__ == "__main__":
    main()
