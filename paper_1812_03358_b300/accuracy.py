"""Angular-plane discretisation study (Sec. VI-A): accuracy and cost of the
pillbox and Dirac angular bases against a fine Dirac (pinhole) rendering.

For each basis and K = n x n cells of the main lens, the plenoptic image of a
seeded plume volume is rendered with the CUDA projector and compared with the
reference through the normalised squared difference
    NSD(y) = ||y - y_ref||^2 / ||y_ref||^2,
and the forward projection is timed with CUDA events.  The camera is the
plenoptic camera of the simulated-plenoptic table with fewer lenslets (the
reference rendering keeps a few thousand cells) and the volume spans the same
128 mm cube.  Marshalling only: every rendering runs in the library's kernels.

Run as a module for one JSON line:
``python -m paper_1812_03358_b300.accuracy --ref 64 --grid 2 4 8 16``.
"""
from __future__ import annotations

import argparse
import json

import numpy as np
import torch

from . import inputs as I
from . import lt


def study_camera(n: int, basis: int, n_lenslets: int = 40) -> I.Camera:
    cam = I.plenoptic_camera(n_lenslets=n_lenslets, ks=n, kt=n)
    cam.basis = basis
    return cam


def render(vol: I.Volume, cam: I.Camera, x, reps: int = 5):
    """(image, mean forward ms, kept cells) of one configuration."""
    plan = lt.Plan(vol, [cam])
    xd = x.reshape(1, -1)
    y = plan.forward(xd)
    ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(reps)]
    for a, b in ev:
        a.record()
        plan.forward(xd, y)
        b.record()
    torch.cuda.synchronize()
    ms = sum(a.elapsed_time(b) for a, b in ev) / reps
    out = y.reshape(-1).double().cpu().numpy()
    cells = plan.cells[0]
    plan.close()
    return out, ms, cells


def nsd(y, ref) -> float:
    return float(np.sum((y - ref) ** 2) / np.sum(ref ** 2))


def angular_study(grid=(2, 4, 8, 16), ref: int = 64, n_vox: int = 64, n_lenslets: int = 40, seed: int = 3000):
    vox = 128.0 / n_vox
    vol = I.Volume(n_vox, n_vox, n_vox, vox, vox, vox)
    x = I.plume_field_torch(vol, seed).contiguous()
    y_ref, ms_ref, k_ref = render(vol, study_camera(ref, I.BASIS_DIRAC, n_lenslets), x, reps=2)
    rows = []
    for n in grid:
        for name, basis in (("pillbox", I.BASIS_PILLBOX), ("dirac", I.BASIS_DIRAC)):
            try:
                y, ms, k = render(vol, study_camera(n, basis, n_lenslets), x)
            except lt.LtError as e:   # e.g. a footprint wider than the kernels' windows
                rows.append({"basis": name, "grid": n, "unsupported": str(e)})
                continue
            rows.append({"basis": name, "grid": n, "cells": k, "nsd": nsd(y, y_ref), "forward_ms": ms})
    return {"reference": {"basis": "dirac", "grid": ref, "cells": k_ref, "forward_ms": ms_ref},
            "volume": [n_vox] * 3, "lenslets": n_lenslets, "rows": rows}


def main(argv=None):
    from . import build
    ap = argparse.ArgumentParser(description="pillbox vs Dirac angular discretisation (accuracy and time)")
    ap.add_argument("--ref", type=int, default=64)
    ap.add_argument("--grid", type=int, nargs="+", default=[2, 4, 8, 16])
    ap.add_argument("--n", type=int, default=64, help="volume edge in voxels (128 mm cube)")
    ap.add_argument("--lenslets", type=int, default=40)
    a = ap.parse_args(argv)
    build.build()
    print(json.dumps(angular_study(tuple(a.grid), a.ref, a.n, a.lenslets)))


if __name__ == "__main__":
    main()
