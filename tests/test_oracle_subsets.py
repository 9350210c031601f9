"""View-subset acceleration (Sec. V, eq. subset) in the oracle.

Pins, independent of the subset code itself:
* the cell subsets partition the angular plane, so the subset operators of a
  partition sum to the full operator (single lens, plenoptic, rotated);
* for one slice exactly at the in-focus distance every angular cell carries
  the same transport (all rays from a point of the focal plane meet at its
  conjugate point), A_k = A / K, so K/|S| sum_{k in S} A_k = A and the subset
  iteration must reproduce the full Table V iteration."""
import math

import numpy as np
import pytest

from oracle import camera as O
from oracle import recon as R
from paper_1812_03358_b300 import inputs as I


def test_subset_cells_partition_the_angular_plane():
    for K, N in [(4, 2), (4, 3), (9, 4), (16, 16), (3, 5)]:
        seen = []
        for it in range(N):
            S = R.subset_cells(K, N, it)
            assert all(k % N == it % N for k in S)
            seen += S
        assert sorted(seen) == list(range(K))
        assert R.subset_cells(K, N, N + 1) == R.subset_cells(K, N, 1)   # cyclic


@pytest.mark.parametrize("which", ["single", "plenoptic", "rotated"])
def test_subset_operators_sum_to_the_full_operator(which):
    if which == "plenoptic":
        vol, cam = I.tiny_plenoptic()
    else:
        vol = I.Volume(7, 6, 5, 4.0, 4.5, 5.0)
        cam = I.table_single_lens(12, 0.5, yaw=0.4 if which == "rotated" else 0.0, ks=2, kt=2)
    K = len(O.lens_cells(cam))
    assert K == 4
    x = I.gaussian_blobs(vol, seed=7).ravel()
    y = I.uniform_random(cam.det_ns * cam.det_nt, seed=8)
    full_f, full_a = np.ravel(O.forward(vol, cam, x)), np.ravel(O.adjoint(vol, cam, y))
    for N in (2, 3):
        sf = sum(np.ravel(O.forward(vol, cam, x, cells=R.subset_cells(K, N, s))) for s in range(N))
        sa = sum(np.ravel(O.adjoint(vol, cam, y, cells=R.subset_cells(K, N, s))) for s in range(N))
        assert np.abs(sf - full_f).max() <= 1e-12 * np.abs(full_f).max()
        assert np.abs(sa - full_a).max() <= 1e-12 * np.abs(full_a).max()
    # a subset really is a part: one cell alone differs from the whole
    one = np.ravel(O.forward(vol, cam, x, cells=[0]))
    assert np.abs(one - full_f).max() > 0.1 * np.abs(full_f).max()


def _in_focus_problem():
    f, D = 30.0, 31.3
    cam = I.table_single_lens(10, 0.4, ks=2, kt=2)
    cam.d_obj = 1.0 / (1.0 / f - 1.0 / D)      # exact conjugate of the detector plane
    vol = I.Volume(8, 8, 1, 3.0, 3.0, 3.0)     # one slice, centred at d_obj
    return vol, cam


def test_cells_carry_equal_transport_at_focus():
    vol, cam = _in_focus_problem()
    x = I.gaussian_blobs(vol, seed=3).ravel() + 0.1
    full = np.ravel(O.forward(vol, cam, x))
    for k in range(4):
        part = np.ravel(O.forward(vol, cam, x, cells=[k]))
        assert np.abs(4.0 * part - full).max() <= 1e-9 * np.abs(full).max()


@pytest.mark.parametrize("N", [2, 4])
def test_subset_iterations_equal_full_iterations_at_focus(N):
    vol, cam = _in_focus_problem()
    x_true = I.gaussian_blobs(vol, seed=4).ravel() + 0.05
    y = np.ravel(O.forward(vol, cam, x_true))
    ops = [(lambda z, cells=None: np.ravel(O.forward(vol, cam, z, cells=cells)),
            lambda r, cells=None: np.ravel(O.adjoint(vol, cam, r, cells=cells)))]
    full = R.fista(ops, [y], [None], vol.shape, 8, beta=1e-3, history=True)
    sub = R.fista(ops, [y], [None], vol.shape, 8, beta=1e-3, history=True, n_subset=N, n_cells=[4])
    assert np.abs(sub["x"] - full["x"]).max() <= 1e-9 * np.abs(full["x"]).max()
    assert np.allclose(sub["fits"], full["fits"], rtol=1e-8)


def test_subsets_differ_from_full_iterations_out_of_focus():
    """Away from focus the cells see different transports and the subset
    iterates differ (the approximation is an approximation)."""
    vol = I.Volume(7, 6, 5, 4.0, 4.5, 5.0)
    cam = I.table_single_lens(12, 0.5, ks=2, kt=2)
    x_true = I.gaussian_blobs(vol, seed=5).ravel()
    y = np.ravel(O.forward(vol, cam, x_true))
    ops = [(lambda z, cells=None: np.ravel(O.forward(vol, cam, z, cells=cells)),
            lambda r, cells=None: np.ravel(O.adjoint(vol, cam, r, cells=cells)))]
    full = R.fista(ops, [y], [None], vol.shape, 3)
    sub = R.fista(ops, [y], [None], vol.shape, 3, n_subset=2, n_cells=[4])
    assert np.abs(sub["x"] - full["x"]).max() > 1e-3 * np.abs(full["x"]).max()
