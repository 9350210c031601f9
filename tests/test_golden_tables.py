"""The synthetic cameras use the optics printed in the paper's camera tables
(Sec. VI); detector sizes and pitches follow the workloads and are not pinned."""
import json
import os

import numpy as np

from paper_1812_03358_b300 import inputs as I

GOLDEN = os.path.join(os.path.dirname(__file__), "golden", "camera_tables.json")


def test_plenoptic_optics_match_table():
    t = json.load(open(GOLDEN))["plenoptic"]
    cam = I.plenoptic_camera()
    assert cam.f_main == t["main_lens_focal_length"] and cam.r_main == t["main_lens_radius"]
    assert cam.d_lens_mla == t["D_mu_m"] and cam.d_mla_det == t["D_mu_d"]
    assert abs(cam.mla_radius - t["microlens_radius"]) < 1e-15
    assert sorted(set(np.unique(cam.mla_focal).tolist())) == t["microlens_focal_lengths"]


def test_single_lens_optics_match_table():
    t = json.load(open(GOLDEN))["single_lens"]
    cam = I.table_single_lens(t["detector_pixels"], t["detector_pixel_pitch"])
    assert cam.f_main == t["lens_focal_length"] and cam.r_main == t["lens_radius"]
    assert cam.d_lens_det == t["D"]
    assert cam.det_ns == 1024 and cam.det_ps == 0.005
