"""Seeded synthetic inputs shared by the CUDA path, the oracle and the benchmark.

This module holds descriptors (plain numbers), camera/volume configurations
shaped like the paper's camera tables (Sec. VI, the "simulated plenoptic camera"
and "simulated single-lens camera" tables) and the phantom / noise generators.
It deliberately contains none of the light-transport arithmetic: it neither
imports the oracle nor the CUDA binding, and both of those consume its output.

Units: millimetres and radians.  Volumes are stored x fastest: index
((iz * ny) + iy) * nx + ix, voxel (ix, iy, iz) centred at
((ix - (nx-1)/2) dx, (iy - (ny-1)/2) dy, (iz - (nz-1)/2) dz) in the object frame.
"""
from __future__ import annotations

from dataclasses import dataclass, field, replace
from typing import List, Optional

import numpy as np

CAM_SINGLE = 0
CAM_PLENOPTIC = 1
BASIS_PILLBOX = 0
BASIS_DIRAC = 1
MLA_SQUARE = 0
MLA_HEX = 1


@dataclass
class Volume:
    """Pillbox voxel grid (Sec. III, eq. voxel)."""
    nx: int
    ny: int
    nz: int
    dx: float
    dy: float
    dz: float

    @property
    def n(self) -> int:
        return self.nx * self.ny * self.nz

    @property
    def shape(self):
        return (self.nz, self.ny, self.nx)


@dataclass
class Camera:
    """One camera (Sec. II-F).  The optical axis passes through the volume
    centre; the main lens sits ``d_obj`` in front of it.  The camera is turned
    by the angles ``yaw`` (about the volume's y axis), ``pitch`` (about x) and
    ``roll`` (about z, the optical axis), radians: Theta = R_y(yaw) R_x(pitch)
    R_z(roll), p = Theta p^r (Sec. III-A)."""
    kind: int = CAM_SINGLE
    basis: int = BASIS_PILLBOX
    f_main: float = 30.0
    r_main: float = 5.0
    d_obj: float = 722.3
    yaw: float = 0.0
    pitch: float = 0.0      # rotation angle about x (not a pixel pitch)
    roll: float = 0.0
    det_ns: int = 64
    det_nt: int = 64
    det_ps: float = 0.08
    det_pt: float = 0.08
    d_lens_det: float = 31.3
    ks: int = 1
    kt: int = 1
    # plenoptic only
    d_lens_mla: float = 0.0
    d_mla_det: float = 0.0
    mla_ns: int = 0
    mla_nt: int = 0
    mla_pitch: float = 0.0
    mla_radius: float = 0.0
    mla_focal: Optional[np.ndarray] = None   # [mla_nt, mla_ns] mm
    arr_ns: int = 0
    arr_nt: int = 0
    arr_ps: float = 0.0
    arr_pt: float = 0.0
    mla_layout: int = 0                      # MLA_SQUARE or MLA_HEX
    arr_mask: Optional[np.ndarray] = None    # [arr_nt, arr_ns] transmission in [0, 1] (coded mask), None = 1

    @property
    def m(self) -> int:
        return self.det_ns * self.det_nt


def in_focus_distance(f: float, d_image: float) -> float:
    """Object distance conjugate to an image distance for a thin lens
    (the lens law; used only to place synthetic volumes in focus)."""
    return 1.0 / (1.0 / f - 1.0 / d_image)


def hex_mla_focal(mla_nt: int, mla_ns: int, focals=(2.8, 3.0, 3.2)) -> np.ndarray:
    """Three focal lengths on the hexagonal (odd rows shifted) lattice with no
    two neighbours alike: type (q - r) mod 3 of the axial coordinates
    q = col - (row - (row & 1)) / 2, r = row."""
    r, c = np.meshgrid(np.arange(mla_nt), np.arange(mla_ns), indexing="ij")
    q = c - (r - (r & 1)) // 2
    return np.asarray(focals, dtype=np.float64)[(q - r) % 3]


def hex_plenoptic_camera(n_cols: int = 40, n_rows: int = 46, n_px: int = 400, pitch_px: float = 0.02,
                         ks: int = 2, kt: int = 2) -> Camera:
    """The plenoptic camera with the paper's hexagonal three-focal MLA (rows
    pitch * sqrt(3)/2 apart, odd rows shifted by half a pitch), 200 um
    pitch, radius 100 um, over an n_px^2 detector / array plane."""
    cam = plenoptic_camera(n_lenslets=1, px_per_lenslet=n_px, pitch_px=pitch_px, ks=ks, kt=kt)
    cam.mla_ns, cam.mla_nt = n_cols, n_rows
    cam.mla_pitch, cam.mla_radius = 0.2, 0.1
    cam.mla_layout = MLA_HEX
    cam.mla_focal = hex_mla_focal(n_rows, n_cols)
    return cam


def square_mla_focal(mla_nt: int, mla_ns: int, focals=(2.8, 3.0, 3.2)) -> np.ndarray:
    """Three interleaved microlens focal lengths on a square grid:
    f[row, col] = focals[(row + col) mod 3]."""
    r, c = np.meshgrid(np.arange(mla_nt), np.arange(mla_ns), indexing="ij")
    return np.asarray(focals, dtype=np.float64)[(r + c) % 3]


# ---------------------------------------------------------------------------
# Configurations.  Geometry follows the paper's camera tables; sizes follow the
# workload descriptions (64^2 single lens at 32^3, plenoptic 1000^2 at 128^3 ...)
# ---------------------------------------------------------------------------

def config_single_small() -> (Volume, Camera):
    """Single thin-lens camera, 64x64 detector at 80 um, K = 1 pillbox,
    32^3 volume of 3.125 mm voxels (a 100 mm cube), lens of the single-lens
    table (f = 30 mm, r = 5 mm, D = 31.3 mm)."""
    vol = Volume(32, 32, 32, 3.125, 3.125, 3.125)
    cam = Camera(kind=CAM_SINGLE, f_main=30.0, r_main=5.0, d_obj=722.3,
                 det_ns=64, det_nt=64, det_ps=0.08, det_pt=0.08,
                 d_lens_det=31.3, ks=1, kt=1)
    return vol, cam


def plenoptic_camera(n_lenslets: int = 100, px_per_lenslet: int = 10,
                     pitch_px: float = 0.02, ks: int = 2, kt: int = 2) -> Camera:
    """Plenoptic camera of the simulated-plenoptic table: main lens f = 105 mm,
    r = 4.5 mm, D_mu_m = 112 mm, D_mu_d = 2.2 mm, microlens radius 100 um on a
    square 200 um grid with focal lengths 2.8/3.0/3.2 mm interleaved.  The
    array-plane grid uses the detector pitch."""
    n_px = n_lenslets * px_per_lenslet
    pitch = pitch_px * px_per_lenslet
    return Camera(kind=CAM_PLENOPTIC, f_main=105.0, r_main=4.5, d_obj=1680.0,
                  det_ns=n_px, det_nt=n_px, det_ps=pitch_px, det_pt=pitch_px,
                  d_lens_det=0.0, ks=ks, kt=kt,
                  d_lens_mla=112.0, d_mla_det=2.2,
                  mla_ns=n_lenslets, mla_nt=n_lenslets, mla_pitch=pitch,
                  mla_radius=pitch / 2.0,
                  mla_focal=square_mla_focal(n_lenslets, n_lenslets),
                  arr_ns=n_px, arr_nt=n_px, arr_ps=pitch_px, arr_pt=pitch_px)


def config_plenoptic() -> (Volume, Camera):
    """Plenoptic 100x100 lenslets x 10x10 px (1000^2 detector), K = 2x2,
    128^3 volume of 1 mm voxels."""
    return Volume(128, 128, 128, 1.0, 1.0, 1.0), plenoptic_camera()


def table_single_lens(n_px: int, pitch: float, yaw: float = 0.0,
                      ks: int = 1, kt: int = 1) -> Camera:
    """Single-lens table camera (f = 30 mm, r = 5 mm, D = 31.3 mm)."""
    return Camera(kind=CAM_SINGLE, f_main=30.0, r_main=5.0, d_obj=722.3, yaw=yaw,
                  det_ns=n_px, det_nt=n_px, det_ps=pitch, det_pt=pitch,
                  d_lens_det=31.3, ks=ks, kt=kt)


def config_multiview(seed: int = 3000, n_views: int = 4, n_px: int = 2048,
                     pitch: float = 0.005, n_lenslets: int = 200):
    """Batched multi-view workload: four single-lens cameras at seeded yaw in
    [0, 180) degrees plus one plenoptic camera, 256^3 volume at 0.5 mm."""
    rng = np.random.Generator(np.random.PCG64(seed))
    yaws = np.deg2rad(rng.uniform(0.0, 180.0, size=n_views))
    cams = [table_single_lens(n_px, pitch, float(y), 2, 2) for y in yaws]
    cams.append(plenoptic_camera(n_lenslets=n_lenslets))
    return Volume(256, 256, 256, 0.5, 0.5, 0.5), cams


def config_differentiable(n_views: int = 4, n_px: int = 1024, pitch: float = 0.01):
    """Differentiable-reconstruction workload: four single-lens 1024 x 1024
    cameras (2 x 2 cells) at yaw 0, 45, 90 and 135 degrees around a 256^3
    volume at 0.5 mm."""
    yaws = np.deg2rad(np.arange(n_views) * 180.0 / n_views)
    cams = [table_single_lens(n_px, pitch, float(y), 2, 2) for y in yaws]
    return Volume(256, 256, 256, 0.5, 0.5, 0.5), cams


def tiny_plenoptic(n_lenslets=4, px_per_lenslet=6, ks=2, kt=2) -> (Volume, Camera):
    """A plenoptic camera small enough for an explicit system matrix."""
    cam = plenoptic_camera(n_lenslets=n_lenslets, px_per_lenslet=px_per_lenslet,
                           pitch_px=0.2 / px_per_lenslet, ks=ks, kt=kt)
    return Volume(8, 8, 6, 0.9, 0.9, 4.0), cam


def tiny_hex_plenoptic(n_cols=4, n_rows=5, n_px=24, ks=2, kt=2) -> (Volume, Camera):
    """A hexagonal-MLA plenoptic camera small enough for an explicit matrix
    (n_px^2 array / detector pixels over the lattice)."""
    cam = plenoptic_camera(n_lenslets=1, px_per_lenslet=n_px, pitch_px=0.8 / n_px, ks=ks, kt=kt)
    cam.mla_ns, cam.mla_nt = n_cols, n_rows
    cam.mla_pitch, cam.mla_radius = 0.2, 0.1
    cam.mla_layout = MLA_HEX
    cam.mla_focal = hex_mla_focal(n_rows, n_cols)
    return Volume(8, 8, 6, 0.9, 0.9, 4.0), cam


# ---------------------------------------------------------------------------
# Phantoms and noise (seeded; PCG64, seed = workload index * 1000 + frame)
# ---------------------------------------------------------------------------

def _unit_grid(vol: Volume):
    z = (np.arange(vol.nz) + 0.5) / vol.nz
    y = (np.arange(vol.ny) + 0.5) / vol.ny
    x = (np.arange(vol.nx) + 0.5) / vol.nx
    return np.meshgrid(z, y, x, indexing="ij")


def gaussian_blobs(vol: Volume, seed: int = 1000, n_blobs: int = 3) -> np.ndarray:
    """Isotropic Gaussian blobs in unit-cube coordinates, centres U[0.25,0.75]^3,
    sigma U[0.05,0.15], amplitude U[0.5,1], sampled at voxel centres (float32)."""
    rng = np.random.Generator(np.random.PCG64(seed))
    Z, Y, X = _unit_grid(vol)
    out = np.zeros(vol.shape, dtype=np.float64)
    for _ in range(n_blobs):
        c = rng.uniform(0.25, 0.75, size=3)
        s = rng.uniform(0.05, 0.15)
        a = rng.uniform(0.5, 1.0)
        r2 = (X - c[0]) ** 2 + (Y - c[1]) ** 2 + (Z - c[2]) ** 2
        out += a * np.exp(-0.5 * r2 / s ** 2)
    return out.astype(np.float32)


def plume_field(vol: Volume, seed: int = 2000, n_plumes: int = 20,
                drift_voxels: float = 0.0, turbulence: float = 0.3) -> np.ndarray:
    """Elongated Gaussian plumes: axis within 20 degrees of +y, sigma_perp
    U[0.02,0.06], sigma_par U[0.1,0.3], amplitude U[0.5,1], centres U[0.2,0.8]^3,
    times i.i.d. lognormal(0, turbulence) per voxel.  ``drift_voxels`` shifts
    every plume along +y (time frames of a drifting field)."""
    rng = np.random.Generator(np.random.PCG64(seed))
    Z, Y, X = _unit_grid(vol)
    Y = Y - drift_voxels / vol.ny
    out = np.zeros(vol.shape, dtype=np.float64)
    for _ in range(n_plumes):
        c = rng.uniform(0.2, 0.8, size=3)
        tilt = np.deg2rad(rng.uniform(0.0, 20.0))
        az = rng.uniform(0.0, 2 * np.pi)
        axis = np.array([np.sin(tilt) * np.cos(az), np.cos(tilt), np.sin(tilt) * np.sin(az)])
        sp = rng.uniform(0.02, 0.06)
        sl = rng.uniform(0.1, 0.3)
        a = rng.uniform(0.5, 1.0)
        dxv, dyv, dzv = X - c[0], Y - c[1], Z - c[2]
        along = dxv * axis[0] + dyv * axis[1] + dzv * axis[2]
        perp2 = dxv ** 2 + dyv ** 2 + dzv ** 2 - along ** 2
        out += a * np.exp(-0.5 * (along ** 2 / sl ** 2 + perp2 / sp ** 2))
    noise_rng = np.random.Generator(np.random.PCG64(seed + 1))
    if turbulence > 0:
        out *= noise_rng.lognormal(0.0, turbulence, size=out.shape)
    return out.astype(np.float32)


def poisson_images(y: np.ndarray, peak_photons: float = 1e4, seed: int = 7) -> np.ndarray:
    """y_noisy = Poisson(s*y)/s with s = peak_photons / max(y)."""
    rng = np.random.Generator(np.random.PCG64(seed))
    y = np.asarray(y, dtype=np.float64)
    s = peak_photons / max(float(y.max()), 1e-30)
    return (rng.poisson(np.clip(y, 0, None) * s) / s).astype(np.float32)


def uniform_random(shape, seed: int, lo: float = 0.0, hi: float = 1.0) -> np.ndarray:
    rng = np.random.Generator(np.random.PCG64(seed))
    return rng.uniform(lo, hi, size=shape).astype(np.float32)


def plume_field_torch(vol: Volume, seed: int, n_plumes: int = 20, turbulence: float = 0.3, device="cuda",
                      drift_voxels: float = 0.0):
    """The plume distribution of ``plume_field`` evaluated on the GPU with
    torch (for generating many training volumes and full-size frames);
    parameters drawn from the same PCG64 recipe, turbulence from a seeded
    torch generator, ``drift_voxels`` as in ``plume_field``."""
    import torch
    rng = np.random.Generator(np.random.PCG64(seed))
    z = (torch.arange(vol.nz, device=device, dtype=torch.float32) + 0.5) / vol.nz
    y = (torch.arange(vol.ny, device=device, dtype=torch.float32) + 0.5) / vol.ny - drift_voxels / vol.ny
    x = (torch.arange(vol.nx, device=device, dtype=torch.float32) + 0.5) / vol.nx
    Z, Y, X = torch.meshgrid(z, y, x, indexing="ij")
    out = torch.zeros(vol.shape, device=device, dtype=torch.float32)
    for _ in range(n_plumes):
        c = rng.uniform(0.2, 0.8, size=3)
        tilt = np.deg2rad(rng.uniform(0.0, 20.0))
        az = rng.uniform(0.0, 2 * np.pi)
        axis = (float(np.sin(tilt) * np.cos(az)), float(np.cos(tilt)), float(np.sin(tilt) * np.sin(az)))
        sp = float(rng.uniform(0.02, 0.06))
        sl = float(rng.uniform(0.1, 0.3))
        a = float(rng.uniform(0.5, 1.0))
        dx, dy, dz = X - float(c[0]), Y - float(c[1]), Z - float(c[2])
        along = dx * axis[0] + dy * axis[1] + dz * axis[2]
        perp2 = dx * dx + dy * dy + dz * dz - along * along
        out += a * torch.exp(-0.5 * (along * along / (sl * sl) + perp2 / (sp * sp)))
    if turbulence > 0:
        g = torch.Generator(device=device).manual_seed(seed + 1)
        out *= torch.exp(turbulence * torch.randn(vol.shape, device=device, generator=g))
    return out.reshape(-1)


def poisson_images_torch(y, peak_photons: float = 1e4, seed: int = 7):
    """Poisson(s y)/s with s = peak_photons / max(y), on the GPU."""
    import torch
    g = torch.Generator(device=y.device).manual_seed(seed)
    s = peak_photons / max(float(y.max()), 1e-30)
    return torch.poisson(torch.clamp(y, min=0) * s, generator=g) / s
