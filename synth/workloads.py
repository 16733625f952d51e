"""Workload recipes shaped like the paper's 4D Camera experiments.

The paper's data (4D Camera, 87 kHz, 576x576 pixels; 1024x1024 scans cropped to
less than 32x32 detector pixels for SSB, Sec. IV) is not available, so every
workload is synthetic: a weak phase object, an aperture-limited probe and
Poisson electron counts stored as linear-index EER (Sec. II, Fig. 1b).

Units: lengths in Angstrom, angles in radians.  ``k`` coordinates are binned
detector pixels measured from the optical axis.

Geometry conventions (the paper is silent on them; these are the readings the
whole repository uses):

* The simulation grid is the binned detector grid: ``sim_px`` binned pixels of
  ``dalpha = bin * dalpha_raw`` each.  Its real-space pixel is
  ``dx = lambda / (sim_px * dalpha)``.
* A scan step of ``step_px`` simulation pixels maps scan frequency index ``m``
  (numpy ``fftfreq`` order) to ``K' = m * kpm`` binned pixels with
  ``kpm = sim_px / (N * step_px)``.
* The optical axis sits at binned pixel ``sim_px // 2``; the crop origin
  ``crop_x0/crop_y0`` is the raw pixel where binned pixel 0 starts.
"""

from __future__ import annotations

import math
from dataclasses import dataclass, field, replace

import numpy as np

LAMBDA_300KV_A = 0.019687  # electron wavelength at 300 keV (Angstrom)


@dataclass(frozen=True)
class Workload:
    name: str
    seed: int
    det_w: int
    det_h: int
    dalpha_raw: float          # raw detector pixel (rad)
    bin: int                   # binning factor b
    sim_px: int                # binned simulation grid (pixels per side)
    alpha: float               # convergence semi-angle (rad)
    lam: float                 # wavelength (Angstrom)
    scan_ny: int
    scan_nx: int
    step_px: int               # scan step in simulation pixels
    e_per_frame: float         # mean electrons per frame (Poisson)
    obj_h: int
    obj_w: int
    phase_std: float = 0.1     # object phase standard deviation (rad)
    sigma_px: float = 1.0      # Gaussian filter of the object phase (sim px)
    crop_margin: float = 0.0   # crop radius = k0 + margin (binned px)
    aberr: tuple = (0.0, 0.0, 0.0, 0.0, 0.0)  # C1, C12a, C12b, C3 (A), rot (rad)
    periodic: bool = False     # object periodic over the scan (N*step)
    scan_rot: float = 0.0      # scan axes rotated by this angle (rad, counter-clockwise in the
                               # detector's (x, y)) against the object and detector axes

    # derived quantities -------------------------------------------------
    @property
    def dalpha(self) -> float:
        return self.bin * self.dalpha_raw

    @property
    def k0(self) -> float:
        return self.alpha / self.dalpha

    @property
    def dx(self) -> float:
        return self.lam / (self.sim_px * self.dalpha)

    @property
    def step_A(self) -> float:
        return self.step_px * self.dx

    @property
    def n_frames(self) -> int:
        return self.scan_ny * self.scan_nx

    def scan_corners(self):
        """Offsets (y, x) in sim px of the scan's extreme positions: frame (iy, ix)
        sits at R = R(scan_rot) (ix step, iy step), R(t) = [[cos t, -sin t],
        [sin t, cos t]] acting on (x, y)."""
        c, s = math.cos(self.scan_rot), math.sin(self.scan_rot)
        X = (self.scan_nx - 1) * self.step_px
        Y = (self.scan_ny - 1) * self.step_px
        pts = [(0.0, 0.0), (X, 0.0), (0.0, Y), (X, Y)]
        xs = [c * x - s * y for x, y in pts]
        ys = [s * x + c * y for x, y in pts]
        return min(ys), max(ys), min(xs), max(xs)

    @property
    def crop_x0(self) -> int:
        # binned pixel sim_px//2 holds the optical axis at raw pixel det_w//2
        return self.det_w // 2 - self.bin * (self.sim_px // 2)

    @property
    def crop_y0(self) -> int:
        return self.det_h // 2 - self.bin * (self.sim_px // 2)


def _obj(n, step, sim):
    return (n - 1) * step + sim


_BASE = dict(lam=LAMBDA_300KV_A)


def workload(cfg: int, **over) -> Workload:
    """The five workloads (1 tiny, 2 precision, 3 differentiation, 4 batching,
    5 full scale), with their seeds 0..4.  Keyword overrides return a variant
    (e.g. a smaller scan for a quick parity case)."""
    if cfg == 1:
        w = Workload(name="tiny-32x32-det64", seed=0, det_w=64, det_h=64, dalpha_raw=1e-3,
                     bin=1, sim_px=64, alpha=20e-3, scan_ny=32, scan_nx=32, step_px=1,
                     e_per_frame=30.0, obj_h=96, obj_w=96, **_BASE)
    elif cfg == 2:
        w = Workload(name="precision-256x256-det576-bin4", seed=1, det_w=576, det_h=576,
                     dalpha_raw=0.25e-3, bin=4, sim_px=144, alpha=20e-3, scan_ny=256,
                     scan_nx=256, step_px=2, e_per_frame=20.0,
                     obj_h=_obj(256, 2, 144), obj_w=_obj(256, 2, 144), **_BASE)
    elif cfg == 3:
        c12, az = 30.0, math.radians(30.0)
        w = Workload(name="differentiation-512x512-det576-bin4", seed=2, det_w=576, det_h=576,
                     dalpha_raw=0.25e-3, bin=4, sim_px=144, alpha=25e-3, scan_ny=512,
                     scan_nx=512, step_px=2, e_per_frame=40.0,
                     obj_h=_obj(512, 2, 144), obj_w=_obj(512, 2, 144),
                     aberr=(80.0, c12 * math.cos(2 * az), c12 * math.sin(2 * az), 1.0e4, 0.0),
                     **_BASE)
    elif cfg == 4:
        w = Workload(name="batching-512x512-det576-bin4", seed=3, det_w=576, det_h=576,
                     dalpha_raw=0.25e-3, bin=4, sim_px=144, alpha=20e-3, scan_ny=512,
                     scan_nx=512, step_px=2, e_per_frame=30.0,
                     obj_h=_obj(512, 2, 144), obj_w=_obj(512, 2, 144), **_BASE)
    elif cfg == 5:
        w = Workload(name="full-1024x1024-det576-bin6", seed=4, det_w=576, det_h=576,
                     dalpha_raw=0.25e-3, bin=6, sim_px=96, alpha=20e-3, scan_ny=1024,
                     scan_nx=1024, step_px=2, e_per_frame=50.0,
                     obj_h=_obj(1024, 2, 96), obj_w=_obj(1024, 2, 96), **_BASE)
    else:
        raise ValueError(f"unknown workload {cfg}")
    user_obj = "obj_h" in over
    if over:
        if ("scan_ny" in over or "scan_nx" in over or "step_px" in over) and "obj_h" not in over:
            ny = over.get("scan_ny", w.scan_ny)
            nx = over.get("scan_nx", w.scan_nx)
            st = over.get("step_px", w.step_px)
            over = dict(over, obj_h=_obj(ny, st, w.sim_px), obj_w=_obj(nx, st, w.sim_px))
        w = replace(w, **over)
    if w.periodic:
        if w.scan_rot != 0.0:
            raise ValueError("a rotated scan does not tile a periodic object")
        w = replace(w, obj_h=w.scan_ny * w.step_px, obj_w=w.scan_nx * w.step_px)
    elif w.scan_rot != 0.0 and not user_obj:
        y0, y1, x0, x1 = w.scan_corners()
        w = replace(w, obj_h=int(math.ceil(y1 - y0)) + w.sim_px + 2,
                    obj_w=int(math.ceil(x1 - x0)) + w.sim_px + 2)
    return w


def geometry(w: Workload) -> dict:
    """Plan geometry in the field names of ``eer4d_geom`` (include/eer4d.h).

    ``kpm`` is the exact rational sim_px/(N*step_px) evaluated in double;
    ``k0`` is alpha/dalpha in double.  Both the oracle and the CUDA plan take
    these numbers as given."""
    return dict(
        det_w=w.det_w, det_h=w.det_h, bin=w.bin,
        crop_x0=w.crop_x0, crop_y0=w.crop_y0,
        pw=w.sim_px, ph=w.sim_px, dc_u=w.sim_px // 2, dc_v=w.sim_px // 2,
        k0_px=w.k0, crop_px=w.k0 + w.crop_margin,
        scan_ny=w.scan_ny, scan_nx=w.scan_nx,
        kpm_y=w.sim_px / (w.scan_ny * w.step_px), kpm_x=w.sim_px / (w.scan_nx * w.step_px),
        lambda_A=w.lam, dalpha_rad=w.dalpha, step_A=w.step_A, dalpha_raw_rad=w.dalpha_raw,
    )


def batching_datasets(seed: int = 3, n: int = 16):
    """Uneven scans for the batching workload: N_i = 16*round(exp(U(ln64, ln512))/16),
    electrons per frame e_i ~ U{10..50}."""
    rng = np.random.default_rng(seed)
    out = []
    for i in range(n):
        N = int(16 * round(math.exp(rng.uniform(math.log(64), math.log(512))) / 16))
        e = int(rng.integers(10, 51))
        out.append(workload(4, scan_ny=N, scan_nx=N, e_per_frame=float(e), seed=1000 * seed + i,
                            name=f"batch{i}-{N}x{N}"))
    return out


def candidate_aberrations(seed: int = 3, n: int = 64) -> np.ndarray:
    """Random aberration candidates: C1 ~ U(-20, 20) nm, C12a, C12b ~ U(-5, 5) nm,
    C3 = 0, rot = 0.  Returns float64 [n][5] in Angstrom/rad."""
    rng = np.random.default_rng(seed + 7)
    out = np.zeros((n, 5))
    out[:, 0] = rng.uniform(-200.0, 200.0, n)
    out[:, 1] = rng.uniform(-50.0, 50.0, n)
    out[:, 2] = rng.uniform(-50.0, 50.0, n)
    return out
