"""Forward model (projection approximation, Eq. 1) and Poisson electron events.

For every scan position R the exit wave a(r) T(r + R) of an aperture-limited
probe a and a weak phase object T = exp(i phi) is propagated to the detector
with a 2D FFT; the normalised intensity times the dose is the mean of the
per-pixel Poisson counts.  Counts are drawn as a Poisson total per frame and a
categorical draw per electron, which has the same joint law as independent
Poisson pixels.  Each electron lands on a uniformly random raw pixel inside its
binned simulation pixel, so binning by ``bin`` recovers the simulated pixel
exactly while the stored indices are genuine ``y*det_w + x`` raw linear indices
(EER linear-index encoding, Sec. II and Fig. 1b).

With ``scan_rot`` the scan axes are rotated against the object (and the
detector, which shares the object's axes): frame (iy, ix) sits at
R = R(scan_rot) (ix, iy) * step.  The window is taken at the integer part of R
and the probe is shifted by the fractional part with a Fourier phase ramp
(exact for the aperture-limited probe), so positions need no interpolation of
the object.

The generator runs with torch on CPU or CUDA.  It is deterministic for a given
(workload, seed, device); CPU and CUDA draw different streams.  It holds no
reconstruction arithmetic.
"""

from __future__ import annotations

import math
from dataclasses import dataclass

import numpy as np
import torch

from .workloads import Workload


@dataclass
class EventData:
    idx: torch.Tensor        # int32 [C]  (raw linear index y*det_w + x, read as uint32)
    off: torch.Tensor        # int64 [F+1] CSR frame offsets
    phi_scan: torch.Tensor   # float64 [Ny][Nx] true object phase under the probe centre
    intensity: torch.Tensor | None = None  # float64 [F][sim][sim] expected counts (optional)

    @property
    def n_events(self) -> int:
        return int(self.idx.numel())

    def rle(self):
        """The same frames in run-length encoding (the format of detectors that
        store the distance between hits, Fig. 1c): hits sorted by linear index
        within each frame, each run the distance from the previous hit (the
        first run from pixel 0).  Returns (runs, off) on the events' device."""
        idx = self.idx.to(torch.int64) & 0xFFFFFFFF
        F = self.off.numel() - 1
        frame = torch.repeat_interleave(torch.arange(F, device=idx.device),
                                        self.off[1:] - self.off[:-1])
        key = frame * (1 << 32) + idx
        srt = torch.sort(key).values & 0xFFFFFFFF
        prev = torch.zeros_like(srt)
        prev[1:] = srt[:-1]
        first = torch.zeros_like(srt, dtype=torch.bool)
        starts = self.off[:-1][self.off[:-1] < self.off[1:]]
        first[starts] = True
        runs = torch.where(first, srt, srt - prev)
        return runs.to(torch.int32), self.off.clone()

    def numpy(self):
        """(idx uint32, off uint64) numpy views for the oracle."""
        idx = self.idx.cpu().numpy().view(np.uint32)
        off = self.off.cpu().numpy().view(np.uint64)
        return idx, off


def _aperture_probe(w: Workload, device, cdtype):
    """Probe in reciprocal space A(k) = [|k| < k0] exp(-i chi(k)) on the binned
    simulation grid, and its centred real-space form a(r)."""
    P = w.sim_px
    j = torch.arange(P, dtype=torch.float64, device=device) - P // 2
    ky, kx = torch.meshgrid(j, j, indexing="ij")
    ap = (kx * kx + ky * ky) < (w.k0 * w.k0)
    C1, C12a, C12b, C3, _rot = w.aberr
    wx, wy = kx * w.dalpha, ky * w.dalpha
    w2 = wx * wx + wy * wy
    chi = (2 * math.pi / w.lam) * (0.5 * C1 * w2 + 0.5 * (C12a * (wx * wx - wy * wy) + C12b * 2 * wx * wy)
                                   + 0.25 * C3 * w2 * w2)
    A = ap.to(torch.float64) * torch.exp(-1j * chi)
    a = torch.fft.fftshift(torch.fft.ifft2(torch.fft.ifftshift(A)))
    return A.to(cdtype), a.to(cdtype)


def _rotated_positions(w: Workload, fr: torch.Tensor):
    """Window corner (y, x) in object px (float64) of the frames ``fr`` of a
    rotated scan, shifted so every window lies inside the object grid."""
    c, s = math.cos(w.scan_rot), math.sin(w.scan_rot)
    y0, _y1, x0, _x1 = w.scan_corners()
    X = (fr % w.scan_nx).to(torch.float64) * w.step_px
    Y = (fr // w.scan_nx).to(torch.float64) * w.step_px
    return s * X + c * Y - y0 + 1.0, c * X - s * Y - x0 + 1.0


def _shifted_probes(A: torch.Tensor, fy: torch.Tensor, fx: torch.Tensor) -> torch.Tensor:
    """Centred real-space probes a(r - f) for fractional shifts f = (fy, fx)
    [n] in px: the spectrum times exp(-2 pi i k.f / P), k the signed
    frequency index."""
    P = A.shape[-1]
    k = torch.fft.fftfreq(P, d=1.0 / P, device=A.device, dtype=torch.float64)
    ramp = torch.exp(-2j * math.pi * (fy[:, None, None] * k[None, :, None]
                                      + fx[:, None, None] * k[None, None, :]) / P)
    A0 = torch.fft.ifftshift(A).to(torch.complex128)
    a = torch.fft.fftshift(torch.fft.ifft2(A0[None] * ramp), dim=(-2, -1))
    return a.to(A.dtype)


def _fourier_sample(phi: torch.Tensor, y: torch.Tensor, x: torch.Tensor) -> torch.Tensor:
    """phi (periodic on its grid) at real positions (y, x) by its Fourier
    series."""
    H, W = phi.shape
    Phi = torch.fft.fft2(phi) / (H * W)
    ky = torch.fft.fftfreq(H, device=phi.device, dtype=torch.float64)
    kx = torch.fft.fftfreq(W, device=phi.device, dtype=torch.float64)
    Ey = torch.exp(2j * math.pi * y[:, None] * ky[None, :])
    Ex = torch.exp(2j * math.pi * x[:, None] * kx[None, :])
    return ((Ey @ Phi) * Ex).sum(dim=1).real


def object_phase(w: Workload, gen: torch.Generator, device) -> torch.Tensor:
    """Gaussian-filtered (sigma in sim px, periodic) N(0,1) noise, zero mean,
    scaled to ``phase_std``."""
    H, W = w.obj_h, w.obj_w
    z = torch.randn((H, W), generator=gen, dtype=torch.float64, device=device)
    fy = torch.fft.fftfreq(H, device=device, dtype=torch.float64)
    fx = torch.fft.fftfreq(W, device=device, dtype=torch.float64)
    filt = torch.exp(-2 * math.pi ** 2 * w.sigma_px ** 2 * (fy[:, None] ** 2 + fx[None, :] ** 2))
    phi = torch.fft.ifft2(torch.fft.fft2(z) * filt).real
    phi = phi - phi.mean()
    s = phi.std()
    if float(s) > 0:
        phi = phi * (w.phase_std / s)
    return phi


def generate(w: Workload, device: str | torch.device = "cpu", *, seed: int | None = None,
             frames: tuple[int, int] | None = None, want_intensity: bool = False,
             phase: torch.Tensor | None = None, chunk: int | None = None) -> EventData:
    """Generate EER events for workload ``w``.

    ``frames=(f0, f1)`` restricts the output to scan positions f0..f1-1 (raster
    order f = y*Nx + x) with offsets starting at 0; the object and the random
    streams are those of the full scan, so a slice equals the same frames of the
    full generation.  ``want_intensity`` also returns the expected counts
    (dose x normalised intensity) on the binned simulation grid.
    ``phase`` replaces the random object phase (shape obj_h x obj_w)."""
    device = torch.device(device)
    seed = w.seed if seed is None else seed
    cdtype = torch.complex128 if device.type == "cpu" else torch.complex64
    gobj = torch.Generator(device=device).manual_seed(seed * 7919 + 1)
    phi = object_phase(w, gobj, device) if phase is None else phase.to(device=device, dtype=torch.float64)
    T = torch.exp(1j * phi).to(cdtype)
    A, a = _aperture_probe(w, device, cdtype)
    P, Ny, Nx, s = w.sim_px, w.scan_ny, w.scan_nx, w.step_px
    rotated = w.scan_rot != 0.0
    F = Ny * Nx
    f0, f1 = (0, F) if frames is None else frames
    if chunk is None:
        chunk = 4096 if device.type == "cpu" else max(1024, (1 << 27) // (P * P))
    # per-frame random streams are drawn per chunk of the FULL scan so that any
    # frame slice reproduces the full generation
    gcnt = torch.Generator(device=device)
    ar = torch.arange(P, device=device)
    idx_parts, n_parts, inten_parts = [], [], []
    c0 = (f0 // chunk) * chunk
    for cs in range(c0, f1, chunk):
        ce = min(cs + chunk, F)
        fr = torch.arange(cs, ce, device=device)
        if rotated:
            ry, rx = _rotated_positions(w, fr)
            iy, ix = torch.floor(ry), torch.floor(rx)
            probe = _shifted_probes(A, ry - iy, rx - ix)
            rows = iy.to(torch.int64)[:, None] + ar[None, :]
            cols = ix.to(torch.int64)[:, None] + ar[None, :]
        else:
            yy, xx = fr // Nx, fr % Nx
            rows = (yy[:, None] * s + ar[None, :])
            cols = (xx[:, None] * s + ar[None, :])
            probe = a[None]
        if w.periodic:
            rows, cols = rows % w.obj_h, cols % w.obj_w
        win = T[rows[:, :, None], cols[:, None, :]]                    # [n][P][P]
        psi = torch.fft.fftshift(torch.fft.fft2(probe * win), dim=(-2, -1))
        I = (psi.real ** 2 + psi.imag ** 2).to(torch.float64)
        I = I / I.sum(dim=(-2, -1), keepdim=True)
        gcnt.manual_seed(seed * 104729 + cs // chunk)
        n_f = torch.poisson(torch.full((ce - cs,), float(w.e_per_frame), dtype=torch.float64,
                                       device=device), generator=gcnt).to(torch.int64)
        cdf = torch.cumsum(I.reshape(ce - cs, P * P), dim=1)
        cdf = cdf / cdf[:, -1:]
        nloc = ce - cs
        fid = torch.repeat_interleave(torch.arange(nloc, device=device), n_f)
        u = torch.rand(fid.numel(), generator=gcnt, dtype=torch.float64, device=device)
        glob = (cdf + torch.arange(nloc, device=device, dtype=torch.float64)[:, None]).reshape(-1)
        pos = torch.searchsorted(glob, fid.to(torch.float64) + u, right=True)
        pix = (pos - fid * (P * P)).clamp_(0, P * P - 1)
        jy, jx = pix // P, pix % P
        sub = torch.randint(0, w.bin, (2, fid.numel()), generator=gcnt, device=device)
        rx = w.crop_x0 + jx * w.bin + sub[0]
        ry = w.crop_y0 + jy * w.bin + sub[1]
        lin = (ry * w.det_w + rx).to(torch.int32)
        # keep only frames inside [f0, f1)
        lo, hi = max(f0, cs) - cs, min(f1, ce) - cs
        if lo > 0 or hi < nloc:
            ends = torch.cumsum(n_f, 0)
            starts = ends - n_f
            e_lo = int(starts[lo]) if lo < nloc else int(ends[-1])
            e_hi = int(ends[hi - 1]) if hi > 0 else 0
            lin = lin[e_lo:e_hi]
            n_f = n_f[lo:hi]
            I = I[lo:hi]
        idx_parts.append(lin)
        n_parts.append(n_f)
        if want_intensity:
            inten_parts.append(I * float(w.e_per_frame))
    idx = torch.cat(idx_parts) if idx_parts else torch.zeros(0, dtype=torch.int32, device=device)
    n_all = torch.cat(n_parts) if n_parts else torch.zeros(0, dtype=torch.int64, device=device)
    off = torch.zeros(n_all.numel() + 1, dtype=torch.int64, device=device)
    off[1:] = torch.cumsum(n_all, 0)
    c = P // 2
    if rotated:
        ry, rx = _rotated_positions(w, torch.arange(F, device=device))
        phi_scan = _fourier_sample(phi, ry + c, rx + c).reshape(Ny, Nx)
    else:
        gy = (torch.arange(Ny, device=device) * s + c) % w.obj_h
        gx = (torch.arange(Nx, device=device) * s + c) % w.obj_w
        phi_scan = phi[gy[:, None], gx[None, :]]
    inten = torch.cat(inten_parts) if want_intensity else None
    return EventData(idx=idx, off=off, phi_scan=phi_scan, intensity=inten)
