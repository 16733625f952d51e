"""Plain FP64 NumPy oracle for the EER -> COM-DPC / SSB phase path.

TEST INFRASTRUCTURE.  Only ``tests/``, ``__graft_entry__.smoke()`` and
``bench.py`` (CPU baseline and reference arm) may import this module.  It
shares no code, tables or helpers with the CUDA path and imports nothing from
it.  Every function is the textbook definition written out step by step, in
the paper's order and notation; numpy's FFT is used as a library primitive.

Paper: Pelz, Johnson, Ophus, Ercius, Scott, "Real-time interactive 4D-STEM
phase-contrast imaging from electron event representation data" (arXiv
2104.06336).  Readings of garbled or silent passages (the list is repeated in
the design notes of the repository):

* The set K of Sec. IV is printed with every vector as ``q``.  Read as
  K(K) = {k : |k| < k0  and  |k + K| > k0  and  |k - K| < k0}, the lune of
  A(k) and A(k - K) that excludes A(k + K).
* Eq. 3 is printed with every vector as ``q``.  Read as
  T(K) = sum_{k in K(K)} G(k, K) / (A(k) A*(k - K)).  With numpy's FFT sign
  (exp(-2 pi i)) and A = |A| exp(-i chi) the sideband is proportional to
  A*(k) A(k - K), so the correction multiplies by A(k) A*(k - K) =
  exp(-i (chi(k) - chi(k - K'))) with |A| = 1 inside the aperture.
* The aberration function is not given; Krivanek notation is used with
  omega = lambda |k| (rad): chi = 2 pi / lambda [C1 w^2/2 + (C12a (wx^2 - wy^2)
  + C12b 2 wx wy)/2 + C3 w^4/4].
* The phase image from T(K) is not given: phi = (N_R / Gbar0) Im(IFFT2(S)),
  Gbar0 = mean of G(k, 0) over bright-field pixels.
* Aperture inequalities are strict.  Mask membership is an integer decided by
  floating point, so it is evaluated in float32 with a fixed operation order
  (no fused multiply-add), the precision the kernels use; a pin checks it
  against the exact rational definition at zero rotation.
* The DPC update of Sec. V has no residual term as printed; its fixed point,
  the regularised Fourier integration, is computed in one shot.

Parity pins: every function here is checked in ``tests/test_oracle_pins.py``
against closed forms, brute force or invariants that do not reuse its code.
"""

from __future__ import annotations

import math

import numpy as np

__all__ = [
    "rle_decode", "rle_decode_fast", "virtual_detector_counts", "dpc_iterative", "pixel_table", "frame_of_events", "event_pixels", "densify", "densify_pixels", "g_column", "g_slices",
    "bin_crop_dense", "com_sums", "com_sums_dense",
    "pacbed", "pacbed_centre", "com_maps", "idpc", "g_function", "gbar0", "chi_turns",
    "kprime_f32", "kprime_f64", "trotter_mask", "ssb_spectrum", "ssb_phase", "ssb_grad",
    "variance", "ssb_value_and_grad_var", "fftfreq_index", "ssb_phase_from_events",
]

TWO_PI = 2.0 * math.pi


# --------------------------------------------------------------------------
# Pixels of the binned, cropped detector (Sec. III bin/crop; Sec. IV "centering,
# cropping and binning to a diffraction pattern size smaller than 32x32")
# --------------------------------------------------------------------------
def pixel_table(geom: dict) -> dict:
    """Binned pixels kept by the crop, numbered row-major (v outer, u inner).

    k = (u - dc_u, v - dc_v) in binned pixels.  A pixel is kept when
    |k| < crop_px (double), and is bright-field (bf) when |k|^2 < k0^2 with both
    sides in float32 (integers are exact there)."""
    pw, ph = geom["pw"], geom["ph"]
    lut = -np.ones((ph, pw), dtype=np.int64)
    us, vs = [], []
    crop2 = geom["crop_px"] * geom["crop_px"]
    for v in range(ph):
        for u in range(pw):
            kx, ky = u - geom["dc_u"], v - geom["dc_v"]
            if float(kx * kx + ky * ky) < crop2:
                lut[v, u] = len(us)
                us.append(u)
                vs.append(v)
    u = np.array(us, dtype=np.int64)
    v = np.array(vs, dtype=np.int64)
    kx = u - geom["dc_u"]
    ky = v - geom["dc_v"]
    k0sq = np.float32(geom["k0_px"] * geom["k0_px"])
    bf = (np.float32(1.0) * (kx * kx + ky * ky).astype(np.float32)) < k0sq
    return dict(u=u, v=v, kx=kx, ky=ky, bf=bf, lut=lut, P=len(us))


def frame_of_events(off: np.ndarray) -> np.ndarray:
    """Frame number of every event of a CSR event list (Fig. 1b)."""
    off = np.asarray(off, dtype=np.int64)
    return np.repeat(np.arange(len(off) - 1, dtype=np.int64), np.diff(off))


def _xy(idx, det_w):
    idx = np.asarray(idx, dtype=np.int64)
    return idx % det_w, idx // det_w


# --------------------------------------------------------------------------
# Bin + crop + densify from linear-index EER (Table 1 rows "bin", "crop";
# Sec. IV "densify the binned and cropped data")
# --------------------------------------------------------------------------
def event_pixels(idx, off, geom):
    """(p, f): the binned, cropped pixel (-1 when dropped) and the frame of
    every event.  Binned pixel u = floor((x - crop_x0) / bin), v likewise;
    events with an index >= det_w*det_h, outside the binned window or outside
    the crop are dropped."""
    pt = pixel_table(geom)
    idx = np.asarray(idx, dtype=np.int64)
    f = frame_of_events(off)
    valid = idx < geom["det_w"] * geom["det_h"]
    x, y = _xy(idx, geom["det_w"])
    u = np.floor_divide(x - geom["crop_x0"], geom["bin"])
    v = np.floor_divide(y - geom["crop_y0"], geom["bin"])
    inside = valid & (u >= 0) & (u < geom["pw"]) & (v >= 0) & (v < geom["ph"])
    p = np.full(idx.shape, -1, dtype=np.int64)
    p[inside] = pt["lut"][v[inside], u[inside]]
    return p, f


def densify(idx, off, geom) -> np.ndarray:
    """counts[p][f] = number of events of frame f whose binned, cropped pixel is p."""
    P = pixel_table(geom)["P"]
    F = len(off) - 1
    p, f = event_pixels(idx, off, geom)
    keep = p >= 0
    flat = np.bincount(p[keep] * F + f[keep], minlength=P * F)
    return flat.reshape(P, F).astype(np.int64)


def densify_pixels(idx, off, geom, pixels) -> np.ndarray:
    """The rows ``pixels`` of densify (counts[i][f] of pixel pixels[i]) without
    forming the others, for scans whose full count array does not fit."""
    pixels = np.asarray(pixels, dtype=np.int64)
    P = pixel_table(geom)["P"]
    F = len(off) - 1
    p, f = event_pixels(idx, off, geom)
    row = np.full(P + 1, -1, dtype=np.int64)
    row[pixels] = np.arange(len(pixels))
    r = row[p]  # p = -1 maps to row[-1] = -1 (dropped)
    keep = r >= 0
    flat = np.bincount(r[keep] * F + f[keep], minlength=len(pixels) * F)
    return flat.reshape(len(pixels), F).astype(np.int64)


def bin_crop_dense(cube: np.ndarray, geom) -> np.ndarray:
    """The dense-format path of Table 1: bin and crop a dense cube
    cube[f][y][x] (raw detector) into counts[p][f] by summing bin x bin blocks."""
    F = cube.shape[0]
    pt = pixel_table(geom)
    b = geom["bin"]
    out = np.zeros((pt["P"], F), dtype=cube.dtype)
    for p in range(pt["P"]):
        x0 = geom["crop_x0"] + pt["u"][p] * b
        y0 = geom["crop_y0"] + pt["v"][p] * b
        xs = slice(max(x0, 0), max(min(x0 + b, geom["det_w"]), 0))
        ys = slice(max(y0, 0), max(min(y0 + b, geom["det_h"]), 0))
        out[p] = cube[:, ys, xs].sum(axis=(1, 2))
    return out


# --------------------------------------------------------------------------
# Run-length encoding (Sec. II, Fig. 1c: only the distance between hits is kept)
# --------------------------------------------------------------------------
def rle_decode(runs, off) -> np.ndarray:
    """Linear indices from run-length-encoded frames: within each frame the
    index of hit j is the sum of runs 0..j (the first run counts from pixel
    0).  Python-int sums per frame; returned as int64."""
    runs = np.asarray(runs, dtype=np.int64)
    off = np.asarray(off, dtype=np.int64)
    out = np.empty_like(runs)
    for f in range(len(off) - 1):
        acc = 0
        for j in range(int(off[f]), int(off[f + 1])):
            acc += int(runs[j])
            out[j] = acc
    return out


def rle_decode_fast(runs, off) -> np.ndarray:
    """The same sums as rle_decode for large inputs: one cumulative sum minus
    the running total at each frame start."""
    runs = np.asarray(runs, dtype=np.int64)
    off = np.asarray(off, dtype=np.int64)
    c = np.cumsum(runs)
    before = np.concatenate(([0], c))[off[:-1]]
    return c - np.repeat(before, np.diff(off))


# --------------------------------------------------------------------------
# Centre of mass (Eq. 4; Table 1 "center of mass"; Sec. V)
# --------------------------------------------------------------------------
def com_sums(idx, off, det_w, det_h):
    """Per-frame integer sums Sx = sum x, Sy = sum y, N = count over the frame's
    events (x = idx mod W, y = idx div W); indices >= W*H are dropped."""
    idx = np.asarray(idx, dtype=np.int64)
    off = np.asarray(off, dtype=np.int64)
    valid = idx < det_w * det_h
    x, y = _xy(idx, det_w)
    x = np.where(valid, x, 0)
    y = np.where(valid, y, 0)
    n = valid.astype(np.int64)

    def seg(a):
        cs = np.zeros(len(a) + 1, dtype=np.int64)
        cs[1:] = np.cumsum(a, dtype=np.int64)
        return cs[off[1:]] - cs[off[:-1]]

    return seg(x), seg(y), seg(n)


def com_sums_dense(cube: np.ndarray):
    """Eq. 4 on a dense cube cube[f][y][x]: sums of x*I, y*I and I (int64 for an
    integer cube, float64 for expected intensities)."""
    F, H, W = cube.shape
    dt = np.int64 if np.issubdtype(cube.dtype, np.integer) else np.float64
    c = cube.astype(dt)
    xs = np.arange(W, dtype=dt)
    ys = np.arange(H, dtype=dt)
    return ((c * xs[None, None, :]).sum(axis=(1, 2)), (c * ys[None, :, None]).sum(axis=(1, 2)),
            c.sum(axis=(1, 2)))


def virtual_detector_counts(idx, off, det_w, det_h, radii, cx, cy) -> np.ndarray:
    """Virtual annular detectors (Table 1, O(C) on linear-index EER): counts
    [n_rings][F], ring j = raw pixels with radii[j]^2 <= (x-cx)^2 + (y-cy)^2
    < radii[j+1]^2 (float64 squares and sums, one rounding each)."""
    idx = np.asarray(idx, dtype=np.int64)
    F = len(off) - 1
    f = frame_of_events(off)
    ok = idx < det_w * det_h
    x, y = _xy(idx[ok], det_w)
    dx = x.astype(np.float64) - cx
    dy = y.astype(np.float64) - cy
    r2 = dx * dx + dy * dy
    edges = np.array([float(r) * float(r) for r in radii])
    ring = np.searchsorted(edges, r2, side="right") - 1
    keep = (ring >= 0) & (ring < len(radii) - 1)
    n_rings = len(radii) - 1
    flat = np.bincount(ring[keep] * F + f[ok][keep], minlength=n_rings * F)
    return flat.reshape(n_rings, F).astype(np.int64)


def pacbed(idx, det_w, det_h) -> np.ndarray:
    """Sum of all frames (Table 1 "sum all frames"): int64 histogram [H*W]."""
    idx = np.asarray(idx, dtype=np.int64)
    idx = idx[idx < det_w * det_h]
    return np.bincount(idx, minlength=det_w * det_h).astype(np.int64)


def pacbed_centre(Sx, Sy, N):
    """Centre of mass of the PACBED = total sums over all frames (raw px)."""
    tot = int(np.sum(N))
    if tot == 0:
        return 0.0, 0.0
    return int(np.sum(Sx)) / tot, int(np.sum(Sy)) / tot


def com_maps(Sx, Sy, N, cx, cy):
    """COM per frame relative to (cx, cy) in raw pixels; a frame with no events
    has COM 0."""
    Sx, Sy, N = (np.asarray(a, dtype=np.float64) for a in (Sx, Sy, N))
    with np.errstate(invalid="ignore", divide="ignore"):
        comx = np.where(N > 0, Sx / np.where(N > 0, N, 1) - cx, 0.0)
        comy = np.where(N > 0, Sy / np.where(N > 0, N, 1) - cy, 0.0)
    return comx, comy


def idpc(comx, comy, geom, lam1=0.0, lam2=0.0) -> np.ndarray:
    """Regularised Fourier integration of the COM field (Sec. V).

    The COM (raw px) is converted to a spatial frequency in 1/A by
    dalpha_raw / lambda; with C = grad(phi) / (2 pi),
    phi = IFFT[-i (Kx Cx^ + Ky Cy^) / (lam1 + K^2 + lam2 K^4)], DC set to 0,
    K from fftfreq(N, d=step_A).  Real part of the inverse transform."""
    Ny, Nx = geom["scan_ny"], geom["scan_nx"]
    s = geom["dalpha_raw_rad"] / geom["lambda_A"]
    cx = np.asarray(comx, dtype=np.float64).reshape(Ny, Nx) * s
    cy = np.asarray(comy, dtype=np.float64).reshape(Ny, Nx) * s
    Kx = np.fft.fftfreq(Nx, d=geom["step_A"])[None, :]
    Ky = np.fft.fftfreq(Ny, d=geom["step_A"])[:, None]
    K2 = Kx * Kx + Ky * Ky
    den = lam1 + K2 + lam2 * K2 * K2
    num = -1j * (Kx * np.fft.fft2(cx) + Ky * np.fft.fft2(cy))
    Phi = np.zeros((Ny, Nx), dtype=np.complex128)
    nz = den != 0
    Phi[nz] = num[nz] / den[nz]
    Phi[0, 0] = 0.0
    return np.fft.ifft2(Phi).real


def dpc_iterative(comx, comy, geom, n_iter, mu=0.5, lam1=0.0, lam2=0.0, pad=2) -> np.ndarray:
    """The gradient-descent DPC of Sec. V, step by step.  The printed update
    has no residual term; it is read as
      R = M (C - grad(phi^l) / 2 pi),
      phi^{l+1} = phi^l + mu IFFT[-i (Kx FFT(Rx) + Ky FFT(Ry)) / (lam1 + K^2 + lam2 K^4)],
    phi^0 = 0, on a periodic grid of pad x the scan with the scan in the
    top-left corner and M its indicator.  Gradients are spectral (FFT, times
    i K, inverse FFT); the DC and Nyquist bins of the update and of the
    derivative are zero.  Returns phi^{n_iter} on the scan."""
    Ny, Nx = geom["scan_ny"], geom["scan_nx"]
    My, Mx = pad * Ny, pad * Nx
    s = geom["dalpha_raw_rad"] / geom["lambda_A"]
    Cx = np.zeros((My, Mx))
    Cy = np.zeros((My, Mx))
    Cx[:Ny, :Nx] = np.asarray(comx, dtype=np.float64).reshape(Ny, Nx) * s
    Cy[:Ny, :Nx] = np.asarray(comy, dtype=np.float64).reshape(Ny, Nx) * s
    M = np.zeros((My, Mx))
    M[:Ny, :Nx] = 1.0
    Kx = np.fft.fftfreq(Mx, d=geom["step_A"])[None, :]
    Ky = np.fft.fftfreq(My, d=geom["step_A"])[:, None]
    K2 = Kx * Kx + Ky * Ky
    den = lam1 + K2 + lam2 * K2 * K2
    zero = np.zeros((My, Mx), dtype=bool)
    zero[:, Mx // 2] = True
    zero[My // 2, :] = True
    upd_zero = zero | (den == 0)
    upd_zero[0, 0] = True
    phi = np.zeros((My, Mx))
    for _ in range(n_iter):
        P = np.fft.fft2(phi)
        P[zero] = 0.0
        gx = np.fft.ifft2(1j * Kx * P).real
        gy = np.fft.ifft2(1j * Ky * P).real
        Rx = M * (Cx - gx)
        Ry = M * (Cy - gy)
        num = -1j * (Kx * np.fft.fft2(Rx) + Ky * np.fft.fft2(Ry))
        U = np.zeros((My, Mx), dtype=np.complex128)
        U[~upd_zero] = num[~upd_zero] / den[~upd_zero]
        phi = phi + mu * np.fft.ifft2(U).real
    return phi[:Ny, :Nx]


# --------------------------------------------------------------------------
# G function (Sec. IV: G(k, K) = F_{R->K} I(k, R))
# --------------------------------------------------------------------------
def g_function(counts, geom) -> np.ndarray:
    """G[p] = 2D DFT over the scan axes of counts[p] reshaped to (Ny, Nx)."""
    Ny, Nx = geom["scan_ny"], geom["scan_nx"]
    c = np.asarray(counts, dtype=np.float64).reshape(-1, Ny, Nx)
    return np.fft.fft2(c, axes=(1, 2))


def g_column(idx, off, geom, ky, kx) -> np.ndarray:
    """G(p, K) for every pixel p at the one scan frequency K = (ky, kx) (DFT
    bin indices), straight from the definition as a sum over events:
    G(p, K) = sum over events e of pixel p of exp(-2 pi i (ky y_f/Ny + kx x_f/Nx)),
    with (y_f, x_f) the raster position of the event's frame."""
    Ny, Nx = geom["scan_ny"], geom["scan_nx"]
    P = pixel_table(geom)["P"]
    p, f = event_pixels(idx, off, geom)
    keep = p >= 0
    y, x = np.divmod(f[keep], Nx)
    ph = -TWO_PI * (((ky * y) % Ny) / Ny + ((kx * x) % Nx) / Nx)
    re = np.bincount(p[keep], weights=np.cos(ph), minlength=P)
    im = np.bincount(p[keep], weights=np.sin(ph), minlength=P)
    return re + 1j * im


def g_slices(G, geom, bins) -> np.ndarray:
    """G(k, K) at the DFT bins (m_y, m_x) laid out on the binned detector
    window [n][ph][pw] (zero outside the kept pixels), the G-function view of
    Fig. 2.  G is the full [P][Ny][Nx] array of g_function."""
    pt = pixel_table(geom)
    out = np.zeros((len(bins), geom["ph"], geom["pw"]), dtype=np.complex128)
    for s, (my, mx) in enumerate(bins):
        out[s, pt["v"], pt["u"]] = G[:, my, mx]
    return out


def gbar0(G, geom) -> float:
    """Mean over bright-field pixels of G(k, K=0) (the summed BF count per pixel)."""
    bf = pixel_table(geom)["bf"]
    if not bf.any():
        return 0.0
    return float(np.mean(G[bf, 0, 0].real))


# --------------------------------------------------------------------------
# Aberrations and the trotter set
# --------------------------------------------------------------------------
def chi_turns(qx, qy, aberr, geom):
    """chi / (2 pi) at detector offset q (binned px), Krivanek notation."""
    C1, C12a, C12b, C3 = aberr[0], aberr[1], aberr[2], aberr[3]
    da, lam = geom["dalpha_rad"], geom["lambda_A"]
    wx = np.asarray(qx, dtype=np.float64) * da
    wy = np.asarray(qy, dtype=np.float64) * da
    w2 = wx * wx + wy * wy
    return (0.5 * C1 * w2 + 0.5 * (C12a * (wx * wx - wy * wy) + C12b * 2.0 * wx * wy)
            + 0.25 * C3 * w2 * w2) / lam


def fftfreq_index(N):
    """Signed frequency index of each DFT bin (numpy fftfreq order)."""
    return np.round(np.fft.fftfreq(N) * N).astype(np.int64)


def kprime_f32(geom, rot):
    """K' (binned px) of every scan bin, float32 with the fixed operation order
    Kx0 = m_x*kpm_x, Ky0 = m_y*kpm_y, Kx = c*Kx0 - s*Ky0, Ky = s*Kx0 + c*Ky0,
    c, s = float32(cos(rot)), float32(sin(rot)).  Arrays [Ny][Nx]."""
    f = np.float32
    my = fftfreq_index(geom["scan_ny"]).astype(f)[:, None]
    mx = fftfreq_index(geom["scan_nx"]).astype(f)[None, :]
    kx0 = mx * f(geom["kpm_x"])
    ky0 = my * f(geom["kpm_y"])
    kx0, ky0 = np.broadcast_arrays(kx0, ky0)
    c, s = f(math.cos(rot)), f(math.sin(rot))
    kx = (c * kx0) - (s * ky0)
    ky = (s * kx0) + (c * ky0)
    return kx.astype(f), ky.astype(f)


def kprime_f64(geom, rot):
    """K' (binned px) of every scan bin in double: R(rot) (m_x kpm_x, m_y kpm_y)."""
    my = fftfreq_index(geom["scan_ny"]).astype(np.float64)[:, None]
    mx = fftfreq_index(geom["scan_nx"]).astype(np.float64)[None, :]
    kx0 = np.broadcast_to(mx * geom["kpm_x"], (geom["scan_ny"], geom["scan_nx"]))
    ky0 = np.broadcast_to(my * geom["kpm_y"], (geom["scan_ny"], geom["scan_nx"]))
    c, s = math.cos(rot), math.sin(rot)
    return c * kx0 - s * ky0, s * kx0 + c * ky0


def trotter_mask(kx_p, ky_p, KX, KY, k0sq):
    """Membership of pixel k in K(K) for every bin (float32 evaluation):
    |k - K'|^2 < k0^2 and |k + K'|^2 > k0^2 (|k| < k0 is the caller's bf flag)."""
    f = np.float32
    dxm, dym = f(kx_p) - KX, f(ky_p) - KY
    dxp, dyp = f(kx_p) + KX, f(ky_p) + KY
    dminus = (dxm * dxm) + (dym * dym)
    dplus = (dxp * dxp) + (dyp * dyp)
    return (dminus < k0sq) & (dplus > k0sq)


# --------------------------------------------------------------------------
# SSB (Eq. 2, set K, Eq. 3) and the phase image
# --------------------------------------------------------------------------
def ssb_spectrum(G, geom, aberr, norm="none", mask_rot=None, pixels=None):
    """S(K) = sum_{p in K(K)} G(p, K) exp(-i (chi(k_p) - chi(k_p - K'))).

    norm = "none" (Eq. 3 as printed) or "area" (divide by |K(K)|, 0 when
    empty).  The mask uses rotation ``mask_rot`` (default: aberr[4]); the
    aberration phase always uses aberr[4].  ``pixels`` (default: every kept
    pixel, in order) names the kept pixel of each row of G; the sum then runs
    over the bright-field pixels among them only.  Returns S [Ny][Nx] and
    |K(K)| (both over those pixels)."""
    pt = pixel_table(geom)
    rows = np.arange(pt["P"]) if pixels is None else np.asarray(pixels, dtype=np.int64)
    rot = float(aberr[4])
    mrot = rot if mask_rot is None else float(mask_rot)
    KXf, KYf = kprime_f32(geom, mrot)
    KX, KY = kprime_f64(geom, rot)
    k0sq = np.float32(geom["k0_px"] * geom["k0_px"])
    Ny, Nx = geom["scan_ny"], geom["scan_nx"]
    S = np.zeros((Ny, Nx), dtype=np.complex128)
    nK = np.zeros((Ny, Nx), dtype=np.int64)
    for i, p in enumerate(rows):
        if not pt["bf"][p]:
            continue
        kx, ky = pt["kx"][p], pt["ky"][p]
        member = trotter_mask(kx, ky, KXf, KYf, k0sq)
        if not member.any():
            continue
        psi = TWO_PI * (chi_turns(kx, ky, aberr, geom) - chi_turns(kx - KX, ky - KY, aberr, geom))
        S += np.where(member, G[i] * np.exp(-1j * psi), 0.0)
        nK += member
    if norm == "area":
        S = np.where(nK > 0, S / np.maximum(nK, 1), 0.0)
    elif norm != "none":
        raise ValueError(norm)
    return S, nK


def ssb_phase(G, geom, aberr, norm="none", mask_rot=None):
    """phi = (N_R / Gbar0) Im(IFFT2(S)) and its population variance V."""
    S, _ = ssb_spectrum(G, geom, aberr, norm, mask_rot)
    g0 = gbar0(G, geom)
    NR = geom["scan_ny"] * geom["scan_nx"]
    scale = NR / g0 if g0 != 0 else 0.0
    phi = scale * np.fft.ifft2(S).imag
    return phi, variance(phi)


def ssb_phase_from_events(idx, off, geom, aberr, norm="none", chunk=16):
    """phi and V of ssb_phase for scans whose full G does not fit in memory:
    the bright-field pixels are taken chunk by chunk, each chunk's count rows
    densified from the events, transformed over the scan and its trotter
    terms added to S(K) (the same sums as ssb_spectrum, grouped by pixel);
    Gbar0 collects G(k, 0) of the same pixels."""
    pt = pixel_table(geom)
    Ny, Nx = geom["scan_ny"], geom["scan_nx"]
    F = Ny * Nx
    p_ev, f_ev = event_pixels(idx, off, geom)
    bf = np.flatnonzero(pt["bf"])
    S = np.zeros((Ny, Nx), dtype=np.complex128)
    nK = np.zeros((Ny, Nx), dtype=np.int64)
    g0 = 0.0
    for c0 in range(0, len(bf), chunk):
        pix = bf[c0:c0 + chunk]
        lo, hi = int(pix[0]), int(pix[-1]) + 1
        sel = (p_ev >= lo) & (p_ev < hi)
        rows = np.bincount((p_ev[sel] - lo) * F + f_ev[sel], minlength=(hi - lo) * F).reshape(hi - lo, F)
        G = g_function(rows[pix - lo], geom)
        s, n = ssb_spectrum(G, geom, aberr, "none", pixels=pix)
        S += s
        nK += n
        g0 += float(np.sum(G[:, 0, 0].real))
    if norm == "area":
        S = np.where(nK > 0, S / np.maximum(nK, 1), 0.0)
    elif norm != "none":
        raise ValueError(norm)
    gbar = g0 / len(bf) if len(bf) else 0.0
    scale = F / gbar if gbar != 0 else 0.0
    phi = scale * np.fft.ifft2(S).imag
    return phi, variance(phi)


def variance(phi) -> float:
    """V = mean((phi - mean(phi))^2) over all scan positions."""
    phi = np.asarray(phi, dtype=np.float64)
    return float(np.mean((phi - phi.mean()) ** 2))


def _dpsi(kx, ky, QX, QY, KX, KY, aberr, geom):
    """d psi / d theta for psi = 2 pi (t(k) - t(q)), q = k - K'(rot), theta =
    (C1, C12a, C12b, C3, rot).  Returns a list of five arrays."""
    da, lam = geom["dalpha_rad"], geom["lambda_A"]
    C1, C12a, C12b, C3 = aberr[0], aberr[1], aberr[2], aberr[3]
    d2 = da * da

    def parts(x, y):
        r2 = x * x + y * y
        return (d2 * r2 / (2 * lam), d2 * (x * x - y * y) / (2 * lam), d2 * x * y / lam,
                d2 * d2 * r2 * r2 / (4 * lam))

    pk = parts(float(kx), float(ky))
    pq = parts(QX, QY)
    out = [TWO_PI * (a - b) for a, b in zip(pk, pq)]
    # rotation: d t(q)/d rot = grad t(q) . dq/drot, dq/drot = -dK'/drot = -(-K'y, K'x)
    r2 = QX * QX + QY * QY
    gx = (C1 * d2 * QX + d2 * (C12a * QX + C12b * QY) + C3 * d2 * d2 * r2 * QX) / lam
    gy = (C1 * d2 * QY + d2 * (-C12a * QY + C12b * QX) + C3 * d2 * d2 * r2 * QY) / lam
    dt_drot = gx * KY + gy * (-KX)
    out.append(-TWO_PI * dt_drot)
    return out


def ssb_grad(G, geom, aberr, grad_phi, norm="none", mask_rot=None):
    """Adjoint of phi with respect to (C1, C12a, C12b, C3, rot), mask held fixed:
    dL/dtheta_j = sum_R g(R) dphi(R)/dtheta_j with
    dphi/dtheta_j = (N_R/Gbar0) Im(IFFT2(dS/dtheta_j)) and
    dS/dtheta_j = sum_{p in K} G exp(-i psi) (-i dpsi/dtheta_j)."""
    pt = pixel_table(geom)
    rot = float(aberr[4])
    mrot = rot if mask_rot is None else float(mask_rot)
    KXf, KYf = kprime_f32(geom, mrot)
    KX, KY = kprime_f64(geom, rot)
    k0sq = np.float32(geom["k0_px"] * geom["k0_px"])
    Ny, Nx = geom["scan_ny"], geom["scan_nx"]
    dS = np.zeros((5, Ny, Nx), dtype=np.complex128)
    nK = np.zeros((Ny, Nx), dtype=np.int64)
    for p in range(pt["P"]):
        if not pt["bf"][p]:
            continue
        kx, ky = pt["kx"][p], pt["ky"][p]
        member = trotter_mask(kx, ky, KXf, KYf, k0sq)
        if not member.any():
            continue
        QX, QY = kx - KX, ky - KY
        psi = TWO_PI * (chi_turns(kx, ky, aberr, geom) - chi_turns(QX, QY, aberr, geom))
        term = np.where(member, G[p] * np.exp(-1j * psi), 0.0)
        for j, d in enumerate(_dpsi(kx, ky, QX, QY, KX, KY, aberr, geom)):
            dS[j] += term * (-1j * d)
        nK += member
    if norm == "area":
        dS = np.where(nK[None] > 0, dS / np.maximum(nK, 1)[None], 0.0)
    g0 = gbar0(G, geom)
    NR = Ny * Nx
    scale = NR / g0 if g0 != 0 else 0.0
    g = np.asarray(grad_phi, dtype=np.float64).reshape(Ny, Nx)
    out = np.zeros(5)
    for j in range(5):
        dphi = scale * np.fft.ifft2(dS[j]).imag
        out[j] = float(np.sum(g * dphi))
    return out


def ssb_value_and_grad_var(G, geom, aberr, norm="none", mask_rot=None):
    """V and dV/dtheta via the chain rule dV/dphi = 2 (phi - mean phi) / N_R."""
    phi, V = ssb_phase(G, geom, aberr, norm, mask_rot)
    g = 2.0 * (phi - phi.mean()) / phi.size
    return V, ssb_grad(G, geom, aberr, g, norm, mask_rot), phi
