"""Pins of the FP64 oracle against what the paper and the mathematics fix.

None of these tests reuses the oracle's own formula to check itself: each one
compares against a closed form, a brute-force sum, an invariant, a
hand-derived worked example or the physics of the forward model (Eq. 1).
"""

import json
import math
import os

import numpy as np
import pytest
import torch

import oracle as orc
import synth

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


def _dense_cube(idx, off, W, H, dtype=np.int64):
    F = len(off) - 1
    f = np.repeat(np.arange(F), np.diff(off.astype(np.int64)))
    i = idx.astype(np.int64)
    ok = i < W * H
    flat = np.bincount(f[ok] * (W * H) + i[ok], minlength=F * W * H)
    return flat.reshape(F, H, W).astype(dtype)


# ---------------------------------------------------------------- golden ---
def test_golden_tiny_worked_example():
    g = json.load(open(os.path.join(GOLDEN, "tiny_eer.json")))
    idx = np.array(g["idx"], dtype=np.uint32)
    off = np.array(g["off"], dtype=np.uint64)
    W, H = g["det_w"], g["det_h"]
    e = g["expect"]
    Sx, Sy, N = orc.com_sums(idx, off, W, H)
    assert Sx.tolist() == e["Sx"] and Sy.tolist() == e["Sy"] and N.tolist() == e["N"]
    pac = orc.pacbed(idx, W, H)
    assert {str(k): int(v) for k, v in enumerate(pac) if v} == e["pacbed_nonzero"]
    assert orc.pacbed_centre(Sx, Sy, N) == tuple(e["centre"])
    geom = dict(g["geom"], det_w=W, det_h=H, scan_ny=2, scan_nx=2)
    pt = orc.pixel_table(geom)
    assert pt["P"] == e["P"]
    assert [[int(u), int(v)] for u, v in zip(pt["u"], pt["v"])] == e["pixel_uv"]
    assert orc.densify(idx, off, geom).tolist() == e["counts"]


# ------------------------------------------------ events vs dense format ---
@pytest.mark.parametrize("cfg,over", [(1, {}), (2, dict(scan_ny=8, scan_nx=8))])
def test_events_equal_dense_format(cfg, over):
    """Table 1: the linear-index path and the dense path give the same binned,
    cropped counts and the same COM sums, exactly."""
    w = synth.workload(cfg, **over)
    d = synth.generate(w)
    idx, off = d.numpy()
    geom = synth.geometry(w)
    cube = _dense_cube(idx, off, w.det_w, w.det_h, np.int32)
    c_ev = orc.densify(idx, off, geom)
    c_de = orc.bin_crop_dense(cube, geom)
    assert c_ev.sum() > 0
    np.testing.assert_array_equal(c_ev, c_de)
    for a, b in zip(orc.com_sums(idx, off, w.det_w, w.det_h), orc.com_sums_dense(cube)):
        np.testing.assert_array_equal(a, b)
    # G from events equals G from the dense path bit for bit (same FP64 ops)
    if cfg == 1:
        np.testing.assert_array_equal(orc.g_function(c_ev, geom), orc.g_function(c_de, geom))


# ------------------------------------------------------------------- FFT ---
def test_g_function_brute_force_dft_8x8():
    rng = np.random.default_rng(0)
    counts = rng.integers(0, 5, size=(3, 64)).astype(np.float64)
    geom = dict(scan_ny=8, scan_nx=8)
    G = orc.g_function(counts, geom)
    ref = np.zeros((3, 8, 8), dtype=np.complex128)
    c = counts.reshape(3, 8, 8)
    for ky in range(8):
        for kx in range(8):
            for y in range(8):
                for x in range(8):
                    ref[:, ky, kx] += c[:, y, x] * complex(math.cos(2 * math.pi * (ky * y + kx * x) / 8),
                                                           -math.sin(2 * math.pi * (ky * y + kx * x) / 8))
    assert np.abs(G - ref).max() <= 1e-12 * np.abs(ref).max()


def test_g_function_parseval_rectangular():
    rng = np.random.default_rng(1)
    counts = rng.poisson(0.3, size=(5, 24 * 40)).astype(np.float64)
    G = orc.g_function(counts, dict(scan_ny=24, scan_nx=40))
    lhs = (np.abs(G) ** 2).sum(axis=(1, 2))
    rhs = 24 * 40 * (counts ** 2).sum(axis=1)
    np.testing.assert_allclose(lhs, rhs, rtol=1e-12)


def test_densify_pixels_are_rows_of_the_dense_path():
    """The sampled-pixel densify equals the dense-format binning (Table 1) on
    the chosen rows, including the first and last pixel and repeats of none."""
    w = synth.workload(1)
    d = synth.generate(w)
    idx, off = d.numpy()
    geom = synth.geometry(w)
    cube = _dense_cube(idx, off, w.det_w, w.det_h, np.int32)
    dense = orc.bin_crop_dense(cube, geom)
    P = dense.shape[0]
    sel = np.array([0, 7, P // 2, P - 2, P - 1])
    np.testing.assert_array_equal(orc.densify_pixels(idx, off, geom, sel), dense[sel])


def test_g_column_equals_brute_force_sum():
    """G(p, K) at single scan frequencies from the event sum equals the DFT
    written as an explicit sum over scan positions of the dense-path counts."""
    w = synth.workload(1)
    d = synth.generate(w)
    idx, off = d.numpy()
    geom = synth.geometry(w)
    Ny, Nx = w.scan_ny, w.scan_nx
    dense = orc.bin_crop_dense(_dense_cube(idx, off, w.det_w, w.det_h, np.int32), geom)
    c = dense.reshape(-1, Ny, Nx).astype(np.float64)
    y = np.arange(Ny)[:, None]
    x = np.arange(Nx)[None, :]
    for ky, kx in [(0, 0), (1, 0), (0, 3), (5, 7), (Ny // 2, Nx // 2), (Ny - 1, 1)]:
        e = np.cos(2 * math.pi * (ky * y / Ny + kx * x / Nx)) - 1j * np.sin(2 * math.pi * (ky * y / Ny + kx * x / Nx))
        ref = (c * e[None]).sum(axis=(1, 2))
        got = orc.g_column(idx, off, geom, ky, kx)
        assert np.abs(got - ref).max() <= 1e-11 * max(1.0, np.abs(ref).max())


def test_rle_decode_golden_frames():
    """Hand-worked frames of run-length encoding (Fig. 1c), including an
    empty frame, a hit at pixel 0, a repeated hit and a hit at the last pixel
    of a 576x576 detector."""
    g = json.load(open(os.path.join(GOLDEN, "rle_frames.json")))
    runs = [r for fr in g["frames"] for r in fr["runs"]]
    off = np.cumsum([0] + [len(fr["runs"]) for fr in g["frames"]])
    hits = [h for fr in g["frames"] for h in fr["hits"]]
    assert orc.rle_decode(runs, off).tolist() == hits
    assert orc.rle_decode_fast(runs, off).tolist() == hits


def test_rle_round_trip_of_generated_frames():
    """Decoding the generator's run-length form returns each frame's hits in
    ascending order (the multiset of the linear-index frame)."""
    w = synth.workload(1)
    d = synth.generate(w)
    idx, off = d.numpy()
    runs, roff = d.rle()
    dec = orc.rle_decode_fast(runs.numpy().view(np.uint32), roff.numpy())
    o = off.astype(np.int64)
    for f in range(len(o) - 1):
        np.testing.assert_array_equal(dec[o[f]:o[f + 1]], np.sort(idx[o[f]:o[f + 1]].astype(np.int64)))
    small = slice(0, int(o[40]))
    np.testing.assert_array_equal(orc.rle_decode(runs.numpy()[small].view(np.uint32), roff.numpy()[:41]),
                                  dec[small])


def test_virtual_detectors_equal_dense_masks():
    """Annular virtual detectors from events equal the dense-format sums over
    boolean ring masks built pixel by pixel with Python floats; rings that
    cover the whole detector add up to the frame's event count."""
    w = synth.workload(1)
    d = synth.generate(w)
    idx, off = d.numpy()
    cube = _dense_cube(idx, off, w.det_w, w.det_h)
    Sx, Sy, N = orc.com_sums(idx, off, w.det_w, w.det_h)
    cx, cy = orc.pacbed_centre(Sx, Sy, N)
    radii = [0.0, 5.0, 12.5, 20.0, 31.0, 100.0]
    got = orc.virtual_detector_counts(idx, off, w.det_w, w.det_h, radii, cx, cy)
    ring = np.full((w.det_h, w.det_w), -1)
    for yy in range(w.det_h):
        for xx in range(w.det_w):
            r2 = (xx - cx) * (xx - cx) + (yy - cy) * (yy - cy)
            for j in range(len(radii) - 1):
                if radii[j] * radii[j] <= r2 < radii[j + 1] * radii[j + 1]:
                    ring[yy, xx] = j
    for j in range(len(radii) - 1):
        np.testing.assert_array_equal(got[j], cube[:, ring == j].sum(axis=1))
    np.testing.assert_array_equal(got.sum(axis=0), N)  # 100 px covers the 64x64 detector


def test_g_slices_place_event_sums_on_the_detector():
    """The G-function view at nine bins (DC, positive, negative, Nyquist) equals
    the event-sum DFT of each kept pixel written at its detector position."""
    w = synth.workload(1)
    d = synth.generate(w)
    idx, off = d.numpy()
    geom = synth.geometry(w)
    G = orc.g_function(orc.densify(idx, off, geom), geom)
    Ny, Nx = w.scan_ny, w.scan_nx
    bins = [(0, 0), (1, 0), (0, 1), (3, 5), (Ny - 3, Nx - 5), (Ny // 2, 0), (0, Nx // 2),
            (Ny - 1, 2), (7, Nx - 1)]
    got = orc.g_slices(G, geom, bins)
    pt = orc.pixel_table(geom)
    for s, (my, mx) in enumerate(bins):
        col = orc.g_column(idx, off, geom, my, mx)
        ref = np.zeros((geom["ph"], geom["pw"]), dtype=np.complex128)
        for p in range(pt["P"]):
            ref[pt["v"][p], pt["u"][p]] = col[p]
        assert np.abs(got[s] - ref).max() <= 1e-10 * max(1.0, np.abs(ref).max())


# ------------------------------------------------------------------- COM ---
@pytest.mark.parametrize("g", [(3, -2), (0, 5), (-4, -4)])
def test_com_of_phase_ramp_is_its_tilt(g):
    """A phase ramp exp(2 pi i g.r / P) shifts the diffraction pattern by g
    pixels, so Eq. 4 on the noise-free intensity moves by exactly g."""
    w = synth.workload(1, scan_ny=4, scan_nx=4)
    yy, xx = np.mgrid[0:w.obj_h, 0:w.obj_w]
    ramp = 2 * math.pi * (g[0] * xx + g[1] * yy) / w.sim_px
    d0 = synth.generate(w, want_intensity=True, phase=torch.zeros(w.obj_h, w.obj_w))
    d1 = synth.generate(w, want_intensity=True, phase=torch.from_numpy(ramp))
    I0 = d0.intensity.numpy()
    I1 = d1.intensity.numpy()
    sx0, sy0, n0 = orc.com_sums_dense(I0)
    sx1, sy1, n1 = orc.com_sums_dense(I1)
    c0 = orc.com_maps(sx0, sy0, n0, 0.0, 0.0)
    c1 = orc.com_maps(sx1, sy1, n1, 0.0, 0.0)
    np.testing.assert_allclose(c1[0] - c0[0], g[0], atol=1e-11)
    np.testing.assert_allclose(c1[1] - c0[1], g[1], atol=1e-11)
    # on Poisson events the mean COM shift agrees within 4 standard errors
    idx, off = d1.numpy()
    sx, sy, n = orc.com_sums(idx, off, w.det_w, w.det_h)
    ev = np.concatenate([idx.astype(np.int64) % w.det_w])
    cx, cy = orc.com_maps(sx, sy, n, 0.0, 0.0)
    se = np.std(ev) / math.sqrt(len(ev))
    assert abs(np.mean(sx.sum() / n.sum()) - (c0[0][0] + g[0])) < 4 * se + 1e-9


def test_com_empty_frames_are_zero():
    idx = np.array([5, 6], dtype=np.uint32)
    off = np.array([0, 0, 2, 2], dtype=np.uint64)
    sx, sy, n = orc.com_sums(idx, off, 4, 4)
    cx, cy = orc.com_maps(sx, sy, n, 1.0, 1.0)
    assert n.tolist() == [0, 2, 0]
    assert cx.tolist() == [0.0, 0.5, 0.0] and cy.tolist() == [0.0, 0.0, 0.0]


# ------------------------------------------------------------------ iDPC ---
def test_idpc_recovers_band_limited_phase():
    """C = grad(phi) / 2 pi in closed form (sums of sinusoids with integer
    wave numbers): Fourier integration returns phi - mean(phi) to 1e-10."""
    w = synth.workload(1, scan_ny=24, scan_nx=40)
    geom = synth.geometry(w)
    Ny, Nx, st = w.scan_ny, w.scan_nx, w.step_A
    Y, X = np.mgrid[0:Ny, 0:Nx].astype(np.float64)
    rng = np.random.default_rng(2)
    phi = np.zeros((Ny, Nx))
    gx = np.zeros((Ny, Nx))
    gy = np.zeros((Ny, Nx))
    for _ in range(12):
        nx, ny = int(rng.integers(-Nx // 2 + 1, Nx // 2)), int(rng.integers(-Ny // 2 + 1, Ny // 2))
        a, c = rng.normal(), rng.uniform(0, 2 * math.pi)
        arg = 2 * math.pi * (nx * X / Nx + ny * Y / Ny) + c
        phi += a * np.cos(arg)
        gx += -a * np.sin(arg) * 2 * math.pi * nx / (Nx * st)
        gy += -a * np.sin(arg) * 2 * math.pi * ny / (Ny * st)
    s = w.lam / w.dalpha_raw  # 1/A -> raw px
    comx = gx / (2 * math.pi) * s
    comy = gy / (2 * math.pi) * s
    out = orc.idpc(comx.ravel(), comy.ravel(), geom)
    np.testing.assert_allclose(out, phi - phi.mean(), atol=1e-10 * np.abs(phi).max())


def _band_limited_com(Ny, Nx, st, w, seed=2, terms=12):
    Y, X = np.mgrid[0:Ny, 0:Nx].astype(np.float64)
    rng = np.random.default_rng(seed)
    phi = np.zeros((Ny, Nx))
    gx = np.zeros((Ny, Nx))
    gy = np.zeros((Ny, Nx))
    for _ in range(terms):
        nx, ny = int(rng.integers(-Nx // 2 + 1, Nx // 2)), int(rng.integers(-Ny // 2 + 1, Ny // 2))
        a, c = rng.normal(), rng.uniform(0, 2 * math.pi)
        arg = 2 * math.pi * (nx * X / Nx + ny * Y / Ny) + c
        phi += a * np.cos(arg)
        gx += -a * np.sin(arg) * 2 * math.pi * nx / (Nx * st)
        gy += -a * np.sin(arg) * 2 * math.pi * ny / (Ny * st)
    s = w.lam / w.dalpha_raw
    return phi, gx / (2 * math.pi) * s, gy / (2 * math.pi) * s


def test_iterative_dpc_geometric_convergence():
    """Without padding and regularisation each step removes the fraction mu
    of the remaining error at every frequency: after L steps the literal
    iteration equals (1 - (1 - mu)^L) (phi - mean phi), to 1e-10."""
    w = synth.workload(1, scan_ny=24, scan_nx=40)
    geom = synth.geometry(w)
    phi, comx, comy = _band_limited_com(24, 40, w.step_A, w)
    for L, mu in [(1, 0.5), (5, 0.5), (3, 1.0), (20, 0.3)]:
        out = orc.dpc_iterative(comx.ravel(), comy.ravel(), geom, L, mu=mu, pad=1)
        ref = (1 - (1 - mu) ** L) * (phi - phi.mean())
        np.testing.assert_allclose(out, ref, atol=1e-10 * np.abs(phi).max())


def test_iterative_dpc_regularised_per_frequency_factor():
    """With lam1 > 0 the preconditioner 1/(lam1 + K^2) scales the step per
    frequency: phi_L(K) = phi(K) (1 - (1 - mu K^2/(lam1 + K^2))^L), the
    closed form of the linear recursion, to 1e-10."""
    w = synth.workload(1, scan_ny=24, scan_nx=40)
    geom = synth.geometry(w)
    phi, comx, comy = _band_limited_com(24, 40, w.step_A, w, seed=5)
    lam1, mu, L = 0.5, 0.5, 7
    out = orc.dpc_iterative(comx.ravel(), comy.ravel(), geom, L, mu=mu, lam1=lam1, pad=1)
    Kx = np.fft.fftfreq(40, d=w.step_A)[None, :]
    Ky = np.fft.fftfreq(24, d=w.step_A)[:, None]
    K2 = Kx * Kx + Ky * Ky
    fac = np.zeros_like(K2)
    nz = K2 > 0
    fac[nz] = 1 - (1 - mu * K2[nz] / (lam1 + K2[nz])) ** L
    ref = np.fft.ifft2(np.fft.fft2(phi) * fac).real
    np.testing.assert_allclose(out, ref, atol=1e-10 * np.abs(phi).max())


def test_iterative_dpc_padding_removes_wraparound():
    """A tilted, non-periodic phase: the one-shot periodic integration cannot
    represent the tilt, the zero-padded iteration with the residual on the
    scan only does much better (error relative to phi - mean over the scan)."""
    w = synth.workload(1, scan_ny=32, scan_nx=32)
    geom = synth.geometry(w)
    st = w.step_A
    Y, X = np.mgrid[0:32, 0:32].astype(np.float64)
    tilt = 0.15
    bump = np.exp(-((X - 12.0) ** 2 + (Y - 20.0) ** 2) / (2 * 4.0 ** 2))
    phi = tilt * X + 2.0 * bump
    gx = (tilt + 2.0 * bump * (-(X - 12.0) / 4.0 ** 2)) / st
    gy = (2.0 * bump * (-(Y - 20.0) / 4.0 ** 2)) / st
    s = w.lam / w.dalpha_raw
    comx, comy = gx / (2 * math.pi) * s, gy / (2 * math.pi) * s
    ref = phi - phi.mean()

    def err(a):
        a = a - a.mean()
        return np.linalg.norm(a - ref) / np.linalg.norm(ref)

    e_closed = err(orc.idpc(comx.ravel(), comy.ravel(), geom))
    e_iter = err(orc.dpc_iterative(comx.ravel(), comy.ravel(), geom, 100, mu=0.5, pad=2))
    assert e_iter < 0.02 and e_closed > 0.5, (e_iter, e_closed)


def test_idpc_sign_from_forward_model():
    """COM of the simulated diffraction patterns of a smooth weak phase object,
    integrated, correlates positively with the object phase."""
    w = synth.workload(1, periodic=True, sigma_px=2.0, phase_std=0.05)
    d = synth.generate(w, want_intensity=True)
    geom = synth.geometry(w)
    sx, sy, n = orc.com_sums_dense(d.intensity.numpy())
    cx, cy = orc.pacbed_centre(sx, sy, n)
    comx, comy = orc.com_maps(sx, sy, n, cx, cy)
    phi = orc.idpc(comx, comy, geom)
    truth = d.phi_scan.numpy()
    r = np.corrcoef(phi.ravel(), truth.ravel())[0, 1]
    assert r > 0.9


# -------------------------------------------------------------- trotter ---
def _exact_mask(kx, ky, m_y, m_x, kpm_num_y, kpm_num_x, kpm_den, k0_num, k0_den):
    """Exact rational membership in K(K) at zero rotation: K' = m*num/den."""
    D = kpm_den * k0_den
    ax = kx * D - k0_den * kpm_num_x * m_x
    ay = ky * D - k0_den * kpm_num_y * m_y
    bx = kx * D + k0_den * kpm_num_x * m_x
    by = ky * D + k0_den * kpm_num_y * m_y
    r2 = (k0_num * kpm_den) ** 2
    return (ax * ax + ay * ay < r2) & (bx * bx + by * by > r2)


@pytest.mark.parametrize("cfg,over,kpm,k0", [
    (1, {}, ((2, 2), 1), (20, 1)),
    (2, {}, ((9, 9), 32), (20, 1)),
    (5, dict(scan_ny=1024, scan_nx=1024), ((3, 3), 64), (40, 3)),
    (2, dict(scan_ny=64, scan_nx=128), ((36, 18), 32), (20, 1)),
])
def test_float32_mask_equals_exact_rational_mask(cfg, over, kpm, k0):
    w = synth.workload(cfg, **over)
    geom = synth.geometry(w)
    (ny_num, nx_num), den = kpm
    assert geom["kpm_x"] == nx_num / den and geom["kpm_y"] == ny_num / den
    pt = orc.pixel_table(geom)
    KXf, KYf = orc.kprime_f32(geom, 0.0)
    k0sq = np.float32(geom["k0_px"] ** 2)
    my = orc.fftfreq_index(w.scan_ny)[:, None]
    mx = orc.fftfreq_index(w.scan_nx)[None, :]
    rng = np.random.default_rng(3)
    ps = np.flatnonzero(pt["bf"])
    if len(ps) * w.n_frames > 3e7:
        ps = rng.choice(ps, 30, replace=False)
    bad = 0
    for p in ps:
        kx, ky = int(pt["kx"][p]), int(pt["ky"][p])
        m32 = orc.trotter_mask(kx, ky, KXf, KYf, k0sq)
        mex = _exact_mask(kx, ky, my, mx, ny_num, nx_num, den, k0[0], k0[1])
        bad += int((m32 != mex).sum())
    assert bad == 0


def _lens(d, k0):
    d = np.minimum(d, 2 * k0)
    return 2 * k0 * k0 * np.arccos(d / (2 * k0)) - 0.5 * d * np.sqrt(np.maximum(4 * k0 * k0 - d * d, 0))


def test_trotter_counts_match_lune_area():
    """|K(K)| counts pixels of the lune D(0) & D(K') minus D(-K'); its area is
    lens(|K'|) - lens(2|K'|).  Lattice counts agree within a perimeter."""
    w = synth.workload(2, scan_ny=64, scan_nx=64)
    geom = synth.geometry(w)
    G = np.ones((orc.pixel_table(geom)["P"], 64, 64), dtype=np.complex128)
    _, nK = orc.ssb_spectrum(G, geom, (0, 0, 0, 0, 0))
    KX, KY = orc.kprime_f64(geom, 0.0)
    s = np.hypot(KX, KY)
    k0 = geom["k0_px"]
    area = _lens(s, k0) - _lens(2 * s, k0)
    per = 4 * math.pi * k0
    assert np.all(np.abs(nK - area) <= per)
    # the exclusion of D(-K') matters: a lens-only count would be far off
    assert np.abs(nK - _lens(s, k0))[s < k0 / 2].min() > per


# ------------------------------------------------------------------- SSB ---
def _weak_phase_case(std, aberr=(0.0, 0.0, 0.0, 0.0, 0.0), ny=32, nx=32, recon_aberr=None, norm="area"):
    # sigma = 2 px keeps the object spectrum inside what the 64-px detector
    # holds without circular aliasing of A(k - K)
    w = synth.workload(1, scan_ny=ny, scan_nx=nx, periodic=True, phase_std=std, aberr=aberr,
                       sigma_px=2.0)
    geom = synth.geometry(w)
    d = synth.generate(w, want_intensity=True)
    counts = orc.bin_crop_dense(d.intensity.numpy(), geom)
    G = orc.g_function(counts, geom)
    ra = aberr if recon_aberr is None else recon_aberr
    phi, V = orc.ssb_phase(G, geom, ra, norm)
    _, nK = orc.ssb_spectrum(G, geom, ra, norm)
    truth = d.phi_scan.numpy()
    T = np.fft.fft2(truth)
    if norm == "area":
        ref = np.fft.ifft2(T * (nK > 0)).real
    else:
        ref = np.fft.ifft2(T * nK).real
    return phi, ref, V


@pytest.mark.parametrize("ny,nx", [(32, 32), (32, 16)])
def test_ssb_recovers_weak_phase_object(ny, nx):
    """Eq. 2/3 on noise-free intensities of a periodic weak phase object: the
    trotter-area SSB image equals the band-limited object to first order, so
    the relative error vanishes with the phase amplitude."""
    errs = []
    for std in (0.1, 0.01, 0.001):
        phi, ref, _ = _weak_phase_case(std, ny=ny, nx=nx)
        errs.append(np.linalg.norm(phi - ref) / np.linalg.norm(ref))
    assert errs[0] <= 0.15 and errs[1] <= 0.02 and errs[2] <= 1e-4
    assert errs[1] / errs[0] <= 0.2 and errs[2] / errs[1] <= 0.2


def test_ssb_unnormalised_transfer_is_trotter_count():
    phi, ref, _ = _weak_phase_case(0.01, norm="none")
    assert np.linalg.norm(phi - ref) / np.linalg.norm(ref) <= 0.02


def _poisson_ssb_corr(e_per_frame, shuffle=False):
    w = synth.workload(1, periodic=True, phase_std=0.1, sigma_px=2.0, e_per_frame=e_per_frame)
    geom = synth.geometry(w)
    d = synth.generate(w)
    idx, off = d.numpy()
    counts = orc.densify(idx, off, geom)
    if shuffle:  # frames at the wrong scan positions: no object information left
        counts = counts[:, np.random.default_rng(0).permutation(counts.shape[1])]
    G = orc.g_function(counts, geom)
    phi, _ = orc.ssb_phase(G, geom, (0, 0, 0, 0, 0), "none")
    _, nK = orc.ssb_spectrum(G, geom, (0, 0, 0, 0, 0), "none")
    ref = np.fft.ifft2(np.fft.fft2(d.phi_scan.numpy()) * nK).real
    return np.corrcoef(phi.ravel(), ref.ravel())[0, 1]


def test_ssb_on_poisson_events_follows_shot_noise():
    """SSB from Poisson electron events (the tiny workload's 30 e-/frame, and
    ten times that): the image correlates with the trotter-filtered object far
    above the shuffled-frame control, and the gain with dose follows shot
    noise: for signal plus independent noise of variance proportional to
    1/dose, r(d2) = 1 / sqrt(1 + (1/r(d1)^2 - 1) d1/d2)."""
    r30, r300 = _poisson_ssb_corr(30.0), _poisson_ssb_corr(300.0)
    ctrl = _poisson_ssb_corr(30.0, shuffle=True)
    assert r30 > 0.15 and r30 > 5 * abs(ctrl), (r30, ctrl)
    pred = 1.0 / math.sqrt(1.0 + (1.0 / r30 ** 2 - 1.0) * 0.1)
    assert abs(r300 - pred) <= 0.06, (r30, r300, pred)


@pytest.mark.parametrize("norm", ["none", "area"])
def test_ssb_from_events_by_pixel_chunks_equals_full_path(norm):
    """The pixel-chunked path (densify a few bright-field pixels at a time,
    transform, add their trotter terms) gives the phase of the full path
    (densify all pixels, G of every pixel, one trotter sum), to rounding."""
    w = synth.workload(2, scan_ny=16, scan_nx=24)
    geom = synth.geometry(w)
    idx, off = synth.generate(w).numpy()
    ab = (60.0, 10.0, -20.0, 5.0e3, 0.2)
    phi, V = orc.ssb_phase(orc.g_function(orc.densify(idx, off, geom), geom), geom, ab, norm)
    phc, Vc = orc.ssb_phase_from_events(idx, off, geom, ab, norm, chunk=37)
    assert np.abs(phc - phi).max() <= 1e-10 * np.abs(phi).max()
    assert abs(Vc - V) <= 1e-10 * V


def test_ssb_spectrum_is_a_sum_over_pixels():
    """S(K) and |K(K)| over disjoint pixel subsets add up to the full ones
    (Eq. 3 is a sum over k): the property a pixel-sharded reconstruction rests
    on."""
    w = synth.workload(1)
    geom = synth.geometry(w)
    idx, off = synth.generate(w).numpy()
    G = orc.g_function(orc.densify(idx, off, geom), geom)
    ab = (40.0, 5.0, -5.0, 0.0, 0.3)
    S, nK = orc.ssb_spectrum(G, geom, ab)
    P_ = G.shape[0]
    a, b = np.arange(0, P_ // 3), np.arange(P_ // 3, P_)
    Sa, na = orc.ssb_spectrum(G[a], geom, ab, pixels=a)
    Sb, nb = orc.ssb_spectrum(G[b], geom, ab, pixels=b)
    assert na.sum() > 0 and nb.sum() > 0
    np.testing.assert_array_equal(na + nb, nK)
    assert np.abs(Sa + Sb - S).max() <= 1e-10 * np.abs(S).max()


def test_aberration_correction_sign():
    """Reading of Eq. 3 under numpy's sign: reconstructing with the true
    aberrations beats no correction and the conjugate correction."""
    ab = (80.0, 20.0, -15.0, 0.0, 0.0)
    r = {}
    for name, ra in [("true", ab), ("zero", (0, 0, 0, 0, 0)), ("conj", tuple(-a for a in ab))]:
        phi, ref, _ = _weak_phase_case(0.01, aberr=ab, recon_aberr=ra)
        r[name] = np.corrcoef(phi.ravel(), ref.ravel())[0, 1]
    assert r["true"] > 0.98
    assert r["true"] > r["zero"] + 0.2 and r["true"] > r["conj"] + 0.2


def test_spherical_aberration_term_from_forward_model():
    """The C3 term of the aberration function (Sec. IV, A(k) of Eq. 3): the
    forward model (its own chi, written separately) makes data with C3 = 50 um
    and C1 = 4 nm; reconstructing with the true C3 reaches the weak-phase
    error floor, while 0.75 C3, 1.25 C3, 0 and 2 C3 are far off.  A wrong
    coefficient, power or sign of the C3 term moves the minimum."""
    ab = (40.0, 0.0, 0.0, 5.0e5, 0.0)
    err = {}
    for s in (0.0, 0.75, 1.0, 1.25, 2.0):
        ra = (ab[0], 0.0, 0.0, s * ab[3], 0.0)
        phi, ref, _ = _weak_phase_case(0.01, aberr=ab, recon_aberr=ra)
        err[s] = np.linalg.norm(phi - ref) / np.linalg.norm(ref)
    assert err[1.0] <= 0.01, err
    assert min(err[0.75], err[1.25]) >= 0.1, err
    assert min(err[0.0], err[2.0]) >= 1.0, err


def _rotated_scan_case(theta, ab=(200.0, 0.0, 0.0, 0.0, 0.0), n=32):
    w = synth.workload(1, scan_ny=n, scan_nx=n, phase_std=0.01, sigma_px=2.0, aberr=ab,
                       scan_rot=theta)
    geom = synth.geometry(w)
    d = synth.generate(w, want_intensity=True)
    G = orc.g_function(orc.bin_crop_dense(d.intensity.numpy(), geom), geom)
    return G, geom, d.phi_scan.numpy()


def test_scan_rotation_direction_from_forward_model():
    """Scan rotation (K' = R(rot) K, counter-clockwise in the detector's x, y):
    the forward model places frame (iy, ix) at R(theta) (ix, iy) step in the
    object frame.  With defocus present the aberration phase depends on the
    direction of K', so only the right rotation recovers the object:
    rot = theta beats -theta, 0 and theta +- 0.1 by correlation with the true
    phase at the probe positions."""
    th = 0.35
    ab = (200.0, 0.0, 0.0, 0.0, 0.0)
    G, geom, truth = _rotated_scan_case(th, ab)
    r = {}
    for rot in (th, -th, 0.0, th - 0.1, th + 0.1):
        phi, _ = orc.ssb_phase(G, geom, ab[:4] + (rot,), "area")
        r[rot] = np.corrcoef(phi.ravel(), truth.ravel())[0, 1]
    assert r[th] > 0.75, r
    assert r[th] > r[-th] + 0.5 and r[th] > r[0.0] + 0.2, r
    assert r[th] > max(r[th - 0.1], r[th + 0.1]) + 0.01, r


# --------------------------------------------------------------- adjoint ---
SCALES = np.array([100.0, 50.0, 50.0, 1.0e4, 0.1])


def _grad_case():
    w = synth.workload(1, scan_ny=16, scan_nx=16, e_per_frame=200.0)
    geom = synth.geometry(w)
    d = synth.generate(w)
    idx, off = d.numpy()
    G = orc.g_function(orc.densify(idx, off, geom), geom)
    return G, geom


def _fd(fun, theta, j, h):
    tp, tm = theta.copy(), theta.copy()
    tp[j] += h
    tm[j] -= h
    return (fun(tp) - fun(tm)) / (2 * h)


def _check_fd(fun, theta, g):
    """Central differences with h = 1e-3 of each scale agree to 1e-5 (their
    O(h^2) truncation), and the Richardson combination of h and h/2 (O(h^4))
    agrees to 1e-8: the analytic gradient is the limit."""
    gmax = np.max(np.abs(g) * SCALES)
    for j in range(5):
        h = 1e-3 * SCALES[j]
        f1 = _fd(fun, theta, j, h)
        f2 = _fd(fun, theta, j, h / 2)
        rich = (4 * f2 - f1) / 3
        floor = 1e-9 * gmax / SCALES[j]
        assert abs(f1 - g[j]) <= 1e-5 * abs(g[j]) + floor, (j, f1, g[j])
        assert abs(rich - g[j]) <= 1e-8 * abs(g[j]) + floor, (j, rich, g[j])


@pytest.mark.parametrize("norm", ["none", "area"])
def test_adjoint_matches_central_differences(norm):
    G, geom = _grad_case()
    theta = np.array([50.0, 10.0, -20.0, 2.0e3, 0.05])
    V, g, _ = orc.ssb_value_and_grad_var(G, geom, theta, norm, mask_rot=theta[4])
    _check_fd(lambda t: orc.ssb_phase(G, geom, t, norm, mask_rot=theta[4])[1], theta, g)


def test_adjoint_general_upstream_gradient():
    """L = sum(u * phi) for a random u: dL/dtheta from the adjoint equals
    central differences of L."""
    G, geom = _grad_case()
    theta = np.array([-30.0, 5.0, 5.0, 0.0, -0.02])
    u = np.random.default_rng(4).normal(size=(16, 16))
    g = orc.ssb_grad(G, geom, theta, u, "none", mask_rot=theta[4])
    _check_fd(lambda t: np.sum(u * orc.ssb_phase(G, geom, t, "none", mask_rot=theta[4])[0]), theta, g)
