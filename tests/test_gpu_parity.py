"""GPU (CUDA path through the C ABI) versus the FP64 oracle, element by element.

Tolerances (stated per result): COM sums, PACBED, counts, trotter set sizes:
bit-exact.  FP32 G: relative max-norm error <= 2e-6 of max|G|.  FP32 SSB phase,
iDPC phase: relative L2 <= 1e-5.  Variance: relative <= 1e-5.  Adjoint:
per component <= 1e-4 relative to the largest scaled component.
"""

import math

import numpy as np
import pytest
import torch

import oracle as orc
import synth

pytestmark = pytest.mark.gpu

SCALES = np.array([100.0, 50.0, 50.0, 1.0e4, 0.1])


@pytest.fixture(scope="module", autouse=True)
def built():
    from paper_2104_06336_gb300.buildlib import build
    build()
    import paper_2104_06336_gb300 as P
    P.load()
    return P


def rel_l2(a, b):
    a = np.asarray(a, dtype=np.float64)
    b = np.asarray(b, dtype=np.float64)
    return float(np.linalg.norm(a - b) / max(np.linalg.norm(b), 1e-300))


class Case:
    """Events (generated once) + GPU reconstructor + oracle quantities."""

    def __init__(self, w, norm=0, device_gen="cpu", n_cand=1, chunk_frames=None, events=None):
        import paper_2104_06336_gb300 as P
        self.w = w
        self.geom = synth.geometry(w)
        d = synth.generate(w, device_gen) if events is None else events
        self.idx_np, self.off_np = d.numpy() if events is None else events.numpy()
        self.idx = d.idx.to("cuda")
        self.off = d.off.to("cuda")
        self.rec = P.Reconstructor(self.geom, norm=norm, n_cand=n_cand)
        self.rec.load(self.idx, self.off, chunk_frames=chunk_frames)
        torch.cuda.synchronize()
        self._G = None

    @property
    def G_orc(self):
        if self._G is None:
            counts = orc.densify(self.idx_np, self.off_np, self.geom)
            self._G = orc.g_function(counts, self.geom)
        return self._G

    def G_gpu_full(self):
        """GPU half spectrum expanded to [P][Ny][Nx] with G(-K) = conj G(K)."""
        Gh = self.rec.G_complex().cpu().numpy().astype(np.complex128)  # [nkx][P_pad][Ny]
        P = self.rec.info["P"]
        Ny, Nx = self.w.scan_ny, self.w.scan_nx
        out = np.zeros((P, Ny, Nx), dtype=np.complex128)
        nkx = Nx // 2 + 1
        out[:, :, :nkx] = np.transpose(Gh[:, :P, :], (1, 2, 0))
        for mx in range(nkx, Nx):
            src = out[:, :, Nx - mx]
            out[:, :, mx] = np.conj(src[:, (-np.arange(Ny)) % Ny])
        return out


@pytest.fixture(scope="module")
def c1():
    return Case(synth.workload(1))


@pytest.fixture(scope="module")
def c1_area():
    return Case(synth.workload(1), norm=1)


@pytest.fixture(scope="module")
def c2small():
    # detector geometry of the 576x576 workloads (bin 4, 1245 BF pixels) on a
    # rectangular 48x64 scan: several FFT tiles and ragged pixel tiles
    return Case(synth.workload(2, scan_ny=48, scan_nx=64), device_gen="cuda")


# --------------------------------------------------------------- a1 + a2 ---
@pytest.mark.parametrize("which", ["c1", "c2small"])
def test_com_sums_pacbed_bit_exact(which, request):
    c = request.getfixturevalue(which)
    import paper_2104_06336_gb300 as P
    W, H = c.w.det_w, c.w.det_h
    pac = torch.zeros(W * H, dtype=torch.int64, device="cuda")
    tot = torch.zeros(3, dtype=torch.int64, device="cuda")
    P.eer_load_csr(c.rec.plan, c.idx, c.off, pacbed=pac, totals=tot, status=c.rec.status)
    sums, com, ph = c.rec.com_dpc(c.idx, c.off)
    torch.cuda.synchronize()
    sx, sy, n = orc.com_sums(c.idx_np, c.off_np, W, H)
    np.testing.assert_array_equal(sums.cpu().numpy(), np.stack([sx, sy, n]))
    np.testing.assert_array_equal(pac.cpu().numpy(), orc.pacbed(c.idx_np, W, H))
    assert tot.cpu().tolist() == [int(sx.sum()), int(sy.sum()), int(n.sum())]
    cx, cy = orc.pacbed_centre(sx, sy, n)
    ox, oy = orc.com_maps(sx, sy, n, cx, cy)
    assert rel_l2(com.cpu().numpy(), np.stack([ox, oy])) <= 1e-6
    phi = orc.idpc(ox, oy, c.geom)
    assert rel_l2(ph.cpu().numpy(), phi) <= 1e-5
    assert c.rec.check() == 0


def test_idpc_regularised(c1):
    sums, com, ph = c1.rec.com_dpc(c1.idx, c1.off, lam1=0.5, lam2=0.01)
    sx, sy, n = orc.com_sums(c1.idx_np, c1.off_np, c1.w.det_w, c1.w.det_h)
    ox, oy = orc.com_maps(sx, sy, n, *orc.pacbed_centre(sx, sy, n))
    assert rel_l2(ph.cpu().numpy(), orc.idpc(ox, oy, c1.geom, 0.5, 0.01)) <= 1e-5


# ------------------------------------------------------------- a4 + a5 -----
@pytest.mark.parametrize("which", ["c1", "c2small"])
def test_counts_bit_exact(which, request):
    c = request.getfixturevalue(which)
    P_, P_pad = c.rec.info["P"], c.rec.info["P_pad"]
    counts = c.rec.counts.view(P_pad, -1).float().cpu().numpy()
    ref = orc.densify(c.idx_np, c.off_np, c.geom)
    np.testing.assert_array_equal(counts[:P_].astype(np.int64), ref)
    assert np.all(counts[P_:] == 0)


@pytest.mark.parametrize("which", ["c1", "c2small"])
def test_g_function_fp32(which, request):
    c = request.getfixturevalue(which)
    G = c.G_gpu_full()
    ref = c.G_orc
    assert np.abs(G - ref).max() <= 2e-6 * np.abs(ref).max()
    # DC terms are sums of integers: exact
    np.testing.assert_array_equal(G[:, 0, 0].real, ref[:, 0, 0].real)


def test_chunked_accumulate_equals_single_call(c2small):
    w = c2small.w
    import paper_2104_06336_gb300 as P
    rec = P.Reconstructor(c2small.geom)
    rec.load(c2small.idx, c2small.off, chunk_frames=3 * w.scan_nx + 5)  # ragged chunks
    torch.cuda.synchronize()
    assert torch.equal(rec.G, c2small.rec.G)
    assert torch.equal(rec.counts, c2small.rec.counts)


# ------------------------------------------------------------- trotter -----
@pytest.mark.parametrize("rot", [0.0, 0.3, -1.1])
@pytest.mark.parametrize("which", ["c1", "c2small"])
def test_trotter_set_sizes_bit_exact(which, rot, request):
    c = request.getfixturevalue(which)
    cnt = c.rec.trotter_counts(rot).cpu().numpy()
    P_ = orc.pixel_table(c.geom)["P"]
    G1 = np.ones((P_, c.w.scan_ny, c.w.scan_nx), dtype=np.complex128)
    _, nK = orc.ssb_spectrum(G1, c.geom, (0, 0, 0, 0, rot))
    np.testing.assert_array_equal(cnt, nK)


ABERRS = [(0.0, 0.0, 0.0, 0.0, 0.0), (80.0, 15.0, 25.98, 1.0e4, 0.0), (-150.0, 40.0, -30.0, 0.0, 0.2)]


@pytest.mark.parametrize("ab", ABERRS)
@pytest.mark.parametrize("which", ["c1", "c1_area", "c2small"])
def test_ssb_phase_fp32(which, ab, request):
    c = request.getfixturevalue(which)
    norm = "area" if c.rec.plan.norm == 1 else "none"
    ph, var = c.rec.reconstruct(torch.tensor(ab, dtype=torch.float64))
    phi, V = orc.ssb_phase(c.G_orc, c.geom, ab, norm)
    assert rel_l2(ph[0].cpu().numpy(), phi) <= 1e-5
    assert abs(float(var[0]) - V) <= 1e-5 * V
    assert c.rec.check() == 0


@pytest.mark.parametrize("which", ["c1", "c2small"])
def test_many_candidates_several_passes_match_single(which, request):
    """20 candidates: several passes of the multi-candidate kernel (8 or 4
    per pass, chosen by the shared memory their phase tables need), spread
    over a second grid dimension on these small scans.  Every candidate's
    phase equals the one-candidate path bit for bit and its variance matches
    the oracle's (Eq. 3)."""
    import paper_2104_06336_gb300 as P
    c = request.getfixturevalue(which)
    rng = np.random.default_rng(7)
    cands = np.zeros((20, 5))
    cands[:, 0] = np.linspace(-150.0, 150.0, 20)
    cands[:, 1] = rng.uniform(-20.0, 20.0, 20)
    cands[:, 2] = rng.uniform(-20.0, 20.0, 20)
    cands[:, 3] = rng.choice([0.0, 5.0e3], 20)
    cands = torch.tensor(cands)
    rec = P.Reconstructor(c.geom, n_cand=20)
    rec.load(c.idx, c.off)
    ph, var = rec.reconstruct(cands)
    torch.cuda.synchronize()
    assert rec.check() == 0
    for i in (0, 7, 8, 13, 19):
        p1, v1 = c.rec.reconstruct(cands[i])
        assert torch.equal(ph[i], p1[0]), i
        _, V = orc.ssb_phase(c.G_orc, c.geom, cands[i].numpy(), "none")
        assert abs(float(var[i]) - V) <= 1e-5 * V, (i, float(var[i]), V)


def test_batched_candidates_match_single(c1):
    import paper_2104_06336_gb300 as P
    cands = torch.tensor([[80.0, 15.0, 26.0, 1.0e4, 0.1], [0, 0, 0, 0, 0.1], [-200.0, -50.0, 30.0, 0, 0.1],
                          [10.0, 0, 0, 0, 0.1]], dtype=torch.float64)
    rec = P.Reconstructor(c1.geom, n_cand=4)
    rec.load(c1.idx, c1.off)
    ph, var = rec.reconstruct(cands)
    for i in range(4):
        p1, v1 = c1.rec.reconstruct(cands[i])
        assert torch.equal(ph[i], p1[0])
        phi, V = orc.ssb_phase(c1.G_orc, c1.geom, cands[i].numpy(), "none")
        assert rel_l2(ph[i].cpu().numpy(), phi) <= 1e-5
    # a candidate with a different rotation is flagged, never silently mixed
    bad = cands.clone()
    bad[2, 4] = 0.0
    rec.status.zero_()
    rec.reconstruct(bad)
    assert (int(rec.status[0].item()) & P._lib.ST_ROTATION) != 0


# --------------------------------------------------------------- adjoint ---
@pytest.mark.parametrize("which", ["c1", "c1_area", "c2small"])
def test_adjoint_parity(which, request):
    c = request.getfixturevalue(which)
    norm = "area" if c.rec.plan.norm == 1 else "none"
    theta = np.array([50.0, 10.0, -20.0, 2.0e3, 0.05])
    u = np.random.default_rng(5).normal(size=(c.w.scan_ny, c.w.scan_nx)).astype(np.float32)
    g = c.rec.grad(torch.tensor(theta), torch.from_numpy(u).cuda()).cpu().numpy()
    ref = orc.ssb_grad(c.G_orc, c.geom, theta, u.astype(np.float64), norm)
    tol = 1e-4 * np.max(np.abs(ref) * SCALES) / SCALES
    assert np.all(np.abs(g - ref) <= tol + 1e-4 * np.abs(ref)), (g, ref)
    V, gv, ph = c.rec.variance_grad(torch.tensor(theta), phase=True)
    Vr, gr, phr = orc.ssb_value_and_grad_var(c.G_orc, c.geom, theta, norm)
    assert abs(float(V) - Vr) <= 1e-5 * Vr
    tol = 1e-4 * np.max(np.abs(gr) * SCALES) / SCALES
    assert np.all(np.abs(gv.cpu().numpy() - gr) <= tol + 1e-4 * np.abs(gr)), (gv, gr)
    assert rel_l2(ph.cpu().numpy(), phr) <= 1e-5


@pytest.mark.parametrize("which", ["c1_area", "c2small"])
def test_adjoint_run_to_run_identical(which, request):
    """The adjoint's warp tasks come from a work queue in whatever order the
    warps reach it; each task's FP64 share is stored at (task, lane) and summed
    in a fixed order afterwards, so repeated calls give the same bits (both
    normalisations, both gradient entry points)."""
    c = request.getfixturevalue(which)
    theta = torch.tensor([50.0, 10.0, -20.0, 2.0e3, 0.05])
    u = torch.from_numpy(np.random.default_rng(9).normal(size=(c.w.scan_ny, c.w.scan_nx))
                         .astype(np.float32)).cuda()
    g1 = c.rec.grad(theta, u).clone()
    V1, gv1, _ = c.rec.variance_grad(theta)
    gv1 = gv1.clone()
    for _ in range(3):
        assert torch.equal(c.rec.grad(theta, u), g1)
        V2, gv2, _ = c.rec.variance_grad(theta)
        assert torch.equal(gv2, gv1) and torch.equal(V2, V1)
    assert c.rec.check() == 0


def test_autograd_function(c1):
    import paper_2104_06336_gb300 as P
    theta = torch.tensor([30.0, 5.0, -5.0, 0.0, 0.0], dtype=torch.float64, device="cuda", requires_grad=True)
    phi = P.ssb_phase(theta, c1.rec)
    loss = (phi.double() ** 2).mean()
    loss.backward()
    g_ref = c1.rec.grad(theta.detach(), (2 * phi.detach() / phi.numel()).float())
    assert torch.allclose(theta.grad, g_ref, rtol=1e-6, atol=0)


# ------------------------------------------------------------ edge cases ---
def _custom(w, idx, off):
    import paper_2104_06336_gb300 as P
    rec = P.Reconstructor(synth.geometry(w))
    i = torch.tensor(np.asarray(idx, dtype=np.uint32).view(np.int32), device="cuda")
    o = torch.tensor(np.asarray(off, dtype=np.int64), device="cuda")
    return rec, i, o


def test_empty_and_out_of_range_events():
    import paper_2104_06336_gb300 as P
    w = synth.workload(1, scan_ny=4, scan_nx=4)
    # frames: empty, valid, one bad index (dropped), empty ...
    idx = [2080, 2081, 4096 + 7, 2080] + [2079] * 3
    off = [0, 0, 2, 3, 4] + [7] * 12
    rec, i, o = _custom(w, idx, off)
    rec.load(i, o)
    sums, com, ph = rec.com_dpc(i, o)
    torch.cuda.synchronize()
    idx_np = np.array(idx, dtype=np.uint32)
    off_np = np.array(off, dtype=np.uint64)
    sx, sy, n = orc.com_sums(idx_np, off_np, 64, 64)
    np.testing.assert_array_equal(sums.cpu().numpy(), np.stack([sx, sy, n]))
    assert com[:, 0].abs().sum().item() == 0.0  # empty frame -> COM 0
    st = rec.status.cpu().numpy()
    assert st[0] & P._lib.ST_RANGE and st[1] >= 1
    counts = rec.counts.view(rec.info["P_pad"], -1).float().cpu().numpy()
    np.testing.assert_array_equal(counts[:rec.info["P"]], orc.densify(idx_np, off_np, synth.geometry(w)))


def test_all_empty_dataset_gives_zero_phase():
    w = synth.workload(1, scan_ny=4, scan_nx=4)
    rec, i, o = _custom(w, [], [0] * 17)
    rec.load(i, o)
    ph, var = rec.reconstruct(torch.zeros(5, dtype=torch.float64))
    assert ph.abs().max().item() == 0.0 and var.item() == 0.0
    assert rec.check() == 0


def test_corrupt_offsets_flagged_without_fault():
    import paper_2104_06336_gb300 as P
    w = synth.workload(1, scan_ny=4, scan_nx=4)
    idx = [2080] * 10
    off = [0, 5, 3, 10**12, 8] + [10] * 12   # decreasing and beyond the array
    rec, i, o = _custom(w, idx, off)
    rec.load(i, o)
    rec.com_dpc(i, o)
    torch.cuda.synchronize()
    assert int(rec.status[0].item()) & P._lib.ST_OFFSETS
    assert rec.check(raise_on_error=False) == P._lib.EER4D_EOFFSETS


def test_pixel_overflow_flagged():
    import paper_2104_06336_gb300 as P
    w = synth.workload(1, scan_ny=2, scan_nx=2)
    idx = [2080] * 2100 + [2081]
    off = [0, 2101, 2101, 2101, 2101]
    rec, i, o = _custom(w, idx, off)
    rec.load(i, o)
    torch.cuda.synchronize()
    assert int(rec.status[0].item()) & P._lib.ST_OVERFLOW


def test_bounded_wait_gives_up_and_reports(c1):
    """Failure detection without a GPU fault: the fused DFT's device wait on a
    producer that never arrives gives up after its limit (about 1 s), sets
    EER4D_ST_TIMEOUT and returns; the context stays usable."""
    import time
    import paper_2104_06336_gb300 as P
    scr = torch.zeros(2, dtype=torch.int32, device="cuda")
    st = torch.zeros(4, dtype=torch.int32, device="cuda")
    torch.cuda.synchronize()
    t0 = time.time()
    P.eer4d_selftest_wait(scr, st)
    torch.cuda.synchronize()
    dt = time.time() - t0
    assert P.status_code(st) == P._lib.EER4D_ETIMEOUT
    assert 0.5 < dt < 30.0, dt
    ph, var = c1.rec.reconstruct(torch.zeros(5, dtype=torch.float64))
    torch.cuda.synchronize()
    assert c1.rec.check() == 0 and torch.isfinite(ph).all()


def test_binding_rejects_short_or_mistyped_buffers(c1):
    """The library cannot see buffer sizes; the binding refuses a buffer that
    is too short or of the wrong type before any launch."""
    import paper_2104_06336_gb300 as P
    rec = c1.rec
    ab = torch.zeros(5, dtype=torch.float64, device="cuda")
    short = torch.empty(rec.F - 1, dtype=torch.float32, device="cuda")
    var = torch.empty(1, dtype=torch.float64, device="cuda")
    with pytest.raises(ValueError):
        P.ssb_reconstruct(rec.plan, rec.G, ab, rec.scratch, short, var, status=rec.status)
    with pytest.raises(TypeError):
        P.ssb_reconstruct(rec.plan, rec.G, ab.float(), rec.scratch, None, var, status=rec.status)
    with pytest.raises(ValueError):
        P.ssb_reconstruct(rec.plan, rec.G[:10], ab, rec.scratch, None, var, status=rec.status)
    with pytest.raises(ValueError):
        P.com_dpc(rec.plan, c1.idx, c1.off[:-1], torch.empty(3, rec.F, dtype=torch.int64, device="cuda"),
                  torch.empty(2, rec.F, device="cuda"))
    torch.cuda.synchronize()
    assert rec.check() == 0


def test_out_of_order_chunks_rejected(c1):
    import paper_2104_06336_gb300 as P
    with pytest.raises(P.Eer4dError) as e:
        P.ssb_accumulate(c1.rec.plan, c1.idx, c1.off[64:129], 64, c1.rec.work, c1.rec.G, False)
    assert e.value.code == P._lib.EER4D_EORDER


# ------------------------------------------------- precision workload size --
@pytest.fixture(scope="module")
def c2full():
    return Case(synth.workload(2), device_gen="cuda")


def test_precision_workload_full_size(c2full):
    """256x256 scan, 576x576 detector binned 4x, 1245 BF pixels: counts exact,
    FP32 G and SSB phase against the FP64 oracle."""
    c = c2full
    P_, P_pad = c.rec.info["P"], c.rec.info["P_pad"]
    assert P_ == 1245
    counts = c.rec.counts.view(P_pad, -1).float().cpu().numpy()[:P_].astype(np.int64)
    ref = orc.densify(c.idx_np, c.off_np, c.geom)
    np.testing.assert_array_equal(counts, ref)
    G = c.G_orc
    ph, var = c.rec.reconstruct(torch.zeros(5, dtype=torch.float64))
    phi, V = orc.ssb_phase(G, c.geom, (0, 0, 0, 0, 0), "none")
    err = rel_l2(ph[0].cpu().numpy(), phi)
    print(f"precision workload FP32 SSB rel L2 = {err:.3e}")
    assert err <= 1e-5


# ------------------------------------------- fused two-axis scan DFT --------
def _two_pass_G(c):
    import paper_2104_06336_gb300 as P
    rec = P.Reconstructor(c.geom, precision=P.FP32_FFT_2PASS)
    rec.load(c.idx, c.off)
    torch.cuda.synchronize()
    assert rec.check() == 0
    return rec


def test_fused_dft_256_matches_oracle_and_two_pass(c2full):
    """256x256 scan (square power of two: one persistent launch for both
    axes): G to 2e-6 of max|G| of the FP64 oracle, and bit-identical to the
    two-launch form (the same arithmetic per element)."""
    G = c2full.G_gpu_full()
    ref = c2full.G_orc
    err = np.abs(G - ref).max() / np.abs(ref).max()
    print(f"fused 256^2 G max err / max|G| = {err:.2e}")
    assert err <= 2e-6
    assert c2full.rec.check() == 0
    assert torch.equal(_two_pass_G(c2full).G, c2full.rec.G)


def test_stockham_form_matches_fused(c2full):
    """The plain FP32 Stockham form (two launches and a transpose) against the
    fused register FFT on the 256x256 precision workload: G within 2e-6 of
    max|G|."""
    import paper_2104_06336_gb300 as P
    rec = P.Reconstructor(c2full.geom, precision=P.FP32_STOCKHAM)
    rec.load(c2full.idx, c2full.off)
    torch.cuda.synchronize()
    assert rec.check() == 0
    a, b = rec.G_complex(), c2full.rec.G_complex()
    assert float((a - b).abs().max()) <= 2e-6 * float(b.abs().max())


@pytest.mark.parametrize("n", [128, 512])
def test_fused_dft_other_sizes_match_two_pass(n):
    """The 128 (groups of 16 pixels) and 512 (groups of 8) instantiations
    against the two-launch form, bit for bit; chunked ingest gives the same."""
    w = synth.workload(1, scan_ny=n, scan_nx=n)
    c = Case(w, device_gen="cuda")
    assert c.rec.check() == 0
    assert torch.equal(_two_pass_G(c).G, c.rec.G)
    import paper_2104_06336_gb300 as P
    rec = P.Reconstructor(c.geom)
    rec.load(c.idx, c.off, chunk_frames=5 * n + 3)
    torch.cuda.synchronize()
    assert torch.equal(rec.G, c.rec.G)


def test_full_size_workload_sampled_pixels_and_frequencies():
    """The 1024x1024 scan on the 576x576 detector binned 6x (553 pixels,
    about 5.2e7 events; the configuration the benchmark times): counts bit-exact
    and G to 2e-6 of max|G| on sampled pixels (every K, from the oracle's
    per-pixel densify + FFT) and on sampled K (every pixel, from the oracle's
    event sum)."""
    w = synth.workload(5)
    geom = synth.geometry(w)
    d = synth.generate(w, "cuda")
    import paper_2104_06336_gb300 as P
    rec = P.Reconstructor(geom)
    rec.load(d.idx, d.off)
    torch.cuda.synchronize()
    assert rec.check() == 0
    idx, off = d.numpy()
    Pn, P_pad, Ny, Nx = rec.info["P"], rec.info["P_pad"], w.scan_ny, w.scan_nx
    assert Pn == 553
    sel = np.array([0, 1, 7, 8, 15, 16, 200, Pn // 2, Pn - 9, Pn - 1])
    counts_ref = orc.densify_pixels(idx, off, geom, sel)
    counts = rec.counts.view(P_pad, -1)[torch.as_tensor(sel, device=rec.device)].float().cpu().numpy()
    np.testing.assert_array_equal(counts.astype(np.int64), counts_ref)
    Gh = rec.G_complex()  # [nkx][P_pad][Ny]
    nkx = Nx // 2 + 1
    ref = orc.g_function(counts_ref, geom)[:, :, :nkx]  # [s][Ny][nkx]
    got = Gh[:, torch.as_tensor(sel, device=rec.device), :].cpu().numpy().transpose(1, 2, 0)
    err = np.abs(got - ref).max() / np.abs(ref).max()
    print(f"1024^2 sampled-pixel G max err / max|G| = {err:.2e}")
    assert err <= 2e-6
    for ky, kx in [(0, 0), (1, 3), (Ny // 2, Nx // 2), (Ny - 5, 17)]:
        col = orc.g_column(idx, off, geom, ky, kx)
        g = Gh[kx, :Pn, ky].cpu().numpy()
        scale = max(np.abs(ref).max(), np.abs(col).max())
        assert np.abs(g - col).max() <= 2e-6 * scale, (ky, kx)


# ------------------------------------------------------- iterative DPC ------
@pytest.mark.parametrize("which", ["c1", "c2small"])
@pytest.mark.parametrize("pad,n_iter,lam1", [(2, 50, 0.0), (1, 7, 0.3), (2, 0, 0.0)])
def test_dpc_iterative_matches_oracle(which, pad, n_iter, lam1, request):
    """The gradient-descent DPC (mu = 0.5) from the oracle's COM maps, within
    1e-5 relative L2 of the FP64 iteration (zero steps: exactly zero)."""
    c = request.getfixturevalue(which)
    W, H = c.w.det_w, c.w.det_h
    Sx, Sy, N = orc.com_sums(c.idx_np, c.off_np, W, H)
    cx, cy = orc.pacbed_centre(Sx, Sy, N)
    ox, oy = orc.com_maps(Sx, Sy, N, cx, cy)
    com = torch.tensor(np.stack([ox, oy]).astype(np.float32), device="cuda")
    ph = c.rec.dpc_iterative(com, n_iter, mu=0.5, lam1=lam1, pad=pad).cpu().numpy()
    ref = orc.dpc_iterative(com.cpu().numpy()[0].astype(np.float64), com.cpu().numpy()[1].astype(np.float64),
                            c.geom, n_iter, mu=0.5, lam1=lam1, pad=pad)
    if n_iter == 0:
        assert np.all(ph == 0)
    else:
        assert rel_l2(ph, ref) <= 1e-5, rel_l2(ph, ref)


# ---------------------------------------------------- G-function view ------
@pytest.mark.parametrize("which", ["c1", "c2small"])
def test_g_slices_match_oracle(which, request):
    """G(k, K) at nine bins, including bins of the unstored K_x < 0 half
    (conjugate symmetry) and Nyquist bins, on the detector window."""
    c = request.getfixturevalue(which)
    Ny, Nx = c.w.scan_ny, c.w.scan_nx
    bins = [(0, 0), (1, 0), (0, 1), (3, 5), (Ny - 3, Nx - 5), (Ny // 2, 0), (0, Nx // 2),
            (Ny - 1, 2), (7, Nx - 1)]
    got = c.rec.g_slices(bins).cpu().numpy()
    ref = orc.g_slices(c.G_orc, c.geom, bins)
    assert np.abs(got - ref).max() <= 2e-6 * np.abs(c.G_orc).max()
    assert np.all(got[ref == 0] == 0)


# ------------------------------------------------- virtual detectors ------
@pytest.mark.parametrize("which", ["c1", "c2small"])
def test_virtual_detectors_bit_exact(which, request):
    """Bright-field disk, annular and dark-field rings and a 16-ring radial sum
    about the PACBED centre, bit-exact against the oracle."""
    c = request.getfixturevalue(which)
    W, H = c.w.det_w, c.w.det_h
    Sx, Sy, N = orc.com_sums(c.idx_np, c.off_np, W, H)
    cx, cy = orc.pacbed_centre(Sx, Sy, N)
    bf = c.geom["k0_px"] * c.geom["bin"]
    for radii in ([0.0, bf], [0.0, 0.5 * bf, bf, 2 * bf, 4.0 * max(W, H)],
                  list(np.linspace(0.0, 1.5 * bf, 17))):
        got = c.rec.virtual_detectors(c.idx, c.off, radii).cpu().numpy().reshape(len(radii) - 1, -1)
        ref = orc.virtual_detector_counts(c.idx_np, c.off_np, W, H, radii, cx, cy)
        np.testing.assert_array_equal(got, ref)
    assert c.rec.check() == 0


# ------------------------------------------- large crop, chunked scatter ----
def test_large_crop_counts_and_phase():
    """The 576x576 detector binned 6x cropped to the disk of radius 48 binned
    pixels (7209 kept pixels, the residency variant of the full workload) on
    a 48x48 scan: the scatter counts pixel chunk by chunk; counts bit-exact,
    G to 2e-6 of max|G| and the SSB phase to 1e-5 relative L2."""
    import paper_2104_06336_gb300 as P
    w = synth.workload(5, scan_ny=48, scan_nx=48)
    geom = dict(synth.geometry(w), crop_px=48.0)
    d = synth.generate(w, "cuda")
    rec = P.Reconstructor(geom)
    rec.load(d.idx, d.off)
    torch.cuda.synchronize()
    assert rec.check() == 0
    Pn, P_pad = rec.info["P"], rec.info["P_pad"]
    assert Pn == 7209
    idx, off = d.numpy()
    ref = orc.densify(idx, off, geom)
    counts = rec.counts.reshape(P_pad, -1)[:Pn].float().cpu().numpy().astype(np.int64)
    np.testing.assert_array_equal(counts, ref)
    G = orc.g_function(ref, geom)
    Gh = rec.G_complex().cpu().numpy()  # [nkx][P_pad][Ny]
    nkx = w.scan_nx // 2 + 1
    got = np.transpose(Gh[:, :Pn, :], (1, 2, 0))
    assert np.abs(got - G[:, :, :nkx]).max() <= 2e-6 * np.abs(G).max()
    ab = (40.0, 5.0, -5.0, 0.0, 0.0)
    ph, _ = rec.reconstruct(torch.tensor(ab, dtype=torch.float64))
    phi, _ = orc.ssb_phase(G, geom, ab, "none")
    assert rel_l2(ph[0].cpu().numpy(), phi) <= 1e-5


# ------------------------------------------- run-length-encoded ingest -----
@pytest.mark.parametrize("which", ["c1", "c2small"])
def test_rle_decode_bit_exact_and_pipeline(which, request):
    """eer_decode_rle against the oracle's prefix sums, bit for bit; the decoded
    (per-frame sorted) events give the same COM sums and G as the original
    linear-index events; decoding in place gives the same indices."""
    import paper_2104_06336_gb300 as P
    c = request.getfixturevalue(which)
    ev = synth.EventData(idx=c.idx, off=c.off, phi_scan=torch.zeros(1))
    runs, off = ev.rle()
    st = torch.zeros(4, dtype=torch.int32, device="cuda")
    idx = P.eer_decode_rle(runs, off, status=st)
    torch.cuda.synchronize()
    assert P.status_code(st) == 0
    ref = orc.rle_decode_fast(runs.cpu().numpy().view(np.uint32), off.cpu().numpy())
    np.testing.assert_array_equal(idx.cpu().numpy().view(np.uint32).astype(np.int64), ref)
    inplace = runs.clone()
    P.eer_decode_rle(inplace, off, idx=inplace, status=st)
    assert torch.equal(inplace, idx)
    rec = P.Reconstructor(c.geom)
    rec.load(idx, off)
    sums, _, _ = rec.com_dpc(idx, off)
    sums0, _, _ = c.rec.com_dpc(c.idx, c.off)
    torch.cuda.synchronize()
    assert torch.equal(sums, sums0)
    assert torch.equal(rec.counts, c.rec.counts)
    assert torch.equal(rec.G, c.rec.G)


def test_rle_decode_flags_overflow_and_bad_offsets():
    """A frame whose runs add up past 2^32 - 1 is written as 0xFFFFFFFF and
    flagged as out of range; decreasing offsets are flagged and clipped."""
    import paper_2104_06336_gb300 as P
    runs = torch.tensor([5, 10, -1, 3], dtype=torch.int32, device="cuda")  # -1 = 0xFFFFFFFF
    off = torch.tensor([0, 2, 4], dtype=torch.int64, device="cuda")
    st = torch.zeros(4, dtype=torch.int32, device="cuda")
    idx = P.eer_decode_rle(runs, off, status=st)
    torch.cuda.synchronize()
    assert idx.cpu().numpy().view(np.uint32).tolist() == [5, 15, 0xFFFFFFFF, 0xFFFFFFFF]
    assert P.status_code(st) == P._lib.EER4D_ERANGE
    st.zero_()
    bad = torch.tensor([0, 3, 1], dtype=torch.int64, device="cuda")
    P.eer_decode_rle(runs, bad, status=st)
    torch.cuda.synchronize()
    assert P.status_code(st) == P._lib.EER4D_EOFFSETS


# ----------------------------------------- overlapped upload + compute ------
def test_streamed_steps_equal_direct_calls(c2small):
    """Uploading each step's events on a copy stream while the previous step
    computes gives the same COM sums, G and phase as the direct calls, for
    every step (alternating buffers)."""
    import paper_2104_06336_gb300 as P
    c = c2small
    rec = P.Reconstructor(c.geom)
    h_idx = c.idx.cpu().pin_memory()
    h_off = c.off.cpu().pin_memory()
    pipe = P.StreamedSteps(c.idx.numel(), rec.F)
    ab = torch.tensor([30.0, 0.0, 0.0, 0.0, 0.0], dtype=torch.float64)
    outs = []

    def body(di, do):
        rec.load(di, do)
        sums, com, _ = rec.com_dpc(di, do)
        ph, var = rec.reconstruct(ab)
        return sums.cpu(), ph.cpu()

    for _ in range(3):
        outs.append(pipe.run(h_idx, h_off, body))
    torch.cuda.synchronize()
    sums0, _, _ = c.rec.com_dpc(c.idx, c.off)
    ph0, _ = c.rec.reconstruct(ab)
    for sums, ph in outs:
        assert torch.equal(sums, sums0.cpu())
        assert torch.equal(ph, ph0.cpu())


# ------------------------------------------------ launch-shape autotuner ----
@pytest.mark.parametrize("n", [0, 128])
def test_autotune_keeps_results_and_caches(n, c2small, tmp_path):
    """The autotuner's choice changes no result: counts, G and the phase are
    bit-identical to the built-in shapes; a cached choice is applied without
    timing; out-of-range shapes are rejected."""
    import paper_2104_06336_gb300 as P
    c = c2small if n == 0 else Case(synth.workload(2, scan_ny=n, scan_nx=n), device_gen="cuda")
    rec = P.Reconstructor(c.geom)
    cache = str(tmp_path / "tune.json")
    t = P.tuning.autotune(rec, c.idx, c.off, cache=cache)
    assert t["scatter_tf"] in (16, 32, 64, 128) and 1 <= t["scatter_ctas_per_sm"] <= 3
    assert 1 <= t["trotter_ctas_per_sm"] <= 3
    assert (t["dft_ctas_per_sm"] == 0) == (n == 0)
    assert all(m > 0 for m, k in zip(t["ms"], (1, n, 1)) if k)
    rec.load(c.idx, c.off)
    ph, var = rec.reconstruct(torch.tensor([40.0, 5.0, -5.0, 0.0, 0.0], dtype=torch.float64))
    ph0, var0 = c.rec.reconstruct(torch.tensor([40.0, 5.0, -5.0, 0.0, 0.0], dtype=torch.float64))
    torch.cuda.synchronize()
    assert rec.check() == 0
    assert torch.equal(rec.counts, c.rec.counts)
    assert torch.equal(rec.G, c.rec.G)
    assert torch.equal(ph, ph0)
    rec2 = P.Reconstructor(c.geom)
    assert P.tuning.autotune(rec2, c.idx, c.off, cache=cache) == t
    assert P.eer4d_get_tuning(rec2.plan)["scatter_tf"] == t["scatter_tf"]
    with pytest.raises(P.Eer4dError):
        P.eer4d_set_tuning(rec2.plan, dict(t, scatter_tf=48))


# ------------------------------------------ uneven batches, one launch ------
def _batch_cases(sizes, doses, seed=3):
    out = []
    for i, ((ny, nx), e) in enumerate(zip(sizes, doses)):
        w = synth.workload(4, scan_ny=ny, scan_nx=nx, e_per_frame=float(e), seed=1000 * seed + i,
                           name=f"batch{i}-{ny}x{nx}")
        out.append(Case(w, device_gen="cuda"))
    return out


def test_batched_uneven_datasets_match_oracle_and_single():
    """Datasets of the batching workload's detector (576x576 binned 4x, 1245
    BF pixels) with different scan shapes and doses, each with its own
    aberrations and scan rotation, in one ssb_reconstruct_batched call: every
    phase within 1e-5 relative L2 of the FP64 oracle and equal to the
    single-dataset path to 1e-6 of its max; variances within 1e-5."""
    import paper_2104_06336_gb300 as P
    cases = _batch_cases([(32, 32), (48, 64), (64, 48), (16, 16)], [10, 50, 30, 20])
    ab = np.array([[60.0, 10.0, -20.0, 0.0, 0.0],
                   [-40.0, 0.0, 15.0, 5.0e3, 0.0],
                   [0.0, -25.0, 0.0, 0.0, 0.4],
                   [120.0, 5.0, 5.0, 0.0, -0.2]])
    ph, var = P.reconstruct_batched([c.rec for c in cases], torch.tensor(ab))
    torch.cuda.synchronize()
    assert cases[0].rec.check() == 0
    for i, c in enumerate(cases):
        phi, V = orc.ssb_phase(c.G_orc, c.geom, tuple(ab[i]), "none")
        got = ph[i].cpu().numpy()
        err = rel_l2(got, phi)
        assert err <= 1e-5, (i, err)
        assert abs(float(var[i]) - V) <= 1e-5 * V, (i, float(var[i]), V)
        ph1, v1 = c.rec.reconstruct(torch.tensor(ab[i]))
        d = np.abs(ph1[0].cpu().numpy() - got).max()
        assert d <= 1e-6 * np.abs(got).max(), (i, d)


def test_batched_rejects_mixed_detectors(c1):
    """Datasets recorded with different detector geometries cannot share one
    launch: the call returns EINVAL before enqueueing anything."""
    import paper_2104_06336_gb300 as P
    other = _batch_cases([(16, 16)], [10])[0]
    with pytest.raises(P.Eer4dError) as ei:
        P.reconstruct_batched([c1.rec, other.rec], torch.zeros(2, 5, dtype=torch.float64))
    assert ei.value.code == -1


def test_batching_workload_sixteen_datasets():
    """The batching workload: 16 square scans N_i = 16 round(exp U(ln 64, ln 512)/16)
    with 10..50 e-/frame, one launch.  Each dataset equals its single-dataset
    reconstruction to 1e-6 of max|phi|; the smallest one against the oracle."""
    import paper_2104_06336_gb300 as P
    ws = synth.batching_datasets()
    recs, small = [], None
    for w in ws:
        d = synth.generate(w, "cuda")
        rec = P.Reconstructor(synth.geometry(w))
        rec.load(d.idx, d.off)
        recs.append(rec)
        if small is None or w.scan_ny < small[0].scan_ny:
            small = (w, d, rec)
    torch.cuda.synchronize()
    ab = torch.tensor(synth.candidate_aberrations(n=len(ws)))
    ph, var = P.reconstruct_batched(recs, ab)
    torch.cuda.synchronize()
    assert recs[0].check() == 0
    for i, rec in enumerate(recs):
        ph1, v1 = rec.reconstruct(ab[i])
        got = ph[i]
        d = float((ph1[0] - got).abs().max())
        assert d <= 1e-6 * float(got.abs().max()), (i, d)
        assert abs(float(v1[0]) - float(var[i])) <= 1e-9 * float(var[i])
    w, d, rec = small
    i = recs.index(rec)
    idx, off = d.numpy()
    G = orc.g_function(orc.densify(idx, off, synth.geometry(w)), synth.geometry(w))
    phi, V = orc.ssb_phase(G, synth.geometry(w), tuple(ab[i].numpy()), "none")
    assert rel_l2(ph[i].cpu().numpy(), phi) <= 1e-5


# ------------------------------------------ split-FP16 tensor-core DFT ------
@pytest.mark.parametrize("which", ["c1", "c2small"])
def test_split_fp16_dft_matches_fp32(which, request):
    """The x-axis DFT on tcgen05 (counts exact in fp16, DFT factors split hi+lo,
    FP32 accumulation) reproduces the FP32 FFT's G to 1e-6 of max|G| and the
    SSB phase to 1e-4 relative L2 of the FP64 oracle."""
    import paper_2104_06336_gb300 as P
    c = request.getfixturevalue(which)
    rec = P.Reconstructor(c.geom, precision=P.SPLIT_FP16)
    rec.load(c.idx, c.off)
    torch.cuda.synchronize()
    assert rec.check() == 0
    Gt = rec.G_complex().cpu().numpy()
    Gf = c.rec.G_complex().cpu().numpy()
    assert np.abs(Gt - Gf).max() <= 1e-6 * np.abs(Gf).max()
    ab = (80.0, 15.0, 25.98, 1.0e4, 0.0)
    ph, var = rec.reconstruct(torch.tensor(ab, dtype=torch.float64))
    phi, V = orc.ssb_phase(c.G_orc, c.geom, ab, "none")
    assert rel_l2(ph[0].cpu().numpy(), phi) <= 1e-4


# ------------------------------------------------------------- refocusing ---
def test_refocus_recovers_true_defocus():
    """Differentiation workload optics (25 mrad, C1 = 8 nm, C12 = 3 nm at 30 deg,
    C3 = 1 um) on a 128x128 scan: a batched sweep of 64 defocus candidates
    (one launch) seeds Adam ascent on the image variance driven by the adjoint;
    the fitted defocus lands on the true 80 A and V does not decrease."""
    import paper_2104_06336_gb300 as P
    w = synth.workload(3, scan_ny=128, scan_nx=128)
    d = synth.generate(w, "cuda")
    rec = P.Reconstructor(synth.geometry(w), n_cand=64)
    rec.load(d.idx, d.off)
    true = torch.tensor(w.aberr, dtype=torch.float64)
    cands = true.repeat(64, 1)
    cands[:, 0] = torch.linspace(-200.0, 200.0, 64, dtype=torch.float64)
    V = P.refocus.sweep(rec, cands).cpu()
    best = cands[int(torch.argmax(V))].clone()
    assert abs(float(best[0]) - 80.0) < 15.0
    theta, hist = P.refocus.fit(rec, best, steps=25, lr=0.02, mask=(1, 0, 0, 0, 0))
    assert abs(float(theta[0]) - 80.0) < 6.0, (float(theta[0]), hist[-3:])
    assert hist[-1] >= float(V.max()) * (1 - 1e-9)
    # graph-replayed device-side refocus steps move toward the same optimum
    g = P.refocus.RefocusGraph(rec, best, step=[0.02 * 100.0 ** 2 / max(1.0, abs(hist[0])), 0, 0, 0, 0])
    g.replay(10)
    torch.cuda.synchronize()
    assert rec.check() == 0
    assert torch.isfinite(g.theta).all()
