"""One pass over the events: ssb_accumulate_com (scatter + per-frame COM sums +
PACBED totals) followed by com_dpc_sums, against the separate calls
(eer_load_csr, com_dpc, ssb_accumulate) and the FP64 oracle (Eq. 4; Table 1).

The single-pass outputs must be bit-identical to the separate calls: the sums
and totals are integers, the COM maps and the DPC phase come from the same
arithmetic, and the counts and G from the same scatter and DFT."""

import numpy as np
import pytest
import torch

import oracle as orc
import synth

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def built():
    if not torch.cuda.is_available():
        pytest.skip("needs a GPU")
    import paper_2104_06336_gb300 as P
    P.build()


def _separate(rec, idx, off):
    import paper_2104_06336_gb300 as P
    F = rec.F
    tot = torch.zeros(3, dtype=torch.int64, device="cuda")
    P.eer_load_csr(rec.plan, idx, off, totals=tot, status=rec.status)
    sums = torch.empty(3, F, dtype=torch.int64, device="cuda")
    com = torch.empty(2, F, dtype=torch.float32, device="cuda")
    ph = torch.empty(rec.Ny, rec.Nx, dtype=torch.float32, device="cuda")
    P.com_dpc(rec.plan, idx, off, sums, com, ph, totals=tot, scratch=rec.scratch,
              status=rec.status)
    P.ssb_accumulate(rec.plan, idx, off, 0, rec.work, rec.G, True, status=rec.status)
    torch.cuda.synchronize()
    return sums, tot, com, ph


def _single(rec, idx, off, chunk=None):
    import paper_2104_06336_gb300 as P
    F = rec.F
    tot = torch.zeros(3, dtype=torch.int64, device="cuda")
    sums = torch.full((3, F), -1, dtype=torch.int64, device="cuda")
    step = F if chunk is None else chunk
    for f0 in range(0, F, step):
        f1 = min(F, f0 + step)
        P.ssb_accumulate_com(rec.plan, idx, off[f0:f1 + 1], f0, rec.work, rec.G, f1 == F, sums,
                             tot, status=rec.status)
    com = torch.empty(2, F, dtype=torch.float32, device="cuda")
    ph = torch.empty(rec.Ny, rec.Nx, dtype=torch.float32, device="cuda")
    P.com_dpc_sums(rec.plan, sums, com, ph, totals=tot, scratch=rec.scratch, status=rec.status)
    torch.cuda.synchronize()
    return sums, tot, com, ph


def _compare(w, geom, d, chunk=None):
    import paper_2104_06336_gb300 as P
    idx = d.idx.to("cuda")
    off = d.off.to("cuda")
    ra = P.Reconstructor(geom)
    rb = P.Reconstructor(geom)
    sa, ta, ca, pa = _separate(ra, idx, off)
    sb, tb, cb, pb = _single(rb, idx, off, chunk)
    assert torch.equal(sa, sb)
    assert torch.equal(ta, tb)
    assert torch.equal(ca, cb)
    assert torch.equal(pa, pb)
    assert torch.equal(ra.counts, rb.counts)
    assert torch.equal(ra.G, rb.G)
    assert torch.equal(ra.status, rb.status)
    idx_np, off_np = d.numpy()
    sx, sy, n = orc.com_sums(idx_np, off_np, w.det_w, w.det_h)
    np.testing.assert_array_equal(sb.cpu().numpy(), np.stack([sx, sy, n]))
    assert tb.cpu().tolist() == [int(sx.sum()), int(sy.sum()), int(n.sum())]
    assert rb.check() == 0


@pytest.mark.parametrize("shape", [(16, 16), (48, 64), (64, 64)])
def test_single_pass_equals_separate_calls(shape):
    """Square power-of-two scans take the fused DFT, the 48 x 64 scan the
    two-pass DFT; frame tiles of 32 with a ragged last tile at 48 x 64."""
    w = synth.workload(2, scan_ny=shape[0], scan_nx=shape[1])
    _compare(w, synth.geometry(w), synth.generate(w, "cuda"))


@pytest.mark.parametrize("chunk", [1000, 37])
def test_single_pass_chunked(chunk):
    """Chunks that start inside a frame tile (37) and span several (1000)."""
    w = synth.workload(2, scan_ny=48, scan_nx=64)
    _compare(w, synth.geometry(w), synth.generate(w, "cuda"), chunk=chunk)


def test_single_pass_large_crop_sums_once():
    """7209 kept pixels counted chunk by chunk (13 pixel chunks per frame
    tile): each frame's sums are formed once, in chunk 0."""
    w = synth.workload(5, scan_ny=32, scan_nx=32)
    geom = dict(synth.geometry(w), crop_px=48.0)
    _compare(w, geom, synth.generate(w, "cuda"))


def _custom(w, idx, off):
    import paper_2104_06336_gb300 as P
    rec = P.Reconstructor(synth.geometry(w))
    i = torch.tensor(np.asarray(idx, dtype=np.uint32).view(np.int32), device="cuda")
    o = torch.tensor(np.asarray(off, dtype=np.int64), device="cuda")
    return rec, i, o


def test_single_pass_empty_and_out_of_range():
    import paper_2104_06336_gb300 as P
    w = synth.workload(1, scan_ny=4, scan_nx=4)
    idx = [2080, 2081, 4096 + 7, 2080] + [2079] * 3
    off = [0, 0, 2, 3, 4] + [7] * 12
    rec, i, o = _custom(w, idx, off)
    sums, tot, com, ph = _single(rec, i, o)
    sx, sy, n = orc.com_sums(np.array(idx, dtype=np.uint32), np.array(off, dtype=np.uint64),
                             64, 64)
    np.testing.assert_array_equal(sums.cpu().numpy(), np.stack([sx, sy, n]))
    assert com[:, 0].abs().sum().item() == 0.0
    st = rec.status.cpu().numpy()
    assert st[0] & P._lib.ST_RANGE and st[1] >= 1


def test_single_pass_corrupt_offsets_flagged():
    import paper_2104_06336_gb300 as P
    w = synth.workload(1, scan_ny=4, scan_nx=4)
    rec, i, o = _custom(w, [2080] * 10, [0, 5, 3, 10**12, 8] + [10] * 12)
    _single(rec, i, o)
    assert int(rec.status[0].item()) & P._lib.ST_OFFSETS


def test_single_pass_frame_overflow_flagged():
    """A frame of 70000 events: EER4D_ST_OVERFLOW, and its sums cover its
    first 65535 events."""
    import paper_2104_06336_gb300 as P
    w = synth.workload(1, scan_ny=2, scan_nx=2)
    idx = [2080] * 70000 + [2081]
    off = [0, 70000, 70001, 70001, 70001]
    rec, i, o = _custom(w, idx, off)
    sums, tot, _, _ = _single(rec, i, o)
    assert int(rec.status[0].item()) & P._lib.ST_OVERFLOW
    x, y = 2080 % 64, 2080 // 64
    assert sums[:, 0].cpu().tolist() == [65535 * x, 65535 * y, 65535]
    assert sums[:, 1].cpu().tolist() == [2081 % 64, 2081 // 64, 1]


def test_single_pass_rejects_missing_sums():
    import paper_2104_06336_gb300 as P
    w = synth.workload(1, scan_ny=4, scan_nx=4)
    rec, i, o = _custom(w, [2080], [0] + [1] * 16)
    with pytest.raises(ValueError):
        P.ssb_accumulate_com(rec.plan, i, o, 0, rec.work, rec.G, True, None, None)
