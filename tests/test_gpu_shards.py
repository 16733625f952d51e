"""Pixel shards on one GPU (Sec. IV: G(k, K) and the trotter sum of Eq. 3 are
per detector pixel).  A dataset split into 2 or 3 shard plans (each reading
every event and keeping its own pixels) gives, after the shares of the
spectrum and of the Gbar0 sums are added on the host, the phase and variance
of the unsharded plan to FP32 rounding and the oracle's within 1e-5; each
shard's counts are the matching rows of the full counts, bit for bit.
(The ranks are emulated one after another on one GPU; the exchange itself,
an all-reduce, is tested on CPU with gloo in test_shards_gloo.py.)"""

import numpy as np
import pytest
import torch

import oracle as orc
import synth

pytestmark = pytest.mark.gpu


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


@pytest.mark.parametrize("n_shards", [2, 3])
@pytest.mark.parametrize("scan", [(48, 64), (256, 256)])
def test_shards_add_up_to_the_whole(n_shards, scan):
    import paper_2104_06336_gb300 as P
    w = synth.workload(2, scan_ny=scan[0], scan_nx=scan[1])
    geom = synth.geometry(w)
    d = synth.generate(w, "cuda")
    cands = torch.tensor([[60.0, 10.0, -20.0, 5.0e3, 0.0], [-30.0, 0.0, 15.0, 0.0, 0.0]],
                         dtype=torch.float64)
    full = P.Reconstructor(geom, n_cand=2)
    full.load(d.idx, d.off)
    ph0, v0 = full.reconstruct(cands)
    H = torch.zeros(2, w.scan_ny, w.scan_nx // 2 + 1, dtype=torch.complex64, device="cuda")
    g0 = torch.zeros(2, dtype=torch.float64, device="cuda")
    Pfull = full.info["P"]
    counts_full = full.counts.view(full.info["P_pad"], -1)
    shards = []
    for s in range(n_shards):
        r = P.Reconstructor(geom, n_cand=2, shard=(s, n_shards))
        r.load(d.idx, d.off)
        b, e = r.info["p_begin"], r.info["p_end"]
        assert (b, e) == P.eer4d_shard_range(Pfull, s, n_shards)
        assert r.info["P"] == e - b
        assert torch.equal(r.counts.view(r.info["P_pad"], -1)[:e - b], counts_full[b:e])
        Hs, gs = r.spectrum_partial(cands)
        H += Hs
        g0 += gs
        shards.append(r)
    ph, v = shards[-1].image_from_spectrum(H, g0)
    torch.cuda.synchronize()
    for r in shards:
        assert r.check() == 0
    assert float(g0[1]) == full.info["P_bf"]
    idx_np, off_np = d.numpy()
    G = orc.g_function(orc.densify(idx_np, off_np, geom), geom)
    for c in range(2):
        e_full = rel_l2(ph[c].cpu().numpy(), ph0[c].cpu().numpy())
        phi, V = orc.ssb_phase(G, geom, cands[c].numpy(), "none")
        e_orc = rel_l2(ph[c].cpu().numpy(), phi)
        print(f"shards {n_shards} {scan} cand {c}: vs unsharded {e_full:.2e}, vs oracle {e_orc:.2e}")
        assert e_full <= 2e-6 and e_orc <= 1e-5
        assert abs(float(v[c]) - float(v0[c])) <= 1e-5 * float(v0[c])


def test_shard_partial_refuses_area_norm_and_empty_shards():
    import paper_2104_06336_gb300 as P
    w = synth.workload(1, scan_ny=8, scan_nx=8)
    geom = synth.geometry(w)
    r = P.Reconstructor(geom, norm=P.NORM_AREA, shard=(0, 2))
    with pytest.raises(P.Eer4dError):
        r.spectrum_partial(torch.zeros(5, dtype=torch.float64))
    with pytest.raises(P.Eer4dError):
        P.Plan(geom, shard=(2, 2))
    # a crop wider than the bright field: the outer shards hold dark-field
    # pixels only and are refused (they would add nothing to Eq. 3)
    wide = dict(geom, crop_px=31.0)
    with pytest.raises(P.Eer4dError):
        P.Plan(wide, shard=(0, 8))
