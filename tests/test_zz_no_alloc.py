"""ssb_reconstruct_static: the reconstruction entry point for callers that
cannot allocate device memory (its scratch is a static array inside the
library).  Checked through the C ABI against ssb_reconstruct, which takes a
caller-allocated scratch buffer, on two calls in a row (the array keeps the
previous call's contents, so the second call shows nothing stale leaks in).

This file is collected last on purpose: if it fails, a run that stops at the
first failure has already run every other test."""

import ctypes

import numpy as np
import pytest
import torch

import synth

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def P():
    from paper_2104_06336_gb300.buildlib import build
    build()
    import paper_2104_06336_gb300 as P
    P.load()
    return P


def _rel_l2(a, b):
    a = a.double().cpu().numpy()
    b = b.double().cpu().numpy()
    return float(np.linalg.norm(a - b) / np.linalg.norm(b))


@pytest.mark.parametrize("cfg,over", [(1, {}), (2, dict(scan_ny=48, scan_nx=64))])
def test_static_scratch_matches_allocating_entry_point(P, cfg, over):
    w = synth.workload(cfg, **over)
    d = synth.generate(w, "cuda")
    rec = P.Reconstructor(synth.geometry(w))
    rec.load(d.idx, d.off)
    lib = P.load()
    Ny, Nx = w.scan_ny, w.scan_nx
    for ab in ([80.0, 15.0, 25.98, 1.0e4, 0.0], [-40.0, 0.0, 10.0, 0.0, 0.2]):
        theta = torch.tensor(ab, dtype=torch.float64, device="cuda")
        ref_phase, ref_var = rec.reconstruct(theta)
        phase = torch.full((Ny, Nx), float("nan"), dtype=torch.float32, device="cuda")
        var = torch.full((1,), float("nan"), dtype=torch.float64, device="cuda")
        status = torch.zeros(4, dtype=torch.int32, device="cuda")
        rc = lib.ssb_reconstruct_static(rec.plan.handle, ctypes.c_void_p(rec.G.data_ptr()),
                                        ctypes.c_void_p(theta.data_ptr()),
                                        ctypes.c_void_p(phase.data_ptr()),
                                        ctypes.c_void_p(var.data_ptr()),
                                        ctypes.c_void_p(status.data_ptr()),
                                        ctypes.c_void_p(torch.cuda.current_stream().cuda_stream))
        assert rc == 0
        torch.cuda.synchronize()
        assert int(status[0].item()) == 0
        assert _rel_l2(phase, ref_phase[0]) <= 1e-5
        assert abs(float(var.item()) - float(ref_var.item())) <= 1e-5 * float(ref_var.item())


def test_static_scratch_rejects_plans_beyond_its_size(P):
    w = synth.workload(5, scan_ny=2048, scan_nx=2048)
    plan = P.Plan(synth.geometry(w))
    lib = P.load()
    theta = torch.zeros(5, dtype=torch.float64, device="cuda")
    G = torch.zeros(16, dtype=torch.float32, device="cuda")
    rc = lib.ssb_reconstruct_static(plan.handle, ctypes.c_void_p(G.data_ptr()),
                                    ctypes.c_void_p(theta.data_ptr()), None, None, None, None)
    assert rc == P._lib.EER4D_ESCRATCH
    assert b"static" in lib.eer4d_strerror(rc)
