"""The bounds-checking debug build (-DEER4D_CHECKS).

On CPU: the variant compiles for sm_103a and exports the same C ABI as the
release library, and the status word's bounds bit maps to EER4D_EBOUNDS.
On the GPU: the small workloads run through the debug build (a child
process loads it through EER4D_LIBRARY) without a single failed check, and
give the release build's results bit for bit (the checks only guard
accesses)."""

import ctypes
import json
import os
import subprocess
import sys

import numpy as np
import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module")
def checks_lib():
    from paper_2104_06336_gb300.buildlib import build
    return build(checks=True)


def test_debug_build_exports_the_same_abi(checks_lib):
    from paper_2104_06336_gb300 import _lib
    from paper_2104_06336_gb300.buildlib import build
    rel = ctypes.CDLL(build())
    dbg = ctypes.CDLL(checks_lib)
    for name in _lib.EXPORTS:
        assert hasattr(dbg, name) and hasattr(rel, name), name
    st = (ctypes.c_uint32 * 4)(_lib.ST_BOUNDS, 0, 0, 0)
    assert dbg.eer4d_status_code(st) == _lib.EER4D_EBOUNDS
    dbg.eer4d_strerror.restype = ctypes.c_char_p
    assert b"bounds" in dbg.eer4d_strerror(_lib.EER4D_EBOUNDS)


_CHILD = r"""
import json, sys
import numpy as np, torch
sys.path.insert(0, ROOT)
import paper_2104_06336_gb300 as P
import synth
out = {}
for cfg, over, prec in ((1, {}, P.FP32_FFT), (2, dict(scan_ny=48, scan_nx=64), P.FP32_FFT),
                        (1, dict(scan_ny=128, scan_nx=128), P.FP32_FFT),
                        (5, dict(scan_ny=8, scan_nx=1024), P.SPLIT_FP16)):
    w = synth.workload(cfg, **over)
    d = synth.generate(w, "cuda")
    rec = P.Reconstructor(synth.geometry(w), precision=prec, n_cand=2)
    rec.load(d.idx, d.off)
    sums, com, dpc = rec.com_dpc(d.idx, d.off)
    ab = torch.tensor([[40.0, 5.0, -5.0, 1.0e3, 0.0], [-20.0, 0.0, 10.0, 0.0, 0.0]], dtype=torch.float64)
    ph, var = rec.reconstruct(ab)
    V, g, _ = rec.variance_grad(ab[0])
    ph_rot, _ = rec.reconstruct(torch.tensor([10.0, 0, 0, 0, 0.3], dtype=torch.float64))
    torch.cuda.synchronize()
    key = f"{cfg}-{w.scan_ny}x{w.scan_nx}-{prec}"
    out[key] = dict(status=P.status_code(rec.status),
                    G=float(rec.G.double().abs().sum()), counts=float(rec.counts.double().sum()),
                    sums=int(sums.sum()), ph=ph.double().cpu().numpy().ravel()[::97].tolist(),
                    var=var.cpu().numpy().tolist(), g=g.cpu().numpy().tolist(),
                    ph_rot=ph_rot.double().cpu().numpy().ravel()[::89].tolist())
print("RESULT" + json.dumps(out))
"""


def _run(lib):
    env = dict(os.environ)
    if lib:
        env["EER4D_LIBRARY"] = lib
    r = subprocess.run([sys.executable, "-c", "ROOT = %r\n" % ROOT + _CHILD], capture_output=True,
                       text=True, env=env, timeout=900)
    assert r.returncode == 0, r.stderr[-3000:]
    line = [ln for ln in r.stdout.splitlines() if ln.startswith("RESULT")][-1]
    return json.loads(line[len("RESULT"):])


@pytest.mark.gpu
def test_small_workloads_pass_every_bounds_check(checks_lib):
    from paper_2104_06336_gb300.buildlib import build
    rel = _run(build())
    dbg = _run(checks_lib)
    assert rel.keys() == dbg.keys()
    for k in rel:
        assert dbg[k]["status"] == 0, (k, dbg[k]["status"])
        assert rel[k]["status"] == 0
        for f in ("G", "counts", "sums", "ph", "var", "g", "ph_rot"):
            assert dbg[k][f] == rel[k][f], (k, f)
