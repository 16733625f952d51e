"""The C-ABI library builds for sm_103a, loads, and exports every function
include/eer4d.h declares (no GPU needed; nothing here calls into CUDA)."""

import ctypes
import os
import re

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
HEADER = os.path.join(ROOT, "include", "eer4d.h")


def declared_functions():
    text = open(HEADER).read()
    text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
    names = re.findall(r"^\s*(?:const\s+)?[A-Za-z_][A-Za-z0-9_]*\s*\*?\s*([A-Za-z_][A-Za-z0-9_]*)\s*\(",
                       text, flags=re.M)
    return sorted(set(n for n in names if n not in ("if", "defined")))


@pytest.fixture(scope="module")
def lib():
    from paper_2104_06336_gb300.buildlib import build
    path = build()
    return ctypes.CDLL(path)


def test_header_declares_the_paths_entry_points():
    names = declared_functions()
    for n in ("eer_load_csr", "com_dpc", "ssb_accumulate", "ssb_reconstruct", "ssb_grad"):
        assert n in names


def test_library_exports_every_declared_symbol(lib):
    missing = [n for n in declared_functions() if not hasattr(lib, n)]
    assert not missing, missing


def test_binding_covers_the_header(lib):
    from paper_2104_06336_gb300 import _lib
    assert sorted(_lib.EXPORTS) == declared_functions()


def test_host_only_helpers(lib):
    lib.eer4d_strerror.restype = ctypes.c_char_p
    assert lib.eer4d_strerror(0) == b"ok"
    st = (ctypes.c_uint32 * 4)(0x2, 0, 0, 0)
    assert lib.eer4d_status_code(st) == -3
    st = (ctypes.c_uint32 * 4)(0x1, 5, 0, 0)
    assert lib.eer4d_status_code(st) == -2
    st = (ctypes.c_uint32 * 4)(0, 0, 0, 0)
    assert lib.eer4d_status_code(st) == 0


def test_invalid_geometry_rejected_before_any_cuda_call(lib):
    from paper_2104_06336_gb300._lib import Geom
    g = Geom(det_w=64, det_h=64, bin=1, crop_x0=0, crop_y0=0, pw=64, ph=64, dc_u=32, dc_v=32,
             k0_px=20.0, crop_px=10.0, scan_ny=32, scan_nx=32, kpm_y=2.0, kpm_x=2.0, lambda_A=0.02,
             dalpha_rad=1e-3, step_A=0.3, dalpha_raw_rad=1e-3)
    h = ctypes.c_void_p()
    lib.eer4d_plan_create.argtypes = [ctypes.POINTER(Geom), ctypes.c_int, ctypes.c_int,
                                      ctypes.POINTER(ctypes.c_void_p)]
    assert lib.eer4d_plan_create(ctypes.byref(g), 0, 0, ctypes.byref(h)) == -1  # crop < k0
    g.crop_px = 20.0
    g.scan_nx = 33
    assert lib.eer4d_plan_create(ctypes.byref(g), 0, 0, ctypes.byref(h)) == -1  # odd scan
    g.scan_nx = 32
    assert lib.eer4d_plan_create(ctypes.byref(g), 7, 0, ctypes.byref(h)) == -1  # precision


def test_valid_geometries_pass_host_validation(lib):
    """Every workload geometry passes the host checks: plan creation fails only
    for want of a GPU here (ECUDA), or succeeds on a GPU machine."""
    import synth
    from paper_2104_06336_gb300._lib import Geom
    lib.eer4d_plan_create.argtypes = [ctypes.POINTER(Geom), ctypes.c_int, ctypes.c_int,
                                      ctypes.POINTER(ctypes.c_void_p)]
    lib.eer4d_plan_destroy.argtypes = [ctypes.c_void_p]
    for cfg in (1, 2, 3, 4, 5):
        g = synth.geometry(synth.workload(cfg))
        G = Geom(**{k: g[k] for k, _ in Geom._fields_})
        h = ctypes.c_void_p()
        rc = lib.eer4d_plan_create(ctypes.byref(G), 0, 0, ctypes.byref(h))
        assert rc in (0, -6), (cfg, rc)
        if rc == 0:
            lib.eer4d_plan_destroy(h)


@pytest.mark.parametrize("n", [16, 96, 1024])
def test_split_dft_factors_within_bound(lib, n):
    """The tensor-core scan DFT's split factors (Sec. IV: the transform as a
    matrix product; the factors W = exp(-2 pi i k x / n) are split hi + lo
    fp16): every hi + lo is within 2^-22 |w| plus half the fp16 subnormal
    spacing (2^-25) of the FP64 value, hi is the fp16 nearest w, and the phase
    index is the exact integer (k x) mod n (checked at k x far beyond n)."""
    import numpy as np
    from paper_2104_06336_gb300._lib import eer4d_dft_split_factors
    n_k = n // 2 + 1
    hi, lo = eer4d_dft_split_factors(n, n_k)
    k = np.arange(n_k)[:, None]
    x = np.arange(n)[None, :]
    e = (k * x) % n
    w = np.stack([np.cos(2 * np.pi * e / n), -np.sin(2 * np.pi * e / n)], axis=-1)
    h = hi.astype(np.float64)
    err = np.abs(h + lo.astype(np.float64) - w)
    assert np.all(err <= 2.0 ** -22 * np.abs(w) + 2.0 ** -25), err.max()
    # hi is the fp16 nearest w (up to the double -> float -> half rounding of a tie)
    assert np.all(np.abs(h - w) <= np.abs(np.spacing(h.astype(np.float16)).astype(np.float64)) * 0.5
                  + 2.0 ** -25)
    # exact symmetric values
    assert np.all(h[:, 0, 0] == 1.0) and np.all(lo[:, 0, :] == 0.0)
    if n % 4 == 0:
        assert h[1, n // 4, 0] == 0.0 or abs(h[1, n // 4, 0]) < 2.0 ** -24
        assert h[1, n // 4, 1] == -1.0
