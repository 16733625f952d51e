"""ctypes binding of libeer4d.so (include/eer4d.h): argument marshalling only.

Every function here forwards to the C ABI with device pointers taken from
torch CUDA tensors and the current torch stream.  There is no CPU fallback:
if the library is missing or a tensor is not on the GPU, the call raises.
"""

from __future__ import annotations

import ctypes as C
import os

import torch

_PKG = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_PKG, "libeer4d.so")

EER4D_OK, EER4D_EINVAL, EER4D_ERANGE, EER4D_EOFFSETS = 0, -1, -2, -3
EER4D_EOVERFLOW, EER4D_ETIMEOUT, EER4D_ECUDA, EER4D_ENOMEM, EER4D_EORDER = -4, -5, -6, -7, -8
EER4D_ESCRATCH, EER4D_EBOUNDS = -9, -10
STATIC_SCRATCH_BYTES = 8 << 20
ST_RANGE, ST_OFFSETS, ST_OVERFLOW, ST_TIMEOUT, ST_ROTATION = 0x1, 0x2, 0x4, 0x8, 0x10
ST_BOUNDS = 0x20
FP32_FFT, SPLIT_FP16, FP32_FFT_2PASS, FP32_STOCKHAM = 0, 1, 2, 3
NORM_NONE, NORM_AREA = 0, 1

EXPORTS = [
    "eer4d_plan_create", "eer4d_plan_destroy", "eer4d_plan_info", "eer4d_workspace_bytes",
    "eer4d_status_code", "eer4d_strerror", "eer4d_last_error", "eer_load_csr", "com_dpc",
    "ssb_accumulate", "ssb_accumulate_com", "com_dpc_sums", "ssb_reconstruct", "ssb_grad", "ssb_variance_grad", "ssb_trotter_counts",
    "ssb_refocus_step", "eer4d_set_stage_events", "eer4d_launch_count", "ssb_reconstruct_static",
    "eer4d_batched_scratch_bytes", "ssb_reconstruct_batched", "eer_decode_rle",
    "virtual_detectors", "ssb_g_slices", "dpc_iterative", "eer4d_autotune", "eer4d_set_tuning",
    "eer4d_get_tuning", "eer4d_selftest_wait", "eer4d_dft_split_factors",
    "eer4d_shard_range", "eer4d_plan_create_shard", "ssb_spectrum_partial", "ssb_image_from_spectrum",
    "ssb_refocus_step_adam",
]
MAX_SHARDS = 64
MAX_SLICES = 64
MAX_RINGS = 64
MAX_SETS = 32
STAGES = ["validate", "com", "dpc", "scatter", "dft_x", "dft_y", "trotter", "image", "dft_xy"]


class Geom(C.Structure):
    _fields_ = [
        ("det_w", C.c_uint32), ("det_h", C.c_uint32), ("bin", C.c_uint32),
        ("crop_x0", C.c_int32), ("crop_y0", C.c_int32),
        ("pw", C.c_uint32), ("ph", C.c_uint32), ("dc_u", C.c_uint32), ("dc_v", C.c_uint32),
        ("k0_px", C.c_double), ("crop_px", C.c_double),
        ("scan_ny", C.c_uint32), ("scan_nx", C.c_uint32),
        ("kpm_y", C.c_double), ("kpm_x", C.c_double),
        ("lambda_A", C.c_double), ("dalpha_rad", C.c_double), ("step_A", C.c_double),
        ("dalpha_raw_rad", C.c_double),
    ]


class Tuning(C.Structure):
    _fields_ = [("scatter_tf", C.c_int32), ("scatter_ctas_per_sm", C.c_int32),
                ("dft_ctas_per_sm", C.c_int32), ("trotter_ctas_per_sm", C.c_int32),
                ("ms", C.c_float * 3)]

    def as_dict(self) -> dict:
        return {"scatter_tf": self.scatter_tf, "scatter_ctas_per_sm": self.scatter_ctas_per_sm,
                "dft_ctas_per_sm": self.dft_ctas_per_sm,
                "trotter_ctas_per_sm": self.trotter_ctas_per_sm, "ms": list(self.ms)}

    @classmethod
    def from_dict(cls, d: dict) -> "Tuning":
        t = cls()
        t.scatter_tf = int(d.get("scatter_tf", 0))
        t.scatter_ctas_per_sm = int(d.get("scatter_ctas_per_sm", 0))
        t.dft_ctas_per_sm = int(d.get("dft_ctas_per_sm", 0))
        t.trotter_ctas_per_sm = int(d.get("trotter_ctas_per_sm", 0))
        for i, v in enumerate(list(d.get("ms", [0, 0, 0]))[:3]):
            t.ms[i] = float(v)
        return t


class Info(C.Structure):
    _fields_ = [("P", C.c_int32), ("P_pad", C.c_int32), ("P_bf", C.c_int32), ("n_rows", C.c_int32),
                ("nkx", C.c_int32), ("trotter_list_max", C.c_int32), ("p_begin", C.c_int32),
                ("p_end", C.c_int32)]


_lib = None


class Eer4dError(RuntimeError):
    def __init__(self, code: int, where: str):
        lib = load()
        msg = lib.eer4d_strerror(code).decode()
        if code == EER4D_ECUDA:
            msg += ": " + lib.eer4d_last_error().decode()
        super().__init__(f"{where}: {msg} ({code})")
        self.code = code


def load(path: str | None = None):
    """Loads libeer4d.so (building it first is the caller's job: build.build()).
    The environment variable EER4D_LIBRARY names another build of the same
    library (for example the bounds-checking debug build) to load instead."""
    global _lib
    if _lib is not None:
        return _lib
    path = path or os.environ.get("EER4D_LIBRARY") or LIB_PATH
    if not os.path.exists(path):
        raise RuntimeError(f"libeer4d.so not found at {path}; run paper_2104_06336_gb300.build.build()")
    lib = C.CDLL(path)
    P, U32, U64, I32, D, S = C.c_void_p, C.c_uint32, C.c_uint64, C.c_int, C.c_double, C.c_size_t
    sig = {
        "eer4d_plan_create": (I32, [C.POINTER(Geom), I32, I32, C.POINTER(C.c_void_p)]),
        "eer4d_plan_destroy": (None, [P]),
        "eer4d_plan_info": (I32, [P, C.POINTER(Info)]),
        "eer4d_workspace_bytes": (I32, [P, I32, C.POINTER(S), C.POINTER(S), C.POINTER(S)]),
        "eer4d_status_code": (I32, [C.POINTER(U32)]),
        "eer4d_strerror": (C.c_char_p, [I32]),
        "eer4d_last_error": (C.c_char_p, []),
        "eer_load_csr": (I32, [P, P, U64, P, U64, P, P, P, P]),
        "com_dpc": (I32, [P, P, U64, P, P, P, P, P, D, D, D, D, P, P, P]),
        "ssb_accumulate": (I32, [P, P, U64, P, U64, U64, P, P, I32, P, P]),
        "ssb_accumulate_com": (I32, [P, P, U64, P, U64, U64, P, P, I32, P, P, P, P]),
        "com_dpc_sums": (I32, [P, P, P, P, P, D, D, D, D, P, P, P]),
        "ssb_reconstruct": (I32, [P, P, P, I32, P, P, P, P, P]),
        "ssb_grad": (I32, [P, P, P, P, P, P, P, P]),
        "ssb_variance_grad": (I32, [P, P, P, P, P, P, P, P, P]),
        "ssb_trotter_counts": (I32, [P, P, P, P, P]),
        "ssb_refocus_step": (I32, [P, P, P, P, P, P, P, P, P, P]),
        "ssb_refocus_step_adam": (I32, [P, P, P, P, P, P, P, P, P, P, P]),
        "eer4d_set_stage_events": (I32, [P, P, P]),
        "eer4d_launch_count": (C.c_uint64, []),
        "ssb_reconstruct_static": (I32, [P, P, P, P, P, P, P]),
        "eer4d_batched_scratch_bytes": (I32, [P, I32, C.POINTER(S)]),
        "ssb_reconstruct_batched": (I32, [P, P, I32, P, P, P, P, P, P]),
        "eer_decode_rle": (I32, [P, U64, P, U64, P, P, P]),
        "dpc_iterative": (I32, [P, P, D, D, D, I32, I32, P, S, P, P]),
        "eer4d_autotune": (I32, [P, P, U64, P, P, P, P, P, P, P, C.POINTER(Tuning)]),
        "eer4d_set_tuning": (I32, [P, C.POINTER(Tuning)]),
        "eer4d_selftest_wait": (I32, [P, P, P]),
        "eer4d_dft_split_factors": (I32, [I32, I32, P, P]),
        "eer4d_shard_range": (I32, [I32, I32, I32, C.POINTER(I32), C.POINTER(I32)]),
        "eer4d_plan_create_shard": (I32, [C.POINTER(Geom), I32, I32, I32, I32, C.POINTER(C.c_void_p)]),
        "ssb_spectrum_partial": (I32, [P, P, P, I32, P, P, P, P, P]),
        "ssb_image_from_spectrum": (I32, [P, P, P, I32, P, P, P, P]),
        "eer4d_get_tuning": (I32, [P, C.POINTER(Tuning)]),
        "ssb_g_slices": (I32, [P, P, C.POINTER(C.c_int32), I32, P, P]),
        "virtual_detectors": (I32, [P, P, U64, P, U64, C.POINTER(D), I32, P, D, D, P, P, P, P]),
    }
    for name, (res, args) in sig.items():
        f = getattr(lib, name)
        f.restype = res
        f.argtypes = args
    _lib = lib
    return lib


def _ptr(t: torch.Tensor | None, name: str):
    if t is None:
        return None
    if not t.is_cuda:
        raise ValueError(f"{name} must be a CUDA tensor")
    if not t.is_contiguous():
        raise ValueError(f"{name} must be contiguous")
    return C.c_void_p(t.data_ptr())


def _need(t, nbytes: int, name: str, dtype=None):
    """Host-side size (and dtype) check of a device buffer before its pointer
    goes to the library, which cannot see buffer sizes."""
    if t is None:
        return
    if dtype is not None and t.dtype not in (dtype if isinstance(dtype, tuple) else (dtype,)):
        raise TypeError(f"{name} must be {dtype}, got {t.dtype}")
    have = t.numel() * t.element_size()
    if have < nbytes:
        raise ValueError(f"{name} holds {have} bytes, needs {nbytes}")


_U32 = (torch.int32, getattr(torch, "uint32", torch.int32))


def _stream():
    return C.c_void_p(torch.cuda.current_stream().cuda_stream)


def _check(rc: int, where: str):
    if rc != EER4D_OK:
        raise Eer4dError(rc, where)


def status_code(status: torch.Tensor) -> int:
    h = status.detach().to("cpu", torch.int64).numpy().astype("uint32")
    arr = (C.c_uint32 * 4)(*[int(v) for v in h[:4]])
    return load().eer4d_status_code(arr)


class Plan:
    """An eer4d_plan on the current CUDA device (geometry dict with the field
    names of eer4d_geom)."""

    def __init__(self, geom: dict, precision: int = FP32_FFT, norm: int = NORM_NONE,
                 shard: tuple[int, int] | None = None):
        lib = load()
        g = Geom(**{k: geom[k] for k, _ in Geom._fields_})
        h = C.c_void_p()
        if shard is None:
            _check(lib.eer4d_plan_create(C.byref(g), precision, norm, C.byref(h)), "eer4d_plan_create")
        else:
            _check(lib.eer4d_plan_create_shard(C.byref(g), precision, norm, int(shard[0]), int(shard[1]),
                                               C.byref(h)), "eer4d_plan_create_shard")
        self.shard = None if shard is None else (int(shard[0]), int(shard[1]))
        self._h = h
        self.geom = dict(geom)
        self.precision = precision
        self.norm = norm
        info = Info()
        _check(lib.eer4d_plan_info(h, C.byref(info)), "eer4d_plan_info")
        self.info = {k: getattr(info, k) for k, _ in Info._fields_}
        self.Ny = int(geom["scan_ny"])
        self.F = int(geom["scan_ny"]) * int(geom["scan_nx"])
        self.WH = int(geom["det_w"]) * int(geom["det_h"])
        self.G_bytes = 8 * self.info["nkx"] * self.info["P_pad"] * int(geom["scan_ny"])

    @property
    def handle(self):
        return self._h

    def workspace_bytes(self, n_cand: int = 1):
        c, g, s = C.c_size_t(), C.c_size_t(), C.c_size_t()
        _check(load().eer4d_workspace_bytes(self._h, n_cand, C.byref(c), C.byref(g), C.byref(s)),
               "eer4d_workspace_bytes")
        return c.value, g.value, s.value

    def close(self):
        if getattr(self, "_h", None) is not None and self._h.value:
            load().eer4d_plan_destroy(self._h)
            self._h = C.c_void_p()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


# ---- entry points, same names as the C ABI ---------------------------------
def eer_load_csr(plan: Plan, idx, off, pacbed=None, totals=None, status=None):
    _need(idx, 0, "idx", _U32)
    _need(off, 16, "off", torch.int64)
    _need(pacbed, 8 * plan.WH, "pacbed", torch.int64)
    _need(totals, 24, "totals", torch.int64)
    _need(status, 16, "status")
    _check(load().eer_load_csr(plan.handle, _ptr(idx, "idx"), idx.numel(), _ptr(off, "off"),
                               off.numel() - 1, _ptr(pacbed, "pacbed"), _ptr(totals, "totals"),
                               _ptr(status, "status"), _stream()), "eer_load_csr")


def com_dpc(plan: Plan, idx, off, sums, com, phase=None, totals=None, cx=0.0, cy=0.0, lam1=0.0,
            lam2=0.0, scratch=None, status=None):
    F = plan.F
    if off.numel() != F + 1:
        raise ValueError("com_dpc takes the whole scan: off must have scan_ny*scan_nx + 1 entries")
    _need(idx, 0, "idx", _U32)
    _need(sums, 24 * F, "sums", torch.int64)
    _need(com, 8 * F, "com", torch.float32)
    _need(phase, 4 * F, "phase", torch.float32)
    _need(totals, 24, "totals", torch.int64)
    if phase is not None:
        if scratch is None:
            raise ValueError("com_dpc needs scratch (8 bytes per frame) for the phase")
        _need(scratch, 8 * F, "scratch")
    _need(status, 16, "status")
    _check(load().com_dpc(plan.handle, _ptr(idx, "idx"), idx.numel(), _ptr(off, "off"),
                          _ptr(sums, "sums"), _ptr(com, "com"), _ptr(phase, "phase"),
                          _ptr(totals, "totals"), float(cx), float(cy), float(lam1), float(lam2),
                          _ptr(scratch, "scratch"), _ptr(status, "status"), _stream()), "com_dpc")


def ssb_accumulate(plan: Plan, idx, off, first_frame: int, counts, G, is_last: bool, status=None):
    _need(idx, 0, "idx", _U32)
    _need(off, 8, "off", torch.int64)
    _need(counts, plan.workspace_bytes(1)[0], "counts (workspace)")
    _need(G, plan.G_bytes, "G")
    _need(status, 16, "status")
    _check(load().ssb_accumulate(plan.handle, _ptr(idx, "idx"), idx.numel(), _ptr(off, "off"),
                                 int(first_frame), off.numel() - 1, _ptr(counts, "counts"),
                                 _ptr(G, "G"), int(bool(is_last)), _ptr(status, "status"),
                                 _stream()), "ssb_accumulate")


def ssb_accumulate_com(plan: Plan, idx, off, first_frame: int, counts, G, is_last: bool, sums,
                       totals, status=None):
    """ssb_accumulate that also forms the per-frame COM sums [3][F] of its
    frames and adds them to totals [3] in the same pass over the events."""
    _need(idx, 0, "idx", _U32)
    _need(off, 8, "off", torch.int64)
    _need(counts, plan.workspace_bytes(1)[0], "counts (workspace)")
    _need(G, plan.G_bytes, "G")
    if sums is None or totals is None:
        raise ValueError("ssb_accumulate_com needs sums and totals")
    _need(sums, 24 * plan.F, "sums", torch.int64)
    _need(totals, 24, "totals", torch.int64)
    _need(status, 16, "status")
    _check(load().ssb_accumulate_com(plan.handle, _ptr(idx, "idx"), idx.numel(), _ptr(off, "off"),
                                     int(first_frame), off.numel() - 1, _ptr(counts, "counts"),
                                     _ptr(G, "G"), int(bool(is_last)), _ptr(sums, "sums"),
                                     _ptr(totals, "totals"), _ptr(status, "status"), _stream()),
           "ssb_accumulate_com")


def com_dpc_sums(plan: Plan, sums, com, phase=None, totals=None, cx=0.0, cy=0.0, lam1=0.0,
                 lam2=0.0, scratch=None, status=None):
    """com_dpc from per-frame sums [3][F] already formed (ssb_accumulate_com)."""
    F = plan.F
    if sums is None:
        raise ValueError("com_dpc_sums needs sums")
    _need(sums, 24 * F, "sums", torch.int64)
    _need(com, 8 * F, "com", torch.float32)
    _need(phase, 4 * F, "phase", torch.float32)
    _need(totals, 24, "totals", torch.int64)
    if phase is not None:
        if scratch is None:
            raise ValueError("com_dpc_sums needs scratch (8 bytes per frame) for the phase")
        _need(scratch, 8 * F, "scratch")
    _need(status, 16, "status")
    _check(load().com_dpc_sums(plan.handle, _ptr(sums, "sums"), _ptr(com, "com"),
                               _ptr(phase, "phase"), _ptr(totals, "totals"), float(cx), float(cy),
                               float(lam1), float(lam2), _ptr(scratch, "scratch"),
                               _ptr(status, "status"), _stream()), "com_dpc_sums")


def ssb_reconstruct(plan: Plan, G, aberr, scratch, phase=None, var=None, status=None):
    n = aberr.numel() // 5
    if n < 1 or aberr.numel() != 5 * n:
        raise ValueError("aberr holds [n][5] float64 values")
    _need(aberr, 40 * n, "aberr", torch.float64)
    _need(G, plan.G_bytes, "G")
    _need(scratch, plan.workspace_bytes(n)[2], "scratch")
    _need(phase, 4 * n * plan.F, "phase", torch.float32)
    _need(var, 8 * n, "var", torch.float64)
    _need(status, 16, "status")
    _check(load().ssb_reconstruct(plan.handle, _ptr(G, "G"), _ptr(aberr, "aberr"), n,
                                  _ptr(scratch, "scratch"), _ptr(phase, "phase"), _ptr(var, "var"),
                                  _ptr(status, "status"), _stream()), "ssb_reconstruct")


def ssb_grad(plan: Plan, G, aberr, grad_phase, grad, scratch, status=None):
    _need(G, plan.G_bytes, "G")
    _need(aberr, 40, "aberr", torch.float64)
    _need(grad_phase, 4 * plan.F, "grad_phase", torch.float32)
    _need(grad, 40, "grad", torch.float64)
    _need(scratch, plan.workspace_bytes(1)[2], "scratch")
    _need(status, 16, "status")
    _check(load().ssb_grad(plan.handle, _ptr(G, "G"), _ptr(aberr, "aberr"),
                           _ptr(grad_phase, "grad_phase"), _ptr(grad, "grad"),
                           _ptr(scratch, "scratch"), _ptr(status, "status"), _stream()), "ssb_grad")


def ssb_variance_grad(plan: Plan, G, aberr, scratch, var, grad, phase=None, status=None):
    _need(G, plan.G_bytes, "G")
    _need(aberr, 40, "aberr", torch.float64)
    _need(scratch, plan.workspace_bytes(1)[2], "scratch")
    _need(var, 8, "var", torch.float64)
    _need(grad, 40, "grad", torch.float64)
    _need(phase, 4 * plan.F, "phase", torch.float32)
    _need(status, 16, "status")
    _check(load().ssb_variance_grad(plan.handle, _ptr(G, "G"), _ptr(aberr, "aberr"),
                                    _ptr(scratch, "scratch"), _ptr(phase, "phase"), _ptr(var, "var"),
                                    _ptr(grad, "grad"), _ptr(status, "status"), _stream()),
           "ssb_variance_grad")


def ssb_trotter_counts(plan: Plan, aberr, count, scratch):
    _need(aberr, 40, "aberr", torch.float64)
    _need(count, 4 * plan.F, "count", torch.int32)
    _need(scratch, plan.workspace_bytes(1)[2], "scratch")
    _check(load().ssb_trotter_counts(plan.handle, _ptr(aberr, "aberr"), _ptr(count, "count"),
                                     _ptr(scratch, "scratch"), _stream()), "ssb_trotter_counts")


def ssb_refocus_step(plan: Plan, G, aberr, step, scratch, var, grad, phase=None, status=None):
    _need(G, plan.G_bytes, "G")
    _need(aberr, 40, "aberr", torch.float64)
    _need(step, 40, "step", torch.float64)
    _need(scratch, plan.workspace_bytes(1)[2], "scratch")
    _need(var, 8, "var", torch.float64)
    _need(grad, 40, "grad", torch.float64)
    _need(phase, 4 * plan.F, "phase", torch.float32)
    _need(status, 16, "status")
    _check(load().ssb_refocus_step(plan.handle, _ptr(G, "G"), _ptr(aberr, "aberr"), _ptr(step, "step"),
                                   _ptr(scratch, "scratch"), _ptr(phase, "phase"), _ptr(var, "var"),
                                   _ptr(grad, "grad"), _ptr(status, "status"), _stream()),
           "ssb_refocus_step")


def ssb_refocus_step_adam(plan: Plan, G, aberr, rate, state, scratch, var, grad, phase=None,
                          status=None):
    """ssb_refocus_step with a device-side Adam update (rate: lr[5] + scale[5];
    state: m1[5], m2[5], t, zeroed before the first step)."""
    _need(G, plan.G_bytes, "G")
    _need(aberr, 40, "aberr", torch.float64)
    _need(rate, 80, "rate", torch.float64)
    _need(state, 88, "state", torch.float64)
    _need(scratch, plan.workspace_bytes(1)[2], "scratch")
    _need(var, 8, "var", torch.float64)
    _need(grad, 40, "grad", torch.float64)
    _need(phase, 4 * plan.F, "phase", torch.float32)
    _need(status, 16, "status")
    _check(load().ssb_refocus_step_adam(plan.handle, _ptr(G, "G"), _ptr(aberr, "aberr"),
                                        _ptr(rate, "rate"), _ptr(state, "state"),
                                        _ptr(scratch, "scratch"), _ptr(phase, "phase"),
                                        _ptr(var, "var"), _ptr(grad, "grad"),
                                        _ptr(status, "status"), _stream()), "ssb_refocus_step_adam")


def eer4d_set_stage_events(plan: Plan, starts=None, stops=None):
    """starts/stops: lists of len(STAGES) torch.cuda.Event (or None) or None to clear."""
    if starts is None:
        _check(load().eer4d_set_stage_events(plan.handle, None, None), "eer4d_set_stage_events")
        return
    arr_t = C.c_void_p * len(STAGES)
    a = arr_t(*[C.c_void_p(e.cuda_event if e is not None else 0) for e in starts])
    b = arr_t(*[C.c_void_p(e.cuda_event if e is not None else 0) for e in stops])
    _check(load().eer4d_set_stage_events(plan.handle, a, b), "eer4d_set_stage_events")


def eer4d_launch_count() -> int:
    return int(load().eer4d_launch_count())


def ssb_reconstruct_static(plan: Plan, G, aberr, phase=None, var=None, status=None):
    """One-candidate ssb_reconstruct whose working memory is the library's
    static device array (no scratch argument, no allocation)."""
    _need(G, plan.G_bytes, "G")
    _need(aberr, 40, "aberr", torch.float64)
    _need(phase, 4 * plan.F, "phase", torch.float32)
    _need(var, 8, "var", torch.float64)
    _need(status, 16, "status")
    _check(load().ssb_reconstruct_static(plan.handle, _ptr(G, "G"), _ptr(aberr, "aberr"),
                                         _ptr(phase, "phase"), _ptr(var, "var"),
                                         _ptr(status, "status"), _stream()), "ssb_reconstruct_static")


def eer4d_shard_range(P: int, shard: int, n_shards: int) -> tuple[int, int]:
    """Kept pixels [begin, end) of shard `shard` of `n_shards` (host only)."""
    b, e = C.c_int(), C.c_int()
    _check(load().eer4d_shard_range(int(P), int(shard), int(n_shards), C.byref(b), C.byref(e)),
           "eer4d_shard_range")
    return b.value, e.value


def ssb_spectrum_partial(plan: Plan, G, aberr, scratch, H, g0, status=None):
    """This plan's share of the spectrum: H complex64 [n][Ny][Nx/2+1] (as
    float32 pairs or complex64) and g0 float64 [2]; see the header."""
    n = aberr.numel() // 5
    if n < 1 or aberr.numel() != 5 * n:
        raise ValueError("aberr holds [n][5] float64 values")
    _need(aberr, 40 * n, "aberr", torch.float64)
    _need(G, plan.G_bytes, "G")
    _need(scratch, plan.workspace_bytes(n)[2], "scratch")
    _need(H, 8 * n * plan.Ny * plan.info["nkx"], "H", (torch.float32, torch.complex64))
    _need(g0, 16, "g0", torch.float64)
    _need(status, 16, "status")
    _check(load().ssb_spectrum_partial(plan.handle, _ptr(G, "G"), _ptr(aberr, "aberr"), n,
                                       _ptr(scratch, "scratch"), _ptr(H, "H"), _ptr(g0, "g0"),
                                       _ptr(status, "status"), _stream()), "ssb_spectrum_partial")


def ssb_image_from_spectrum(plan: Plan, H, g0, n_cand: int, scratch, phase=None, var=None):
    """Phase images and variances from the summed shares of every shard."""
    _need(H, 8 * n_cand * plan.Ny * plan.info["nkx"], "H", (torch.float32, torch.complex64))
    _need(g0, 16, "g0", torch.float64)
    _need(scratch, plan.workspace_bytes(n_cand)[2], "scratch")
    _need(phase, 4 * n_cand * plan.F, "phase", torch.float32)
    _need(var, 8 * n_cand, "var", torch.float64)
    _check(load().ssb_image_from_spectrum(plan.handle, _ptr(H, "H"), _ptr(g0, "g0"), int(n_cand),
                                          _ptr(scratch, "scratch"), _ptr(phase, "phase"),
                                          _ptr(var, "var"), _stream()), "ssb_image_from_spectrum")


def _handles(plans):
    arr = (C.c_void_p * len(plans))(*[p.handle for p in plans])
    return arr


def batched_scratch_bytes(plans) -> int:
    n = C.c_size_t(0)
    _check(load().eer4d_batched_scratch_bytes(_handles(plans), len(plans), C.byref(n)),
           "eer4d_batched_scratch_bytes")
    return int(n.value)


def ssb_reconstruct_batched(plans, Gs, aberr, scratch, phases=None, var=None, status=None):
    """Datasets of one detector geometry in one trotter launch: plans and Gs
    are lists (one per dataset), aberr [n][5] float64 on the device, phases a
    list of [Ny_i][Nx_i] float32 tensors (or None entries) or None."""
    n = len(plans)
    if len(Gs) != n or aberr.numel() != 5 * n:
        raise ValueError("one G and one aberration row per plan")
    _need(aberr, 40 * n, "aberr", torch.float64)
    for pl, g in zip(plans, Gs):
        _need(g, pl.G_bytes, "G")
    _need(scratch, batched_scratch_bytes(plans), "scratch")
    _need(var, 8 * n, "var", torch.float64)
    _need(status, 16, "status")
    if phases is not None:
        for pl, ph in zip(plans, phases):
            _need(ph, 4 * pl.F, "phase", torch.float32)
    g_arr = (C.c_void_p * n)(*[_ptr(g, "G").value for g in Gs])
    ph_arr = None
    if phases is not None:
        if len(phases) != n:
            raise ValueError("one phase output (or None) per plan")
        ph_arr = (C.c_void_p * n)(*[(_ptr(ph, "phase").value if ph is not None else None)
                                    for ph in phases])
    _check(load().ssb_reconstruct_batched(_handles(plans), g_arr, n, _ptr(aberr, "aberr"),
                                          _ptr(scratch, "scratch"), ph_arr, _ptr(var, "var"),
                                          _ptr(status, "status"), _stream()),
           "ssb_reconstruct_batched")


def eer_decode_rle(runs, off, idx=None, status=None):
    """Run-length-encoded frames (uint32 runs, uint64 CSR offsets) to linear
    indices; returns idx (a new int32 tensor of uint32 values unless given;
    ``idx=runs`` decodes in place)."""
    if idx is None:
        idx = torch.empty_like(runs)
    _need(runs, 0, "runs", _U32)
    _need(idx, 4 * runs.numel(), "idx", _U32)
    _need(off, 8, "off", torch.int64)
    _need(status, 16, "status")
    _check(load().eer_decode_rle(_ptr(runs, "runs"), runs.numel(), _ptr(off, "off"),
                                 off.numel() - 1, _ptr(idx, "idx"), _ptr(status, "status"),
                                 _stream()), "eer_decode_rle")
    return idx


def virtual_detectors(plan: Plan, idx, off, radii, out, scratch, totals=None, cx=0.0, cy=0.0,
                      status=None):
    """Per-frame event counts in the annuli radii[j] <= r < radii[j+1] (raw px)
    about the PACBED centre (totals) or (cx, cy); out int32 [n_rings][F]."""
    r = [float(x) for x in radii]
    arr = (C.c_double * len(r))(*r)
    _need(out, 4 * (len(r) - 1) * plan.F, "out", torch.int32)
    _need(scratch, plan.WH, "scratch")
    _need(status, 16, "status")
    _check(load().virtual_detectors(plan.handle, _ptr(idx, "idx"), idx.numel(), _ptr(off, "off"),
                                    off.numel() - 1, arr, len(r) - 1, _ptr(totals, "totals"),
                                    float(cx), float(cy), _ptr(scratch, "scratch"),
                                    _ptr(out, "out"), _ptr(status, "status"), _stream()),
           "virtual_detectors")


def ssb_g_slices(plan: Plan, G, bins, out):
    """G(k, K) at the DFT bins [(m_y, m_x), ...] on the binned detector window:
    out complex64 [n][ph][pw] (as a float32 [n][ph][pw][2] or complex tensor)."""
    flat = [int(v) for b in bins for v in b]
    arr = (C.c_int32 * len(flat))(*flat)
    _need(G, plan.G_bytes, "G")
    _need(out, 8 * len(bins) * int(plan.geom["ph"]) * int(plan.geom["pw"]), "out")
    _check(load().ssb_g_slices(plan.handle, _ptr(G, "G"), arr, len(bins), _ptr(out, "out"),
                               _stream()), "ssb_g_slices")


def dpc_iterative(plan: Plan, com, phase, scratch, n_iter: int, mu: float = 0.5, lam1: float = 0.0,
                  lam2: float = 0.0, pad: int = 2):
    """Iterative regularised DPC from COM maps (float32 [2][F], raw px)."""
    _need(com, 8 * plan.F, "com", torch.float32)
    _need(phase, 4 * plan.F, "phase", torch.float32)
    _check(load().dpc_iterative(plan.handle, _ptr(com, "com"), float(lam1), float(lam2), float(mu),
                                int(n_iter), int(pad), _ptr(scratch, "scratch"),
                                scratch.numel() * scratch.element_size(), _ptr(phase, "phase"),
                                _stream()), "dpc_iterative")


def eer4d_autotune(plan: Plan, idx, off, work, G, scratch, aberr, status=None) -> dict:
    """Times the launch-shape candidates on this data and keeps the fastest in
    the plan (synchronises the current stream).  Returns the choice."""
    t = Tuning()
    _need(work, plan.workspace_bytes(1)[0], "work")
    _need(G, plan.G_bytes, "G")
    _need(scratch, plan.workspace_bytes(1)[2], "scratch")
    _need(aberr, 40, "aberr", torch.float64)
    _need(status, 16, "status")
    _check(load().eer4d_autotune(plan.handle, _ptr(idx, "idx"), idx.numel(), _ptr(off, "off"),
                                 _ptr(work, "work"), _ptr(G, "G"), _ptr(scratch, "scratch"),
                                 _ptr(aberr, "aberr"), _ptr(status, "status"), _stream(),
                                 C.byref(t)), "eer4d_autotune")
    return t.as_dict()


def eer4d_set_tuning(plan: Plan, tuning: dict):
    t = Tuning.from_dict(tuning)
    _check(load().eer4d_set_tuning(plan.handle, C.byref(t)), "eer4d_set_tuning")


def eer4d_get_tuning(plan: Plan) -> dict:
    t = Tuning()
    _check(load().eer4d_get_tuning(plan.handle, C.byref(t)), "eer4d_get_tuning")
    return t.as_dict()


def eer4d_selftest_wait(scratch, status):
    """Runs the library's bounded device wait against a counter that nothing
    increments (see the header): status then holds EER4D_ST_TIMEOUT."""
    _need(scratch, 8, "scratch")
    _need(status, 16, "status")
    _check(load().eer4d_selftest_wait(_ptr(scratch, "scratch"), _ptr(status, "status"), _stream()),
           "eer4d_selftest_wait")


def eer4d_dft_split_factors(n: int, n_k: int):
    """The split hi + lo fp16 DFT factors of the tensor-core scan transform
    (host only): two float16 arrays [n_k][n][2] (cos, -sin)."""
    import numpy as np
    hi = np.zeros((n_k, n, 2), dtype=np.uint16)
    lo = np.zeros_like(hi)
    _check(load().eer4d_dft_split_factors(n, n_k, C.c_void_p(hi.ctypes.data), C.c_void_p(lo.ctypes.data)),
           "eer4d_dft_split_factors")
    return hi.view(np.float16), lo.view(np.float16)
