"""Device buffers around one plan: the user-facing path EER -> COM/DPC and SSB.

PyTorch only allocates device memory and supplies the stream; every step runs
in libeer4d's kernels through the C ABI (``_lib``).
"""

from __future__ import annotations

import torch

from . import _lib as L


def as_u32(idx: torch.Tensor) -> torch.Tensor:
    """int32 or uint32 storage of raw linear indices, as the C ABI reads them."""
    if idx.dtype not in (torch.int32, getattr(torch, "uint32", torch.int32)):
        raise TypeError("event indices must be 32-bit integers (uint32 values)")
    return idx.contiguous()


class Reconstructor:
    """Plan + workspace for one scan geometry on one GPU.

    ``geom`` uses the field names of eer4d_geom.  Buffers: ``work`` (the
    accumulation workspace of ssb_accumulate; ``counts`` is its fp16
    [P_pad][F] head), G complex64 [nkx][P_pad][Ny], scratch bytes, status
    int32[4] (zeroed at construction; see ``check``)."""

    def __init__(self, geom: dict, precision: int = L.FP32_FFT, norm: int = L.NORM_NONE,
                 n_cand: int = 1, device=None, alloc_counts: bool = True,
                 shard: tuple[int, int] | None = None):
        if not torch.cuda.is_available():
            raise RuntimeError("Reconstructor needs a CUDA GPU; there is no CPU path")
        self.device = torch.device(device or "cuda")
        with torch.cuda.device(self.device):
            self.plan = L.Plan(geom, precision, norm, shard=shard)
            cb, gb, sb = self.plan.workspace_bytes(n_cand)
            self.n_cand = n_cand
            self.work = torch.empty(cb, dtype=torch.uint8, device=self.device) if alloc_counts else None
            info = self.plan.info
            n_counts = info["P_pad"] * geom["scan_ny"] * geom["scan_nx"]
            self.counts = self.work[:2 * n_counts].view(torch.float16) if alloc_counts else None
            self.G = torch.empty(gb // 4, dtype=torch.float32, device=self.device)
            self.scratch = torch.empty(sb, dtype=torch.uint8, device=self.device)
            self.status = torch.zeros(4, dtype=torch.int32, device=self.device)
            self.totals = torch.zeros(3, dtype=torch.int64, device=self.device)
        self.geom = dict(geom)
        self.Ny, self.Nx = geom["scan_ny"], geom["scan_nx"]
        self.F = self.Ny * self.Nx
        self.info = self.plan.info

    # -- ingest ---------------------------------------------------------------
    def load(self, idx: torch.Tensor, off: torch.Tensor, chunk_frames: int | None = None,
             pacbed: torch.Tensor | None = None):
        """Validates the CSR (totals for the PACBED centre) and builds G
        (ssb_accumulate over chunks of ``chunk_frames`` frames)."""
        idx = as_u32(idx)
        off = off.contiguous()
        self.totals.zero_()
        L.eer_load_csr(self.plan, idx, off, pacbed=pacbed, totals=self.totals, status=self.status)
        self.accumulate(idx, off, chunk_frames)

    def accumulate(self, idx: torch.Tensor, off: torch.Tensor, chunk_frames: int | None = None):
        F = self.F
        step = F if chunk_frames is None else int(chunk_frames)
        for f0 in range(0, F, step):
            f1 = min(F, f0 + step)
            L.ssb_accumulate(self.plan, idx, off[f0:f1 + 1], f0, self.work, self.G, f1 == F,
                             status=self.status)

    def com_dpc(self, idx: torch.Tensor, off: torch.Tensor, lam1=0.0, lam2=0.0, use_totals=True,
                cx=0.0, cy=0.0, phase=True):
        """Per-frame COM sums, COM maps and the Fourier-integrated DPC phase."""
        sums = torch.empty(3, self.F, dtype=torch.int64, device=self.device)
        com = torch.empty(2, self.F, dtype=torch.float32, device=self.device)
        ph = torch.empty(self.Ny, self.Nx, dtype=torch.float32, device=self.device) if phase else None
        L.com_dpc(self.plan, as_u32(idx), off.contiguous(), sums, com, ph,
                  totals=self.totals if use_totals else None, cx=cx, cy=cy, lam1=lam1, lam2=lam2,
                  scratch=self.scratch, status=self.status)
        return sums, com, ph

    def dpc_iterative(self, com: torch.Tensor, n_iter: int, mu: float = 0.5, lam1: float = 0.0,
                      lam2: float = 0.0, pad: int = 2) -> torch.Tensor:
        """Iterative regularised DPC phase [Ny][Nx] from COM maps [2][F]."""
        scr = torch.empty(24 * pad * pad * self.F, dtype=torch.uint8, device=self.device)
        ph = torch.empty(self.Ny, self.Nx, dtype=torch.float32, device=self.device)
        L.dpc_iterative(self.plan, com.to(torch.float32).contiguous(), ph, scr, n_iter, mu=mu,
                        lam1=lam1, lam2=lam2, pad=pad)
        return ph

    def virtual_detectors(self, idx: torch.Tensor, off: torch.Tensor, radii, use_totals=True,
                          cx=0.0, cy=0.0) -> torch.Tensor:
        """Per-frame event counts in annuli radii[j] <= r < radii[j+1] (raw px)
        about the PACBED centre: int32 [n_rings][Ny][Nx] images."""
        out = torch.empty(len(radii) - 1, self.F, dtype=torch.int32, device=self.device)
        L.virtual_detectors(self.plan, as_u32(idx), off.contiguous(), radii, out, self.scratch,
                            totals=self.totals if use_totals else None, cx=cx, cy=cy,
                            status=self.status)
        return out.view(-1, self.Ny, self.Nx)

    # -- SSB -----------------------------------------------------------------
    def reconstruct(self, aberr: torch.Tensor, phase: bool = True):
        """SSB phase images and variances for aberration candidates [n][5]."""
        ab = aberr.to(self.device, torch.float64).reshape(-1, 5).contiguous()
        n = ab.shape[0]
        if n > self.n_cand:
            raise ValueError(f"{n} candidates but workspace sized for {self.n_cand}")
        ph = torch.empty(n, self.Ny, self.Nx, dtype=torch.float32, device=self.device) if phase else None
        var = torch.empty(n, dtype=torch.float64, device=self.device)
        L.ssb_reconstruct(self.plan, self.G, ab, self.scratch, ph, var, status=self.status)
        return ph, var

    def spectrum_partial(self, aberr: torch.Tensor):
        """This plan's share of the spectrum for candidates [n][5]: H complex64
        [n][Ny][Nx/2+1] and g0 float64 [2] (summable over pixel shards)."""
        ab = aberr.to(self.device, torch.float64).reshape(-1, 5).contiguous()
        n = ab.shape[0]
        if n > self.n_cand:
            raise ValueError(f"{n} candidates but workspace sized for {self.n_cand}")
        H = torch.empty(n, self.Ny, self.info["nkx"], dtype=torch.complex64, device=self.device)
        g0 = torch.empty(2, dtype=torch.float64, device=self.device)
        L.ssb_spectrum_partial(self.plan, self.G, ab, self.scratch, H, g0, status=self.status)
        return H, g0

    def image_from_spectrum(self, H: torch.Tensor, g0: torch.Tensor, phase: bool = True):
        """Phase images and variances from shares summed over every shard."""
        n = H.shape[0]
        if n > self.n_cand:
            raise ValueError(f"{n} candidates but workspace sized for {self.n_cand}")
        ph = torch.empty(n, self.Ny, self.Nx, dtype=torch.float32, device=self.device) if phase else None
        var = torch.empty(n, dtype=torch.float64, device=self.device)
        L.ssb_image_from_spectrum(self.plan, H.contiguous(), g0.contiguous(), n, self.scratch, ph, var)
        return ph, var

    def grad(self, aberr: torch.Tensor, grad_phase: torch.Tensor):
        ab = aberr.to(self.device, torch.float64).reshape(5).contiguous()
        g = torch.empty(5, dtype=torch.float64, device=self.device)
        L.ssb_grad(self.plan, self.G, ab, grad_phase.to(torch.float32).contiguous(), g, self.scratch,
                   status=self.status)
        return g

    def variance_grad(self, aberr: torch.Tensor, phase: bool = False):
        ab = aberr.to(self.device, torch.float64).reshape(5).contiguous()
        var = torch.empty(1, dtype=torch.float64, device=self.device)
        g = torch.empty(5, dtype=torch.float64, device=self.device)
        ph = torch.empty(self.Ny, self.Nx, dtype=torch.float32, device=self.device) if phase else None
        L.ssb_variance_grad(self.plan, self.G, ab, self.scratch, var, g, ph, status=self.status)
        return var, g, ph

    def trotter_counts(self, rot: float = 0.0):
        ab = torch.zeros(5, dtype=torch.float64, device=self.device)
        ab[4] = rot
        cnt = torch.empty(self.Ny, self.Nx, dtype=torch.int32, device=self.device)
        L.ssb_trotter_counts(self.plan, ab, cnt, self.scratch)
        return cnt

    def g_slices(self, bins) -> torch.Tensor:
        """G(k, K) at DFT bins [(m_y, m_x), ...] on the binned detector window:
        complex64 [n][ph][pw] (zero outside the crop)."""
        out = torch.empty(len(bins), self.geom["ph"], self.geom["pw"], dtype=torch.complex64,
                          device=self.device)
        L.ssb_g_slices(self.plan, self.G, bins, out)
        return out

    # -- views -----------------------------------------------------------------
    def G_complex(self) -> torch.Tensor:
        """G as complex64 [nkx][P_pad][Ny] (K_x >= 0 half, K_y innermost)."""
        nkx, P_pad = self.info["nkx"], self.info["P_pad"]
        return torch.view_as_complex(self.G.view(nkx, P_pad, self.Ny, 2))

    def check(self, raise_on_error: bool = True) -> int:
        code = L.status_code(self.status)
        if code != L.EER4D_OK and raise_on_error:
            raise L.Eer4dError(code, "device status")
        return code


def reconstruct_batched(recs, aberr: torch.Tensor, phase: bool = True, scratch=None):
    """SSB phase images and variances of several datasets (one Reconstructor
    each, same detector geometry, any scan sizes) in one trotter launch.
    aberr: [n][5], row i for dataset i.  Returns (list of phases or None, var)."""
    if not recs:
        raise ValueError("no datasets")
    dev = recs[0].device
    ab = aberr.to(dev, torch.float64).reshape(len(recs), 5).contiguous()
    plans = [r.plan for r in recs]
    if scratch is None:
        scratch = torch.empty(L.batched_scratch_bytes(plans), dtype=torch.uint8, device=dev)
    ph = [torch.empty(r.Ny, r.Nx, dtype=torch.float32, device=dev) for r in recs] if phase else None
    var = torch.empty(len(recs), dtype=torch.float64, device=dev)
    L.ssb_reconstruct_batched(plans, [r.G for r in recs], ab, scratch, ph, var,
                              status=recs[0].status)
    return ph, var


class StreamedSteps:
    """Double-buffered upload of each step's events, overlapped with the
    previous step's computation.

    ``run(h_idx, h_off, fn)`` copies the pinned host CSR (uint32 indices as an
    int32 tensor, int64 offsets) into one of two device buffer pairs on a copy
    stream, makes the current stream wait for that copy, calls
    ``fn(d_idx, d_off)`` on the current stream (the whole path: library calls
    and the device-to-host read of its results) and marks the buffer free when
    the current stream has used it.  The next call's upload therefore runs on
    the copy engine while this step computes; every step still uploads its own
    events.  ``start(event)`` makes the next uploads wait for an event recorded
    on the current stream (the start of a timed region)."""

    def __init__(self, max_events: int, max_frames: int, device=None):
        self.device = torch.device(device or "cuda")
        self.bufs = [(torch.empty(max_events, dtype=torch.int32, device=self.device),
                      torch.empty(max_frames + 1, dtype=torch.int64, device=self.device))
                     for _ in range(2)]
        self.copy_stream = torch.cuda.Stream(device=self.device)
        self.copied = [torch.cuda.Event(), torch.cuda.Event()]
        self.free = [torch.cuda.Event(), torch.cuda.Event()]
        self.k = 0

    def start(self, event: torch.cuda.Event):
        self.copy_stream.wait_event(event)

    def run(self, h_idx: torch.Tensor, h_off: torch.Tensor, fn):
        i = self.k % 2
        self.k += 1
        d_idx, d_off = self.bufs[i]
        if h_idx.numel() > d_idx.numel() or h_off.numel() > d_off.numel():
            raise ValueError("step larger than the buffers")
        cur = torch.cuda.current_stream(self.device)
        self.copy_stream.wait_event(self.free[i])
        with torch.cuda.stream(self.copy_stream):
            di = d_idx[:h_idx.numel()]
            do = d_off[:h_off.numel()]
            di.copy_(h_idx, non_blocking=True)
            do.copy_(h_off, non_blocking=True)
            self.copied[i].record(self.copy_stream)
        cur.wait_event(self.copied[i])
        out = fn(di, do)
        self.free[i].record(cur)
        return out
