"""One dataset over several GPUs by detector pixel (Sec. IV: G(k, K) and the
trotter sum of Eq. 3 are per pixel k, so pixels split between devices that
exchange only partial spectra).

Each rank builds a shard plan (``Reconstructor(..., shard=(rank, world))``):
its ssb_accumulate reads every event and keeps its own pixels, its G covers
them only.  ``sharded_reconstruct`` then forms the rank's share of the
spectrum (ssb_spectrum_partial), sums the shares of all ranks with one
all-reduce of the spectrum and one of the two Gbar0 sums, and forms the image
(ssb_image_from_spectrum) on every rank.  The COM/DPC path does not depend on
the pixels and is computed per frame by any plan.
"""

from __future__ import annotations

import torch


def allreduce_partials(H: torch.Tensor, g0: torch.Tensor, group=None):
    """Sums the shares of every rank in place: H (complex64 [n][Ny][Nx/2+1],
    summed as its float32 pairs) and g0 (float64 [2]).  No-op without an
    initialised process group or with one rank."""
    import torch.distributed as dist
    if not dist.is_available() or not dist.is_initialized() or dist.get_world_size(group) == 1:
        return H, g0
    dist.all_reduce(torch.view_as_real(H), op=dist.ReduceOp.SUM, group=group)
    dist.all_reduce(g0, op=dist.ReduceOp.SUM, group=group)
    return H, g0


def sharded_reconstruct(rec, aberr: torch.Tensor, group=None, phase: bool = True):
    """SSB phase images and variances of the whole pixel set from this rank's
    shard plan (``rec``) and the other ranks' shares."""
    H, g0 = rec.spectrum_partial(aberr)
    allreduce_partials(H, g0, group)
    return rec.image_from_spectrum(H, g0, phase=phase)
