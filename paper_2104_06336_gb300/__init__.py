"""GB300-native EER -> COM-DPC / SSB phase-contrast imaging (arXiv 2104.06336).

The compute path is libeer4d.so (hand-written sm_103a CUDA kernels behind the
C ABI of include/eer4d.h); this package is its Python binding.
"""

from . import _lib
from ._lib import (  # noqa: F401  (C-ABI names)
    Plan, Eer4dError, eer_load_csr, com_dpc, com_dpc_sums, ssb_accumulate, ssb_accumulate_com,
    ssb_reconstruct, ssb_grad,
    ssb_variance_grad, ssb_trotter_counts, ssb_refocus_step, eer4d_set_stage_events,
    eer4d_launch_count, status_code, FP32_FFT, SPLIT_FP16, FP32_FFT_2PASS, FP32_STOCKHAM, NORM_NONE, NORM_AREA,
    ssb_reconstruct_batched, batched_scratch_bytes, MAX_SETS, eer_decode_rle,
    virtual_detectors, MAX_RINGS, ssb_g_slices, MAX_SLICES, dpc_iterative, eer4d_autotune,
    eer4d_set_tuning, eer4d_get_tuning, eer4d_selftest_wait, eer4d_dft_split_factors,
    eer4d_shard_range, ssb_spectrum_partial, ssb_image_from_spectrum, MAX_SHARDS,
    ssb_refocus_step_adam,
)
from .pipeline import Reconstructor, reconstruct_batched, StreamedSteps  # noqa: F401
from .autograd import SSBPhase, ssb_phase  # noqa: F401
from . import refocus  # noqa: F401
from . import tuning  # noqa: F401
from . import sharding  # noqa: F401


def build(force: bool = False) -> str:
    """Compiles libeer4d.so in-tree for sm_103a and returns its path."""
    from .buildlib import build as _build
    return _build(force=force)


def load():
    return _lib.load()
