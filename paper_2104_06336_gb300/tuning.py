"""Launch-shape autotuning with an on-disk cache.

``autotune(rec, idx, off)`` times the candidate tile/grid shapes of the
scatter, fused scan-DFT and trotter kernels on the given data
(``eer4d_autotune``) and keeps the fastest in the Reconstructor's plan.  With
``cache`` (a JSON file path) the choice is stored under a key made of the GPU
name, the plan's precision and the geometry, and later calls with the same
key apply it without timing.
"""

from __future__ import annotations

import json
import os

import torch

from . import _lib as L


def cache_key(geom: dict, precision: int, device_name: str) -> str:
    fields = ("det_w", "det_h", "bin", "pw", "ph", "k0_px", "crop_px", "scan_ny", "scan_nx")
    parts = [device_name, f"prec={precision}"] + [f"{f}={geom[f]}" for f in fields]
    return "|".join(str(p) for p in parts)


def load_cache(path: str) -> dict:
    try:
        with open(path) as fh:
            d = json.load(fh)
        return d if isinstance(d, dict) else {}
    except (OSError, ValueError):
        return {}


def store_cache(path: str, key: str, tuning: dict) -> None:
    d = load_cache(path)
    d[key] = tuning
    tmp = path + ".tmp"
    with open(tmp, "w") as fh:
        json.dump(d, fh, indent=1, sort_keys=True)
    os.replace(tmp, path)


def autotune(rec, idx: torch.Tensor, off: torch.Tensor, aberr=None, cache: str | None = None,
             force: bool = False) -> dict:
    """Chooses and applies the launch shapes for ``rec`` (see module doc)."""
    name = torch.cuda.get_device_name(rec.device)
    key = cache_key(rec.geom, rec.plan.precision, name)
    if cache and not force:
        hit = load_cache(cache).get(key)
        if hit is not None:
            L.eer4d_set_tuning(rec.plan, hit)
            return hit
    ab = torch.zeros(5, dtype=torch.float64, device=rec.device) if aberr is None else \
        torch.as_tensor(aberr, dtype=torch.float64).to(rec.device).contiguous()
    t = L.eer4d_autotune(rec.plan, idx.contiguous(), off.contiguous(), rec.work, rec.G, rec.scratch,
                         ab, status=rec.status)
    if cache:
        store_cache(cache, key, t)
    return t
