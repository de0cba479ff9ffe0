"""Launch-shape autotuning of the batched ensemble, with a JSON cache.

The timing itself runs in the library (lbm_batch_autotune tries both batch
forms, the persistent kernel at every (threads per CTA, CTAs per SM) shape and
the member grids on 4, 8 and 16 streams, and keeps the fastest); this module
remembers the winner per (GPU, storage precision, member grids) so that later
runs apply it without re-timing.
"""
from __future__ import annotations

import hashlib
import json
import os

from . import build as _build

DEFAULT_CACHE = os.path.join(_build.BUILD, "autotune.json")


def batch_key(batch) -> str:
    import torch
    dev = torch.cuda.get_device_name(torch.cuda.current_device())
    grids = ";".join(f"{c.nx}x{c.ny}x{c.nz}" for c in batch.cases)
    h = hashlib.sha1(grids.encode()).hexdigest()[:16]
    return f"{dev}|prec{batch.precision}|n{len(batch.cases)}|{h}"


def _load(path):
    try:
        with open(path) as fh:
            return json.load(fh)
    except (OSError, ValueError):
        return {}


def tune_batch(batch, cache_path: str | None = None, steps: int = 3, retune: bool = False) -> dict:
    """Apply the cached launch shape for this batch, or time all shapes and cache
    the fastest. Timing advances the members, so call it before initialising them.
    Returns {"threads", "ctas_per_sm", "ms_per_step" (None if from cache), "cached"}."""
    path = cache_path or DEFAULT_CACHE
    cache = _load(path)
    key = batch_key(batch)
    if key in cache and not retune and "streams" in cache[key]:
        cfg = cache[key]
        batch.set_form(cfg["form"], cfg["streams"])
        batch.set_config(cfg["threads"], cfg["ctas_per_sm"])
        return {**cfg, "cached": True}
    ms = batch.autotune(steps)
    c = batch.config()
    cfg = {"form": c["form"], "streams": c["streams"], "threads": c["threads"], "ctas_per_sm": c["ctas_per_sm"],
           "ms_per_step": ms}
    cache[key] = cfg
    os.makedirs(os.path.dirname(path), exist_ok=True)
    tmp = f"{path}.tmp{os.getpid()}"
    with open(tmp, "w") as fh:
        json.dump(cache, fh, indent=1, sort_keys=True)
    os.replace(tmp, path)
    return {**cfg, "cached": False}
