"""Launch-shape autotuning of single channels and of the batched ensemble,
with a JSON cache.

The timing itself runs in the library: lbm_autotune times every kernel form
a channel's grid allows (one, two or four cells per thread, or the
row-pipelined CTA) and keeps the fastest; lbm_batch_autotune tries both batch
forms, the persistent kernel at every (threads per CTA, CTAs per SM) shape and
the member grids on 4, 8 and 16 streams. This module remembers the winners
per GPU and problem so that later runs apply them without re-timing.
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


def channel_key(ch) -> str:
    import torch
    dev = torch.cuda.get_device_name(torch.cuda.current_device())
    return (f"{dev}|channel|prec{ch.precision}|layout{ch.layout}|{ch.nx}x{ch.ny}x{ch.nz}|wall{ch.wall}"
            f"|coll{ch.collision}")


def tune_channel(ch, cache_path: str | None = None, steps: int = 16, retune: bool = False) -> dict:
    """Apply the cached kernel form for this channel, or time every form and
    cache the fastest. Timing advances the state, so call it before
    initialising the channel. Returns {"kernel", "ms_per_step" (None if from
    cache), "cached"}."""
    path = cache_path or DEFAULT_CACHE
    cache = _load(path)
    key = channel_key(ch)
    if key in cache and not retune:
        ch.set_kernel(cache[key]["kernel"])
        return {**cache[key], "cached": True}
    kernel, ms = ch.autotune(steps)
    cfg = {"kernel": kernel, "ms_per_step": ms}
    _store(path, cache, key, cfg)
    return {**cfg, "cached": False}


def _store(path, cache, key, cfg):
    cache[key] = cfg
    os.makedirs(os.path.dirname(path), exist_ok=True)
    tmp = f"{path}.tmp{os.getpid()}"
    with open(tmp, "w") as fh:
        json.dump(cache, fh, indent=1, sort_keys=True)
    os.replace(tmp, path)


def tune_batch(batch, cache_path: str | None = None, steps: int = 16, retune: bool = False) -> dict:
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
    _store(path, cache, key, cfg)
    return {**cfg, "cached": False}
