"""Autotuner for the launch shapes that the kernels leave open, with a cache.

What is tuned: the form of the MED recovery wavefront -- the row-band pipeline (0) or
tiles of 32 rows and 64, 128 or 256 columns.  The paper's own path has no free tile shape: its 64 x 64 tiles follow
from the rotation's per-bit closed form (levels 1..6 inside a tile).

How: for a batch of decode jobs, each candidate width gets its own plan; the first
three stages of rdhei_decrypt_recover run once to stage the pixels, then the
wavefront stage is timed with CUDA events over a few repetitions (it rewrites the
output from the staged pixels, so every repetition does the full work).  The fastest
width is cached under a key made of the device name and the batch's shape signature
(sizes and variants), in ``_build/tune_cache.json`` next to the library.
"""
from __future__ import annotations

import hashlib
import json
import os

import torch

from . import build as _build
from . import rdhei as rd

WAVE_WIDTHS = (0, 64, 128, 256)          # 0: row-band pipeline
_CACHE = os.path.join(_build.OUT, "tune_cache.json")


def _load() -> dict:
    try:
        with open(_CACHE) as f:
            return json.load(f)
    except Exception:
        return {}


def _store(cache: dict):
    os.makedirs(os.path.dirname(_CACHE), exist_ok=True)
    tmp = _CACHE + f".{os.getpid()}.tmp"
    with open(tmp, "w") as f:
        json.dump(cache, f, indent=1, sort_keys=True)
    os.replace(tmp, _CACHE)


def signature(jobs) -> str:
    """Device name + the multiset of (H, W, variant) of the jobs."""
    shapes = sorted((int(j.H), int(j.W), int(j.variant)) for j in jobs)
    h = hashlib.sha256(json.dumps(shapes).encode()).hexdigest()[:16]
    return f"{torch.cuda.get_device_name()}|{len(shapes)}|{h}"


def time_wave(jobs, cols: int, reps: int = 5, stream=None) -> float:
    """Mean milliseconds of the wavefront stage for this batch at tile width cols."""
    st = stream or torch.cuda.current_stream()
    plan = rd.Plan(jobs, st, wave_cols=cols)
    for s in (0, 1, 2):
        plan.run_stage(rd.OP_DECRYPT_RECOVER, s, st)
    plan.run_stage(rd.OP_DECRYPT_RECOVER, 3, st)          # warm-up
    a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    ms = 0.0
    for _ in range(reps):
        # the wavefront reads the staged pixels it overwrites: stage them again, untimed
        plan.run_stage(rd.OP_DECRYPT_RECOVER, 2, st)
        a.record(st)
        plan.run_stage(rd.OP_DECRYPT_RECOVER, 3, st)
        b.record(st)
        b.synchronize()
        ms += a.elapsed_time(b)
    if plan.status(st) != 0:
        raise rd.RdheiError("wavefront reported an error while tuning")
    return ms / reps


def best_wave_cols(jobs, stream=None, refresh: bool = False) -> tuple[int, dict]:
    """Tile width for the MED wavefront of this batch of decrypt_recover jobs, and the
    measured milliseconds per width ({} when taken from the cache)."""
    if not any(int(j.variant) >> 1 for j in jobs):
        return 128, {}
    key = "wave_cols|" + signature(jobs)
    cache = _load()
    if not refresh and key in cache:
        return int(cache[key]["best"]), cache[key].get("ms", {})
    times = {str(c): time_wave(jobs, c, stream=stream) for c in WAVE_WIDTHS}
    best = int(min(times, key=times.get))
    cache[key] = {"best": best, "ms": times}
    _store(cache)
    return best, times
