"""Autotuner for the launch shapes that the kernels leave open, with a cache.

What is tuned (none of it changes a result bit):
  * the form of the MED recovery wavefront -- the row-band pipeline (0) or tiles of
    32 rows and 64, 128 or 256 columns;
  * the rows of a 64-row strip that one CTA of the fused decode's extraction handles
    (64 .. 4): whole strips give the longest runs, smaller parts more CTAs for wide
    images and small batches;
  * the CTAs that share one tile row of the owner's gather (rdhei_label_encrypt), 1..64.
The paper's own tile is not free: its 64 x 64 tiles follow from the rotation's per-bit
closed form (levels 1..6 inside a tile).

How: for a batch of jobs, the operation runs once, then the stages a knob acts on are
timed with CUDA events over a few repetitions for each candidate (the stages tuned
here rewrite their whole output from inputs they do not modify, so every repetition
does the full work).  The fastest candidate is cached under a key made of the device name
and the batch's shape signature (sizes and variants), in ``_build/tune_cache.json``
next to the library.
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


EXTRACT_ROWS = (64, 32, 16, 8, 4)
ENC_SPLITS = (1, 2, 4, 8, 16, 32, 64)


def time_param(jobs, op: int, stages, param: int, values, reps: int = 5, stream=None) -> dict:
    """Mean milliseconds of the given stages of op (run in order) for each value of a
    plan parameter, on one plan over the jobs (the whole operation runs once first)."""
    st = stream or torch.cuda.current_stream()
    plan = rd.Plan(jobs, st)
    plan.run(op, st)
    a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    out = {}
    for v in values:
        plan.set_param(param, v)
        for stage in stages:                                # warm-up at this value
            plan.run_stage(op, stage, st)
        ms = 0.0
        for _ in range(reps):
            a.record(st)
            for stage in stages:
                plan.run_stage(op, stage, st)
            b.record(st)
            b.synchronize()
            ms += a.elapsed_time(b)
        out[str(v)] = ms / reps
    if plan.status(st) not in (0, rd.RDHEI_ECAPACITY):
        raise rd.RdheiError("a tuned stage reported an error")
    return out


def _best(kind: str, jobs, op, stages, param, values, stream, refresh) -> tuple[int, dict]:
    key = f"{kind}|" + signature(jobs)
    cache = _load()
    if not refresh and key in cache:
        return int(cache[key]["best"]), cache[key].get("ms", {})
    times = time_param(jobs, op, stages, param, values, stream=stream)
    best = int(min(times, key=times.get))
    cache[key] = {"best": best, "ms": times}
    _store(cache)
    return best, times


def best_extract_rows(decode_jobs, stream=None, refresh: bool = False) -> tuple[int, dict]:
    """Rows per extraction CTA for this batch of rdhei_decode jobs.  Timed: the top-level
    pass, which derives each part's first bit (more parts, more work there), and the
    extraction itself (stages 1 and 2)."""
    return _best("extract_rows", decode_jobs, rd.OP_DECODE, (1, 2), rd.PARAM_EXTRACT_ROWS, EXTRACT_ROWS, stream,
                 refresh)


def best_enc_split(label_encrypt_jobs, stream=None, refresh: bool = False) -> tuple[int, dict]:
    """CTAs per tile row of rdhei_label_encrypt's gather for this batch (stage 2 timed)."""
    return _best("enc_split", label_encrypt_jobs, rd.OP_LABEL_ENCRYPT, (2,), rd.PARAM_ENC_SPLIT, ENC_SPLITS, stream,
                 refresh)
