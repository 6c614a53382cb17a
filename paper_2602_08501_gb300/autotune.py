"""Autotuner for the launch parameters of a libmpwsd code handle.

The tunable is MPWSD_TUNE_SPLIT_ITEMS: how many work items a tensor-core
scoring launch aims at when it has few 256-row units (each unit's pattern
tiles are then split across CTAs). The best value depends on the code (pattern
tiles per unit), the list size, the batch sizes a caller uses and how many
decodes run concurrently, so it is measured, not guessed: every candidate is
timed on the caller's representative frames (CUDA graph replays, CUDA events)
at each batch size, the candidate with the smallest summed time wins, and the
choice is cached on disk keyed by the code, L, T, batch sizes and GPU.
Tuning changes speed only; the decoded output is identical for every value.
"""
from __future__ import annotations

import hashlib
import json
import os
import threading

import numpy as np

from . import mpwsd

_lock = threading.Lock()


def cache_path() -> str:
    p = os.environ.get("MPWSD_TUNE_CACHE")
    if p:
        return p
    return os.path.join(os.path.expanduser("~"), ".cache", "mpwsd", "tune.json")


def _load_cache(path: str) -> dict:
    try:
        with open(path) as fh:
            return json.load(fh)
    except (OSError, ValueError):
        return {}


def _store_cache(path: str, data: dict) -> None:
    os.makedirs(os.path.dirname(path) or ".", exist_ok=True)
    tmp = f"{path}.tmp{os.getpid()}"
    with open(tmp, "w") as fh:
        json.dump(data, fh, indent=1, sort_keys=True)
    os.replace(tmp, path)


def tune_key(code: "mpwsd.Code", L: int, T: int, batch_sizes, device_name: str, sms: int) -> str:
    h = hashlib.sha256()
    h.update(code.frozen.tobytes())
    h.update(np.ascontiguousarray(code.patterns).tobytes())
    return f"n{code.n}-P{code.n_patterns}-{h.hexdigest()[:12]}-L{L}-T{T}-B{'_'.join(map(str, batch_sizes))}-" \
           f"{device_name.replace(' ', '_')}-{sms}sm"


def candidates(sms: int) -> list[int]:
    return sorted({0, max(1, sms // 4), max(1, sms // 2), sms, 2 * sms})


def measure(code, y, L: int, T: int, batch_sizes, value: int, reps: int = 10) -> float:
    """Summed mean decode time (ms) over the batch sizes with the knob at value."""
    import torch

    code.tune_set(mpwsd.TUNE_SPLIT_ITEMS, value)
    total = 0.0
    for B in batch_sizes:
        yb = y[:B]
        ws = code.workspace(B, L)
        cw = torch.empty((B, code.W), dtype=torch.int64, device="cuda")
        fl = torch.empty((B,), dtype=torch.int16, device="cuda")
        for _ in range(3):
            code.decode(yb, L, T, cw_out=cw, flags_out=fl, workspace=ws, use_graph=True)
        torch.cuda.synchronize()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record()
        for _ in range(reps):
            code.decode(yb, L, T, cw_out=cw, flags_out=fl, workspace=ws, use_graph=True)
        e1.record()
        torch.cuda.synchronize()
        total += e0.elapsed_time(e1) / reps
        ws.close()
    return total


def tune(code: "mpwsd.Code", y, L: int, T: int, batch_sizes=(256, 2048, 16384), use_cache: bool = True,
         reps: int = 10) -> dict:
    """Choose MPWSD_TUNE_SPLIT_ITEMS for `code` from the representative frames
    `y` (CUDA float32 tensor, at least max(batch_sizes) rows), apply it to the
    handle and return {"value", "times_ms", "cached"}."""
    import torch

    props = torch.cuda.get_device_properties(torch.cuda.current_device())
    sms = int(props.multi_processor_count)
    batch_sizes = sorted(int(b) for b in batch_sizes)
    if y.shape[0] < batch_sizes[-1]:
        raise ValueError(f"need at least {batch_sizes[-1]} representative frames, got {y.shape[0]}")
    key = tune_key(code, L, T, batch_sizes, props.name, sms)
    path = cache_path()
    with _lock:
        cache = _load_cache(path) if use_cache else {}
        if key in cache:
            code.tune_set(mpwsd.TUNE_SPLIT_ITEMS, int(cache[key]["value"]))
            return {"value": int(cache[key]["value"]), "times_ms": cache[key]["times_ms"], "cached": True}
    times = {v: measure(code, y, L, T, batch_sizes, v, reps) for v in candidates(sms)}
    best = min(times, key=lambda v: (times[v], v))
    code.tune_set(mpwsd.TUNE_SPLIT_ITEMS, best)
    if use_cache:
        with _lock:
            cache = _load_cache(path)
            cache[key] = {"value": best, "times_ms": {str(k): v for k, v in times.items()}}
            _store_cache(path, cache)
    return {"value": best, "times_ms": {str(k): v for k, v in times.items()}, "cached": False}
