"""Autotuner for the launch parameters of a libmpwsd code handle.

Two knobs of the tensor-core scoring kernel are tuned:

* MPWSD_TUNE_TC_SHAPE -- the kernel's tile shape among the instantiated ones
  (pattern tile 256 or 128 wide, two or four A-builder warps, a two- or
  four-stage pattern-tile ring; see include/mpwsd.h);
* MPWSD_TUNE_SPLIT_ITEMS -- how many work items a launch aims at when it has
  few 256-row units (each unit's pattern tiles are then split across CTAs).

The best values depend on the code (pattern tiles per unit), the list size,
the batch sizes a caller uses and how many decodes run concurrently, so they
are measured, not guessed: every candidate is timed on the caller's
representative frames (CUDA graph replays, CUDA events) at each batch size and
the one with the smallest summed time wins. The shape is chosen first (at two
split targets), then the split target for that shape. The choice is cached on
disk keyed by the code, L, T, batch sizes and GPU, and records both knobs.
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


def shapes(code: "mpwsd.Code") -> list[int]:
    """The MPWSD_TUNE_TC_SHAPE values instantiated for this code length."""
    out = []
    for v in range(8):
        try:
            code.tune_set(mpwsd.TUNE_TC_SHAPE, v)
        except mpwsd.MpwsdError:
            continue
        out.append(v)
    code.tune_set(mpwsd.TUNE_TC_SHAPE, 0)
    return out


def choose(shape_list, split_list, default_split: int, run) -> tuple[int, int]:
    """The two-pass search: the shape with the smallest time at the default
    split target or at no split, then the split target (candidates plus the
    default) with the smallest time for that shape; ties go to the lower
    value. run(shape, split) returns the time of one setting."""
    best_shape = min(shape_list, key=lambda sh: (min(run(sh, default_split), run(sh, 0)), sh))
    best_split = min(sorted(set(split_list) | {default_split}), key=lambda v: (run(best_shape, v), v))
    return best_shape, best_split


def measure(code, y, L: int, T: int, batch_sizes, value: int, reps: int = 10, shape: int | None = None) -> float:
    """Summed mean decode time (ms) over the batch sizes with the split target
    at `value` (and the scoring shape at `shape`, if given)."""
    import torch

    if shape is not None:
        code.tune_set(mpwsd.TUNE_TC_SHAPE, shape)
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
    """Choose the scoring shape and split target for `code` from the
    representative frames `y` (CUDA float32 tensor, at least max(batch_sizes)
    rows), apply them to the handle and return {"shape", "value", "times_ms",
    "default_ms", "cached"}; times_ms maps "shape/split" to the summed time."""
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
        ent = cache.get(key)
        if ent and "shape" in ent:
            code.tune_set(mpwsd.TUNE_TC_SHAPE, int(ent["shape"]))
            code.tune_set(mpwsd.TUNE_SPLIT_ITEMS, int(ent["value"]))
            return {"shape": int(ent["shape"]), "value": int(ent["value"]), "times_ms": ent["times_ms"],
                    "default_ms": ent.get("default_ms"), "cached": True}
    default_split = code.tune_get(mpwsd.TUNE_SPLIT_ITEMS)
    times = {}

    def run(shape, split):
        k = f"{shape}/{split}"
        if k not in times:
            times[k] = measure(code, y, L, T, batch_sizes, split, reps, shape=shape)
        return times[k]

    default_ms = run(0, default_split)
    best_shape, best_split = choose(shapes(code), candidates(sms), default_split, run)
    code.tune_set(mpwsd.TUNE_TC_SHAPE, best_shape)
    code.tune_set(mpwsd.TUNE_SPLIT_ITEMS, best_split)
    out = {"shape": best_shape, "value": best_split, "times_ms": dict(times), "default_ms": default_ms}
    if use_cache:
        with _lock:
            cache = _load_cache(path)
            cache[key] = out
            _store_cache(path, cache)
    return dict(out, cached=False)
