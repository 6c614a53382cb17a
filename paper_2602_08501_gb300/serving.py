"""Continuous-batching request loop over libmpwsd (frames of several codes).

Frames arrive over time, each for one of several codes. The loop:

* admits work by device memory: every code owns a few *slots* (a decoder
  workspace, device buffers for y / codewords / flags, a CUDA stream), created
  up front while the memory budget allows -- a slot that does not fit
  (over budget, or MPWSD_ENOMEM) is not created, so frames wait instead;
* batches as work accrues: whenever a code has pending frames and a free slot,
  it dispatches up to ``max_batch`` of them -- as soon as ``min_batch`` have
  accrued or the oldest has waited ``max_wait_s`` -- so frames that arrive while
  others are on the GPU are admitted as slots free up and their decodes overlap
  on the device (one stream per slot). Each dispatch runs the whole two-stage
  decode, whose stage 2 gathers the CRC-failing frames of the batch;
* keeps decoder state on the GPU: inputs come straight from pinned host memory
  into the slot's device buffer, the decode leaves results on the device and
  one copy brings them back; batches are padded to size buckets so that the
  decode's CUDA graph is replayed;
* reports per-frame latency (completion, from CUDA events, minus arrival) and
  throughput.

Padding frames are all-zero observations; frames are decoded independently,
so a frame's result does not depend on what it was batched with.
"""
from __future__ import annotations

import time
from collections import deque
from dataclasses import dataclass, field

import numpy as np

from . import mpwsd


@dataclass
class CodeSpec:
    code: "mpwsd.Code"
    L: int
    T: int


@dataclass
class _Slot:
    name: str
    ws: "mpwsd.Workspace"
    y: object
    cw: object
    fl: object
    stream: object
    done: object
    busy: bool = False
    lo: int = 0
    hi: int = 0
    t_dispatch: float = 0.0


@dataclass
class ServeResult:
    latency_s: dict            # code -> per-frame latency (s), arrival order of that code
    cw: dict                   # code -> B x W uint64 codewords
    flags: dict                # code -> B uint16 flags
    served: int
    wall_s: float
    dispatches: int
    slots: dict                # code -> slots admitted
    refused_slots: dict        # code -> slots refused by the memory budget
    batch_sizes: list = field(default_factory=list)

    def percentiles(self, qs=(50, 99)):
        lat = np.concatenate([v for v in self.latency_s.values() if v.size]) if self.latency_s else np.zeros(0)
        return {f"p{q}": float(np.percentile(lat, q)) if lat.size else None for q in qs}


def _bucket(b: int, lo: int = 256) -> int:
    n = lo
    while n < b:
        n *= 2
    return n


class Server:
    def __init__(self, specs: dict, max_batch: int = 65536, slots_per_code: int = 4,
                 mem_budget_bytes: int | None = None, min_batch: int = 4096, max_wait_s: float = 200e-6,
                 score_mode: str = "bf16x2", use_graph: bool = True):
        import torch

        self.torch = torch
        self.specs = specs
        self.max_batch = int(max_batch)
        self.min_batch = int(min_batch)
        self.max_wait_s = float(max_wait_s)
        self.score_mode = score_mode
        self.use_graph = use_graph
        self.slots: dict[str, list[_Slot]] = {}
        self.refused: dict[str, int] = {}
        budget = mem_budget_bytes
        used = 0
        per_slot = {}
        for name, sp in specs.items():
            self.slots[name] = []
            self.refused[name] = 0
            per_slot[name] = sp.code.workspace_bytes(self.max_batch, sp.L) + \
                self.max_batch * (sp.code.n * 4 + sp.code.W * 8 + 2)
        # round-robin over the codes, so every code gets a slot before any gets a second
        for _ in range(slots_per_code):
            for name, sp in specs.items():
                n, W = sp.code.n, sp.code.W
                if budget is not None and used + per_slot[name] > budget:
                    self.refused[name] += 1
                    continue
                try:
                    ws = sp.code.workspace(self.max_batch, sp.L)
                except mpwsd.MpwsdError as e:
                    if e.status != mpwsd.ENOMEM:
                        raise
                    self.refused[name] += 1
                    continue
                used += per_slot[name]
                self.slots[name].append(_Slot(
                    name=name, ws=ws,
                    y=torch.zeros((self.max_batch, n), dtype=torch.float32, device="cuda"),
                    cw=torch.empty((self.max_batch, W), dtype=torch.int64, device="cuda"),
                    fl=torch.empty((self.max_batch,), dtype=torch.int16, device="cuda"),
                    stream=torch.cuda.Stream(), done=torch.cuda.Event(enable_timing=True)))
        self.mem_used = used

    def warmup(self):
        """Record the decode graph of every batch bucket on every slot (all-zero
        frames), so no capture happens while requests are being served."""
        torch = self.torch
        for nm, slots in self.slots.items():
            sp = self.specs[nm]
            for s in slots:
                b = 256
                while True:
                    bp = min(b, self.max_batch)
                    with torch.cuda.stream(s.stream):
                        s.y[:bp].zero_()
                        sp.code.decode(s.y[:bp], sp.L, sp.T, score_mode=self.score_mode, cw_out=s.cw[:bp],
                                       flags_out=s.fl[:bp], stream=s.stream, workspace=s.ws, use_graph=self.use_graph)
                    if bp >= self.max_batch:
                        break
                    b *= 2
        torch.cuda.synchronize()

    def run(self, arrivals: dict, y_pinned: dict) -> ServeResult:
        """arrivals[code]: sorted arrival times (s) of that code's frames;
        y_pinned[code]: matching pinned CPU tensor, frames in arrival order."""
        torch = self.torch
        names = list(self.specs)
        for nm in names:
            if len(arrivals[nm]) and not self.slots[nm]:
                raise RuntimeError(f"no decoder slot fits the memory budget for code {nm}")
        pending = {nm: deque() for nm in names}      # (lo, hi) ranges of arrived, undispatched frames
        nxt = {nm: 0 for nm in names}                # next frame index not yet arrived
        total = {nm: len(arrivals[nm]) for nm in names}
        cw_out = {nm: torch.empty((total[nm], self.specs[nm].code.W), dtype=torch.int64).pin_memory() for nm in names}
        fl_out = {nm: torch.empty((total[nm],), dtype=torch.int16).pin_memory() for nm in names}
        done_t = {nm: np.full(total[nm], np.nan) for nm in names}
        disp_queue = {nm: 0 for nm in names}          # frames dispatched so far (FIFO)
        busy = []
        dispatches = 0
        batch_sizes = []
        ref = torch.cuda.Event(enable_timing=True)
        ref.record(torch.cuda.current_stream())
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        remaining = sum(total.values())
        while remaining > 0:
            now = time.perf_counter() - t0
            for nm in names:  # arrivals up to now
                arr = arrivals[nm]
                j = nxt[nm]
                k = int(np.searchsorted(arr, now, side="right"))
                if k > j:
                    nxt[nm] = k
            for s in list(busy):  # completions
                if s.done.query():
                    t_done = ref.elapsed_time(s.done) / 1e3
                    done_t[s.name][s.lo:s.hi] = t_done
                    remaining -= s.hi - s.lo
                    s.busy = False
                    busy.remove(s)
            for nm in names:  # dispatch
                avail = nxt[nm] - disp_queue[nm]
                if avail <= 0:
                    continue
                oldest = arrivals[nm][disp_queue[nm]]
                if avail < self.min_batch and now - oldest < self.max_wait_s and nxt[nm] < total[nm]:
                    continue
                free = [s for s in self.slots[nm] if not s.busy]
                if not free:
                    continue
                s = free[0]
                lo = disp_queue[nm]
                hi = min(lo + self.max_batch, nxt[nm])
                b = hi - lo
                bp = min(_bucket(b), self.max_batch)
                sp = self.specs[nm]
                with torch.cuda.stream(s.stream):
                    s.y[:b].copy_(y_pinned[nm][lo:hi], non_blocking=True)
                    if bp > b:
                        s.y[b:bp].zero_()
                    sp.code.decode(s.y[:bp], sp.L, sp.T, score_mode=self.score_mode, cw_out=s.cw[:bp],
                                   flags_out=s.fl[:bp], stream=s.stream, workspace=s.ws, use_graph=self.use_graph)
                    cw_out[nm][lo:hi].copy_(s.cw[:b], non_blocking=True)
                    fl_out[nm][lo:hi].copy_(s.fl[:b], non_blocking=True)
                    s.done.record(s.stream)
                s.busy, s.lo, s.hi = True, lo, hi
                busy.append(s)
                disp_queue[nm] = hi
                dispatches += 1
                batch_sizes.append(b)
        torch.cuda.synchronize()
        first = min(arrivals[nm][0] for nm in names if total[nm])
        last = max(np.nanmax(done_t[nm]) for nm in names if total[nm])
        lat = {nm: done_t[nm] - arrivals[nm] for nm in names}
        return ServeResult(latency_s=lat, cw={nm: cw_out[nm].numpy().view(np.uint64) for nm in names},
                           flags={nm: fl_out[nm].numpy().view(np.uint16) for nm in names},
                           served=sum(total.values()), wall_s=last - first, dispatches=dispatches,
                           slots={nm: len(v) for nm, v in self.slots.items()}, refused_slots=dict(self.refused),
                           batch_sizes=batch_sizes)


def poisson_arrivals(rate_hz: float, count: int, seed: int) -> np.ndarray:
    """Arrival times of a Poisson process (exponential gaps from a seeded stream)."""
    rng = np.random.Generator(np.random.Philox(seed))
    return np.cumsum(rng.exponential(1.0 / rate_hz, count))
