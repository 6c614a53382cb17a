"""Continuous-batching request loop over libmpwsd (frames of several codes).

Frames arrive over time, each for one of several codes. The loop:

* admits work by device memory: every code owns ``pools_per_code`` stage-2
  pools (``mpwsd_pool_*``) whose slot counts -- the frames they hold in
  flight -- are what the device-memory budget allows; a code whose smallest
  pool does not fit gets none (its frames are refused). Frames wait on the
  host while the pools are full and enter as earlier frames finish;
* batches stage-2 work as it accrues: arrived frames of a code are submitted
  (stage 1 runs on them at once) as soon as ``min_batch`` have accrued or the
  oldest has waited ``max_wait_s``; their CRC-failing frames join the pool, and
  every pool step runs one iteration of Algorithm 1 on all rows of the pool --
  trajectories of frames from many submissions, at different iterations --
  so the scoring launches grow with the load instead of with one submission;
* keeps decoder state on the GPU: y goes from pinned host memory into a
  device staging buffer, each frame's result is written on the device where
  the loop asked, and one copy brings all of them back at the end; every pool
  runs on its own stream (submissions go to the pool with the most free
  slots), so stage 1 of one pool overlaps the scoring of another and the
  codes' work overlaps on the device; the pool step is replayed from a CUDA
  graph;
* reports per-frame latency (the CUDA event of the submission or step that
  finished the frame, minus its arrival), throughput and the mean stage-2
  rows per pool step.

Frames are decoded independently, so a frame's result does not depend on what
it was batched with (the tests check it against a one-batch decode and against
decoding the frame alone).
"""
from __future__ import annotations

import time
from dataclasses import dataclass, field

import numpy as np

from . import mpwsd


@dataclass
class CodeSpec:
    code: "mpwsd.Code"
    L: int
    T: int


@dataclass
class ServeResult:
    latency_s: dict            # code -> per-frame latency (s), arrival order of that code
    cw: dict                   # code -> B x W uint64 codewords
    flags: dict                # code -> B uint16 flags
    served: int
    wall_s: float
    dispatches: int            # submissions
    slots: dict                # code -> frames its pools hold in flight
    refused_slots: dict        # code -> 1 if the budget fit no pool for it
    batch_sizes: list = field(default_factory=list)
    steps: dict = field(default_factory=dict)           # code -> pool steps (all its pools)
    stage2_rows: dict = field(default_factory=dict)     # code -> trajectory rows scored over all steps
    submissions: dict = field(default_factory=dict)     # code -> submissions

    def percentiles(self, qs=(50, 99)):
        lat = np.concatenate([v for v in self.latency_s.values() if v.size]) if self.latency_s else np.zeros(0)
        return {f"p{q}": float(np.percentile(lat, q)) if lat.size else None for q in qs}

    def rows_per_step(self):
        steps = sum(self.steps.values())
        return sum(self.stage2_rows.values()) / steps if steps else 0.0


def _bucket(b: int, lo: int = 256) -> int:
    n = lo
    while n < b:
        n *= 2
    return n


def pool_frames_for_budget(code, L: int, want: int, budget: int | None, floor: int) -> int:
    """The largest pool size <= want (halving from it) whose device memory fits
    the budget, or 0 when not even `floor` frames fit."""
    f = int(want)
    while f >= floor:
        if budget is None or code.pool_bytes(f, L) <= budget:
            return f
        f //= 2
    return 0


class Server:
    def __init__(self, specs: dict, max_batch: int = 65536, pool_frames: int | None = None,
                 mem_budget_bytes: int | None = None, min_batch: int = 4096, max_wait_s: float = 200e-6,
                 score_mode: str = "bf16x2", use_graph: bool = True, steps_ahead: int = 2,
                 pools_per_code: int = 1):
        import torch

        self.torch = torch
        self.specs = specs
        self.max_batch = int(max_batch)
        self.min_batch = int(min_batch)
        self.max_wait_s = float(max_wait_s)
        self.steps_ahead = int(steps_ahead)
        want = int(pool_frames) if pool_frames else 4 * self.max_batch
        npc = max(1, int(pools_per_code))
        share = None if mem_budget_bytes is None else int(mem_budget_bytes) // max(1, len(specs) * npc)
        self.pools, self.refused = {}, {}
        self.mem_used = 0
        for name, sp in specs.items():
            self.pools[name] = []
            self.refused[name] = 0
            for _ in range(npc):
                # the staging buffer for y counts against the budget too
                stage = self.max_batch * sp.code.n * 4
                frames = pool_frames_for_budget(sp.code, sp.L, want, None if share is None else share - stage,
                                                floor=min(256, want))
                pool = None
                if frames:
                    try:
                        pool = sp.code.pool(frames, sp.L, sp.T, score_mode=score_mode, use_graph=use_graph)
                    except mpwsd.MpwsdError as e:
                        if e.status != mpwsd.ENOMEM:
                            raise
                if pool is None:
                    self.refused[name] += 1
                    continue
                self.mem_used += sp.code.pool_bytes(frames, sp.L) + stage
                self.pools[name].append(_Lane(pool=pool, stream=torch.cuda.Stream(),
                                              y=torch.zeros((self.max_batch, sp.code.n), dtype=torch.float32,
                                                            device="cuda")))

    @property
    def slots(self):
        return {nm: sum(ln.pool.max_frames for ln in lanes) for nm, lanes in self.pools.items()}

    def warmup(self):
        """Record every pool's step graph and run one submission through each
        (all-zero frames), so nothing is captured while requests are served."""
        torch = self.torch
        for nm, lanes in self.pools.items():
            sp = self.specs[nm]
            for ln in lanes:
                b = min(256, self.max_batch)
                cw = torch.empty((b, sp.code.W), dtype=torch.int64, device="cuda")
                fl = torch.empty((b,), dtype=torch.int16, device="cuda")
                with torch.cuda.stream(ln.stream):
                    ln.y[:b].zero_()
                    ln.pool.submit(ln.y[:b], cw, fl, stream=ln.stream)
                    for _ in range(sp.T):
                        ln.pool.step(stream=ln.stream)
        torch.cuda.synchronize()

    def run(self, arrivals: dict, y_pinned: dict) -> ServeResult:
        """arrivals[code]: sorted arrival times (s) of that code's frames;
        y_pinned[code]: matching pinned CPU tensor, frames in arrival order."""
        torch = self.torch
        names = list(self.specs)
        for nm in names:
            if len(arrivals[nm]) and not self.pools[nm]:
                raise RuntimeError(f"no stage-2 pool fits the memory budget for code {nm}")
        total = {nm: len(arrivals[nm]) for nm in names}
        dev = {nm: dict(cw=torch.empty((total[nm], self.specs[nm].code.W), dtype=torch.int64, device="cuda"),
                        fl=torch.empty((total[nm],), dtype=torch.int16, device="cuda"),
                        done=torch.zeros((total[nm],), dtype=torch.int32, device="cuda")) for nm in names}
        # which lane decoded each frame (its done entry counts that pool's submissions / steps)
        lane_of = {nm: np.zeros(total[nm], np.int32) for nm in names}
        sub = {nm: 0 for nm in names}        # frames submitted so far
        lanes = [(nm, i, ln) for nm in names for i, ln in enumerate(self.pools[nm])]
        for _, _, ln in lanes:
            ln.sub_ev, ln.step_ev = [], []
            ln.sub0, ln.step0 = ln.pool.submits, ln.pool.steps
            ln.last_sub_step = -10 ** 9
        batch_sizes = []
        for nm in names:
            self.specs[nm].code.reset_stats()
        # events are made up front (one per submission or step at most), so the loop allocates nothing
        ev_free = [torch.cuda.Event(enable_timing=True) for _ in range(2 * sum(total.values()) // 64 + 4096)]
        ref = torch.cuda.Event(enable_timing=True)
        ref.record(torch.cuda.current_stream())
        torch.cuda.synchronize()
        t0 = time.perf_counter()

        def busy(ln):
            return ln.pool.steps - ln.last_sub_step < ln.pool.T

        while any(sub[nm] < total[nm] for nm in names) or any(busy(ln) for _, _, ln in lanes):
            now = time.perf_counter() - t0
            for nm in names:
                if not self.pools[nm]:
                    continue
                arrived = int(np.searchsorted(arrivals[nm], now, side="right"))
                pend = arrived - sub[nm]
                if pend <= 0:
                    continue
                oldest = arrivals[nm][sub[nm]]
                if not (pend >= self.min_batch or now - oldest >= self.max_wait_s or arrived == total[nm]):
                    continue
                lanes_nm = self.pools[nm]
                if len(lanes_nm) == 1:
                    i, ln = 0, lanes_nm[0]
                    free = ln.pool.free_frames()
                else:
                    i, ln = max(enumerate(lanes_nm), key=lambda t: t[1].pool.free_frames())
                    free = ln.pool.free_frames()
                b = min(pend, self.max_batch, free)
                if b <= 0:
                    continue
                lo, hi = sub[nm], sub[nm] + b
                with torch.cuda.stream(ln.stream):
                    ln.y[:b].copy_(y_pinned[nm][lo:hi], non_blocking=True)
                ln.pool.submit(ln.y[:b], dev[nm]["cw"][lo:hi], dev[nm]["fl"][lo:hi], dev[nm]["done"][lo:hi],
                               stream=ln.stream)
                ev = ev_free.pop() if ev_free else torch.cuda.Event(enable_timing=True)
                ev.record(ln.stream)
                ln.sub_ev.append(ev)
                lane_of[nm][lo:hi] = i
                sub[nm] = hi
                ln.last_sub_step = ln.pool.steps
                batch_sizes.append(b)
            for nm, i, ln in lanes:
                if not busy(ln):
                    continue
                # keep at most `steps_ahead` steps queued on the device per pool
                evs = ln.step_ev
                if len(evs) >= self.steps_ahead and not evs[-self.steps_ahead].query():
                    continue
                ln.pool.step(stream=ln.stream)
                ev = ev_free.pop() if ev_free else torch.cuda.Event(enable_timing=True)
                ev.record(ln.stream)
                evs.append(ev)
        torch.cuda.synchronize()
        lat, cws, fls, steps, rows, subs = {}, {}, {}, {}, {}, {}
        first = min((arrivals[nm][0] for nm in names if total[nm]), default=0.0)
        last = first
        for nm in names:
            sp = self.specs[nm]
            steps[nm] = sum(ln.pool.steps - ln.step0 for ln in self.pools[nm])
            subs[nm] = sum(len(ln.sub_ev) for ln in self.pools[nm])
            rows[nm] = sp.code.stats()["pattern_evals"] // max(sp.code.n_patterns, 1)
            if not total[nm]:
                lat[nm], cws[nm], fls[nm] = np.zeros(0), np.zeros((0, sp.code.W), np.uint64), np.zeros(0, np.uint16)
                continue
            done = dev[nm]["done"].cpu().numpy()
            t_done = np.zeros(total[nm])
            for i, ln in enumerate(self.pools[nm]):
                sel = lane_of[nm] == i
                if not sel.any():
                    continue
                t_sub = np.array([ref.elapsed_time(e) / 1e3 for e in ln.sub_ev])
                t_step = np.array([ref.elapsed_time(e) / 1e3 for e in ln.step_ev]) if ln.step_ev else np.zeros(1)
                d = done[sel]
                # done entries count the pool's submissions and steps from its creation
                t_done[sel] = np.where(d < 0, t_sub[np.clip(-d - 1 - ln.sub0, 0, len(t_sub) - 1)],
                                       t_step[np.clip(d - 1 - ln.step0, 0, len(t_step) - 1)])
            lat[nm] = t_done - arrivals[nm]
            last = max(last, float(t_done.max()))
            cws[nm] = dev[nm]["cw"].cpu().numpy().view(np.uint64)
            fls[nm] = dev[nm]["fl"].cpu().numpy().view(np.uint16)
        return ServeResult(latency_s=lat, cw=cws, flags=fls, served=sum(total.values()), wall_s=last - first,
                           dispatches=len(batch_sizes), slots=self.slots, refused_slots=dict(self.refused),
                           batch_sizes=batch_sizes, steps=steps, stage2_rows=rows, submissions=subs)


@dataclass
class _Lane:
    """One pool of a code with its stream and its device staging buffer for y."""
    pool: "mpwsd.Pool"
    stream: object
    y: object
    sub_ev: list = field(default_factory=list)
    step_ev: list = field(default_factory=list)
    sub0: int = 0
    step0: int = 0
    last_sub_step: int = 0


def poisson_arrivals(rate_hz: float, count: int, seed: int) -> np.ndarray:
    """Arrival times of a Poisson process (exponential gaps from a seeded stream)."""
    rng = np.random.Generator(np.random.Philox(seed))
    return np.cumsum(rng.exponential(1.0 / rate_hz, count))
