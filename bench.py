#!/usr/bin/env python
"""Throughput of the two-stage SCL + MP-WSD decoder on GB300 (one JSON line).

A step decodes one batch of synthetic frames through the whole hot path
(stage-1 SC-list + CRC + compaction, T iterations of scoring / FP64 re-rank /
hop, final select). Default workload: RM(2,6)+CRC-6 (x^6+x^5+1), Eb/N0 = 1 dB,
10^6 frames from seed 1, L = 8, T = 4, all 2604 weight-16 patterns, BF16
hi+lo tensor-core scoring. y (256 MB) is larger than L2, so no flush is
needed between steps.

    python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference]
                    [--workload NAME] [--ebn0 DB] [--seed S] [--frames B]

Under torchrun the batches of one seeded stream are dealt round-robin over the
ranks (batch b to rank b mod N; each rank decodes one batch per step, so the
per-GPU work is fixed: weak scaling); the only collectives are a barrier and
the max / sum of the timers and counters.
"""
from __future__ import annotations

import argparse
import hashlib
import json
import math
import os
import re
import statistics
import subprocess
import sys
import threading
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "decoded frames/s and pattern-evals/s at 1 GB300 at oracle-equal FER; p99 latency"

_CRC6 = dict(crc_poly=0x21, crc_len=6)   # x^6 + x^5 + 1
_NOCRC = dict(crc_poly=0x0, crc_len=0)

WORKLOADS = {
    "rm26_crc6_1db": dict(steps=200, code="rm26_crc6", m=6, r=2, ebn0=1.0, frames=1_000_000, seed=1, L=8, T=4, weights=[16],
                          **_CRC6, desc="RM(2,6)+CRC-6, Eb/N0 {ebn0} dB, {frames} frames, seed {seed}, L=8, T=4, "
                                        "2604 w16 patterns"),
    "rm26_crc6_cfg1": dict(steps=200, code="rm26_crc6", m=6, r=2, ebn0=1.0, frames=10_000, seed=0, L=8, T=4, weights=[16],
                           **_CRC6, mode="fp32",
                           desc="RM(2,6)+CRC-6, Eb/N0 {ebn0} dB, {frames} frames, seed {seed}, L=8, T=4, "
                                "2604 w16 patterns, FP32 scoring"),
    "rm27_crc6_1p5db": dict(steps=50, code="rm27_crc6", m=7, r=2, ebn0=1.5, frames=1_000_000, seed=2, L=16, T=6,
                            weights=[32], **_CRC6, desc="RM(2,7)+CRC-6, Eb/N0 {ebn0} dB, {frames} frames, seed {seed}, "
                                                        "L=16, T=6, 10668 w32 patterns"),
    "rm27_crc6_osd2": dict(steps=30, code="rm27_crc6", m=7, r=2, ebn0=1.5, frames=1_000_000, seed=2, L=16, T=6,
                           weights=[32], osd=2, **_CRC6,
                           desc="RM(2,7)+CRC-6 with CRC early exit, Eb/N0 {ebn0} dB, {frames} frames, seed {seed}, "
                                "OSD(2) stage 1, L=16, T=6, 10668 w32 patterns"),
    "rm26_crc6_l32": dict(steps=10, code="rm26_crc6", m=6, r=2, ebn0=0.5, frames=200_000, seed=3, L=32, T=8,
                          weights=[16, 24], **_CRC6,
                          desc="RM(2,6)+CRC-6, Eb/N0 {ebn0} dB, {frames} frames, seed {seed}, L=32, T=8, "
                               "294252 w16+w24 patterns"),
}
# The paper's RM experiment (Sec. IV-A settings, Table II): RM(128, 29) with no CRC, stage 2
# always on (P_act = 1, Sec. III-C), OSD(order) anchors, J = 4, the r = 1 sphere
# (the 10,668 weight-32 codewords). The list size and Eb/N0 are not printed in
# the text; L = 16 and 1 dB (oracle FER about 2.5 %) are this workload's choice.
for _o in (2, 3, 4):
    WORKLOADS[f"rm27_osd{_o}_aom"] = dict(
        code="rm27", m=7, r=2, ebn0=1.0, frames=1_000_000, seed=6, L=16, T=4, steps=10, weights=[32], osd=_o, aom=True,
        **_NOCRC, desc=f"RM(128,29) no CRC, always-on stage 2, Eb/N0 {{ebn0}} dB, {{frames}} frames, seed {{seed}}, "
                       f"OSD({_o}) stage 1, L=16, J=4, 10668 w32 patterns")


def resolve_workload(name: str, args) -> dict:
    """The named workload with the command line's overrides applied."""
    w = dict(WORKLOADS[name])
    if getattr(args, "ebn0", None) is not None:
        w["ebn0"] = float(args.ebn0)
    if getattr(args, "seed", None) is not None:
        w["seed"] = int(args.seed)
    if getattr(args, "frames", 0):
        w["frames"] = int(args.frames)
    if getattr(args, "mode", None) is None:
        args.mode = w.get("mode", "bf16x2")
    w["name"] = name
    w["desc"] = w["desc"].format(ebn0=f"{w['ebn0']:g}", frames=f"{w['frames']:.0e}".replace("+0", ""), seed=w["seed"])
    return w


def workload_config(w: dict, args, world: int) -> dict:
    """The `config` object of the JSON line; both arms print the same one."""
    return {"workload": w["desc"], "name": w["name"], "frames_per_rank": w["frames"], "L": w["L"], "T": w["T"],
            "stage1": f"OSD({w['osd']})" if w.get("osd") is not None else "SC-list",
            "always_on": bool(w.get("aom", False)), "scoring": args.mode,
            "l2": "inputs larger than L2 (y is %.0f MB per step)" % (w["frames"] * (1 << w["m"]) * 4 / 1e6),
            "parallelism": f"replicas x{world} (batch b of the seed-{w['seed']} stream on rank b mod {world})"}


def load_peaks():
    p = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(p):
        with open(p) as fh:
            d = json.load(fh)
        return dict(hbm_gbs=d["hbm_gbs"], bf16=d["bf16_tflops"], bf16_sus=d["bf16_tflops_sustained"],
                    sm_max_mhz=d.get("sm_max_mhz", 2070.0), source="measured")
    return dict(hbm_gbs=6800.0, bf16=1900.0, bf16_sus=1700.0, sm_max_mhz=2070.0, source="fallback")


# ---- clocks -------------------------------------------------------------------

class ClockSampler:
    """SM clock and throttle reasons of one GPU, sampled during the timed region.

    Reads NVML through ctypes every 5 ms (nothing is set); without NVML it
    falls back to `nvidia-smi -lms 100`."""
    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")
    # throttle-reason bits of nvmlDeviceGetCurrentClocksEventReasons
    _BITS = {"sw_power_cap": 0x4, "hw_slowdown": 0x8, "sw_thermal_slowdown": 0x20, "hw_thermal_slowdown": 0x40}

    def __init__(self, gpu_index: int, period_s: float = 0.005):
        self.gpu = gpu_index
        self.period = period_s
        self.proc = None
        self.lines = []
        self.samples = []   # (time, sm_mhz, reasons bitmask, power_w) from NVML
        self.t = None
        self._stop = threading.Event()
        self.nvml = None
        self.source = None

    def _nvml_open(self):
        import ctypes

        try:
            lib = ctypes.CDLL("libnvidia-ml.so.1")
        except OSError:
            return None
        if lib.nvmlInit_v2() != 0:
            return None
        # the process sees its GPU by CUDA ordinal; map it to NVML through the PCI bus id
        h = ctypes.c_void_p()
        bus = None
        try:
            import torch

            p = torch.cuda.get_device_properties(self.gpu)
            bus = "%08x:%02x:%02x.0" % (getattr(p, "pci_domain_id", 0), p.pci_bus_id, p.pci_device_id)
        except Exception:
            bus = None
        ok = bus is not None and lib.nvmlDeviceGetHandleByPciBusId_v2(bus.encode(), ctypes.byref(h)) == 0
        if not ok and lib.nvmlDeviceGetHandleByIndex_v2(self.gpu, ctypes.byref(h)) != 0:
            return None
        return lib, h

    def start(self):
        self.nvml = self._nvml_open()
        if self.nvml is not None:
            self.source = "nvml 5 ms"
            self.t = threading.Thread(target=self._poll_nvml, daemon=True)
            self.t.start()
            return
        try:
            self.proc = subprocess.Popen(["nvidia-smi", "-i", str(self.gpu), f"--query-gpu={self.FIELDS}",
                                          "--format=csv,noheader,nounits", "-lms", "100"],
                                         stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
        except (OSError, ValueError):
            self.proc = None
            return
        self.source = "nvidia-smi 100 ms"
        self.t = threading.Thread(target=self._read, daemon=True)
        self.t.start()

    def _poll_nvml(self):
        import ctypes

        lib, h = self.nvml
        clk, mx, pw = ctypes.c_uint(), ctypes.c_uint(), ctypes.c_uint()
        rs = ctypes.c_ulonglong()
        reasons_fn = getattr(lib, "nvmlDeviceGetCurrentClocksEventReasons", None) or \
            getattr(lib, "nvmlDeviceGetCurrentClocksThrottleReasons")
        if lib.nvmlDeviceGetMaxClockInfo(h, 1, ctypes.byref(mx)) == 0:  # NVML_CLOCK_SM = 1
            self.max_mhz = float(mx.value)
        while not self._stop.is_set():
            a = lib.nvmlDeviceGetClockInfo(h, 1, ctypes.byref(clk))
            b = reasons_fn(h, ctypes.byref(rs))
            c = lib.nvmlDeviceGetPowerUsage(h, ctypes.byref(pw))
            if a == 0:
                self.samples.append((time.time(), float(clk.value), int(rs.value) if b == 0 else 0,
                                     pw.value / 1000.0 if c == 0 else 0.0))
            time.sleep(self.period)

    def _read(self):
        for ln in self.proc.stdout:
            self.lines.append((time.time(), ln.strip()))

    def stop(self):
        self._stop.set()
        if self.proc is not None:
            self.proc.terminate()
            try:
                self.proc.wait(timeout=5)
            except subprocess.TimeoutExpired:
                self.proc.kill()
        if self.t is not None:
            self.t.join(timeout=5)

    def summary(self, t0: float, t1: float):
        if self.samples:
            inside = [s for s in self.samples if t0 <= s[0] <= t1] or self.samples
            sm = [s[1] for s in inside]
            reasons = sorted({nm for s in inside for nm, bit in self._BITS.items() if s[2] & bit})
            return {"sm_mhz": statistics.median(sm), "sm_max_mhz": getattr(self, "max_mhz", None),
                    "sm_mhz_min": min(sm), "reasons": reasons, "samples": len(inside), "source": self.source,
                    "power_w_max": max(s[3] for s in inside)}
        rows = []
        for ts, ln in self.lines:
            parts = [x.strip() for x in ln.split(",")]
            if len(parts) < 9:
                continue
            rows.append((ts, parts))
        inside = [p for ts, p in rows if t0 <= ts <= t1] or [p for _, p in rows]
        if not inside:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"], "samples": 0,
                    "source": None}

        def num(x):
            try:
                return float(x)
            except ValueError:
                return None

        sm = [num(p[1]) for p in inside if num(p[1]) is not None]
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        reasons = sorted({names[i] for p in inside for i in range(4) if p[5 + i].lower() == "active"})
        return {"sm_mhz": statistics.median(sm) if sm else None, "sm_max_mhz": num(inside[0][2]),
                "sm_mhz_min": min(sm) if sm else None, "reasons": reasons, "samples": len(inside),
                "source": self.source, "power_w_max": max((num(p[3]) or 0.0) for p in inside)}


# ---- helpers ------------------------------------------------------------------

def rank_first_frame(frames_per_rank: int, world: int, rank: int) -> int:
    """First frame of this rank's batch: batches of `frames_per_rank` frames of
    one seeded stream are dealt round-robin (batch b to rank b mod world), one
    batch per rank, so rank r decodes frames [r B, (r + 1) B)."""
    import synth

    (b,) = synth.shard_batches(world, world, rank)
    return b * frames_per_rank


class RankReduce:
    """Timer / counter reductions over ranks (a barrier, max and sum of scalars).
    With no process group everything is local."""

    def __init__(self, dist=None, device: str = "cpu"):
        self.dist = dist
        self.device = device

    def barrier(self):
        if self.dist is not None:
            self.dist.barrier()

    def _reduce(self, x: float, op) -> float:
        if self.dist is None:
            return float(x)
        import torch

        t = torch.tensor([float(x)], dtype=torch.float64, device=self.device)
        self.dist.all_reduce(t, op=op)
        return float(t.item())

    def max(self, x: float) -> float:
        return self._reduce(x, None if self.dist is None else self.dist.ReduceOp.MAX)

    def sum(self, x: float) -> float:
        return self._reduce(x, None if self.dist is None else self.dist.ReduceOp.SUM)


def clopper_pearson(k: int, n: int, alpha: float = 0.05):
    from scipy.stats import beta

    lo = 0.0 if k == 0 else float(beta.ppf(alpha / 2, k, n - k + 1))
    hi = 1.0 if k == n else float(beta.ppf(1 - alpha / 2, k + 1, n - k))
    return lo, hi


def src_hash(*rel):
    h = hashlib.sha256()
    for r in rel:
        with open(os.path.join(ROOT, r), "rb") as fh:
            h.update(fh.read())
    return h.hexdigest()[:16]


def recorded_traffic(kernel: str, source_hash: str, unit: str):
    """DRAM bytes per unit (row or frame) from the committed ncu summary of this
    kernel, if it was taken on the current kernel source; else None."""
    p = os.path.join(ROOT, "profiles", f"{kernel}_ncu.md")
    if not os.path.exists(p):
        return None
    with open(p) as fh:
        txt = fh.read()
    m_src = re.search(r"source_hash:\s*([0-9a-f]+)", txt)
    m_b = re.search(rf"dram_bytes_per_{unit}:\s*([0-9.eE+]+)", txt)
    if not m_src or not m_b or m_src.group(1) != source_hash:
        return None
    return float(m_b.group(1))


def oracle_code_for(wl_cfg):
    import oracle

    code = oracle.rm_code(wl_cfg["m"], wl_cfg["r"], crc_poly=wl_cfg["crc_poly"], crc_len=wl_cfg["crc_len"])
    return code.with_patterns(code.enumerate_codewords(wl_cfg["weights"]))


def oracle_run(code, wl_cfg, y, threads):
    return code.decode(y, wl_cfg["L"], wl_cfg["T"], threads=threads, osd_order=wl_cfg.get("osd"),
                       aom=bool(wl_cfg.get("aom", False)))


def time_oracle(wl_cfg, seconds: float, threads: int):
    """Oracle frames/s on a bounded sample (first frames of the same stream)."""
    import oracle  # noqa: F401  (test infrastructure; cpu_baseline leg only)
    import synth

    probe = synth.make_workload(wl_cfg["code"], wl_cfg["ebn0"], 500, seed=wl_cfg["seed"])
    code = oracle_code_for(wl_cfg)
    oracle_run(code, wl_cfg, probe.y[:50], threads)  # builds the oracle
    t = time.perf_counter()
    oracle_run(code, wl_cfg, probe.y, threads)
    rate = probe.B / max(time.perf_counter() - t, 1e-6)
    n = int(min(max(500, rate * seconds), wl_cfg["frames"]))
    wl = synth.make_workload(wl_cfg["code"], wl_cfg["ebn0"], n, seed=wl_cfg["seed"])
    t = time.perf_counter()
    out = oracle_run(code, wl_cfg, wl.y, threads)
    dt = time.perf_counter() - t
    return wl, out, dt


# ---- reference arm (the oracle on host cores) ---------------------------------

def run_reference(args, wl_cfg):
    rank = int(os.environ.get("RANK", "0"))
    world = int(os.environ.get("WORLD_SIZE", "1"))
    if rank != 0:
        return None
    import oracle  # noqa: F401  (the reference arm is the oracle on host cores)
    import synth

    threads = os.cpu_count() or 1
    code = oracle_code_for(wl_cfg)
    probe = synth.make_workload(wl_cfg["code"], wl_cfg["ebn0"], 500, seed=wl_cfg["seed"])
    oracle_run(code, wl_cfg, probe.y[:50], threads)
    t = time.perf_counter()
    oracle_run(code, wl_cfg, probe.y, threads)
    rate = probe.B / max(time.perf_counter() - t, 1e-6)
    per_step = int(min(max(200, rate * args.ref_step_seconds), wl_cfg["frames"]))
    wl = synth.make_workload(wl_cfg["code"], wl_cfg["ebn0"], per_step, seed=wl_cfg["seed"])
    for _ in range(args.warmup):
        oracle_run(code, wl_cfg, wl.y[:min(per_step, 200)], threads)
    times = []
    for _ in range(args.steps):
        t = time.perf_counter()
        oracle_run(code, wl_cfg, wl.y, threads)
        times.append(time.perf_counter() - t)
    total = sum(times)
    value = per_step * args.steps / total
    line = {
        "metric": METRIC, "value": value, "unit": "frames/s", "n_gpus": args.gpus, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": 1e3 * total / args.steps, "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
        "impl": "reference",
        "config": workload_config(wl_cfg, args, world),
        "cpu_baseline": {"value": value, "unit": "frames/s", "cores": threads, "kind": "oracle",
                         "sample": f"first {per_step} frames of the workload stream per step (each step a bounded "
                                   f"sample of the {wl_cfg['frames']}-frame batch)"},
        "e2e": {"value": value, "unit": "frames/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }
    print(json.dumps(line), flush=True)
    return line


# ---- our arm ------------------------------------------------------------------

def run_ours(args, wl_cfg):
    import torch

    import synth
    from paper_2602_08501_gb300 import mpwsd

    rank = int(os.environ.get("RANK", "0"))
    world = int(os.environ.get("WORLD_SIZE", "1"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    torch.cuda.set_device(local)
    dist = None
    if world > 1:
        import torch.distributed as dist

        dist.init_process_group("nccl", device_id=torch.device("cuda", local))
    red = RankReduce(dist, "cuda")
    barrier, allmax, allsum = red.barrier, red.max, red.sum

    frames = wl_cfg["frames"]
    first = rank_first_frame(frames, world, rank)
    wl = synth.make_workload(wl_cfg["code"], wl_cfg["ebn0"], frames, seed=wl_cfg["seed"], first_frame=first)
    n, L, T = wl.n, wl_cfg["L"], wl_cfg["T"]
    W = (n + 63) // 64
    aom = bool(wl_cfg.get("aom", False))
    osd = wl_cfg.get("osd")
    code = mpwsd.Code.rm(wl_cfg["m"], wl_cfg["r"], crc_poly=wl_cfg["crc_poly"], crc_len=wl_cfg["crc_len"],
                         weights=wl_cfg["weights"])
    P = code.n_patterns
    y_host = torch.from_numpy(wl.y).pin_memory()
    y_dev = y_host.to("cuda", non_blocking=False)
    cw_dev = torch.empty((frames, W), dtype=torch.int64, device="cuda")
    fl_dev = torch.empty((frames,), dtype=torch.int16, device="cuda")
    stream = torch.cuda.current_stream()

    tuning = None
    if args.tune:
        # the autotuner times every scoring shape and split target on this batch
        # (graph replays), applies the fastest and reports it beside the default
        from paper_2602_08501_gb300 import autotune

        if osd is None and not aom:
            r = autotune.tune(code, y_dev, L, T, batch_sizes=(frames,), use_cache=False, reps=3)
            tuning = {"shape": r["shape"], "split_items": r["value"], "default_ms": r["default_ms"],
                      "tuned_ms": r["times_ms"][f"{r['shape']}/{r['value']}"], "times_ms": r["times_ms"]}

    def step():
        code.decode(y_dev, L, T, score_mode=args.mode, cw_out=cw_dev, flags_out=fl_dev, osd_order=osd,
                    always_on=aom)

    for _ in range(args.warmup):
        step()
    torch.cuda.synchronize()

    clocks = ClockSampler(local)
    clocks.start()
    time.sleep(0.2)
    code.reset_stats()
    code.profile_begin()
    evs = [torch.cuda.Event(enable_timing=True) for _ in range(args.steps + 1)]
    barrier()
    torch.cuda.synchronize()
    t_wall0 = time.time()
    evs[0].record(stream)
    for k in range(args.steps):
        step()
        evs[k + 1].record(stream)
    torch.cuda.synchronize()
    t_wall1 = time.time()
    barrier()
    prof = code.profile_end()
    stats = code.stats()
    step_ms = [evs[k].elapsed_time(evs[k + 1]) for k in range(args.steps)]
    total_ms = evs[0].elapsed_time(evs[-1])
    time.sleep(0.05)
    clocks.stop()
    clk = clocks.summary(t_wall0, t_wall1)

    # end to end through the binding with pinned host buffers
    cw_host = torch.empty((frames, W), dtype=torch.int64).pin_memory()
    fl_host = torch.empty((frames,), dtype=torch.int16).pin_memory()

    def e2e_step():
        # the library's host-buffer entry point: y in, codewords and flags out, with
        # the input copies overlapping stage 1
        code.decode_host(y_host, L, T, score_mode=args.mode, cw_out=cw_host, flags_out=fl_host, osd_order=osd,
                         always_on=aom)

    e2e_steps = max(1, args.steps)
    e2e_step()
    torch.cuda.synchronize()
    barrier()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    for _ in range(e2e_steps):
        e2e_step()
    e1.record(stream)
    torch.cuda.synchronize()
    e2e_ms = allmax(e0.elapsed_time(e1))

    max_ms = allmax(total_ms)
    total_frames = allsum(frames * args.steps)
    total_evals = allsum(stats["pattern_evals"])
    value = total_frames / (max_ms / 1e3)
    timed_s = max_ms / 1e3

    # outcome of the last step (identical every step)
    cw = cw_host.numpy().view(np.uint64)
    fl = fl_host.numpy().view(np.uint16)
    tx = synth.pack_bits(wl.cw)
    err = np.any(cw != tx, axis=1)
    fer = float(err.mean())
    p_act = float(np.mean(fl & 1))

    peaks = load_peaks()
    kinds = {k: v for k, v in prof.items() if v["launches"]}
    busy = sum(v["ms"] for v in kinds.values())
    dominant = max(kinds, key=lambda k: kinds[k]["ms"])
    shares = {k: {"launches": v["launches"], "ms": round(v["ms"], 4), "share": round(v["ms"] / busy, 4)}
              for k, v in kinds.items()}
    sm_clock_max = peaks["sm_max_mhz"] * 1e6
    alu_peak = 152 * 128 * sm_clock_max  # lane-ops/s: 152 SMs x 128 INT32/FP32 lanes x max SM clock
    evals = stats["pattern_evals"]
    wts = [bin(int(p[0])).count("1") + (bin(int(p[1])).count("1") if W > 1 else 0) for p in code.patterns]
    wbar = float(np.mean(wts)) if P else 0.0
    wmax = max(wts) if P else 0
    # the scoring launches run inside a timed region of a few seconds at most: the
    # burst peak (a GEMM timed alone) is the denominator, the sustained one beside it
    long_region = timed_s > 5.0
    tc_peak = peaks["bf16_sus"] if long_region else peaks["bf16"]
    tc_kind = ("bf16 sustained" if long_region else "bf16 burst") + \
        f" ({peaks['source']}; timed region {timed_s:.2f} s)"

    def roofline_for(kname):
        ms = kinds[kname]["ms"]
        launches = kinds[kname]["launches"]
        per_launch_s = ms / 1e3 / launches
        traffic_note = "ncu dram__bytes_read.sum + dram__bytes_write.sum of a smaller capture (profiles/), " \
                       "scaled per launch by the units it processes; null when the kernel source changed since"
        if kname == "score_tc":
            flops = evals * 2 * n * 2 / launches  # dense bf16 work per launch: 2 n flops x 2 splits per pattern-eval
            ach = flops / per_launch_s / 1e12
            src = src_hash("paper_2602_08501_gb300/csrc/score_tc.cu", "paper_2602_08501_gb300/csrc/score_tc_impl.cuh",
                           "paper_2602_08501_gb300/csrc/common.cuh", "paper_2602_08501_gb300/csrc/internal.h")
            bpr = recorded_traffic("score_tc", src, "row")
            tr = None if bpr is None else bpr * (evals / P) / launches  # scaled by active rows per launch
            return {"bound": "tensor", "achieved": ach, "peak": tc_peak, "unit": "TFLOP/s",
                    "frac": ach / tc_peak, "frac_of_sustained": ach / peaks["bf16_sus"], "traffic": tr,
                    "traffic_source": traffic_note, "kernel": "score_tc", "peak_kind": tc_kind,
                    "flops_per_launch": flops}
        if kname == "score_fp32":
            adds = evals * wbar / launches
            ach = adds / per_launch_s / 1e12
            return {"bound": "alu", "achieved": ach, "peak": alu_peak / 1e12, "unit": "Tadd/s",
                    "frac": ach / (alu_peak / 1e12), "traffic": None, "kernel": "score_fp32",
                    "peak_kind": "152 SMs x 128 FP32 lanes x max SM clock"}
        if kname == "score_flats":
            # the transform's additions: n log2 n per row, then kd 2^kd per complement (kd = m - log2 w)
            kd = wl_cfg["m"] - int(math.log2(wmax))
            adds = evals / P * (n * math.log2(n) + (P >> kd) * kd * (1 << kd)) / launches
            ach = adds / per_launch_s / 1e12
            src = src_hash("paper_2602_08501_gb300/csrc/score_flats.cu", "paper_2602_08501_gb300/csrc/common.cuh",
                           "paper_2602_08501_gb300/csrc/internal.h")
            bpr = recorded_traffic("score_flats", src, "row")
            tr = None if bpr is None else bpr * (evals / P) / launches
            return {"bound": "alu", "achieved": ach, "peak": alu_peak / 1e12, "unit": "Tadd/s",
                    "frac": ach / (alu_peak / 1e12), "traffic": tr, "traffic_source": traffic_note,
                    "kernel": "score_flats",
                    "peak_kind": "152 SMs x 128 INT32 lanes x max SM clock",
                    "adds_per_launch": adds, "pattern_sums_per_s": evals / launches / per_launch_s}
        if kname == "scl":
            ops = frames * 4 * L * n * math.log2(n)  # per launch (one per step): Table I, (4/3) L log2 N ED units x 3N
            ach = ops / per_launch_s / 1e12
            src = src_hash("paper_2602_08501_gb300/csrc/scl_impl.cuh", "paper_2602_08501_gb300/csrc/internal.h")
            bpf = recorded_traffic("scl", src, "frame")
            tr = None if bpf is None else bpf * frames
            return {"bound": "alu", "achieved": ach, "peak": alu_peak / 1e12, "unit": "Top/s",
                    "frac": ach / (alu_peak / 1e12), "traffic": tr, "traffic_source": traffic_note, "kernel": "scl",
                    "peak_kind": "152 SMs x 128 INT32 lanes x max SM clock", "ops_per_launch": ops}
        if kname == "osd":
            # per frame: the discrepancy of every candidate (n weighted adds each) and the elimination (n k)
            kk = int(code.k)
            order = int(osd or 0)
            ncand = sum(math.comb(kk, w) for w in range(order + 1))
            ops = frames * n * (ncand + kk)  # per launch (one per step)
            ach = ops / per_launch_s / 1e12
            src = src_hash("paper_2602_08501_gb300/csrc/osd.cu", "paper_2602_08501_gb300/csrc/common.cuh",
                           "paper_2602_08501_gb300/csrc/internal.h")
            # the recorded capture is of the always-on workload (every frame writes trajectories)
            bpf = recorded_traffic("osd", src, "frame") if aom else None
            tr = None if bpf is None else bpf * frames
            return {"bound": "alu", "achieved": ach, "peak": alu_peak / 1e12, "unit": "Top/s",
                    "frac": ach / (alu_peak / 1e12), "traffic": tr, "traffic_source": traffic_note, "kernel": "osd",
                    "peak_kind": "152 SMs x 128 INT32 lanes x max SM clock", "ops_per_launch": ops}
        if kname == "hop":
            rows = evals / P if P else 0.0
            wq = math.ceil(wmax / 4)
            cand = stats["rerank_candidates"] / rows if rows else 0.0
            hopf = stats["hops"] / rows if rows else 0.0
            src = src_hash("paper_2602_08501_gb300/csrc/traj.cu", "paper_2602_08501_gb300/csrc/common.cuh",
                           "paper_2602_08501_gb300/csrc/internal.h")
            if args.mode == "bf16x2":
                # the class holds the twin retirement alone (the resolution kernel takes the
                # hop decisions): per hopped row its entry, its centre, the centres and states
                # of the (L - 1) / 2 lower-numbered trajectories of its frame on average, and
                # its next-iteration entry
                units = stats["hops"]
                bpr = 4 + 8 * W + (L - 1) / 2 * (8 * W + 4) + 4
                ach = bpr * units / launches / per_launch_s / 1e9
                return {"bound": "hbm", "achieved": ach, "peak": peaks["hbm_gbs"], "unit": "GB/s",
                        "frac": ach / peaks["hbm_gbs"], "traffic": None, "kernel": "hop",
                        "peak_kind": f"HBM copy, {peaks['source']}", "bytes_per_hopped_row": bpr,
                        "note": "twin retirement only (the resolution kernel takes the hop decisions)"}
            # bytes a row needs: its list entry (4 + 32), centre, D, state, 1/L of its frame's y row and
            # slot data, the supports of its candidates, and on a hop the written centre, D, state, entry
            bpr = 36 + 8 * W + 12 + (4 * n + 8) / L + cand * 4 * wq + hopf * (8 * W + 16)
            ach = bpr * rows / launches / per_launch_s / 1e9
            rec = recorded_traffic("hop", src, "row")
            tr = None if rec is None else rec * rows / launches
            return {"bound": "hbm", "achieved": ach, "peak": peaks["hbm_gbs"], "unit": "GB/s",
                    "frac": ach / peaks["hbm_gbs"], "traffic": tr, "traffic_source": traffic_note, "kernel": "hop",
                    "peak_kind": f"HBM copy, {peaks['source']}", "bytes_per_row": bpr}
        if kname == "resolve":
            # bytes a row needs: its list (32), row / slot / frame ids and ||y||_1 (12), centre, D and
            # state (12), 1/L of its frame's y row, the supports of one group of kGroupCols = 8
            # patterns, and on a hop the written centre, D and state plus its entry (8W + 16)
            rows = evals / P if P else 0.0
            wq = math.ceil(wmax / 4)
            hopf = stats["hops"] / rows if rows else 0.0
            bpr = 32 + 12 + 8 * W + 12 + (4 * n + 8) / L + 8 * 4 * wq + hopf * (8 * W + 16)
            ach = bpr * rows / launches / per_launch_s / 1e9
            src = src_hash("paper_2602_08501_gb300/csrc/score_tc.cu", "paper_2602_08501_gb300/csrc/common.cuh",
                           "paper_2602_08501_gb300/csrc/internal.h")
            rec = recorded_traffic("resolve", src, "row")
            tr = None if rec is None else rec * rows / launches
            return {"bound": "hbm", "achieved": ach, "peak": peaks["hbm_gbs"], "unit": "GB/s",
                    "frac": ach / peaks["hbm_gbs"], "traffic": tr, "traffic_source": traffic_note,
                    "kernel": "resolve", "peak_kind": f"HBM copy, {peaks['source']}", "bytes_per_row": bpr}
        return {"bound": "alu", "achieved": None, "peak": None, "unit": None, "frac": None, "traffic": None,
                "kernel": kname}

    roof = roofline_for(dominant)
    others = [roofline_for(k) for k in ("scl", "osd", "score_tc", "resolve", "score_fp32", "score_flats", "hop")
              if k in kinds and k != dominant]

    line = {
        "metric": METRIC, "value": value, "unit": "frames/s", "n_gpus": world, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": max_ms / args.steps, "higher_is_better": True, "scaling": "weak",
        "vs_baseline": None, "data": "synthetic",
        "dtype": {"bf16x2": "bf16x2+f64", "fp32": "f32+f64", "flats": "i32+f64"}[args.mode],
        "config": workload_config(wl_cfg, args, world),
        "pattern_evals_per_s": {
            "scored": total_evals / timed_s,
            "what": "(trajectory, pattern) pairs the GPU scored per second; trajectories that hop onto the "
                    "centre of a live lower-numbered one of their frame are retired and not scored"},
        "latency_ms": {"p50": statistics.median(step_ms), "p99": float(np.percentile(step_ms, 99)),
                       "what": "per batch step of %d frames" % frames},
        "fer": fer, "p_act": p_act,
        "roofline": roof, "roofline_other": others, "kernels": shares,
        "e2e": {"value": total_frames / args.steps * e2e_steps / (e2e_ms / 1e3), "unit": "frames/s",
                "h2d_bytes_per_step": int(y_host.numel() * 4),
                "d2h_bytes_per_step": int(cw_host.numel() * 8 + fl_host.numel() * 2)},
        "gpu_launches": int(stats["kernel_launches"]),
        "clocks": {k: clk.get(k) for k in ("sm_mhz", "sm_max_mhz", "sm_mhz_min", "reasons", "samples", "source")},
        "stats": {k: stats[k] for k in ("stage2_frames", "trajectories", "hops", "rerank_candidates", "rescans")},
        "tuning": tuning if tuning else {"shape": code.tune_get(mpwsd.TUNE_TC_SHAPE),
                                         "split_items": code.tune_get(mpwsd.TUNE_SPLIT_ITEMS), "tuned": False},
    }

    if rank == 0 and not args.no_cpu:
        threads = os.cpu_count() or 1
        owl, oout, odt = time_oracle(wl_cfg, args.cpu_seconds, threads)
        nb = owl.B
        # rank 0 decodes frames [0, B) of the stream, the oracle's sample is its first nb frames
        mism = np.any(oout["cw"] != cw[:nb], axis=1) | ((oout["flags"] & 0x1F3) != (fl[:nb] & 0x1F3))
        tie = oout["min_gap"] < 1e-6 * np.sum(owl.y.astype(np.float64) ** 2, axis=1)
        oerr = np.any(oout["cw"] != tx[:nb], axis=1)
        lo, hi = clopper_pearson(int(oerr.sum()), nb)
        alg1_per_frame = float(oout["evals"].sum()) / nb
        line["cpu_baseline"] = {"value": nb / odt, "unit": "frames/s", "cores": threads, "kind": "oracle",
                                "sample": f"first {nb} frames of the same stream (seed {wl_cfg['seed']})",
                                "pattern_evals_per_s_algorithm1": float(oout["evals"].sum()) / odt}
        line["pattern_evals_per_s"]["algorithm1_equivalent"] = value * alg1_per_frame
        line["pattern_evals_per_s"]["algorithm1_what"] = (
            "GPU frames/s x the (trajectory, pattern) pairs per frame that Algorithm 1 scores (twins included), "
            "counted by the oracle on its sample; comparable with cpu_baseline.pattern_evals_per_s_algorithm1")
        line["parity"] = {"frames": nb, "mismatches": int(mism.sum()), "mismatches_outside_near_ties":
                          int((mism & ~tie).sum()), "near_ties": int(tie.sum()),
                          "flags_compared": "stage 2, CRC ok, iterations, error"}
        line["fer_check"] = {"gpu_fer": fer, "oracle_fer_sample": float(oerr.mean()), "oracle_ci95": [lo, hi],
                             "gpu_in_ci": bool(lo <= fer <= hi)}
    if rank == 0:
        print(json.dumps(line), flush=True)
    if dist is not None:
        dist.destroy_process_group()
    return line


def run_serving(args):
    """Workload 5: Poisson arrivals of mixed RM(2,6)+CRC-6 / RM(2,7)+CRC-6 frames
    (50/50), Eb/N0 uniform in [0.5, 3] dB, through the continuous-batching loop
    (one stage-2 pool per code); one JSON line with throughput, p50/p99
    per-frame latency and stage-2 rows per pool step for each arrival rate."""
    import torch

    import synth
    from paper_2602_08501_gb300 import mpwsd, serving

    torch.cuda.set_device(int(os.environ.get("LOCAL_RANK", "0")))
    rates = [float(r) * 1e6 for r in args.rates.split(",")]
    n_max = int(max(rates) * args.serve_seconds / 2) + 1
    specs = {"rm26": serving.CodeSpec(mpwsd.Code.rm(6, 2, crc_poly=0x21, crc_len=6, weights=[16]), 8, 4),
             "rm27": serving.CodeSpec(mpwsd.Code.rm(7, 2, crc_poly=0x21, crc_len=6, weights=[32]), 16, 6)}
    pools = {"rm26": synth.make_workload("rm26_crc6", (0.5, 3.0), n_max, seed=4),
             "rm27": synth.make_workload("rm27_crc6", (0.5, 3.0), n_max, seed=5)}
    ys = {nm: torch.from_numpy(pools[nm].y).pin_memory() for nm in specs}
    from paper_2602_08501_gb300 import autotune

    tuned = {}
    for nm, sp in specs.items():  # scoring shape and split target on a sample of each code's frames
        sample = ys[nm][:min(n_max, 32768)].cuda()
        sizes = [b for b in (256, 4096, 32768) if b <= sample.shape[0]]
        tuned[nm] = autotune.tune(sp.code, sample, sp.L, sp.T, batch_sizes=sizes, reps=3, use_cache=False)
    srv = serving.Server(specs, max_batch=args.serve_batch, pool_frames=4 * args.serve_batch,
                         min_batch=args.serve_batch // 8, max_wait_s=args.serve_wait_us * 1e-6,
                         pools_per_code=args.serve_pools)
    srv.warmup()  # records each pool's step graph
    out = []
    for rate in rates:
        n_each = int(rate * args.serve_seconds / 2)
        arr = {nm: serving.poisson_arrivals(rate / 2, n_each, seed=100 + i) for i, nm in enumerate(specs)}
        res = srv.run(arr, {nm: ys[nm][:n_each] for nm in specs})
        p = res.percentiles((50, 99))
        fer = {nm: float(np.mean(np.any(res.cw[nm] != synth.pack_bits(pools[nm].cw[:n_each]), axis=1))) for nm in specs}
        # the same rows with a stage 2 run per submission: T scoring passes per submission of a code
        per_sub_launches = sum(res.submissions[nm] * specs[nm].T for nm in specs)
        out.append({"offered_frames_per_s": rate, "served_frames_per_s": res.served / res.wall_s,
                    "p50_ms": p["p50"] * 1e3, "p99_ms": p["p99"] * 1e3, "frames": res.served,
                    "submissions": res.submissions, "mean_submission": float(np.mean(res.batch_sizes)),
                    "pool_steps": res.steps, "stage2_rows_per_step": res.rows_per_step(),
                    "stage2_rows_per_launch_if_per_submission": sum(res.stage2_rows.values()) / max(1, per_sub_launches),
                    "fer": fer})
    line = {"metric": METRIC + " (serving)", "value": max(o["served_frames_per_s"] for o in out), "unit": "frames/s",
            "n_gpus": 1, "higher_is_better": True, "dtype": "bf16x2+f64", "data": "synthetic",
            "config": {"workload": "serving: Poisson arrivals, 50/50 RM(2,6)+CRC-6 (L=8,T=4) / RM(2,7)+CRC-6 (L=16,T=6), "
                                   "Eb/N0 U[0.5,3] dB; one stage-2 pool per code (continuous batching)",
                       "max_batch": args.serve_batch, "pool_frames": srv.slots, "pools_per_code": args.serve_pools,
                       "max_wait_us": args.serve_wait_us, "seconds_per_rate": args.serve_seconds,
                       "tuned": {nm: {"shape": t["shape"], "split_items": t["value"]} for nm, t in tuned.items()}},
            "rates": out}
    print(json.dumps(line), flush=True)


def main():
    ap = argparse.ArgumentParser(description=__doc__, formatter_class=argparse.RawDescriptionHelpFormatter)
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=None,
                    help="timed steps (default: the workload's, about one second of decoding)")
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", choices=["ours", "reference"], default="ours")
    ap.add_argument("--workload", choices=sorted(WORKLOADS) + ["serving"], default="rm26_crc6_1db")
    ap.add_argument("--mode", choices=["bf16x2", "fp32", "flats"], default=None)
    ap.add_argument("--frames", type=int, default=0, help="override frames per step")
    ap.add_argument("--ebn0", type=float, default=None, help="override the workload's Eb/N0 (dB)")
    ap.add_argument("--seed", type=int, default=None, help="override the workload's seed")
    ap.add_argument("--cpu-seconds", type=float, default=12.0, help="oracle sample size in CPU seconds")
    ap.add_argument("--ref-step-seconds", type=float, default=6.0)
    ap.add_argument("--no-cpu", action="store_true")
    ap.add_argument("--tune", action="store_true", help="autotune the scoring shape and split target first")
    ap.add_argument("--rates", default="1,2,5,10,20", help="serving: offered M frames/s")
    ap.add_argument("--serve-seconds", type=float, default=0.1, help="serving: seconds of traffic per rate")
    ap.add_argument("--serve-batch", type=int, default=65536)
    ap.add_argument("--serve-wait-us", type=float, default=200.0)
    ap.add_argument("--serve-pools", type=int, default=1, help="serving: stage-2 pools per code (one stream each)")
    args = ap.parse_args()
    args.warmup = max(args.warmup, 3)  # at least 3 untimed warm-up steps
    if args.workload == "serving":
        args.steps = args.steps or 1
        args.mode = args.mode or "bf16x2"
        run_serving(args)
        return
    wl_cfg = resolve_workload(args.workload, args)
    if args.steps is None:
        args.steps = wl_cfg.get("steps", 20) if args.impl == "ours" else 3
    if args.impl == "reference":
        run_reference(args, wl_cfg)
    else:
        run_ours(args, wl_cfg)


if __name__ == "__main__":
    main()
