#!/usr/bin/env python
"""Throughput of the two-stage SCL + MP-WSD decoder on GB300 (one JSON line).

A step decodes one batch of synthetic frames through the whole hot path
(stage-1 SC-list + CRC + compaction, T iterations of scoring / FP64 re-rank /
hop, final select). Default workload: RM(2,6)+CRC-6 (x^6+x^5+1), Eb/N0 = 1 dB,
10^6 frames from seed 1, L = 8, T = 4, all 2604 weight-16 patterns, BF16
hi+lo tensor-core scoring. y (256 MB) is larger than L2, so no flush is
needed between steps.

    python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference]

Under torchrun each rank decodes its own batch (seed + rank); the only
collectives are a barrier and the max of the timers.
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

WORKLOADS = {
    "rm26_crc6_1db": dict(code="rm26_crc6", m=6, r=2, ebn0=1.0, frames=1_000_000, seed=1, L=8, T=4, weights=[16],
                          desc="RM(2,6)+CRC-6, Eb/N0 1 dB, 1e6 frames, seed 1, L=8, T=4, 2604 w16 patterns"),
    "rm27_crc6_1p5db": dict(code="rm27_crc6", m=7, r=2, ebn0=1.5, frames=1_000_000, seed=2, L=16, T=6,
                            weights=[32], desc="RM(2,7)+CRC-6, Eb/N0 1.5 dB, 1e6 frames, seed 2, L=16, T=6, "
                                               "10668 w32 patterns"),
    "rm27_crc6_osd2": dict(code="rm27_crc6", m=7, r=2, ebn0=1.5, frames=1_000_000, seed=2, L=16, T=6,
                           weights=[32], osd=2, desc="RM(2,7)+CRC-6, Eb/N0 1.5 dB, 1e6 frames, seed 2, OSD(2) "
                                                     "stage 1, L=16, T=6, 10668 w32 patterns"),
    "rm26_crc6_l32": dict(code="rm26_crc6", m=6, r=2, ebn0=0.5, frames=200_000, seed=3, L=32, T=8,
                          weights=[16, 24], desc="RM(2,6)+CRC-6, Eb/N0 0.5 dB, 2e5 frames, seed 3, L=32, T=8, "
                                                 "294252 w16+w24 patterns"),
}


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
    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_index: int):
        self.gpu = gpu_index
        self.proc = None
        self.lines = []
        self.t = None

    def start(self):
        try:
            self.proc = subprocess.Popen(["nvidia-smi", "-i", str(self.gpu), f"--query-gpu={self.FIELDS}",
                                          "--format=csv,noheader,nounits", "-lms", "100"],
                                         stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
        except (OSError, ValueError):
            self.proc = None
            return
        self.t = threading.Thread(target=self._read, daemon=True)
        self.t.start()

    def _read(self):
        for ln in self.proc.stdout:
            self.lines.append((time.time(), ln.strip()))

    def stop(self):
        if self.proc is not None:
            self.proc.terminate()
            try:
                self.proc.wait(timeout=5)
            except subprocess.TimeoutExpired:
                self.proc.kill()
            self.t.join(timeout=5)

    def summary(self, t0: float, t1: float):
        rows = []
        for ts, ln in self.lines:
            parts = [x.strip() for x in ln.split(",")]
            if len(parts) < 9:
                continue
            rows.append((ts, parts))
        inside = [p for ts, p in rows if t0 <= ts <= t1] or [p for _, p in rows]
        if not inside:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"], "samples": 0}

        def num(x):
            try:
                return float(x)
            except ValueError:
                return None

        sm = [num(p[1]) for p in inside if num(p[1]) is not None]
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        reasons = sorted({names[i] for p in inside for i in range(4) if p[5 + i].lower() == "active"})
        return {"sm_mhz": statistics.median(sm) if sm else None, "sm_max_mhz": num(inside[0][2]),
                "reasons": reasons, "samples": len(inside),
                "power_w_max": max((num(p[3]) or 0.0) for p in inside)}


# ---- helpers ------------------------------------------------------------------

def rank_seed(base_seed: int, rank: int) -> int:
    """Each rank decodes its own frames: the workload stream of seed base + rank."""
    return base_seed + rank


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


def oracle_decode(wl_cfg, y, threads):
    import oracle

    code = oracle.rm_code(wl_cfg["m"], wl_cfg["r"], crc_poly=0x21, crc_len=6)
    code = code.with_patterns(code.enumerate_codewords(wl_cfg["weights"]))
    return code, code.decode(y, wl_cfg["L"], wl_cfg["T"], threads=threads, osd_order=wl_cfg.get("osd"))


def time_oracle(wl_cfg, seconds: float, threads: int):
    """Oracle frames/s on a bounded sample (first frames of the same stream)."""
    import oracle  # noqa: F401  (test infrastructure; cpu_baseline leg only)
    import synth

    probe = synth.make_workload(wl_cfg["code"], wl_cfg["ebn0"], 2000, seed=wl_cfg["seed"])
    code, _ = oracle_decode(wl_cfg, probe.y[:200], threads)  # builds the oracle and its pattern set
    t = time.perf_counter()
    code.decode(probe.y, wl_cfg["L"], wl_cfg["T"], threads=threads, osd_order=wl_cfg.get("osd"))
    rate = probe.B / max(time.perf_counter() - t, 1e-6)
    n = int(min(max(2000, rate * seconds), wl_cfg["frames"]))
    wl = synth.make_workload(wl_cfg["code"], wl_cfg["ebn0"], n, seed=wl_cfg["seed"])
    t = time.perf_counter()
    out = code.decode(wl.y, wl_cfg["L"], wl_cfg["T"], threads=threads, osd_order=wl_cfg.get("osd"))
    dt = time.perf_counter() - t
    return wl, out, dt


# ---- reference arm (the oracle on host cores) ---------------------------------

def run_reference(args, wl_cfg):
    rank = int(os.environ.get("RANK", "0"))
    if rank != 0:
        return None
    import oracle  # noqa: F401
    import synth

    threads = os.cpu_count() or 1
    probe = synth.make_workload(wl_cfg["code"], wl_cfg["ebn0"], 1000, seed=wl_cfg["seed"])
    code, _ = oracle_decode(wl_cfg, probe.y[:100], threads)
    t = time.perf_counter()
    code.decode(probe.y, wl_cfg["L"], wl_cfg["T"], threads=threads, osd_order=wl_cfg.get("osd"))
    rate = probe.B / max(time.perf_counter() - t, 1e-6)
    per_step = int(min(max(1000, rate * args.ref_step_seconds), wl_cfg["frames"]))
    wl = synth.make_workload(wl_cfg["code"], wl_cfg["ebn0"], per_step, seed=wl_cfg["seed"])
    for _ in range(args.warmup):
        code.decode(wl.y[:min(per_step, 500)], wl_cfg["L"], wl_cfg["T"], threads=threads, osd_order=wl_cfg.get("osd"))
    times = []
    for _ in range(args.steps):
        t = time.perf_counter()
        code.decode(wl.y, wl_cfg["L"], wl_cfg["T"], threads=threads, osd_order=wl_cfg.get("osd"))
        times.append(time.perf_counter() - t)
    total = sum(times)
    value = per_step * args.steps / total
    line = {
        "metric": METRIC, "value": value, "unit": "frames/s", "n_gpus": args.gpus, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": 1e3 * total / args.steps, "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
        "impl": "reference",
        "config": {"workload": wl_cfg["desc"], "frames_per_step": per_step,
                   "l2": "inputs larger than L2 on the GPU arm; host-only here"},
        "cpu_baseline": {"value": value, "unit": "frames/s", "cores": threads, "kind": "oracle",
                         "sample": f"first {per_step} frames of the workload stream per step"},
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

    frames = args.frames or wl_cfg["frames"]
    seed = rank_seed(wl_cfg["seed"], rank)
    wl = synth.make_workload(wl_cfg["code"], wl_cfg["ebn0"], frames, seed=seed)
    n, L, T = wl.n, wl_cfg["L"], wl_cfg["T"]
    W = (n + 63) // 64
    code = mpwsd.Code.rm(wl_cfg["m"], wl_cfg["r"], crc_poly=0x21, crc_len=6, weights=wl_cfg["weights"])
    P = code.n_patterns
    y_host = torch.from_numpy(wl.y).pin_memory()
    y_dev = y_host.to("cuda", non_blocking=False)
    cw_dev = torch.empty((frames, W), dtype=torch.int64, device="cuda")
    fl_dev = torch.empty((frames,), dtype=torch.int16, device="cuda")
    stream = torch.cuda.current_stream()

    def step():
        code.decode(y_dev, L, T, score_mode=args.mode, cw_out=cw_dev, flags_out=fl_dev, osd_order=wl_cfg.get("osd"))

    for _ in range(args.warmup):
        step()
    torch.cuda.synchronize()

    clocks = ClockSampler(local)
    clocks.start()
    time.sleep(0.3)
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
    time.sleep(0.2)
    clocks.stop()
    clk = clocks.summary(t_wall0, t_wall1)

    # end to end through the binding with pinned host buffers
    cw_host = torch.empty((frames, W), dtype=torch.int64).pin_memory()
    fl_host = torch.empty((frames,), dtype=torch.int16).pin_memory()

    def e2e_step():
        # the library's host-buffer entry point: y in, codewords and flags out, with
        # the input copies overlapping stage 1
        code.decode_host(y_host, L, T, score_mode=args.mode, cw_out=cw_host, flags_out=fl_host,
                         osd_order=wl_cfg.get("osd"))

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

    def roofline_for(kname):
        ms = kinds[kname]["ms"]
        launches = kinds[kname]["launches"]
        per_launch_s = ms / 1e3 / launches
        if kname == "score_tc":
            flops = evals * 2 * n * 2 / launches  # dense bf16 work per launch: 2 n flops x 2 splits per pattern-eval
            ach = flops / per_launch_s / 1e12
            src = src_hash("paper_2602_08501_gb300/csrc/score_tc.cu", "paper_2602_08501_gb300/csrc/common.cuh",
                           "paper_2602_08501_gb300/csrc/internal.h")
            bpr = recorded_traffic("score_tc", src, "row")
            tr = None if bpr is None else bpr * (evals / P) / launches  # scaled by active rows per launch
            return {"bound": "tensor", "achieved": ach, "peak": peaks["bf16_sus"], "unit": "TFLOP/s",
                    "frac": ach / peaks["bf16_sus"], "traffic": tr, "kernel": "score_tc",
                    "peak_kind": f"bf16 sustained, {peaks['source']}", "flops_per_launch": flops}
        if kname == "score_fp32":
            adds = evals * wbar / launches
            ach = adds / per_launch_s / 1e12
            return {"bound": "alu", "achieved": ach, "peak": alu_peak / 1e12, "unit": "Tadd/s",
                    "frac": ach / (alu_peak / 1e12), "traffic": None, "kernel": "score_fp32",
                    "peak_kind": "152 SMs x 128 FP32 lanes x max SM clock"}
        if kname == "scl":
            ops = frames * 4 * L * n * math.log2(n)  # per launch (one per step): Table I, (4/3) L log2 N ED units x 3N
            ach = ops / per_launch_s / 1e12
            src = src_hash("paper_2602_08501_gb300/csrc/scl_impl.cuh", "paper_2602_08501_gb300/csrc/internal.h")
            bpf = recorded_traffic("scl", src, "frame")
            tr = None if bpf is None else bpf * frames
            return {"bound": "alu", "achieved": ach, "peak": alu_peak / 1e12, "unit": "Top/s",
                    "frac": ach / (alu_peak / 1e12), "traffic": tr, "kernel": "scl",
                    "peak_kind": "152 SMs x 128 INT32 lanes x max SM clock", "ops_per_launch": ops}
        if kname == "osd":
            # per frame: the discrepancy of every candidate (n weighted adds each) and the elimination (n k)
            kk = int(code.k)
            order = int(wl_cfg.get("osd", 0))
            ncand = sum(math.comb(kk, w) for w in range(order + 1))
            ops = frames * n * (ncand + kk)  # per launch (one per step)
            ach = ops / per_launch_s / 1e12
            src = src_hash("paper_2602_08501_gb300/csrc/osd.cu", "paper_2602_08501_gb300/csrc/common.cuh",
                           "paper_2602_08501_gb300/csrc/internal.h")
            bpf = recorded_traffic("osd", src, "frame")
            tr = None if bpf is None else bpf * frames
            return {"bound": "alu", "achieved": ach, "peak": alu_peak / 1e12, "unit": "Top/s",
                    "frac": ach / (alu_peak / 1e12), "traffic": tr, "kernel": "osd",
                    "peak_kind": "152 SMs x 128 INT32 lanes x max SM clock", "ops_per_launch": ops}
        if kname == "hop":
            # bytes a row needs: its list entry (4 + 32), centre, D, state, 1/L of its frame's y row and
            # slot data, the supports of its candidates, and on a hop the written centre, D, state, entry
            rows = evals / P if P else 0.0
            wq = math.ceil(wmax / 4)
            cand = stats["rerank_candidates"] / rows if rows else 0.0
            hopf = stats["hops"] / rows if rows else 0.0
            bpr = 36 + 8 * W + 12 + (4 * n + 8) / L + cand * 4 * wq + hopf * (8 * W + 16)
            ach = bpr * rows / launches / per_launch_s / 1e9
            src = src_hash("paper_2602_08501_gb300/csrc/traj.cu", "paper_2602_08501_gb300/csrc/common.cuh",
                           "paper_2602_08501_gb300/csrc/internal.h")
            rec = recorded_traffic("hop", src, "row")
            tr = None if rec is None else rec * rows / launches
            return {"bound": "hbm", "achieved": ach, "peak": peaks["hbm_gbs"], "unit": "GB/s",
                    "frac": ach / peaks["hbm_gbs"],
                    "traffic": tr, "kernel": "hop", "peak_kind": f"HBM copy, {peaks['source']}",
                    "bytes_per_row": bpr}
        return {"bound": "alu", "achieved": None, "peak": None, "unit": None, "frac": None, "traffic": None,
                "kernel": kname}

    roof = roofline_for(dominant)
    others = [roofline_for(k) for k in ("scl", "osd", "score_tc", "score_fp32", "hop") if k in kinds and k != dominant]

    line = {
        "metric": METRIC, "value": value, "unit": "frames/s", "n_gpus": world, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": max_ms / args.steps, "higher_is_better": True, "scaling": "weak",
        "vs_baseline": None, "dtype": "bf16x2+f64" if args.mode == "bf16x2" else "f32+f64", "data": "synthetic",
        "config": {"workload": wl_cfg["desc"], "frames_per_rank": frames, "L": L, "T": T, "patterns": P,
                   "scoring": args.mode, "l2": "inputs larger than L2 (y is %.0f MB per step)" % (frames * n * 4 / 1e6),
                   "parallelism": f"replicas x{world} (frames sharded by seed)"},
        "pattern_evals_per_s": total_evals / (max_ms / 1e3),
        "latency_ms": {"p50": statistics.median(step_ms), "p99": float(np.percentile(step_ms, 99)),
                       "what": "per batch step of %d frames" % frames},
        "fer": fer, "p_act": p_act,
        "roofline": roof, "roofline_other": others, "kernels": shares,
        "e2e": {"value": total_frames / args.steps * e2e_steps / (e2e_ms / 1e3), "unit": "frames/s",
                "h2d_bytes_per_step": int(y_host.numel() * 4),
                "d2h_bytes_per_step": int(cw_host.numel() * 8 + fl_host.numel() * 2)},
        "gpu_launches": int(stats["kernel_launches"]),
        "clocks": {k: clk[k] for k in ("sm_mhz", "sm_max_mhz", "reasons")} | {"samples": clk["samples"]},
        "stats": {k: stats[k] for k in ("stage2_frames", "trajectories", "hops", "rerank_candidates", "rescans")},
    }

    if rank == 0 and not args.no_cpu:
        threads = os.cpu_count() or 1
        owl, oout, odt = time_oracle(wl_cfg, args.cpu_seconds, threads)
        nb = owl.B
        mism = np.any(oout["cw"] != cw[:nb], axis=1) | ((oout["flags"] & 0xF3) != (fl[:nb] & 0xF3))
        tie = oout["min_gap"] < 1e-6 * np.sum(owl.y.astype(np.float64) ** 2, axis=1)
        oerr = np.any(oout["cw"] != tx[:nb], axis=1)
        lo, hi = clopper_pearson(int(oerr.sum()), nb)
        line["cpu_baseline"] = {"value": nb / odt, "unit": "frames/s", "cores": threads, "kind": "oracle",
                                "sample": f"first {nb} frames of the same stream (seed {wl_cfg['seed']})",
                                "pattern_evals_per_s": float(oout["evals"].sum()) / odt}
        line["parity"] = {"frames": nb, "mismatches": int(mism.sum()), "mismatches_outside_near_ties":
                          int((mism & ~tie).sum()), "near_ties": int(tie.sum())}
        line["fer_check"] = {"gpu_fer": fer, "oracle_fer_sample": float(oerr.mean()), "oracle_ci95": [lo, hi],
                             "gpu_in_ci": bool(lo <= fer <= hi)}
    if rank == 0:
        print(json.dumps(line), flush=True)
    if dist is not None:
        dist.destroy_process_group()
    return line


def run_serving(args):
    """Workload 5: Poisson arrivals of mixed RM(2,6)+CRC-6 / RM(2,7)+CRC-6 frames
    (50/50), Eb/N0 uniform in [0.5, 3] dB, through the continuous-batching loop;
    one JSON line with throughput and p50/p99 per-frame latency per arrival rate."""
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
    for nm, sp in specs.items():  # choose the pattern-split target on a sample of each code's frames
        sample = ys[nm][:min(n_max, 32768)].cuda()
        sizes = [b for b in (256, 4096, 32768) if b <= sample.shape[0]]
        tuned[nm] = autotune.tune(sp.code, sample, sp.L, sp.T, batch_sizes=sizes, reps=5)
    srv = serving.Server(specs, max_batch=args.serve_batch, slots_per_code=4, min_batch=args.serve_batch // 8,
                         max_wait_s=args.serve_wait_us * 1e-6)
    srv.warmup()  # records the decode graph of every batch bucket on every slot
    out = []
    for rate in rates:
        n_each = int(rate * args.serve_seconds / 2)
        arr = {nm: serving.poisson_arrivals(rate / 2, n_each, seed=100 + i) for i, nm in enumerate(specs)}
        res = srv.run(arr, {nm: ys[nm][:n_each] for nm in specs})
        p = res.percentiles((50, 99))
        fer = {nm: float(np.mean(np.any(res.cw[nm] != synth.pack_bits(pools[nm].cw[:n_each]), axis=1))) for nm in specs}
        out.append({"offered_frames_per_s": rate, "served_frames_per_s": res.served / res.wall_s,
                    "p50_ms": p["p50"] * 1e3, "p99_ms": p["p99"] * 1e3, "frames": res.served,
                    "dispatches": res.dispatches, "mean_batch": float(np.mean(res.batch_sizes)), "fer": fer})
    line = {"metric": METRIC + " (serving)", "value": max(o["served_frames_per_s"] for o in out), "unit": "frames/s",
            "n_gpus": 1, "higher_is_better": True, "dtype": "bf16x2+f64", "data": "synthetic",
            "config": {"workload": "serving: Poisson arrivals, 50/50 RM(2,6)+CRC-6 (L=8,T=4) / RM(2,7)+CRC-6 (L=16,T=6), "
                                   "Eb/N0 U[0.5,3] dB", "max_batch": args.serve_batch, "slots_per_code": {nm: len(v) for nm, v in srv.slots.items()},
                       "max_wait_us": args.serve_wait_us, "seconds_per_rate": args.serve_seconds,
                       "tuned_split_items": {nm: t["value"] for nm, t in tuned.items()}},
            "rates": out}
    print(json.dumps(line), flush=True)


def main():
    ap = argparse.ArgumentParser(description=__doc__, formatter_class=argparse.RawDescriptionHelpFormatter)
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=20)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", choices=["ours", "reference"], default="ours")
    ap.add_argument("--workload", choices=sorted(WORKLOADS) + ["serving"], default="rm26_crc6_1db")
    ap.add_argument("--mode", choices=["bf16x2", "fp32"], default="bf16x2")
    ap.add_argument("--frames", type=int, default=0, help="override frames per step")
    ap.add_argument("--cpu-seconds", type=float, default=12.0, help="oracle sample size in CPU seconds")
    ap.add_argument("--ref-step-seconds", type=float, default=6.0)
    ap.add_argument("--no-cpu", action="store_true")
    ap.add_argument("--rates", default="1,2,5,10,20", help="serving: offered M frames/s")
    ap.add_argument("--serve-seconds", type=float, default=0.1, help="serving: seconds of traffic per rate")
    ap.add_argument("--serve-batch", type=int, default=65536)
    ap.add_argument("--serve-wait-us", type=float, default=200.0)
    args = ap.parse_args()
    args.warmup = max(args.warmup, 3)  # at least 3 untimed warm-up steps
    if args.workload == "serving":
        run_serving(args)
        return
    wl_cfg = WORKLOADS[args.workload]
    if args.impl == "reference":
        run_reference(args, wl_cfg)
    else:
        run_ours(args, wl_cfg)


if __name__ == "__main__":
    main()
