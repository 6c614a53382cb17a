"""Python binding of libmpwsd (include/mpwsd.h): argument marshalling only.

Device buffers are torch CUDA tensors; their ``data_ptr()`` and the current
torch stream are handed to the C ABI. Every step of a decode runs in the
library's CUDA kernels; nothing here computes. If the shared library has not
been built this module raises on first use -- there is no other code path.
"""
from __future__ import annotations

import ctypes
import os
import re
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "libmpwsd.so")
HEADER = os.path.join(os.path.dirname(_HERE), "include", "mpwsd.h")

OK, EINVAL, ENOMEM, ECUDA, ETIMEOUT, EUNSUPPORTED = 0, -1, -2, -3, -4, -5
SCORE_BF16X2, SCORE_FP32, SCORE_FLATS = 0, 1, 2
RULE_TOP1, RULE_ANY = 0, 1
STAGE1_SCL, STAGE1_OSD = 0, 1
FLAG_STAGE2, FLAG_CRC_OK, FLAG_RESCAN, FLAG_ERROR = 0x1, 0x2, 0x4, 0x100
ITERS_SHIFT = 4
MAX_L, MAX_T, TOPK = 32, 15, 4
TUNE_SPLIT_ITEMS = 0
TUNE_TC_SHAPE = 1

_lock = threading.Lock()
_lib = None


class MpwsdError(RuntimeError):
    def __init__(self, status: int, msg: str):
        super().__init__(f"{msg} (status {status})")
        self.status = status


class _Opts(ctypes.Structure):
    _fields_ = [("score_mode", ctypes.c_int), ("stage1_rule", ctypes.c_int), ("always_on", ctypes.c_int),
                ("use_graph", ctypes.c_int), ("stage1", ctypes.c_int), ("osd_order", ctypes.c_int),
                ("reserved", ctypes.c_int * 2)]


class _KTime(ctypes.Structure):
    _fields_ = [("launches", ctypes.c_int64), ("ms", ctypes.c_double)]


KERNEL_NAMES = ("scl", "score_tc", "score_fp32", "hop", "rescan", "final", "osd", "score_flats", "resolve")


class _Stats(ctypes.Structure):
    _fields_ = [(k, ctypes.c_int64) for k in ("frames", "stage2_frames", "trajectories", "pattern_evals",
                                               "rerank_candidates", "rescans", "hops", "kernel_launches")]


def declared_symbols() -> list[str]:
    """Entry points declared in include/mpwsd.h."""
    with open(HEADER) as fh:
        txt = fh.read()
    return sorted(set(re.findall(r"MPWSD_API\s+[^;(]*?\b(mpwsd_\w+)\s*\(", txt)))


def lib():
    global _lib
    with _lock:
        if _lib is not None:
            return _lib
        if not os.path.exists(LIB_PATH):
            raise ImportError(f"{LIB_PATH} is missing: build it with "
                              "`python -c 'import __graft_entry__ as g; g.build()'` (needs nvcc)")
        L = ctypes.CDLL(LIB_PATH)
        P, i32, i64, u32 = ctypes.c_void_p, ctypes.c_int, ctypes.c_int64, ctypes.c_uint32
        sig = {
            "mpwsd_strerror": (ctypes.c_char_p, [i32]),
            "mpwsd_last_error": (ctypes.c_char_p, []),
            "mpwsd_load_code": (i32, [i32, P, P, i32, u32, i32, P, i64, ctypes.POINTER(P)]),
            "mpwsd_free_code": (None, [P]),
            "mpwsd_code_info": (i32, [P, P, P, P, P]),
            "mpwsd_decode": (i32, [P, P, i64, i32, i32, P, P, P, P]),
            "mpwsd_decode_host": (i32, [P, P, i64, i32, i32, P, P, P, P]),
            "mpwsd_workspace_create": (i32, [P, i64, i32, ctypes.POINTER(P)]),
            "mpwsd_workspace_free": (None, [P]),
            "mpwsd_workspace_bytes": (i32, [P, i64, i32, ctypes.POINTER(ctypes.c_size_t)]),
            "mpwsd_decode_ws": (i32, [P, P, P, i64, i32, i32, P, P, P, P]),
            "mpwsd_stage1_list": (i32, [P, P, i64, i32, P, P, P]),
            "mpwsd_osd_list": (i32, [P, P, i64, i32, i32, P, P, P]),
            "mpwsd_score_topk": (i32, [P, i32, P, i64, P, P, i64, P, P, P]),
            "mpwsd_sync": (i32, [P, P]),
            "mpwsd_stats_get": (i32, [P, ctypes.POINTER(_Stats)]),
            "mpwsd_stats_reset": (i32, [P]),
            "mpwsd_enumerate_codewords": (i32, [i32, P, P, i32, P, i64, ctypes.POINTER(ctypes.c_int64)]),
            "mpwsd_tune_set": (i32, [P, i32, i32]),
            "mpwsd_tune_get": (i32, [P, i32, ctypes.POINTER(ctypes.c_int)]),
            "mpwsd_profile_begin": (i32, [P]),
            "mpwsd_profile_end": (i32, [P, ctypes.POINTER(_KTime)]),
            "mpwsd_pool_create": (i32, [P, i64, i32, i32, P, ctypes.POINTER(P)]),
            "mpwsd_pool_free": (None, [P]),
            "mpwsd_pool_bytes": (i32, [P, i64, i32, ctypes.POINTER(ctypes.c_size_t)]),
            "mpwsd_pool_free_frames": (i32, [P, ctypes.POINTER(ctypes.c_int64)]),
            "mpwsd_pool_submit": (i32, [P, P, i64, P, P, P, P]),
            "mpwsd_pool_step": (i32, [P, P]),
        }
        for name, (res, args) in sig.items():
            fn = getattr(L, name)
            fn.restype = res
            fn.argtypes = args
        _lib = L
        return L


def _check(status: int, what: str):
    if status != OK:
        msg = lib().mpwsd_last_error().decode() or lib().mpwsd_strerror(status).decode()
        raise MpwsdError(status, f"{what}: {msg}")


def _np_ptr(a: np.ndarray):
    return a.ctypes.data_as(ctypes.c_void_p)


def _stream_ptr(stream):
    import torch

    s = stream if stream is not None else torch.cuda.current_stream()
    return ctypes.c_void_p(s.cuda_stream)


def _dev(t, dtype, name):
    import torch

    if not isinstance(t, torch.Tensor) or not t.is_cuda:
        raise TypeError(f"{name} must be a CUDA tensor")
    if t.dtype != dtype or not t.is_contiguous():
        raise TypeError(f"{name} must be a contiguous {dtype} tensor")
    return ctypes.c_void_p(t.data_ptr())


def _host(t, dtype, name):
    import torch

    if not isinstance(t, torch.Tensor) or t.device.type != "cpu":
        raise TypeError(f"{name} must be a host (CPU) tensor")
    if t.dtype != dtype or not t.is_contiguous():
        raise TypeError(f"{name} must be a contiguous {dtype} tensor")
    return ctypes.c_void_p(t.data_ptr())


def rm_frozen(m: int, r: int) -> np.ndarray:
    """Frozen set of RM(r, m) in the Arikan form (rows of weight < 2^(m-r))."""
    return np.array([1 if bin(i).count("1") < m - r else 0 for i in range(1 << m)], np.uint8)


def enumerate_codewords(n: int, frozen, weights) -> np.ndarray:
    """All codewords with the given weights (host helper of the library)."""
    frozen = np.ascontiguousarray(frozen, np.uint8)
    w = np.ascontiguousarray(sorted(weights), np.int32)
    cnt = ctypes.c_int64(0)
    _check(lib().mpwsd_enumerate_codewords(n, _np_ptr(frozen), _np_ptr(w), int(w.size), None, 0, ctypes.byref(cnt)),
           "enumerate_codewords")
    W = (n + 63) // 64
    out = np.zeros((max(cnt.value, 1), W), np.uint64)
    _check(lib().mpwsd_enumerate_codewords(n, _np_ptr(frozen), _np_ptr(w), int(w.size), _np_ptr(out), cnt.value,
                                           ctypes.byref(cnt)), "enumerate_codewords")
    return out[:cnt.value]


class Workspace:
    def __init__(self, code: "Code", max_B: int, max_L: int):
        h = ctypes.c_void_p()
        _check(lib().mpwsd_workspace_create(code._h, int(max_B), int(max_L), ctypes.byref(h)), "workspace_create")
        self._h = h
        self.max_B, self.max_L = int(max_B), int(max_L)

    def close(self):
        if getattr(self, "_h", None):
            lib().mpwsd_workspace_free(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


class Code:
    """A code handle of the library (mpwsd_load_code)."""

    def __init__(self, n: int, frozen, k_info: int, crc_poly: int, crc_len: int, patterns, G=None):
        self.n = int(n)
        self.W = (self.n + 63) // 64
        self.frozen = np.ascontiguousarray(frozen, np.uint8)
        self.patterns = np.ascontiguousarray(patterns, np.uint64).reshape(-1, self.W)
        g = None if G is None else np.ascontiguousarray(G, np.uint8)
        h = ctypes.c_void_p()
        _check(lib().mpwsd_load_code(self.n, None if g is None else _np_ptr(g), _np_ptr(self.frozen), int(k_info),
                                     int(crc_poly), int(crc_len), _np_ptr(self.patterns), int(self.patterns.shape[0]),
                                     ctypes.byref(h)), "load_code")
        self._h = h
        self.k_info, self.crc_poly, self.crc_len = int(k_info), int(crc_poly), int(crc_len)
        self.k = int((self.frozen == 0).sum())

    @classmethod
    def rm(cls, m: int, r: int, crc_poly: int = 0, crc_len: int = 0, weights=None, patterns=None) -> "Code":
        fz = rm_frozen(m, r)
        k = int((fz == 0).sum())
        if patterns is None:
            patterns = enumerate_codewords(1 << m, fz, weights or [2 ** (m - r)])
        return cls(1 << m, fz, k - crc_len, crc_poly, crc_len, patterns)

    @property
    def n_patterns(self) -> int:
        return int(self.patterns.shape[0])

    def close(self):
        if getattr(self, "_h", None):
            lib().mpwsd_free_code(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    @staticmethod
    def _opts(score_mode, rule, always_on, use_graph=False, osd_order=None):
        o = _Opts()
        o.score_mode = {"bf16x2": SCORE_BF16X2, "fp32": SCORE_FP32, "flats": SCORE_FLATS}.get(score_mode, score_mode)
        o.stage1_rule = {"top1": RULE_TOP1, "any": RULE_ANY}.get(rule, rule)
        o.always_on = int(bool(always_on))
        o.use_graph = int(bool(use_graph))
        o.stage1 = STAGE1_SCL if osd_order is None else STAGE1_OSD
        o.osd_order = 0 if osd_order is None else int(osd_order)
        return o

    def decode(self, y, L: int, T: int, score_mode="bf16x2", rule="top1", always_on=False, cw_out=None,
               flags_out=None, stream=None, workspace: Workspace | None = None, use_graph: bool = False,
               osd_order: int | None = None):
        """Two-stage decode of y (B x n float32 CUDA tensor). Returns (cw, flags)
        as CUDA tensors (B x W int64 bit patterns, B int16); asynchronous.
        Stage 1 is SC-list, or OSD(osd_order) when osd_order is given."""
        import torch

        B = int(y.shape[0]) if y.dim() == 2 else 0
        if y.dim() != 2 or y.shape[1] != self.n:
            raise ValueError(f"y must be B x {self.n}")
        if cw_out is None:
            cw_out = torch.empty((B, self.W), dtype=torch.int64, device=y.device)
        if flags_out is None:
            flags_out = torch.empty((B,), dtype=torch.int16, device=y.device)
        o = self._opts(score_mode, rule, always_on, use_graph, osd_order)
        args = (_dev(y, torch.float32, "y"), B, int(L), int(T), ctypes.byref(o), _dev(cw_out, torch.int64, "cw_out"),
                _dev(flags_out, torch.int16, "flags_out"), _stream_ptr(stream))
        if workspace is None:
            _check(lib().mpwsd_decode(self._h, *args), "decode")
        else:
            _check(lib().mpwsd_decode_ws(self._h, workspace._h, *args), "decode_ws")
        return cw_out, flags_out

    def decode_host(self, y, L: int, T: int, score_mode="bf16x2", rule="top1", always_on=False, cw_out=None,
                    flags_out=None, stream=None, use_graph: bool = False, osd_order: int | None = None):
        """decode() on host (CPU) tensors: the library copies y in chunk by chunk,
        overlapping the copies with stage 1, and copies the results back. Pinned
        tensors let the copies overlap. Returns (cw, flags) host tensors, valid once
        the stream has been synchronised."""
        import torch

        if y.dim() != 2 or y.shape[1] != self.n:
            raise ValueError(f"y must be B x {self.n}")
        B = int(y.shape[0])
        if cw_out is None:
            cw_out = torch.empty((B, self.W), dtype=torch.int64, pin_memory=y.is_pinned())
        if flags_out is None:
            flags_out = torch.empty((B,), dtype=torch.int16, pin_memory=y.is_pinned())
        o = self._opts(score_mode, rule, always_on, use_graph, osd_order)
        _check(lib().mpwsd_decode_host(self._h, _host(y, torch.float32, "y"), B, int(L), int(T), ctypes.byref(o),
                                       _host(cw_out, torch.int64, "cw_out"), _host(flags_out, torch.int16, "flags_out"),
                                       _stream_ptr(stream)), "decode_host")
        return cw_out, flags_out

    def stage1_list(self, y, L: int, stream=None):
        import torch

        B = int(y.shape[0])
        cw = torch.zeros((B, L, self.W), dtype=torch.int64, device=y.device)
        pm = torch.full((B, L), -1, dtype=torch.int64, device=y.device)
        _check(lib().mpwsd_stage1_list(self._h, _dev(y, torch.float32, "y"), B, int(L), _dev(cw, torch.int64, "cw"),
                                       _dev(pm, torch.int64, "pm"), _stream_ptr(stream)), "stage1_list")
        return cw, pm

    def osd_list(self, y, order: int, L: int, stream=None):
        """OSD(order) list of every frame: (cw B x L x W int64, D B x L int64 in units of
        2^-19; entries past the list size keep D = -1)."""
        import torch

        B = int(y.shape[0])
        cw = torch.zeros((B, L, self.W), dtype=torch.int64, device=y.device)
        d = torch.full((B, L), -1, dtype=torch.int64, device=y.device)
        _check(lib().mpwsd_osd_list(self._h, _dev(y, torch.float32, "y"), B, int(order), int(L),
                                    _dev(cw, torch.int64, "cw"), _dev(d, torch.int64, "d"), _stream_ptr(stream)),
               "osd_list")
        return cw, d

    def score_topk(self, y, frame, cw, score_mode="bf16x2", stream=None):
        import torch

        M = int(frame.shape[0])
        vals = torch.empty((M, TOPK), dtype=torch.float32, device=y.device)
        idx = torch.empty((M, TOPK), dtype=torch.int32, device=y.device)
        mode = {"bf16x2": SCORE_BF16X2, "fp32": SCORE_FP32, "flats": SCORE_FLATS}.get(score_mode, score_mode)
        _check(lib().mpwsd_score_topk(self._h, int(mode), _dev(y, torch.float32, "y"), int(y.shape[0]),
                                      _dev(frame, torch.int32, "frame"), _dev(cw, torch.int64, "cw"), M,
                                      _dev(vals, torch.float32, "vals"), _dev(idx, torch.int32, "idx"),
                                      _stream_ptr(stream)), "score_topk")
        return vals, idx

    def workspace(self, max_B: int, max_L: int) -> Workspace:
        return Workspace(self, max_B, max_L)

    def pool_bytes(self, max_frames: int, L: int) -> int:
        b = ctypes.c_size_t(0)
        _check(lib().mpwsd_pool_bytes(self._h, int(max_frames), int(L), ctypes.byref(b)), "pool_bytes")
        return int(b.value)

    def pool(self, max_frames: int, L: int, T: int, score_mode="bf16x2", rule="top1", always_on=False,
             use_graph: bool = True, osd_order: int | None = None) -> "Pool":
        return Pool(self, max_frames, L, T, score_mode, rule, always_on, use_graph, osd_order)

    def workspace_bytes(self, max_B: int, max_L: int) -> int:
        b = ctypes.c_size_t(0)
        _check(lib().mpwsd_workspace_bytes(self._h, int(max_B), int(max_L), ctypes.byref(b)), "workspace_bytes")
        return int(b.value)

    def sync(self, stream=None):
        _check(lib().mpwsd_sync(self._h, _stream_ptr(stream)), "sync")

    def stats(self) -> dict:
        s = _Stats()
        _check(lib().mpwsd_stats_get(self._h, ctypes.byref(s)), "stats_get")
        return {k: int(getattr(s, k)) for k, _ in _Stats._fields_}

    def reset_stats(self):
        _check(lib().mpwsd_stats_reset(self._h), "stats_reset")

    def tune_set(self, knob: int, value: int):
        _check(lib().mpwsd_tune_set(self._h, int(knob), int(value)), "tune_set")

    def tune_get(self, knob: int) -> int:
        v = ctypes.c_int(0)
        _check(lib().mpwsd_tune_get(self._h, int(knob), ctypes.byref(v)), "tune_get")
        return int(v.value)

    def profile_begin(self):
        """Record CUDA events around every kernel this handle launches."""
        _check(lib().mpwsd_profile_begin(self._h), "profile_begin")

    def profile_end(self) -> dict:
        """Per kernel class: {"launches": n, "ms": summed device time}."""
        arr = (_KTime * len(KERNEL_NAMES))()
        _check(lib().mpwsd_profile_end(self._h, arr), "profile_end")
        return {name: {"launches": int(arr[i].launches), "ms": float(arr[i].ms)} for i, name in enumerate(KERNEL_NAMES)}


class Pool:
    """A stage-2 pool of the library (mpwsd_pool_*): continuous batching of
    stage 2 across submissions of one code."""

    def __init__(self, code: Code, max_frames: int, L: int, T: int, score_mode="bf16x2", rule="top1",
                 always_on=False, use_graph: bool = True, osd_order: int | None = None):
        self.code = code
        self.L, self.T, self.max_frames = int(L), int(T), int(max_frames)
        o = Code._opts(score_mode, rule, always_on, use_graph, osd_order)
        h = ctypes.c_void_p()
        _check(lib().mpwsd_pool_create(code._h, self.max_frames, self.L, self.T, ctypes.byref(o), ctypes.byref(h)),
               "pool_create")
        self._h = h
        self.submits = 0
        self.steps = 0

    def free_frames(self) -> int:
        v = ctypes.c_int64(0)
        _check(lib().mpwsd_pool_free_frames(self._h, ctypes.byref(v)), "pool_free_frames")
        return int(v.value)

    def submit(self, y, cw_out, flags_out, done_out=None, stream=None) -> int:
        """Stage 1 on y (B x n float32 CUDA tensor); results land in cw_out /
        flags_out (and done_out, int32) when each frame finishes. Returns the
        submission number."""
        import torch

        B = int(y.shape[0])
        if y.dim() != 2 or y.shape[1] != self.code.n:
            raise ValueError(f"y must be B x {self.code.n}")
        done = _dev(done_out, torch.int32, "done_out") if done_out is not None else None
        _check(lib().mpwsd_pool_submit(self._h, _dev(y, torch.float32, "y"), B, _dev(cw_out, torch.int64, "cw_out"),
                                       _dev(flags_out, torch.int16, "flags_out"), done, _stream_ptr(stream)),
               "pool_submit")
        sid = self.submits
        if B > 0:
            self.submits += 1
        return sid

    def step(self, stream=None) -> int:
        """One iteration of Algorithm 1 on every row of the pool; returns the step number (from 1)."""
        _check(lib().mpwsd_pool_step(self._h, _stream_ptr(stream)), "pool_step")
        self.steps += 1
        return self.steps

    def close(self):
        if getattr(self, "_h", None):
            lib().mpwsd_pool_free(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass
