"""FP64 CPU oracle for two-stage MP-WSD decoding (arXiv 2602.08501).

TEST INFRASTRUCTURE. Only ``tests/``, ``__graft_entry__.smoke()`` and the
``cpu_baseline`` / ``--impl reference`` legs of ``bench.py`` may import this
package. The GPU library never imports, links or calls it, and this package
imports nothing from the GPU library.

The arithmetic lives in ``mpwsd_oracle.c`` (plain C, FP64, one frame and one
path at a time); this module compiles it with gcc on first use and exposes it
through ctypes with numpy arrays. What each function restates:

* ``rm_frozen``, ``kron_power``, ``encode``, ``crc`` -- code model, Sec. II-B
* ``scl`` -- stage-1 list decoding, Sec. III-A (min-sum reading)
* ``enumerate_codewords``, ``weight_distribution`` -- S_r(0), Sec. II-C, Eqs. (1)-(3)
* ``mpwsd`` -- Algorithm 1 with the filter of Eq. (5), Sec. III-B/C
* ``decode`` -- the two-stage decoder, Sec. III
* ``gains`` -- the correlation gain G_k(c) of Eq. (5) for every pattern
* ``ml`` -- brute-force maximum-likelihood decoding (the optimality reference, Sec. IV-A)
"""
from __future__ import annotations

import ctypes
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "mpwsd_oracle.c")
_BUILD = os.path.join(_HERE, "_build")
_LIB_PATH = os.path.join(_BUILD, "liboracle.so")
_lib = None
_lock = threading.Lock()

RULE_TOP1 = 0
RULE_ANY = 1


def build() -> str:
    """Compile the oracle with gcc (portable flags: x86_64 and aarch64)."""
    os.makedirs(_BUILD, exist_ok=True)
    if (not os.path.exists(_LIB_PATH)) or os.path.getmtime(_LIB_PATH) < os.path.getmtime(_SRC):
        tmp = _LIB_PATH + f".tmp{os.getpid()}"
        subprocess.check_call(["gcc", "-O2", "-std=c11", "-shared", "-fPIC", "-o", tmp, _SRC, "-lm", "-lpthread"])
        os.replace(tmp, _LIB_PATH)
    return _LIB_PATH


def _load():
    global _lib
    with _lock:
        if _lib is not None:
            return _lib
        lib = ctypes.CDLL(build())
        P = ctypes.c_void_p
        i32, i64, u32 = ctypes.c_int, ctypes.c_int64, ctypes.c_uint32
        sig = {
            "or_kron_power": (None, [i32, P]),
            "or_rm_frozen": (i32, [i32, i32, P]),
            "or_crc": (None, [P, i32, u32, i32, P]),
            "or_code_create": (P, [i32, P, i32, u32, i32, P, i64]),
            "or_code_free": (None, [P]),
            "or_code_filter_m": (i32, [P]),
            "or_encode": (None, [P, P, P]),
            "or_crc_ok_codeword": (i32, [P, P]),
            "or_leaf_llrs": (None, [P, P, P, P]),
            "or_scl": (i32, [P, P, i32, P, P]),
            "or_enumerate": (i64, [P, P, i32, P, i64]),
            "or_weight_distribution": (None, [P, P]),
            "or_decode": (i32, [P, P, i64, i32, i32, i32, i32, i32, i32, P, P, P, P, P, P]),
            "or_osd": (i32, [P, P, i32, i32, P, P]),
            "or_mpwsd": (None, [P, P, P, i32, i32, P, P, P, P, P]),
            "or_ml": (None, [P, P, P, P]),
            "or_gains": (None, [P, P, P, P]),
        }
        for name, (res, args) in sig.items():
            fn = getattr(lib, name)
            fn.restype = res
            fn.argtypes = args
        _lib = lib
        return lib


def _ptr(a: np.ndarray):
    return a.ctypes.data_as(ctypes.c_void_p)


def kron_power(m: int) -> np.ndarray:
    n = 1 << m
    F = np.zeros((n, n), np.uint8)
    _load().or_kron_power(m, _ptr(F))
    return F


def rm_frozen(m: int, r: int) -> np.ndarray:
    fz = np.zeros(1 << m, np.uint8)
    _load().or_rm_frozen(m, r, _ptr(fz))
    return fz


def crc(msg, poly: int, length: int) -> np.ndarray:
    msg = np.ascontiguousarray(msg, np.uint8)
    r = np.zeros(max(length, 1), np.uint8)
    _load().or_crc(_ptr(msg), int(msg.size), poly, length, _ptr(r))
    return r[:length]


def pack_bits(bits: np.ndarray) -> np.ndarray:
    """(..., n) 0/1 bytes -> (..., W) uint64 words, bit j of word j//64 = bit j."""
    bits = np.asarray(bits, np.uint8)
    n = bits.shape[-1]
    W = (n + 63) // 64
    out = np.zeros(bits.shape[:-1] + (W,), np.uint64)
    for j in range(n):
        out[..., j // 64] |= bits[..., j].astype(np.uint64) << np.uint64(j % 64)
    return out


def unpack_bits(words: np.ndarray, n: int) -> np.ndarray:
    words = np.asarray(words, np.uint64)
    out = np.zeros(words.shape[:-1] + (n,), np.uint8)
    for j in range(n):
        out[..., j] = ((words[..., j // 64] >> np.uint64(j % 64)) & np.uint64(1)).astype(np.uint8)
    return out


class Code:
    """An (n, k) code in the Arikan form with an optional CRC and a pattern set."""

    def __init__(self, n: int, frozen, k_info: int, crc_poly: int = 0, crc_len: int = 0, patterns=None):
        self.n = int(n)
        self.W = (self.n + 63) // 64
        self.frozen = np.ascontiguousarray(frozen, np.uint8)
        self.k = int((self.frozen == 0).sum())
        self.k_info, self.crc_poly, self.crc_len = int(k_info), int(crc_poly), int(crc_len)
        if patterns is None:
            patterns = np.zeros((0, self.W), np.uint64)
        self.patterns = np.ascontiguousarray(patterns, np.uint64).reshape(-1, self.W)
        self._h = _load().or_code_create(self.n, _ptr(self.frozen), self.k_info, self.crc_poly, self.crc_len,
                                         _ptr(self.patterns), int(self.patterns.shape[0]))
        if not self._h:
            raise ValueError("oracle rejected the code parameters")

    def __del__(self):
        h = getattr(self, "_h", None)
        if h and _lib is not None:
            _lib.or_code_free(h)
            self._h = None

    @property
    def filter_m(self) -> int:
        return int(_load().or_code_filter_m(self._h))

    def with_patterns(self, patterns) -> "Code":
        return Code(self.n, self.frozen, self.k_info, self.crc_poly, self.crc_len, patterns)

    def encode(self, u) -> np.ndarray:
        u = np.ascontiguousarray(u, np.uint8)
        c = np.zeros(self.n, np.uint8)
        _load().or_encode(self._h, _ptr(u), _ptr(c))
        return c

    def crc_ok(self, cw) -> bool:
        cw = np.ascontiguousarray(cw, np.uint8)
        return bool(_load().or_crc_ok_codeword(self._h, _ptr(cw)))

    def leaf_llrs(self, y, u) -> np.ndarray:
        y = np.ascontiguousarray(y, np.float64)
        u = np.ascontiguousarray(u, np.uint8)
        out = np.zeros(self.n, np.float64)
        _load().or_leaf_llrs(self._h, _ptr(y), _ptr(u), _ptr(out))
        return out

    def scl(self, y, L: int):
        """Stage-1 list of one frame: (u_list count x n bytes, pm count)."""
        y = np.ascontiguousarray(y, np.float64)
        ul = np.zeros((L, self.n), np.uint8)
        pm = np.zeros(L, np.float64)
        cnt = _load().or_scl(self._h, _ptr(y), L, _ptr(ul), _ptr(pm))
        return ul[:cnt], pm[:cnt]

    def enumerate_codewords(self, weights) -> np.ndarray:
        w = np.ascontiguousarray(weights, np.int32)
        cnt = _load().or_enumerate(self._h, _ptr(w), int(w.size), None, 0)
        out = np.zeros((max(cnt, 1), self.W), np.uint64)
        got = _load().or_enumerate(self._h, _ptr(w), int(w.size), _ptr(out), cnt)
        assert got == cnt
        return out[:cnt]

    def weight_distribution(self) -> np.ndarray:
        A = np.zeros(self.n + 1, np.int64)
        _load().or_weight_distribution(self._h, _ptr(A))
        return A

    def osd(self, y, order: int, L: int):
        """OSD(order) list of one frame: (codewords count x n bytes, discrepancies count)."""
        y = np.ascontiguousarray(y, np.float64)
        cl = np.zeros((L, self.n), np.uint8)
        d = np.zeros(L, np.float64)
        cnt = _load().or_osd(self._h, _ptr(y), int(order), int(L), _ptr(cl), _ptr(d))
        return cl[:cnt], d[:cnt]

    def decode(self, y, L: int, T: int, rule: int = RULE_TOP1, aom: bool = False, threads: int | None = None,
               want_anchors: bool = False, osd_order: int | None = None):
        """Two-stage decode of B frames (y: B x n). Returns a dict of numpy arrays:
        cw (B x W uint64), flags (B uint16), min_gap (B float64), evals (B int64),
        evals_distinct (B int64: evals without the trajectories that hop onto the
        centre of a lower-numbered one of their frame, which decide alike from
        then on) and, if asked, anchors (B x L x n bytes; rows past the list size
        are 0).
        Stage 1 is SC-list, or OSD(osd_order) when osd_order is given."""
        y = np.ascontiguousarray(y, np.float64).reshape(-1, self.n)
        B = y.shape[0]
        cw = np.zeros((B, self.W), np.uint64)
        flags = np.zeros(B, np.uint16)
        gap = np.zeros(B, np.float64)
        evals = np.zeros(B, np.int64)
        evals_distinct = np.zeros(B, np.int64)
        anchors = np.zeros((B, L, self.n), np.uint8) if want_anchors else None
        if threads is None:
            threads = os.cpu_count() or 1
        rc = _load().or_decode(self._h, _ptr(y), B, L, T, rule, int(aom), -1 if osd_order is None else int(osd_order),
                               int(threads), _ptr(cw), _ptr(flags), _ptr(gap),
                               _ptr(anchors) if anchors is not None else None, _ptr(evals), _ptr(evals_distinct))
        if rc != 0:
            raise ValueError("oracle decode rejected its arguments")
        out = dict(cw=cw, flags=flags, min_gap=gap, evals=evals, evals_distinct=evals_distinct)
        if anchors is not None:
            out["anchors"] = anchors
        return out

    def mpwsd(self, y, anchors, T: int):
        """Algorithm 1 on one frame from explicit anchors (count x n bytes)."""
        y = np.ascontiguousarray(y, np.float64)
        a = np.ascontiguousarray(anchors, np.uint8).reshape(-1, self.n)
        out = np.zeros(self.n, np.uint8)
        it = ctypes.c_int(0)
        gap = ctypes.c_double(0)
        ev = ctypes.c_int64(0)
        fk = ctypes.c_int(0)
        _load().or_mpwsd(self._h, _ptr(y), _ptr(a), int(a.shape[0]), T, _ptr(out), ctypes.byref(it),
                         ctypes.byref(gap), ctypes.byref(ev), ctypes.byref(fk))
        return dict(cw=out, iters=it.value, min_gap=gap.value, evals=ev.value, final_k=fk.value)

    def gains(self, y, cw) -> np.ndarray:
        """G(p) of Eq. (5) for every pattern around the centre cw (n bytes)."""
        y = np.ascontiguousarray(y, np.float64)
        cw = np.ascontiguousarray(cw, np.uint8)
        G = np.zeros(max(self.patterns.shape[0], 1), np.float64)
        _load().or_gains(self._h, _ptr(y), _ptr(cw), _ptr(G))
        return G[:self.patterns.shape[0]]

    def ml(self, y):
        y = np.ascontiguousarray(y, np.float64)
        out = np.zeros(self.n, np.uint8)
        ed = ctypes.c_double(0)
        _load().or_ml(self._h, _ptr(y), _ptr(out), ctypes.byref(ed))
        return out, ed.value


def rm_code(m: int, r: int, k_info: int | None = None, crc_poly: int = 0, crc_len: int = 0, patterns=None) -> Code:
    fz = rm_frozen(m, r)
    k = int((fz == 0).sum())
    if k_info is None:
        k_info = k - crc_len
    return Code(1 << m, fz, k_info, crc_poly, crc_len, patterns)
