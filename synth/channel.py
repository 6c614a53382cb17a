"""Transmitter and channel of Sec. II-B, seeded and vectorised with numpy.

Random numbers come from SplitMix64 (G. L. Steele, D. Lea, C. H. Flood,
"Fast splittable pseudorandom number generators", OOPSLA 2014) used as a
counter-based generator: output i of the stream with key s is
``mix64(s + (i + 1) * 0x9E3779B97F4A7C15)``, which is exactly the i-th output
of a SplitMix64 generator seeded with s. Message bits and noise draw from two
streams whose keys derive from the workload seed, so any frame can be
regenerated on its own. Gaussian samples use the Box-Muller transform
(G. E. P. Box, M. E. Muller, 1958) on two uniforms in (0, 1].

Grid: every received sample is rounded to the nearest multiple of 2^-19 and
clamped to |y| <= (2^23 - 1) 2^-19, so it is an exact float32 whose integer
image y * 2^19 fits in 24 bits. All sums a decoder forms from such samples are
then exact in FP64 (and in int32/int64 on the integer image), which is what
lets a GPU decoder match an FP64 oracle bit for bit.
"""
from __future__ import annotations

import math
from dataclasses import dataclass, field

import numpy as np

GAMMA = np.uint64(0x9E3779B97F4A7C15)
_M1 = np.uint64(0xBF58476D1CE4E5B9)
_M2 = np.uint64(0x94D049BB133111EB)
GRID_BITS = 19
GRID_MAX = (1 << 23) - 1


def _mix64(z: np.ndarray) -> np.ndarray:
    z = z.astype(np.uint64, copy=True)
    with np.errstate(over="ignore"):
        z ^= z >> np.uint64(30)
        z *= _M1
        z ^= z >> np.uint64(27)
        z *= _M2
        z ^= z >> np.uint64(31)
    return z


def splitmix64_stream(key: int, counters: np.ndarray) -> np.ndarray:
    """Outputs ``counters`` (0-based) of the SplitMix64 stream seeded with ``key``."""
    c = np.asarray(counters, dtype=np.uint64)
    with np.errstate(over="ignore"):
        s = np.uint64(key & 0xFFFFFFFFFFFFFFFF) + (c + np.uint64(1)) * GAMMA
    return _mix64(s)


def _subkey(seed: int, purpose: int) -> int:
    return int(_mix64(np.array([(seed * 0x100000001B3 + purpose) & 0xFFFFFFFFFFFFFFFF], np.uint64))[0])


def rm_info_set(m: int, r: int) -> np.ndarray:
    """Non-frozen indices of RM(r, m) in the Arikan form: rows of
    [[1,0],[1,1]]^{(x)m} with weight 2^popcount(i) >= 2^(m-r)."""
    idx = [i for i in range(1 << m) if bin(i).count("1") >= m - r]
    return np.array(idx, np.int64)


def encode_arikan(u: np.ndarray) -> np.ndarray:
    """c = u [[1,0],[1,1]]^{(x)m} over F2 for a batch of bit rows (uint8, ... x n)."""
    c = np.array(u, dtype=np.uint8, copy=True)
    n = c.shape[-1]
    lead = c.shape[:-1]
    h = 1
    while h < n:
        v = c.reshape(lead + (n // (2 * h), 2, h))
        v[..., 0, :] ^= v[..., 1, :]
        h *= 2
    return c


def _crc_parity_matrix(k_info: int, poly: int, length: int) -> np.ndarray:
    """Rows = CRC remainders of the unit messages (the CRC is linear: zero
    initial value, no reflection, no final XOR). Message bit 0 is the highest
    power; the generator is x^length + sum_b bit_b(poly) x^b."""
    rows = np.zeros((k_info, length), np.uint8)
    for t in range(k_info):
        # remainder of x^(k_info - 1 - t + length) mod g(x), by shift-and-reduce
        reg = 0
        top = 1 << length
        deg = k_info - 1 - t + length
        val = 1
        for _ in range(deg):
            val <<= 1
            if val & top:
                val ^= top | poly
        reg = val
        for b in range(length):
            rows[t, b] = (reg >> (length - 1 - b)) & 1
    return rows


def grid_quantize(y: np.ndarray) -> np.ndarray:
    """Round to the 2^-19 grid and clamp to 24-bit magnitudes; returns float32."""
    q = np.rint(np.asarray(y, np.float64) * float(1 << GRID_BITS))
    q = np.clip(q, -GRID_MAX, GRID_MAX)
    return (q / float(1 << GRID_BITS)).astype(np.float32)


def sigma_for(ebn0_db: float, rate: float) -> float:
    """sigma^2 = N0/2 with Es = 1 and Eb/N0 = Es/(R N0): sigma^2 = 1/(2 R 10^(Eb/N0 / 10))."""
    return math.sqrt(1.0 / (2.0 * rate * 10.0 ** (ebn0_db / 10.0)))


def pack_bits(bits: np.ndarray) -> np.ndarray:
    bits = np.asarray(bits, np.uint8)
    n = bits.shape[-1]
    W = (n + 63) // 64
    out = np.zeros(bits.shape[:-1] + (W,), np.uint64)
    for q in range(W):
        seg = bits[..., 64 * q: min(n, 64 * (q + 1))].astype(np.uint64)
        sh = np.arange(seg.shape[-1], dtype=np.uint64)
        out[..., q] = np.bitwise_or.reduce(seg << sh, axis=-1)
    return out


# Code families used by the workloads: (m, r, CRC polynomial without the x^len
# term, CRC length). x^6 + x^5 + 1 -> 0x21.
CODES = {
    "rm15": dict(m=5, r=1, crc_poly=0x0, crc_len=0),
    "rm26_crc6": dict(m=6, r=2, crc_poly=0x21, crc_len=6),
    "rm27_crc6": dict(m=7, r=2, crc_poly=0x21, crc_len=6),
    "rm26": dict(m=6, r=2, crc_poly=0x0, crc_len=0),
    # RM(128, 29) with no CRC: all 29 information bits carry the message
    "rm27": dict(m=7, r=2, crc_poly=0x0, crc_len=0),
}


def shard_batches(total_batches: int, world: int, rank: int) -> list:
    """Batches of one stream dealt round-robin over ranks: batch b goes to
    rank b mod world. Returns the batch numbers of ``rank``."""
    return list(range(rank, total_batches, world))


@dataclass
class Workload:
    code: str
    n: int
    k: int
    k_info: int
    crc_poly: int
    crc_len: int
    ebn0_db: np.ndarray     # per frame
    sigma: np.ndarray       # per frame
    seed: int
    first_frame: int
    y: np.ndarray           # B x n float32 on the grid
    cw: np.ndarray          # B x n uint8 transmitted codewords
    msg: np.ndarray         # B x k_info uint8
    frozen: np.ndarray = field(default=None)

    @property
    def B(self) -> int:
        return int(self.y.shape[0])


def make_workload(code: str, ebn0_db, frames: int, seed: int, first_frame: int = 0,
                  chunk: int = 1 << 17) -> Workload:
    """Frames [first_frame, first_frame + frames) of the seeded stream.

    ``ebn0_db`` is a scalar, or a (lo, hi) tuple for Eb/N0 drawn uniformly per
    frame from a third stream. The rate is R = k_info / n (CRC bits counted as
    overhead)."""
    p = CODES[code]
    m, r = p["m"], p["r"]
    n = 1 << m
    info = rm_info_set(m, r)
    k = int(info.size)
    k_info = k - p["crc_len"]
    rate = k_info / n
    frozen = np.ones(n, np.uint8)
    frozen[info] = 0
    C = _crc_parity_matrix(k_info, p["crc_poly"], p["crc_len"]) if p["crc_len"] else None
    key_msg, key_noise, key_snr = _subkey(seed, 1), _subkey(seed, 2), _subkey(seed, 3)

    ys, cws, msgs, snrs, sigs = [], [], [], [], []
    for f0 in range(first_frame, first_frame + frames, chunk):
        f1 = min(first_frame + frames, f0 + chunk)
        fidx = np.arange(f0, f1, dtype=np.uint64)
        B = fidx.size
        words = splitmix64_stream(key_msg, fidx)
        msg = ((words[:, None] >> np.arange(k_info, dtype=np.uint64)[None, :]) & np.uint64(1)).astype(np.uint8)
        if C is not None:
            par = (msg.astype(np.int64) @ C.astype(np.int64)) & 1
            v = np.concatenate([msg, par.astype(np.uint8)], axis=1)
        else:
            v = msg
        u = np.zeros((B, n), np.uint8)
        u[:, info] = v
        c = encode_arikan(u)
        if isinstance(ebn0_db, (tuple, list)):
            lo, hi = float(ebn0_db[0]), float(ebn0_db[1])
            uu = (splitmix64_stream(key_snr, fidx) >> np.uint64(11)).astype(np.float64) * 2.0 ** -53
            snr = lo + (hi - lo) * uu
        else:
            snr = np.full(B, float(ebn0_db))
        sig = np.sqrt(1.0 / (2.0 * rate * 10.0 ** (snr / 10.0)))
        ctr = (fidx[:, None] * np.uint64(n) + np.arange(n, dtype=np.uint64)[None, :]) * np.uint64(2)
        u1 = ((splitmix64_stream(key_noise, ctr) >> np.uint64(11)).astype(np.float64) + 1.0) * 2.0 ** -53
        u2 = ((splitmix64_stream(key_noise, ctr + np.uint64(1)) >> np.uint64(11)).astype(np.float64) + 1.0) * 2.0 ** -53
        g = np.sqrt(-2.0 * np.log(u1)) * np.cos(2.0 * np.pi * u2)
        y = (1.0 - 2.0 * c.astype(np.float64)) + sig[:, None] * g
        ys.append(grid_quantize(y))
        cws.append(c)
        msgs.append(msg)
        snrs.append(snr)
        sigs.append(sig)
    if not ys:
        ys, cws, msgs = [np.zeros((0, n), np.float32)], [np.zeros((0, n), np.uint8)], [np.zeros((0, k_info), np.uint8)]
        snrs, sigs = [np.zeros(0)], [np.zeros(0)]
    return Workload(code=code, n=n, k=k, k_info=k_info, crc_poly=p["crc_poly"], crc_len=p["crc_len"],
                    ebn0_db=np.concatenate(snrs), sigma=np.concatenate(sigs), seed=seed, first_frame=first_frame,
                    y=np.concatenate(ys), cw=np.concatenate(cws), msg=np.concatenate(msgs), frozen=frozen)
