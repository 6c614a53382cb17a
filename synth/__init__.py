"""Seeded synthetic workloads for the MP-WSD decoder (inputs only).

This package is the transmitter side of the paper's system model (Sec. II-B):
messages, CRC precoding, Arikan/Reed-Muller encoding, BPSK and AWGN, with the
received samples rounded to a 2^-19 grid. It holds none of the decoder's
arithmetic and imports neither the oracle nor the GPU library; both of them
consume what it produces.
"""
from .channel import (  # noqa: F401
    CODES,
    Workload,
    encode_arikan,
    grid_quantize,
    make_workload,
    pack_bits,
    rm_info_set,
    shard_batches,
    sigma_for,
    splitmix64_stream,
)
