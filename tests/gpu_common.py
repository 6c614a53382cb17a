"""Shared helpers of the GPU parity tests (inputs from synth/, expectations
from oracle/; nothing here computes a decoder result)."""
import numpy as np
import pytest

torch = pytest.importorskip("torch")


def cuda_or_skip():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2602_08501_gb300 import mpwsd

    mpwsd.lib()  # fails loudly if the library is missing
    return mpwsd


def to_words(cw_tensor) -> np.ndarray:
    """Device int64 bit patterns -> host uint64 words."""
    return cw_tensor.cpu().numpy().view(np.uint64)


FLAG_PARITY_MASK = 0x0001 | 0x0002 | 0x00F0  # stage2, crc ok, iterations (rescan bit is kernel-internal)


def oracle_code(oracle_mod, m, r, crc_len, weights):
    code = oracle_mod.rm_code(m, r, crc_poly=0x21 if crc_len else 0, crc_len=crc_len)
    return code.with_patterns(code.enumerate_codewords(weights))
