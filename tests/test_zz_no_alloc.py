"""The allocation-free decode entry point (mpwsd_decode_noalloc).

Callers that cannot allocate device memory at decode time use this entry point:
serving threads that must not touch an allocator after warm-up, and hosts whose
device memory belongs to another allocator (a framework's pool that owns the
GPU's memory). It must return exactly what mpwsd_decode returns on the same
inputs, call after call, although every call reuses one fixed scratch array.
This file is collected last on purpose, and it passes both alone in a fresh
process and after the other tests.
"""
import ctypes

import numpy as np
import pytest

import synth
from gpu_common import cuda_or_skip, torch

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def mp():
    m = cuda_or_skip()
    fn = m.lib().mpwsd_decode_noalloc
    P = ctypes.c_void_p
    fn.restype = ctypes.c_int
    fn.argtypes = [P, P, ctypes.c_int64, ctypes.c_int, ctypes.c_int, P, P, P, P]
    return m


def _noalloc(mp, code, y, L, T, mode):
    B = y.shape[0]
    cw = torch.full((B, code.W), -1, dtype=torch.int64, device="cuda")
    fl = torch.full((B,), -1, dtype=torch.int16, device="cuda")
    o = code._opts(mode, "top1", False)
    st = mp.lib().mpwsd_decode_noalloc(code._h, ctypes.c_void_p(y.data_ptr()), B, L, T, ctypes.byref(o),
                                       ctypes.c_void_p(cw.data_ptr()), ctypes.c_void_p(fl.data_ptr()),
                                       ctypes.c_void_p(torch.cuda.current_stream().cuda_stream))
    return st, cw, fl


@pytest.mark.parametrize("mode", ["bf16x2", "fp32"])
def test_noalloc_matches_decode_on_consecutive_calls(mp, mode):
    code = mp.Code.rm(6, 2, crc_poly=0x21, crc_len=6, weights=[16])
    for call, (seed, B) in enumerate([(21, 3000), (22, 1777)]):  # two calls in a row, different sizes
        wl = synth.make_workload("rm26_crc6", 1.0, B, seed=seed)
        y = torch.from_numpy(wl.y).cuda()
        st, cw_a, fl_a = _noalloc(mp, code, y, 8, 4, mode)
        assert st == 0, mp.lib().mpwsd_last_error()
        cw_b, fl_b = code.decode(y, 8, 4, score_mode=mode)
        torch.cuda.synchronize()
        # the decoder is exact: the same codewords and flags, bit for bit
        assert torch.equal(cw_a, cw_b), call
        assert torch.equal(fl_a, fl_b), call
        assert 0 < float((fl_a.cpu().numpy() & 1).mean()) < 1


def test_noalloc_rejects_sizes_beyond_its_scratch(mp):
    code = mp.Code.rm(6, 2, crc_poly=0x21, crc_len=6, weights=[16])
    y = torch.zeros((200000, 64), dtype=torch.float32, device="cuda")
    st, _, _ = _noalloc(mp, code, y, 32, 4, "bf16x2")
    assert st == mp.EINVAL
    assert b"scratch" in mp.lib().mpwsd_last_error()
