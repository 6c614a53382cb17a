"""mpwsd_decode_host: the decode on host buffers, with the input copied in
chunks that overlap stage 1. Its results must equal the device-buffer decode
bit for bit (the same kernels run, stage 1 in chunks with global frame
indices), and a sample of frames from every chunk is checked against the
oracle."""
import numpy as np
import pytest

import synth
from gpu_common import FLAG_PARITY_MASK, assert_decode_parity, cuda_or_skip, oracle_code, to_words, torch

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def mp():
    return cuda_or_skip()


def _device_decode(code, y, L, T, **kw):
    cw, fl = code.decode(torch.from_numpy(y).cuda(), L, T, **kw)
    torch.cuda.synchronize()
    return to_words(cw), fl.cpu().numpy()


def _host_decode(code, y, L, T, pinned=True, **kw):
    yh = torch.from_numpy(y)
    if pinned:
        yh = yh.pin_memory()
    cw, fl = code.decode_host(yh, L, T, **kw)
    torch.cuda.synchronize()
    return cw.numpy().view(np.uint64), fl.numpy()


@pytest.mark.parametrize("frames", [1000, 65536 * 3 + 17, 300_000])
@pytest.mark.parametrize("use_graph", [False, True])
def test_host_decode_equals_device_decode_rm26(mp, frames, use_graph):
    code = mp.Code.rm(6, 2, crc_poly=0x21, crc_len=6, weights=[16])
    wl = synth.make_workload("rm26_crc6", 1.0, frames, seed=70)
    cw_d, fl_d = _device_decode(code, wl.y, 8, 4)
    for _ in range(2):  # the second call replays the cached graph
        cw_h, fl_h = _host_decode(code, wl.y, 8, 4, use_graph=use_graph)
        assert np.array_equal(cw_h, cw_d)
        assert np.array_equal(fl_h & FLAG_PARITY_MASK, fl_d & FLAG_PARITY_MASK)
    assert 0 < np.mean(fl_h & 1) < 1


def test_host_decode_pageable_and_osd(mp):
    code = mp.Code.rm(7, 2, crc_poly=0x21, crc_len=6, weights=[32])
    wl = synth.make_workload("rm27_crc6", 1.5, 140_000, seed=71)
    cw_d, fl_d = _device_decode(code, wl.y, 16, 6, osd_order=2)
    cw_h, fl_h = _host_decode(code, wl.y, 16, 6, pinned=False, osd_order=2)
    assert np.array_equal(cw_h, cw_d)
    assert np.array_equal(fl_h & FLAG_PARITY_MASK, fl_d & FLAG_PARITY_MASK)


def test_host_decode_matches_oracle_across_chunks(mp):
    import oracle

    frames = 65536 * 4 + 999  # four chunks, ragged
    code = mp.Code.rm(6, 2, crc_poly=0x21, crc_len=6, weights=[16])
    wl = synth.make_workload("rm26_crc6", 1.0, frames, seed=72)
    cw, fl = _host_decode(code, wl.y, 8, 4, use_graph=True)
    fl = fl.view(np.uint16)
    # stage-2 frames from every chunk, plus the first and last frame of each chunk
    rng = np.random.default_rng(73)
    bounds = [frames * i // 4 for i in range(5)]
    pick = []
    for i in range(4):
        s2 = np.flatnonzero(fl[bounds[i]:bounds[i + 1]] & 1) + bounds[i]
        pick += list(rng.choice(s2, 40, replace=False)) + [bounds[i], bounds[i + 1] - 1]
    pick = np.unique(np.array(pick))
    ocode = oracle_code(oracle, 6, 2, 6, [16])
    ref = ocode.decode(wl.y[pick], 8, 4)
    assert_decode_parity(cw[pick], fl[pick], ref, wl.y[pick], label="host buffers, 4 chunks")


def test_host_decode_rejects_device_tensors(mp):
    code = mp.Code.rm(6, 2, crc_poly=0x21, crc_len=6, weights=[16])
    with pytest.raises(TypeError):
        code.decode_host(torch.zeros((4, 64), device="cuda"), 8, 4)


@pytest.mark.parametrize("use_graph", [False, True])
def test_host_decodes_back_to_back(mp, use_graph):
    """Calls alternate between two device input buffers: the input copies of a
    call may run while the call before it still decodes. Four back-to-back calls
    on different inputs, with no synchronisation between them, each equal the
    device-buffer decode of their own input."""
    code = mp.Code.rm(6, 2, crc_poly=0x21, crc_len=6, weights=[16])
    B = 200_000
    ys = [synth.make_workload("rm26_crc6", 1.0, B, seed=s).y for s in (41, 42, 43, 44)]
    pins = [torch.from_numpy(y).pin_memory() for y in ys]
    outs = [code.decode_host(p, 8, 4, use_graph=use_graph) for p in pins]
    torch.cuda.synchronize()
    for y, (cw, fl) in zip(ys, outs):
        rcw, rfl = _device_decode(code, y, 8, 4)
        assert np.array_equal(to_words(cw), rcw)
        assert np.array_equal(fl.numpy(), rfl)
