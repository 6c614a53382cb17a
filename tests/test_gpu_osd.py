"""GPU OSD(order) stage 1 against the oracle: the list (codewords and integer
discrepancies, bit-exact) and whole decodes with OSD anchors."""
import numpy as np
import pytest

import synth
from gpu_common import assert_decode_parity, cuda_or_skip, oracle_code, to_words, torch

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def mp():
    return cuda_or_skip()


@pytest.fixture(scope="module")
def oracle_mod():
    import oracle

    return oracle


def _dev(a, dtype=torch.float32):
    return torch.from_numpy(np.ascontiguousarray(a)).to(dtype).cuda()


def _check_lists(mp, code, ocode, oracle_mod, y, order, L):
    cw, d = code.osd_list(_dev(y), order, L)
    torch.cuda.synchronize()
    cw, d = to_words(cw), d.cpu().numpy()
    for f in range(y.shape[0]):
        cl, dl = ocode.osd(y[f].astype(np.float64), order, L)
        cnt = cl.shape[0]
        assert np.array_equal(cw[f, :cnt], oracle_mod.pack_bits(cl)), (order, L, f)
        assert np.array_equal(d[f, :cnt], np.rint(dl * 2 ** 19).astype(np.int64)), (order, L, f)
        assert np.all(d[f, cnt:] == -1)


@pytest.mark.parametrize("order,L", [(0, 1), (1, 8), (2, 8), (2, 32), (3, 16), (4, 8)])
def test_osd_list_bit_exact_rm26(mp, oracle_mod, order, L):
    code = mp.Code.rm(6, 2, crc_poly=0x21, crc_len=6, weights=[16])
    ocode = oracle_code(oracle_mod, 6, 2, 6, [16])
    wl = synth.make_workload("rm26_crc6", 1.0, 60 if order < 4 else 12, seed=40 + order)
    _check_lists(mp, code, ocode, oracle_mod, wl.y, order, L)


def test_osd_list_bit_exact_rm27_and_rm15(mp, oracle_mod):
    code = mp.Code.rm(7, 2, crc_poly=0x21, crc_len=6, weights=[32])
    ocode = oracle_code(oracle_mod, 7, 2, 6, [32])
    wl = synth.make_workload("rm27_crc6", 1.5, 40, seed=50)
    _check_lists(mp, code, ocode, oracle_mod, wl.y, 2, 16)
    small = mp.Code.rm(5, 1, weights=[16])
    osmall = oracle_code(oracle_mod, 5, 1, 0, [16])
    rng = np.random.default_rng(51)
    y = synth.grid_quantize(rng.standard_normal((30, 32)) * 1.3)
    _check_lists(mp, small, osmall, oracle_mod, y, 4, 32)  # 57 of the 64 codewords


def test_osd_list_edge_inputs(mp, oracle_mod):
    code = mp.Code.rm(6, 2, crc_poly=0x21, crc_len=6, weights=[16])
    ocode = oracle_code(oracle_mod, 6, 2, 6, [16])
    rng = np.random.default_rng(52)
    for y in (np.zeros((3, 64), np.float32),                                     # every reliability ties
              synth.grid_quantize(rng.standard_normal((5, 64)) * 2e-6),            # a few grid steps
              synth.grid_quantize(np.sign(rng.standard_normal((4, 64))) * 40.0),   # clamped
              synth.grid_quantize(np.round(rng.standard_normal((6, 64)) * 2) / 2)):  # many equal magnitudes
        _check_lists(mp, code, ocode, oracle_mod, np.ascontiguousarray(y, np.float32), 2, 16)


def _decode_parity(mp, code, ocode, y, L, T, order, mode, aom=False):
    cw, fl = code.decode(_dev(y), L, T, score_mode=mode, always_on=aom, osd_order=order)
    torch.cuda.synchronize()
    cw, fl = to_words(cw), fl.cpu().numpy().view(np.uint16)
    ref = ocode.decode(y, L, T, aom=aom, osd_order=order)
    assert_decode_parity(cw, fl, ref, y, label=f"OSD({order}) L={L} T={T} {mode} aom={aom}")
    return fl


@pytest.mark.parametrize("mode", ["bf16x2", "fp32"])
def test_decode_with_osd_anchors_rm26(mp, oracle_mod, mode):
    code = mp.Code.rm(6, 2, crc_poly=0x21, crc_len=6, weights=[16])
    ocode = oracle_code(oracle_mod, 6, 2, 6, [16])
    wl = synth.make_workload("rm26_crc6", 1.0, 1500, seed=53)
    fl = _decode_parity(mp, code, ocode, wl.y, 8, 4, 2, mode)
    assert 0 < np.mean(fl & 1) < 1
    _decode_parity(mp, code, ocode, wl.y[:300], 16, 4, 1, mode, aom=True)


def test_decode_with_osd_anchors_rm27(mp, oracle_mod):
    code = mp.Code.rm(7, 2, crc_poly=0x21, crc_len=6, weights=[32])
    ocode = oracle_code(oracle_mod, 7, 2, 6, [32])
    wl = synth.make_workload("rm27_crc6", 1.5, 200, seed=54)
    _decode_parity(mp, code, ocode, wl.y, 16, 6, 2, "bf16x2")


@pytest.mark.parametrize("order", [2, 3, 4])
def test_decode_rm128_29_always_on(mp, oracle_mod, order):
    """The paper's RM experiment (Sec. IV-A settings, Sec. III-C always-on mode):
    RM(128, 29) with no CRC, stage 2 on every frame, OSD(order) anchors, J = 4,
    the 10,668 weight-32 patterns; bit-exact against the oracle."""
    code = mp.Code.rm(7, 2, weights=[32])
    ocode = oracle_code(oracle_mod, 7, 2, 0, [32])
    wl = synth.make_workload("rm27", 1.0, 400, seed=60 + order)
    fl = _decode_parity(mp, code, ocode, wl.y, 16, 4, order, "bf16x2", aom=True)
    assert np.all(fl & 1) and not np.any(fl & 2)  # no CRC: stage 2 ran everywhere, no CRC-ok flag
    # with no CRC the stage-1 exit cannot happen, so the always-on switch changes nothing
    cw2, fl2 = code.decode(_dev(wl.y), 16, 4, osd_order=order)
    cw1, fl1 = code.decode(_dev(wl.y), 16, 4, osd_order=order, always_on=True)
    torch.cuda.synchronize()
    assert torch.equal(cw1, cw2) and torch.equal(fl1, fl2)
    if order == 2:
        _decode_parity(mp, code, ocode, wl.y[:120], 16, 4, order, "fp32", aom=True)


def test_decode_rm128_29_always_on_list_sizes(mp, oracle_mod):
    """The same pipeline with 1, 8 and 32 anchors and a single iteration."""
    code = mp.Code.rm(7, 2, weights=[32])
    ocode = oracle_code(oracle_mod, 7, 2, 0, [32])
    wl = synth.make_workload("rm27", 0.5, 150, seed=66)
    for L, T in ((1, 4), (8, 1), (32, 4)):
        _decode_parity(mp, code, ocode, wl.y, L, T, 3, "bf16x2", aom=True)


def test_osd_options_are_validated(mp):
    code = mp.Code.rm(6, 2, crc_poly=0x21, crc_len=6, weights=[16])
    y = torch.zeros((4, 64), dtype=torch.float32, device="cuda")
    with pytest.raises(mp.MpwsdError) as ei:
        code.decode(y, 8, 4, osd_order=5)
    assert ei.value.status == mp.EINVAL
