"""CPU-side checks of the C ABI (no GPU needed): the library loads and exports
every entry point that include/mpwsd.h declares; the host helpers agree with
the oracle; argument validation rejects bad inputs before touching CUDA."""
import ctypes

import numpy as np
import pytest

mp = pytest.importorskip("paper_2602_08501_gb300.mpwsd")


@pytest.fixture(scope="module")
def lib():
    import os

    if not os.path.exists(mp.LIB_PATH):
        pytest.skip("libmpwsd.so not built (run __graft_entry__.build())")
    return mp.lib()


def test_exports_every_declared_symbol(lib):
    names = mp.declared_symbols()
    assert len(names) >= 16
    for n in names:
        assert hasattr(lib, n), n


def test_strerror(lib):
    for st in (0, -1, -2, -3, -4, -5):
        assert lib.mpwsd_strerror(st).decode().startswith("MPWSD_")


@pytest.mark.parametrize("m,r,weights", [(5, 1, [16]), (6, 2, [16]), (6, 2, [16, 24]), (5, 1, [8, 16, 32])])
def test_enumerator_matches_oracle(lib, oracle_mod, m, r, weights):
    got = mp.enumerate_codewords(1 << m, mp.rm_frozen(m, r), weights)
    want = oracle_mod.rm_code(m, r).enumerate_codewords(weights)
    assert np.array_equal(got, want)


def test_enumerator_rm27(lib, oracle_mod):
    got = mp.enumerate_codewords(128, mp.rm_frozen(7, 2), [32])
    want = oracle_mod.rm_code(7, 2).enumerate_codewords([32])
    assert got.shape == (10668, 2) and np.array_equal(got, want)


def test_rm_frozen_matches_oracle(oracle_mod):
    for m, r in [(5, 1), (6, 2), (7, 2), (4, 1)]:
        assert np.array_equal(mp.rm_frozen(m, r), oracle_mod.rm_frozen(m, r))


def _load(n, frozen, k_info, poly, crc_len, pats, G=None):
    h = ctypes.c_void_p()
    fz = np.ascontiguousarray(frozen, np.uint8)
    pats = np.ascontiguousarray(pats, np.uint64)
    g = None if G is None else np.ascontiguousarray(G, np.uint8)
    st = mp.lib().mpwsd_load_code(n, None if g is None else g.ctypes.data_as(ctypes.c_void_p),
                                  fz.ctypes.data_as(ctypes.c_void_p), k_info, poly, crc_len,
                                  pats.ctypes.data_as(ctypes.c_void_p), pats.shape[0], ctypes.byref(h))
    if st == 0:
        mp.lib().mpwsd_free_code(h)
    return st


def test_load_code_validation(lib):
    fz = mp.rm_frozen(6, 2)
    pats = mp.enumerate_codewords(64, fz, [16])
    EINVAL = mp.EINVAL
    assert _load(48, fz, 16, 0x21, 6, pats) == EINVAL                 # bad n
    assert _load(64, fz, 17, 0x21, 6, pats) == EINVAL                 # k_info + crc_len != k
    assert _load(64, fz, 16, 0x61, 6, pats) == EINVAL                 # poly bit above crc_len
    bad = pats.copy()
    bad[5, 0] ^= np.uint64(1)                                          # not a codeword
    assert _load(64, fz, 16, 0x21, 6, bad) == EINVAL
    zero = pats.copy()
    zero[3, 0] = 0                                                     # zero pattern
    assert _load(64, fz, 16, 0x21, 6, zero) == EINVAL
    dup = pats.copy()
    dup[10] = dup[11]                                                  # repeated pattern
    assert _load(64, fz, 16, 0x21, 6, dup) == EINVAL
    # G must be the Arikan rows at the information indices
    info = np.flatnonzero(fz == 0)
    G = np.array([[1 if (i & j) == j else 0 for j in range(64)] for i in info], np.uint8)
    Gb = G.copy()
    Gb[0, 0] ^= 1
    assert _load(64, fz, 16, 0x21, 6, pats, Gb) == EINVAL
    assert b"G row" in mp.lib().mpwsd_last_error()


def test_enumerator_validation(lib):
    cnt = ctypes.c_int64(0)
    fz = np.ascontiguousarray(mp.rm_frozen(6, 2), np.uint8)
    w = np.array([24, 16], np.int32)  # not ascending
    st = lib.mpwsd_enumerate_codewords(64, fz.ctypes.data_as(ctypes.c_void_p), w.ctypes.data_as(ctypes.c_void_p), 2,
                                       None, 0, ctypes.byref(cnt))
    assert st == mp.EINVAL
