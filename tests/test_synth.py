"""Checks of the seeded input generator (transmitter + channel, Sec. II-B)."""
import numpy as np
import pytest

import synth


def test_splitmix64_known_outputs():
    # SplitMix64 seeded with 0 (Steele, Lea, Flood 2014): first outputs
    out = synth.splitmix64_stream(0, np.arange(2))
    assert int(out[0]) == 0xE220A8397B1DCDAF
    assert int(out[1]) == 0x6E789E6AA1B965F4


@pytest.mark.parametrize("ebn0,rate,sigma", [
    (1.0, 16 / 64, 1.2604), (2.0, 16 / 64, 1.1233), (3.0, 16 / 64, 1.0012), (0.5, 16 / 64, 1.3351),
    (0.5, 23 / 128, 1.5748), (1.5, 23 / 128, 1.4036), (2.5, 23 / 128, 1.2509)])
def test_sigma_values(ebn0, rate, sigma):
    assert abs(synth.sigma_for(ebn0, rate) - sigma) < 1e-4  # printed to 4 decimals


def test_grid_and_determinism():
    wl = synth.make_workload("rm26_crc6", 1.0, 3000, seed=1)
    q = wl.y.astype(np.float64) * 2 ** 19
    assert np.all(q == np.rint(q)) and np.abs(q).max() <= 2 ** 23 - 1
    part = synth.make_workload("rm26_crc6", 1.0, 500, seed=1, first_frame=1200)
    assert np.array_equal(part.y, wl.y[1200:1700]) and np.array_equal(part.cw, wl.cw[1200:1700])
    other = synth.make_workload("rm26_crc6", 1.0, 500, seed=2)
    assert not np.array_equal(other.y, wl.y[:500])


def test_noise_statistics():
    wl = synth.make_workload("rm26_crc6", 1.0, 20000, seed=3)
    noise = wl.y.astype(np.float64) - (1.0 - 2.0 * wl.cw)
    s = synth.sigma_for(1.0, 0.25)
    assert abs(noise.mean()) < 0.01
    assert abs(noise.std() / s - 1.0) < 0.01
    # Gaussian tails: P(|g| > 2) = 0.0455
    assert abs(np.mean(np.abs(noise / s) > 2.0) - 0.0455) < 0.003
    assert abs(wl.msg.mean() - 0.5) < 0.01


def test_transmitted_words_are_crc_codewords(oracle_mod):
    for name, (m, r) in [("rm26_crc6", (6, 2)), ("rm27_crc6", (7, 2))]:
        wl = synth.make_workload(name, 2.0, 200, seed=0)
        code = oracle_mod.rm_code(m, r, crc_poly=0x21, crc_len=6)
        assert all(code.crc_ok(c) for c in wl.cw)
        F = oracle_mod.kron_power(m)
        u = (wl.cw.astype(np.int64) @ F.astype(np.int64)) % 2
        info = np.flatnonzero(code.frozen == 0)
        assert np.array_equal(u[:, info[:code.k_info]], wl.msg)


def test_encoder_matches_kronecker_matrix(oracle_mod):
    rng = np.random.default_rng(0)
    for m in (1, 3, 5, 7):
        u = rng.integers(0, 2, (50, 1 << m)).astype(np.uint8)
        F = oracle_mod.kron_power(m).astype(np.int64)
        assert np.array_equal(synth.encode_arikan(u), (u.astype(np.int64) @ F) % 2)


def test_snr_range_workload():
    wl = synth.make_workload("rm27_crc6", (0.5, 3.0), 4000, seed=4)
    assert wl.ebn0_db.min() >= 0.5 and wl.ebn0_db.max() <= 3.0
    assert abs(wl.ebn0_db.mean() - 1.75) < 0.05
