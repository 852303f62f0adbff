"""Pins for the oracle's synthetic channel (eq. 16-17) and its counter-based
random numbers: published Philox test vectors, the elementary-function
series against libm in double precision, and the noise statistics."""
import math

import numpy as np
import pytest

import oracle
import synth

# Known-answer vectors for Philox4x32-10 published with the Random123 library
# (Salmon et al., SC'11): (counter, key) -> output.
PHILOX_KAT = [
    ((0, 0, 0, 0), (0, 0), (0x6627E8D5, 0xE169C58D, 0xBC57AC4C, 0x9B00DBD8)),
    ((0xFFFFFFFF,) * 4, (0xFFFFFFFF,) * 2,
     (0x408F276D, 0x41C83B0E, 0xA20BC7C6, 0x6D5451FD)),
    ((0x243F6A88, 0x85A308D3, 0x13198A2E, 0x03707344), (0xA4093822, 0x299F31D0),
     (0xD16CFE09, 0x94FDCCEB, 0x5001E420, 0x24126EA1)),
]


@pytest.mark.parametrize("ctr,key,want", PHILOX_KAT)
def test_philox_known_answers(ctr, key, want):
    assert oracle.philox4x32_10(ctr, key).tolist() == list(want)


def test_lnf_against_libm():
    rng = np.random.default_rng(0)
    us = np.concatenate([(rng.integers(0, 1 << 24, 20000) + 1) / float(1 << 24),
                         [2.0 ** -24, 0.5, 1.0, 0.70710677, 0.7071068, 0.999999]])
    for u in us.astype(np.float32):
        got = oracle.lnf(float(u))
        want = math.log(float(u))
        assert abs(got - want) <= 3e-7 * max(1.0, abs(want)), (u, got, want)
    assert oracle.lnf(1.0) == 0.0


def test_sincos_turn_against_libm():
    rng = np.random.default_rng(1)
    ks = np.concatenate([rng.integers(0, 1 << 24, 20000),
                         [0, 1 << 21, 1 << 22, (1 << 22) + (1 << 21), 1 << 23,
                          3 << 22, (1 << 24) - 1]])
    for k in ks:
        s, c = oracle.sincos_turn(int(k))
        a = 2.0 * math.pi * int(k) / float(1 << 24)
        assert abs(s - math.sin(a)) <= 2.5e-7 and abs(c - math.cos(a)) <= 2.5e-7, k


def test_gaussian_moments():
    """Noise of eq. (16) is standard normal: with an all-zero codeword,
    sigma = 1 and llr_scale = 1, llr - 1 is exactly the Gaussian stream."""
    cw = np.zeros((64, 4096), dtype=np.uint8)
    llr = oracle.awgn_llr(cw, 0, seed=1, sigma=1.0, llr_scale=1.0)
    g = llr.astype(np.float64).ravel() - 1.0
    assert abs(g.mean()) < 5 * (1 / math.sqrt(g.size))
    assert abs(g.var() - 1.0) < 0.01
    assert abs((g ** 3).mean()) < 0.02                      # skew
    assert abs((g ** 4).mean() - 3.0) < 0.05                # kurtosis
    assert abs((np.abs(g) > 2.0).mean() - 0.0455) < 0.002   # two-sided tail


def test_llr_formula_and_sign_convention():
    """eq. (16)-(17): bit 0 -> +1, bit 1 -> -1; llr = 2 y / sigma^2."""
    rng = np.random.default_rng(2)
    cw = rng.integers(0, 2, size=(4, 1000), dtype=np.uint8)
    sigma = synth.ebn0_db_to_sigma(2.0, 0.5)
    llr = oracle.awgn_llr(cw, 10, seed=1, sigma=sigma)
    g = oracle.awgn_llr(np.zeros_like(cw), 10, seed=1, sigma=1.0, llr_scale=1.0) - 1.0
    y = (1.0 - 2.0 * cw) + np.float32(sigma) * g
    np.testing.assert_allclose(llr, 2.0 * y / np.float32(sigma) ** 2, rtol=2e-6, atol=1e-5)
    assert abs(synth.ebn0_db_to_sigma(0.0, 0.5) - 1.0) < 1e-12   # Eb/N0 = 1, R = 1/2


def test_info_bits_counter_layout():
    a = oracle.gen_info(1, 0, 8, 324)
    b = oracle.gen_info(1, 5, 3, 324)
    assert (a[5:] == b).all()                      # frame index is the counter
    w = oracle.philox4x32_10((1, 2, 0, 0), (1, 0x494E464F))
    bit = lambda k: (int(w[(k // 32) % 4]) >> (k % 32)) & 1
    full = oracle.gen_info(1, 2, 1, 324)[0]
    assert [full[128 + t] for t in range(128)] == [bit(t) for t in range(128)]
    big = oracle.gen_info(7, 0, 64, 1620)
    assert abs(big.mean() - 0.5) < 0.01


# ------------------------------------------------ per-frame Eb/N0 and channel

def test_snr_sigma_range_uniformity_and_counter():
    """Eb/N0 recovered from each sigma lies in [lo, hi) and is uniform there
    (Kolmogorov-Smirnov); a frame's draw depends on its index only."""
    from scipy import stats
    lo, hi, rate = 1.0, 4.0, 5 / 6
    sig = oracle.snr_sigma(9, 1000, 20000, lo, hi, rate).astype(np.float64)
    ebn0 = 10 * np.log10(1.0 / (2 * rate * sig ** 2))
    assert ebn0.min() >= lo - 1e-5 and ebn0.max() < hi + 1e-5
    assert stats.kstest((ebn0 - lo) / (hi - lo), "uniform").pvalue > 1e-3
    assert (oracle.snr_sigma(9, 1003, 10, lo, hi, rate) ==
            oracle.snr_sigma(9, 1000, 13, lo, hi, rate)[3:]).all()
    assert not (oracle.snr_sigma(10, 1000, 50, lo, hi, rate) ==
                oracle.snr_sigma(9, 1000, 50, lo, hi, rate)).any()


def test_snr_sigma_degenerate_range_is_the_closed_form():
    for db, rate in ((2.0, 0.5), (4.5, 0.75), (-1.0, 0.625)):   # exact in float32
        sig = oracle.snr_sigma(3, 0, 7, db, db, rate)
        assert (sig == np.float32(synth.ebn0_db_to_sigma(db, rate))).all()


def test_mixed_frames_identities_and_codewords():
    """Frame j of code c is drawn at identity c * 2^32 + j; every codeword
    satisfies H c = 0, and at a very high Eb/N0 the LLR signs are the bits."""
    shapes = [synth.tiny_z2_code(), synth.tiny_z3_code(), synth.wifi_n648_r12()]
    cof = np.array([2, 0, 1, 1, 2, 0, 2, 1], dtype=np.int32)
    info, llr = oracle.mixed_frames(shapes, cof, (40.0, 40.0), seed=5)
    seen = {0: 0, 1: 0, 2: 0}
    for f, c in enumerate(cof):
        rc = oracle.RefCode(shapes[c].hbm, shapes[c].z)
        j = seen[int(c)]
        seen[int(c)] += 1
        assert (info[f] == oracle.gen_info(5, (int(c) << 32) + j, 1, rc.k)[0]).all()
        cw = rc.encode(info[f][None])[0]
        assert rc.syndrome_weight(cw) == 0
        assert ((llr[f] < 0) == (cw == 1)).all()
