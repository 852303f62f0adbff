"""Pins of the oracle's paper variants (Section 3 bitmap encoder, Section 5
int16 wrap-around decoder).

* int16 wrap-around: a hand-worked overflow trace on the Z=2 code; equality
  with the FP32 plain decoder on integer LLRs whenever nothing wraps (min,
  plus and minus are exact there); equality with the saturating int8
  decoder (normalised) whenever neither saturates nor wraps.
* bitmap encoder: the word/bit rotation against a brute-force bit roll; the
  packed codeword against the byte encoder and against H x = 0.
"""
import numpy as np
import pytest

import oracle
import synth


def _pack(bits):
    bits = np.ascontiguousarray(bits, dtype=np.uint8)
    F, n = bits.shape
    return np.packbits(bits.reshape(F, n // 8, 8), axis=2, bitorder="little") \
             .reshape(F, n // 8).view(np.uint32)


def test_int16_wrap_hand_example(golden_z2):
    from tests.conftest import load_golden
    g = load_golden("z2_int16_wrap.txt")
    sh = synth.tiny_z2_code()
    rc = oracle.RefCode(sh.hbm, sh.z)
    llr = np.array(g["llr"], dtype=np.int16)[None]
    h, it, post, ev = rc.decode_layered_i16w(llr, max_iters=1, normalise=False)
    assert post[0].tolist() == [int(x) for x in g["after_iter1"]]
    assert ev == int(g["wrap_events"][0])
    bits = oracle.unpack_hard(h, rc.n)[0]
    assert bits.tolist() == [1] * 8 + [0, 0]
    llr = np.array(g["llr_b"], dtype=np.int16)[None]
    h, it, post, ev = rc.decode_layered_i16w(llr, max_iters=1, normalise=False)
    assert post[0].tolist() == [int(x) for x in g["after_iter1_b"]]
    assert oracle.unpack_hard(h, rc.n)[0].tolist() == [int(x) for x in g["hard_b"]]
    assert ev == int(g["wrap_events_b"][0])


@pytest.mark.parametrize("shape,ebn0,iters", [(synth.wifi_n648_r12(), 2.0, 8),
                                              (synth.wifi_n1944_r56(), 4.0, 6),
                                              (synth.random_small_code(3, 5, 12, 29), 1.5, 10)],
                         ids=["wifi648", "wifi1944", "rand_z29"])
def test_int16_plain_equals_fp32_plain_without_wrap(shape, ebn0, iters):
    rc = oracle.RefCode(shape.hbm, shape.z)
    info = oracle.gen_info(1, 0, 40, rc.k)
    llr = oracle.awgn_llr(rc.encode(info), 0, 1, synth.ebn0_db_to_sigma(ebn0, rc.k / rc.n))
    q = oracle.quantize_i16(llr, 4.0, 10)
    h16, i16, p16, ev = rc.decode_layered_i16w(q, iters, normalise=False, early_stop=True)
    assert ev == 0
    h32, i32, p32 = rc.decode_layered_f32(q.astype(np.float32), iters, 1.0, False, True)
    assert (i16 == i32).all() and (h16 == h32).all()
    assert (p16.astype(np.float32) == p32).all()


def test_int16_normalised_equals_int8_without_saturation():
    shape = synth.wifi_n648_r12()
    rc = oracle.RefCode(shape.hbm, shape.z)
    info = oracle.gen_info(1, 0, 30, rc.k)
    llr = oracle.awgn_llr(rc.encode(info), 0, 1, synth.ebn0_db_to_sigma(1.0, 0.5))
    q8 = oracle.quantize_i8(llr, 1.0, 12)
    h8, i8, p8, sat = rc.decode_layered_i8(q8, 2, True, False)
    assert sat == 0
    h16, i16, p16, ev = rc.decode_layered_i16w(q8.astype(np.int16), 2, normalise=True)
    assert ev == 0
    assert (p16 == p8.astype(np.int16)).all() and (h16 == h8).all()


def test_int16_quantiser():
    x = np.array([0.0, 0.49, 0.5, 1.5, -2.5, 63.99, 64.1, -1e9, 1e9], dtype=np.float32)
    assert oracle.quantize_i16(x, 16.0, 10).tolist() == \
        [0, 8, 8, 24, -40, 1023, 1023, -1023, 1023]
    assert oracle.quantize_i16(np.array([0.5, 1.5, 2.5], np.float32), 1.0, 10).tolist() == \
        [0, 2, 2]


@pytest.mark.parametrize("zw", [1, 2, 3])
def test_block_rotation_brute_force(zw):
    rng = np.random.default_rng(zw)
    z = 32 * zw
    words = rng.integers(0, 2**32, zw, dtype=np.uint64).astype(np.uint32)
    bits = np.unpackbits(words.view(np.uint8), bitorder="little")
    for s in range(z):
        got = np.unpackbits(oracle.rotate_block(words, s).view(np.uint8), bitorder="little")
        assert (got == np.roll(bits, -s)).all(), s     # out[r] = in[(r + s) mod Z]


@pytest.mark.parametrize("z", [32, 64, 96])
def test_bitmap_encoder_matches_byte_encoder(z):
    shapes = [s for s in synth.wimax_mixed_set() if s.z == z]
    assert len(shapes) == 4
    for sh in shapes:
        rc = oracle.RefCode(sh.hbm, sh.z)
        info = oracle.gen_info(9, 0, 12, rc.k)
        cw = rc.encode(info)
        got = rc.encode_bitmap(_pack(info))
        assert (got == _pack(cw)).all()
        bits = oracle.unpack_hard(got, rc.n)
        assert all(rc.syndrome_weight(b) == 0 for b in bits)


def test_bitmap_encoder_rejects_z_not_multiple_of_32():
    sh = synth.wimax_mixed_set()[0]   # Z = 24
    rc = oracle.RefCode(sh.hbm, sh.z)
    with pytest.raises(oracle.OracleError):
        rc.encode_bitmap(np.zeros((1, rc.k // 32), np.uint32))
