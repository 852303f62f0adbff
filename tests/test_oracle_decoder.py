"""Pins for the oracle's decoders (Section 4-5: eq. 18-23 and the layered
schedule).  Each test fixes the oracle against something other than itself:
the hand-derived worked example, closed forms, brute-force maximum
likelihood, exact-arithmetic invariants, or a structural symmetry."""
import numpy as np
import pytest

import oracle
import synth
from helpers import all_codewords, unpack_bits


def _prefix_code(hbm, rows):
    """Block rows 0..rows-1 of H_bm as a decoder-only code: one iteration on
    it performs exactly the first `rows` layers of the full schedule."""
    return oracle.RefCode(hbm[:rows], 2, require_encodable=False)


@pytest.mark.parametrize("layers", [1, 2, 3])
def test_worked_example_alpha1(golden_z2, layers):
    c = synth.tiny_z2_code()
    rc = _prefix_code(c.hbm, layers) if layers < 3 else oracle.RefCode(c.hbm, 2)
    llr = np.array([golden_z2["llr"]], dtype=np.float32)
    hard, iters, post = rc.decode_layered_f32(llr, max_iters=1, normalise=False)
    assert post[0].tolist() == golden_z2[f"alpha1_after_layer{layers - 1}"]


@pytest.mark.parametrize("layers", [1, 2, 3])
def test_worked_example_alpha075(golden_z2, layers):
    c = synth.tiny_z2_code()
    rc = _prefix_code(c.hbm, layers) if layers < 3 else oracle.RefCode(c.hbm, 2)
    llr = np.array([golden_z2["llr"]], dtype=np.float32)
    _, _, post = rc.decode_layered_f32(llr, max_iters=1, alpha=0.75, normalise=True)
    assert post[0].tolist() == golden_z2[f"alpha075_after_layer{layers - 1}"]


@pytest.mark.parametrize("layers", [1, 2, 3])
def test_worked_example_int8(golden_z2, layers):
    c = synth.tiny_z2_code()
    rc = _prefix_code(c.hbm, layers) if layers < 3 else oracle.RefCode(c.hbm, 2)
    q = np.array([golden_z2["int8_llr"]], dtype=np.int8)
    _, _, post, ev = rc.decode_layered_i8(q, max_iters=1, normalise=True)
    assert post[0].tolist() == golden_z2[f"int8_after_layer{layers - 1}"]
    assert ev == 0


def test_worked_example_decision(golden_z2):
    """eq. (21) and the syndrome stop: the one channel error is corrected in
    the first iteration, so early stop reports iters = 1."""
    c = synth.tiny_z2_code()
    rc = oracle.RefCode(c.hbm, 2)
    llr = np.array([golden_z2["llr"]], dtype=np.float32)
    hard, iters, _ = rc.decode_layered_f32(llr, max_iters=20, normalise=False,
                                           early_stop=True)
    assert iters[0] == 1
    assert unpack_bits(hard, 10)[0].tolist() == [int(v) for v in golden_z2["codeword"]]


@pytest.mark.parametrize("shape", [synth.wifi_n648_r12(), synth.wifi_n1944_r56()],
                         ids=lambda s: s.name)
def test_noiseless_one_iteration(shape):
    """LLR = +-A on a codeword: every message agrees with the channel, so the
    syndrome is zero after the first iteration and x_hat = c."""
    rc = oracle.RefCode(shape.hbm, shape.z)
    rng = np.random.default_rng(5)
    info = rng.integers(0, 2, size=(3, rc.k), dtype=np.uint8)
    cw = rc.encode(info)
    llr = (1.0 - 2.0 * cw).astype(np.float32) * 8.0
    hard, iters, post = rc.decode_layered_f32(llr, max_iters=10, early_stop=True)
    assert (iters == 1).all()
    assert (unpack_bits(hard, rc.n) == cw).all()
    assert (np.abs(post) >= 8.0).all()       # |Z| only grows
    q = (1 - 2 * cw.astype(np.int8)) * np.int8(20)
    hard8, iters8, _, _ = rc.decode_layered_i8(q, max_iters=10, early_stop=True)
    assert (iters8 == 1).all() and (unpack_bits(hard8, rc.n) == cw).all()


def test_single_parity_check_is_ml():
    """One block row with every block column used once is a set of Z disjoint
    single-parity-check codes (a tree).  With distinct |LLR|, one min-sum
    iteration (alpha = 1) returns the ML decision: hard decisions, with the
    least reliable bit flipped when the parity is odd."""
    hbm = np.array([[0, 1, 0, 1, 0]], dtype=np.int16)
    rc = oracle.RefCode(hbm, 2, require_encodable=False)
    rng = np.random.default_rng(9)
    for _ in range(200):
        mags = rng.permutation(np.arange(1, 11)).astype(np.float32) * 0.37
        sgn = rng.choice([-1.0, 1.0], size=10).astype(np.float32)
        llr = (mags * sgn)[None]
        hard, _, _ = rc.decode_layered_f32(llr, max_iters=1, normalise=False)
        got = unpack_bits(hard, 10)[0]
        want = (llr[0] <= 0).astype(np.uint8)
        for r in range(2):
            vars_ = rc.row_vars(r)
            if want[vars_].sum() % 2:
                weakest = vars_[np.argmin(np.abs(llr[0, vars_]))]
                want[weakest] ^= 1
        assert (got == want).all()


def _corr(words, llr):
    return ((1.0 - 2.0 * words) * llr).sum(axis=-1)


@pytest.mark.parametrize("shape", [synth.tiny_z2_code(), synth.tiny_z3_code()],
                         ids=lambda s: s.name)
def test_brute_force_ml_bounds_minsum(shape):
    """ML over all codewords maximises the correlation sum (1 - 2 c_n) LLR_n,
    so whenever min-sum outputs a codeword its correlation is no larger, and
    over many frames min-sum cannot beat ML's frame error rate."""
    rc = oracle.RefCode(shape.hbm, shape.z)
    book = all_codewords(shape.hbm, shape.z)
    assert len(book) == 1 << rc.k
    rng = np.random.default_rng(21)
    F = 4000
    info = rng.integers(0, 2, size=(F, rc.k), dtype=np.uint8)
    cw = rc.encode(info)
    sigma = 0.8
    y = (1.0 - 2.0 * cw) + sigma * rng.standard_normal(cw.shape)
    llr = (2.0 * y / sigma ** 2).astype(np.float32)
    hard, _, _ = rc.decode_layered_f32(llr, max_iters=20, alpha=0.75, early_stop=True)
    xh = unpack_bits(hard, rc.n)
    scores = llr.astype(np.float64) @ (1.0 - 2.0 * book.T.astype(np.float64))
    ml = book[np.argmax(scores, axis=1)]
    is_cw = np.array([rc.syndrome_weight(w) == 0 for w in xh])
    c_ms = _corr(xh[is_cw], llr[is_cw].astype(np.float64))
    c_ml = _corr(ml[is_cw], llr[is_cw].astype(np.float64))
    assert (c_ml >= c_ms - 1e-9).all()
    fer_ms = (xh != cw).any(axis=1).mean()
    fer_ml = (ml != cw).any(axis=1).mean()
    sd = np.sqrt(max(fer_ml * (1 - fer_ml), 1e-12) / F)
    assert fer_ms >= fer_ml - 3 * sd


@pytest.mark.parametrize("shape", [synth.wifi_n648_r12(), synth.wifi_n1944_r56()],
                         ids=lambda s: s.name)
def test_int8_equals_f32_in_exact_range(shape):
    """With plain min-sum (no scaling) and small integer LLRs, every FP32
    operation is exact, so while no int8 clamp fires the two decoders must
    agree exactly on posteriors, decisions and iteration counts."""
    rc = oracle.RefCode(shape.hbm, shape.z)
    rng = np.random.default_rng(13)
    info = rng.integers(0, 2, size=(6, rc.k), dtype=np.uint8)
    cw = rc.encode(info)
    noise = rng.integers(-5, 6, size=cw.shape)
    q = np.clip((1 - 2 * cw.astype(np.int64)) * 2 + noise, -7, 7).astype(np.int8)
    h8, it8, p8, ev = rc.decode_layered_i8(q, max_iters=2, normalise=False,
                                           early_stop=True)
    hf, itf, pf = rc.decode_layered_f32(q.astype(np.float32), max_iters=2,
                                        normalise=False, early_stop=True)
    assert ev == 0
    assert (h8 == hf).all() and (it8 == itf).all()
    assert (p8.astype(np.float32) == pf).all()


def test_normalise_alpha_one_is_plain():
    c = synth.wifi_n648_r12()
    rc = oracle.RefCode(c.hbm, c.z)
    rng = np.random.default_rng(1)
    llr = rng.normal(0.5, 2.0, size=(4, rc.n)).astype(np.float32)
    a = rc.decode_layered_f32(llr, max_iters=5, alpha=1.0, normalise=True)
    b = rc.decode_layered_f32(llr, max_iters=5, alpha=0.3, normalise=False)
    assert all((x == y).all() for x, y in zip(a, b))


def test_block_column_permutation_invariance():
    """Min and sign-XOR are order-free and each edge gets exactly one add, so
    relabelling the info block columns (and permuting the channel values with
    them) permutes the decoder output and changes nothing else."""
    c = synth.wifi_n648_r12()
    rc = oracle.RefCode(c.hbm, c.z)
    perm = np.concatenate([np.random.default_rng(2).permutation(c.kb),
                           np.arange(c.kb, c.nb)])
    rc2 = oracle.RefCode(c.hbm[:, perm], c.z)
    var_perm = (perm[:, None] * c.z + np.arange(c.z)[None, :]).reshape(-1)
    rng = np.random.default_rng(4)
    llr = rng.normal(1.0, 2.5, size=(3, rc.n)).astype(np.float32)
    _, it1, p1 = rc.decode_layered_f32(llr, max_iters=6, early_stop=True)
    _, it2, p2 = rc2.decode_layered_f32(llr[:, var_perm], max_iters=6, early_stop=True)
    assert (it1 == it2).all()
    assert (p1[:, var_perm] == p2).all()


def test_early_stop_count_is_first_zero_syndrome():
    """iters = k means the syndrome is nonzero after k-1 full iterations and
    zero after k (the check runs only after complete iterations)."""
    c = synth.wifi_n648_r12()
    rc = oracle.RefCode(c.hbm, c.z)
    rng = np.random.default_rng(8)
    info = rng.integers(0, 2, size=(12, rc.k), dtype=np.uint8)
    cw = rc.encode(info)
    sigma = synth.ebn0_db_to_sigma(2.0, 0.5)
    llr = (2.0 * ((1.0 - 2.0 * cw) + sigma * rng.standard_normal(cw.shape))
           / sigma ** 2).astype(np.float32)
    _, iters, _ = rc.decode_layered_f32(llr, max_iters=20, early_stop=True)
    assert iters.max() > 1
    for f in range(len(info)):
        k = int(iters[f])
        hk, _, _ = rc.decode_layered_f32(llr[f:f + 1], max_iters=k, early_stop=False)
        assert rc.syndrome_weight(unpack_bits(hk, rc.n)[0]) == 0 or k == 20
        if k > 1:
            hp, _, _ = rc.decode_layered_f32(llr[f:f + 1], max_iters=k - 1,
                                             early_stop=False)
            assert rc.syndrome_weight(unpack_bits(hp, rc.n)[0]) > 0


def test_flooding_equals_layered_on_one_layer():
    """With a single block row the layered and flooding schedules coincide;
    with integer LLRs and alpha = 1 the arithmetic is exact."""
    hbm = np.array([[0, 2, 1, 3, 0, 4]], dtype=np.int16)
    rc = oracle.RefCode(hbm, 5, require_encodable=False)
    rng = np.random.default_rng(6)
    llr = rng.integers(-9, 10, size=(20, rc.n)).astype(np.float32)
    a = rc.decode_layered_f32(llr, max_iters=4, normalise=False)
    b = rc.decode_flooding_f32(llr, max_iters=4, normalise=False)
    assert all((x == y).all() for x, y in zip(a, b))


def test_flooding_and_layered_agree_on_decoded_words():
    """Both schedules are min-sum: at moderate noise both return the sent
    codeword on almost every frame (layered in fewer iterations)."""
    c = synth.wifi_n648_r12()
    rc = oracle.RefCode(c.hbm, c.z)
    rng = np.random.default_rng(12)
    info = rng.integers(0, 2, size=(8, rc.k), dtype=np.uint8)
    cw = rc.encode(info)
    sigma = synth.ebn0_db_to_sigma(3.0, 0.5)
    llr = (2.0 * ((1.0 - 2.0 * cw) + sigma * rng.standard_normal(cw.shape))
           / sigma ** 2).astype(np.float32)
    hl, itl, _ = rc.decode_layered_f32(llr, max_iters=30, early_stop=True)
    hf, itf, _ = rc.decode_flooding_f32(llr, max_iters=30, early_stop=True)
    ok_l = (unpack_bits(hl, rc.n) == cw).all(axis=1)
    ok_f = (unpack_bits(hf, rc.n) == cw).all(axis=1)
    assert ok_l.sum() >= 7 and ok_f.sum() >= 7
    both = ok_l & ok_f
    assert itl[both].mean() <= itf[both].mean()


def test_int8_saturation_counted():
    """Posteriors clamp at +-127 and each clamp is counted.  After one
    iteration on a strong all-zero input every posterior is pinned at 127.
    (Later iterations subtract the full stored message from a clamped
    posterior, so values can fall and even change sign: that is the
    arithmetic the saturating rule defines, kept as is.)"""
    c = synth.wifi_n648_r12()
    rc = oracle.RefCode(c.hbm, c.z)
    q = np.full((1, rc.n), 63, dtype=np.int8)
    _, _, post, ev = rc.decode_layered_i8(q, max_iters=1, normalise=True)
    assert ev > 0 and (post == 127).all()
    _, _, post5, _ = rc.decode_layered_i8(q, max_iters=5, normalise=True)
    assert post5.min() >= -127 and post5.max() <= 127


def test_quantizer_rounding_and_clip():
    x = np.array([0.125, 0.375, -0.125, -0.375, 0.3, 100.0, -100.0, 15.8, -15.76],
                 dtype=np.float32)
    q = oracle.quantize_i8(x, 4.0, 63)
    # 0.5 -> 0 and 1.5 -> 2 (half to even), 1.2 -> 1, clip at +-63
    assert q.tolist() == [0, 2, 0, -2, 1, 63, -63, 63, -63]


def test_weighted_worked_example_layer0(golden_z2):
    """Per-edge message weights (learned normalised min-sum) on the first
    layer of the worked example, derived by hand from eq. (23)."""
    c = synth.tiny_z2_code()
    rc = oracle.RefCode(c.hbm[:1], 2, require_encodable=False)
    llr = np.array([golden_z2["llr"]], dtype=np.float32)
    w = np.array([golden_z2["weighted_layer0_weights"]], dtype=np.float32)
    _, _, post = rc.decode_layered_weighted_f32(llr, w, 1, early_stop=False)
    assert post[0].tolist() == golden_z2["weighted_after_layer0"]


@pytest.mark.parametrize("alpha", [1.0, 0.75, 0.6])
def test_weighted_constant_equals_normalised(alpha):
    """Constant weights reduce to the normalised decoder (plain for 1.0)."""
    c = synth.wifi_n648_r12()
    rc = oracle.RefCode(c.hbm, c.z)
    rng = np.random.default_rng(17)
    llr = rng.normal(0.8, 2.2, size=(6, rc.n)).astype(np.float32)
    T = 7
    w = np.full((T, rc.nnz_blocks), alpha, dtype=np.float32)
    a = rc.decode_layered_weighted_f32(llr, w, T, early_stop=True)
    b = rc.decode_layered_f32(llr, T, alpha, alpha != 1.0, True)
    assert all((x == y).all() for x, y in zip(a, b))


def test_weighted_weights_are_per_block_and_iteration():
    """Changing one block's weight in one iteration changes exactly the
    messages of that block from that iteration on (earlier iterations are
    unaffected)."""
    c = synth.wifi_n648_r12()
    rc = oracle.RefCode(c.hbm, c.z)
    rng = np.random.default_rng(19)
    llr = rng.normal(0.5, 2.0, size=(3, rc.n)).astype(np.float32)
    w = np.full((4, rc.nnz_blocks), 0.75, dtype=np.float32)
    w2 = w.copy()
    w2[2, 5] = 0.3
    p_a = [rc.decode_layered_weighted_f32(llr, w, T, early_stop=False)[2] for T in (2, 3)]
    p_b = [rc.decode_layered_weighted_f32(llr, w2, T, early_stop=False)[2] for T in (2, 3)]
    assert (p_a[0] == p_b[0]).all()        # iterations 1-2 identical
    assert not (p_a[1] == p_b[1]).all()    # iteration 3 differs
