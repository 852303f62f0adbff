"""Pins of the oracle's learned decoder in its inference form
(ldpc_ref_decode_learned_f32): fused posterior updates, iterations past the
weight table, give-up checkpoints.  None of it is in the paper (learned
normalised min-sum extends eq. (23), the give-up rule extends the Section 4
stopping test), so each part is fixed against a definition that does not run
through the same code path: an exact-rational trace of the layered schedule
on tiny codes, the alpha-scaled decoder, an explicitly extended weight table,
a shorter decode, and syndrome weights recomputed from the dense parity-check
matrix of eq. (2)."""
from fractions import Fraction

import numpy as np
import pytest

import oracle
import synth
from helpers import dense_h, unpack_bits


def _frames(shape, frames, ebn0, seed=3, frame0=0):
    rc = oracle.RefCode(shape.hbm, shape.z)
    info = oracle.gen_info(seed, frame0, frames, rc.k)
    llr = oracle.awgn_llr(rc.encode(info), frame0, seed,
                          synth.ebn0_db_to_sigma(ebn0, rc.k / rc.n))
    return rc, llr


def _weights(rc, T, seed):
    rng = np.random.default_rng(seed)
    return rng.uniform(0.45, 1.05, size=(T, rc.nnz_blocks)).astype(np.float32)


@pytest.fixture(scope="module")
def case():
    shape = synth.wifi_n648_r12()
    rc, llr = _frames(shape, 240, 1.25)
    return shape, rc, llr


def test_iterations_past_the_table_repeat_its_last_row(case):
    _, rc, llr = case
    w = _weights(rc, 4, 1)
    got = rc.decode_learned_f32(llr, w, max_iters=11)
    explicit = np.concatenate([w, np.repeat(w[-1:], 7, axis=0)])
    want = rc.decode_learned_f32(llr, explicit)
    for a, b in zip(got, want):
        assert (a == b).all()
    # and not the first row, nor a cycle through the table
    cyc = np.concatenate([w, w, w[:3]])
    other = rc.decode_learned_f32(llr, cyc)
    assert not all((a == b).all() for a, b in zip(got, other))


@pytest.mark.parametrize("wval,alpha,normalise", [(0.5, 0.5, True), (1.0, 1.0, False),
                                                  (0.25, 0.25, True)])
def test_power_of_two_weights_are_the_alpha_decoder(case, wval, alpha, normalise):
    """With w a power of two every product w m is exact, so the fused
    updates equal the alpha decoder's (alpha m rounded, then added)."""
    _, rc, llr = case
    w = np.full((3, rc.nnz_blocks), wval, dtype=np.float32)
    got = rc.decode_learned_f32(llr, w, max_iters=15)
    want = rc.decode_layered_f32(llr, 15, alpha, normalise, True)
    for a, b in zip(got, want):
        assert (a == b).all()


def _round_f32(x: Fraction) -> np.float32:
    """x rounded to the nearest float32, ties to even."""
    a = np.float32(float(x))
    best = None
    for c in (np.nextafter(a, np.float32(-np.inf)), a, np.nextafter(a, np.float32(np.inf))):
        d = abs(Fraction(float(c)) - x)
        even = (int(np.array(c, dtype=np.float32).view(np.uint32)) & 1) == 0
        key = (d, not even)
        if best is None or key < best[0]:
            best = (key, c)
    return np.float32(best[1])


def _exact_trace(shape, llr, w, iters, fused):
    """The layered learned decoder written with exact rationals, rounding to
    float32 where the definition rounds: fused, Z - w' m_old and Z + w m
    once each; otherwise w m first.  Rows in natural order, each row's edges
    by increasing column, weight index q = nonzero block of H_bm row by row."""
    H = dense_h(shape.hbm, shape.z)
    mb, z = shape.hbm.shape[0], shape.z
    T = w.shape[0]
    Z = [Fraction(float(v)) for v in llr]
    Lm = {}
    q0 = 0
    qbase = []
    for i in range(mb):
        qbase.append(q0)
        q0 += int((shape.hbm[i] >= 0).sum())
    for k in range(1, iters + 1):
        wk = w[min(k, T) - 1]
        wp = w[min(max(k - 1, 1), T) - 1]
        for i in range(mb):
            for r in range(z):
                row = i * z + r
                vs = list(np.nonzero(H[row])[0])
                Q = []
                for t, v in enumerate(vs):
                    old = Lm.get((row, t), Fraction(0))
                    wq = Fraction(float(wp[qbase[i] + t]))
                    Q.append(_round_f32(Z[v] - wq * old) if fused else _round_f32(Z[v] - old))
                Qf = [Fraction(float(q)) for q in Q]
                for t, v in enumerate(vs):
                    others = [Qf[u] for u in range(len(vs)) if u != t]
                    neg = sum(1 for o in others if o < 0) % 2
                    m = min(abs(o) for o in others) * (-1 if neg else 1)
                    wq = Fraction(float(wk[qbase[i] + t]))
                    if fused:
                        Lm[(row, t)] = m
                        Z[v] = Fraction(float(_round_f32(Qf[t] + wq * m)))
                    else:
                        lw = Fraction(float(_round_f32(wq * m)))
                        Lm[(row, t)] = lw
                        Z[v] = Fraction(float(_round_f32(Qf[t] + lw)))
    return np.array([float(v) for v in Z], dtype=np.float32)


@pytest.mark.parametrize("shape", [synth.tiny_z2_code(), synth.tiny_z3_code()],
                         ids=["z2", "z3"])
def test_fused_and_separate_rounding_against_exact_trace(shape):
    rc = oracle.RefCode(shape.hbm, shape.z)
    rng = np.random.default_rng(11)
    F = 40
    llr = rng.normal(0.3, 2.0, size=(F, rc.n)).astype(np.float32)
    w = rng.uniform(0.3, 1.1, size=(2, rc.nnz_blocks)).astype(np.float32)
    _, _, pf = rc.decode_learned_f32(llr, w, max_iters=3, early_stop=False)
    _, _, ps = rc.decode_layered_weighted_f32(
        llr, np.concatenate([w, w[-1:]]), early_stop=False)
    differ = 0
    for f in range(F):
        ef = _exact_trace(shape, llr[f], w, 3, True)
        es = _exact_trace(shape, llr[f], np.concatenate([w, w[-1:]]), 3, False)
        assert (pf[f] == ef).all(), f
        assert (ps[f] == es).all(), f
        differ += int((ef != es).any())
    assert differ > 0   # the two roundings are told apart on these frames


def test_checkpoint_that_always_fires_is_a_shorter_decode(case):
    _, rc, llr = case
    w = _weights(rc, 8, 2)
    got = rc.decode_learned_f32(llr, w, max_iters=20, stop_iter=(5, 0), stop_frac=(0.0, 0.0))
    want = rc.decode_learned_f32(llr, w, max_iters=5)
    for a, b in zip(got, want):
        assert (a == b).all()
    assert (got[1] == 5).sum() > 20


def test_checkpoint_that_never_fires_changes_nothing(case):
    _, rc, llr = case
    w = _weights(rc, 8, 2)
    got = rc.decode_learned_f32(llr, w, max_iters=20, stop_iter=(3, 9), stop_frac=(1.0, 1.5))
    want = rc.decode_learned_f32(llr, w, max_iters=20)
    for a, b in zip(got, want):
        assert (a == b).all()


def test_checkpoint_decisions_follow_the_unsatisfied_check_count(case):
    """At checkpoint g a frame stops iff its unsatisfied checks u (recounted
    here from the dense H) exceed floor(frac * M); the boundary u = limit
    continues."""
    shape, rc, llr = case
    H = dense_h(shape.hbm, shape.z).astype(np.int64)
    w = _weights(rc, 8, 4)
    g = 4
    h_g, it_g, _ = rc.decode_learned_f32(llr, w, max_iters=g, want_post=False)
    u = ((unpack_bits(h_g, rc.n).astype(np.int64) @ H.T) & 1).sum(axis=1)
    live = u > 0
    assert live.sum() > 30
    limit = int(np.median(u[live]))
    frac = np.float32((limit + 0.5) / rc.m)
    assert int(np.floor(frac * np.float32(rc.m))) == limit
    h, it, _ = rc.decode_learned_f32(llr, w, max_iters=20, stop_iter=(g, 0),
                                     stop_frac=(frac, 0.0), want_post=False)
    stop = live & (u > limit)
    go_on = live & (u <= limit)
    assert stop.sum() > 5 and go_on.sum() > 5 and (u[live] == limit).any()
    assert (it[stop] == g).all() and (h[stop] == h_g[stop]).all()
    assert (it[go_on] > g).all()
    assert (it[~live] == it_g[~live]).all()
    # the second checkpoint acts on the frames the first one let through
    h2, it2, _ = rc.decode_learned_f32(llr, w, max_iters=20, stop_iter=(g, 9),
                                       stop_frac=(frac, 0.0), want_post=False)
    assert (it2[stop] == g).all()
    assert (it2[go_on] <= 9).all()


def test_checkpoints_need_early_stop(case):
    _, rc, llr = case
    w = _weights(rc, 2, 5)
    with pytest.raises(RuntimeError):
        rc.decode_learned_f32(llr[:4], w, max_iters=6, early_stop=False, stop_iter=(3, 0),
                              stop_frac=(0.1, 0.0))
