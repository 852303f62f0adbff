"""Pins of the oracle's learned decoder run past its weight table and with
give-up checkpoints (ldpc_ref_decode_learned_f32).  Neither part is in the
paper (learned normalised min-sum extends eq. (23), the give-up rule extends
the Section 4 stopping test), so each is fixed against a definition that
does not run through the same code path: an explicitly extended weight
table, the alpha-scaled decoder, a shorter decode, and syndrome weights
recomputed from the dense parity-check matrix of eq. (2)."""
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
    want = rc.decode_layered_weighted_f32(llr, explicit, early_stop=True)
    for a, b in zip(got, want):
        assert (a == b).all()
    # and not the first row, nor a cycle through the table
    cyc = np.concatenate([w, w, w[:3]])
    other = rc.decode_layered_weighted_f32(llr, cyc, early_stop=True)
    assert not all((a == b).all() for a, b in zip(got, other))


def test_constant_table_run_long_is_the_alpha_decoder(case):
    _, rc, llr = case
    w = np.full((3, rc.nnz_blocks), 0.75, dtype=np.float32)
    got = rc.decode_learned_f32(llr, w, max_iters=15)
    want = rc.decode_layered_f32(llr, 15, 0.75, True, True)
    for a, b in zip(got, want):
        assert (a == b).all()


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
