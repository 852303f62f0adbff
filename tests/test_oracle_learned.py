"""Pins of the oracle's unrolled learned min-sum and its reference gradient.

* the PyTorch forward in float32 reproduces the C oracle's weighted layered
  decoder bit for bit (that decoder is pinned by the hand-worked Z=2 trace);
* the edge tables match the explicit H the C oracle builds;
* the loss is the textbook cross-entropy of the posterior bit probabilities;
* the float64 gradient matches central finite differences (h = 1e-4) on
  every frame whose discrete choices (argmins, signs) stay unchanged under
  the perturbation: the decoder is piecewise linear in (LLR, w), so away
  from kinks the difference quotient is exact up to the loss's curvature.
"""
import numpy as np
import pytest
import torch

import oracle
import synth
from oracle import learned

H_STEP = 1e-4


def _frames(shape, frames, ebn0, seed=1, frame0=0):
    rc = oracle.RefCode(shape.hbm, shape.z)
    info = oracle.gen_info(seed, frame0, frames, rc.k)
    cw = rc.encode(info)
    llr = oracle.awgn_llr(cw, frame0, seed, synth.ebn0_db_to_sigma(ebn0, rc.k / rc.n))
    return rc, cw, llr


def _weights(rc, T, seed, lo=0.5, hi=1.0):
    return np.random.default_rng(seed).uniform(lo, hi, (T, rc.nnz_blocks))


@pytest.mark.parametrize("shape,T,ebn0,frames", [(synth.tiny_z3_code(), 4, 1.0, 40),
                                                 (synth.wifi_n648_r12(), 5, 2.0, 24),
                                                 (synth.random_small_code(4, 6, 16, 37), 3, 1.5, 9)],
                         ids=["tiny_z3", "wifi648", "rand_z37"])
def test_forward_f32_equals_c_oracle(shape, T, ebn0, frames):
    rc, cw, llr = _frames(shape, frames, ebn0)
    w = _weights(rc, T, 2).astype(np.float32)
    _, _, post = rc.decode_layered_weighted_f32(llr, w, T, early_stop=False)
    _, _, posts, _ = learned.unrolled_forward(
        shape.hbm, shape.z, torch.from_numpy(llr), torch.from_numpy(cw), torch.from_numpy(w))
    assert posts.dtype == torch.float32
    assert (posts[-1].numpy() == post).all()
    # each iteration's posteriors equal a T-iteration run of the C oracle
    _, _, post2 = rc.decode_layered_weighted_f32(llr, w[:2], 2, early_stop=False)
    assert (posts[1].numpy() == post2).all()


def test_layer_tables_are_rows_of_h():
    shape = synth.random_small_code(7, 5, 13, 11)
    rc = oracle.RefCode(shape.hbm, shape.z)
    tabs = learned.layer_tables(shape.hbm, shape.z)
    nb = 0
    for l, (v, blocks) in enumerate(tabs):
        for r in range(shape.z):
            assert sorted(v[r].tolist()) == sorted(rc.row_vars(l * shape.z + r).tolist())
        assert blocks.tolist() == list(range(nb, nb + v.shape[1]))
        nb += v.shape[1]
    assert nb == rc.nnz_blocks


def test_loss_is_textbook_cross_entropy():
    rng = np.random.default_rng(0)
    Z = rng.uniform(-12, 12, 500)
    c = rng.integers(0, 2, 500)
    p1 = 1.0 / (1.0 + np.exp(Z))          # posterior probability of bit 1
    ref = -(c * np.log(p1) + (1 - c) * np.log(1 - p1))
    got = learned.bce_posterior(torch.from_numpy(Z), torch.from_numpy(c.astype(np.float64)))
    np.testing.assert_allclose(got.numpy(), ref, rtol=1e-9, atol=1e-12)
    # large |Z| stays finite and linear
    big = learned.bce_posterior(torch.tensor([800.0, -800.0]), torch.tensor([1.0, 0.0]))
    assert big.tolist() == [800.0, 800.0]


def _fd_check(shape, T, ebn0, frames, n_probe, seed, wrt):
    rc, cw, llr = _frames(shape, frames, ebn0, seed=seed)
    w = _weights(rc, T, seed)
    x = torch.from_numpy(llr.astype(np.float64))
    wt = torch.from_numpy(w)
    b = torch.from_numpy(cw)
    rng = np.random.default_rng(seed + 100)
    checked = 0
    for _ in range(n_probe):
        if wrt == "w":
            i = (int(rng.integers(T)), int(rng.integers(rc.nnz_blocks)))
        else:
            i = (int(rng.integers(frames)), int(rng.integers(rc.n)))

        def run(delta, grad=False):
            xx = x.clone()
            ww = wt.clone()
            (ww if wrt == "w" else xx)[i] += delta
            if grad:
                (ww if wrt == "w" else xx).requires_grad_(True)
            out = learned.unrolled_forward(shape.hbm, shape.z, xx, b, ww)
            return out, (ww if wrt == "w" else xx)

        (_, pf0, _, s0), var = run(0.0, grad=True)
        (_, pfp, _, sp), _ = run(H_STEP)
        (_, pfm, _, sm), _ = run(-H_STEP)
        keep = (s0 == sp) & (s0 == sm)
        if keep.sum() == 0:
            continue
        fd = ((pfp - pfm)[keep].sum() / (2 * H_STEP)).item()
        pf0[keep].sum().backward()
        g = var.grad[i].item()
        assert abs(g - fd) <= 1e-6 * max(abs(fd), 1e-3), (i, g, fd)
        checked += 1
    assert checked >= n_probe // 2


@pytest.mark.parametrize("shape,T,ebn0,frames", [(synth.tiny_z3_code(), 5, 1.0, 64),
                                                 (synth.wifi_n648_r12(), 4, 2.0, 8)],
                         ids=["tiny_z3", "wifi648"])
def test_weight_gradient_matches_central_differences(shape, T, ebn0, frames):
    _fd_check(shape, T, ebn0, frames, n_probe=10, seed=3, wrt="w")


def test_llr_gradient_matches_central_differences():
    _fd_check(synth.wifi_n648_r12(), 3, 1.5, 6, n_probe=10, seed=5, wrt="x")


def test_gradient_with_zero_weights_sees_only_the_channel():
    """w = 0 makes every message 0, so Z^(t) = LLR for all t and the
    gradient of the loss with respect to the LLRs is T (c - sigmoid(-LLR))."""
    shape = synth.tiny_z3_code()
    rc, cw, llr = _frames(shape, 16, 2.0)
    T = 3
    w = np.zeros((T, rc.nnz_blocks))
    loss, pf, gw, gx = learned.reference_gradient(shape.hbm, shape.z, llr, cw, w)
    L = llr.astype(np.float64)
    want = T * (cw - 1.0 / (1.0 + np.exp(L)))
    np.testing.assert_allclose(gx, want, rtol=1e-12, atol=1e-14)
    assert np.isfinite(gw).all() and np.abs(gw).sum() > 0
