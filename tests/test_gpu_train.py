"""Training kernels of learned min-sum against the oracle.

* forward checkpoints: every iteration's posteriors bit-exact against the
  oracle's float32 unrolled forward (and against the inference decoder),
  per-frame loss against the same loss evaluated in float64;
* backward: the weight and LLR gradients against the oracle's float64
  reverse-mode gradient (relative error below 1e-4) on the frames whose
  discrete choices agree in float32 and float64, and against float64
  central differences (h = 1e-4);
* the per-frame noise draw and channel, Adam, the autograd wrapper and a
  short training run (the loss falls; the result is reproducible).
"""
import numpy as np
import pytest

import oracle
import synth
from oracle import learned

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")

REL = 1e-4


@pytest.fixture(scope="module")
def ldpc():
    assert torch.cuda.is_available(), "GPU tests need a CUDA device"
    from paper_2306_12063_gb300 import _build
    _build.build()
    import paper_2306_12063_gb300 as m
    m.load()
    return m


def _batch(shape, frames, seed=1000, lo=1.0, hi=4.0):
    rc = oracle.RefCode(shape.hbm, shape.z)
    info = oracle.gen_info(seed, 0, frames, rc.k)
    cw = rc.encode(info)
    rng = np.random.default_rng(seed)
    llr = np.concatenate([
        oracle.awgn_llr(cw[i:i + 1], i, seed,
                        synth.ebn0_db_to_sigma(rng.uniform(lo, hi), rc.k / rc.n))
        for i in range(frames)])
    return rc, cw, llr


def _w(rc, T, seed=3):
    rng = np.random.default_rng(seed)
    return (0.75 + 0.1 * rng.standard_normal((T, rc.nnz_blocks))).astype(np.float32)


def _cuda(*arrs):
    return [torch.from_numpy(np.ascontiguousarray(a)).cuda() for a in arrs]


@pytest.mark.parametrize("shape,T,frames", [(synth.wifi_n648_r12(), 8, 77),
                                            (synth.wifi_n1944_r56(), 6, 33),
                                            (synth.random_small_code(4, 6, 16, 37), 3, 9)],
                         ids=["wifi648", "wifi1944", "rand_z37"])
def test_forward_checkpoints_bit_exact(ldpc, shape, T, frames):
    rc, cw, llr = _batch(shape, frames)
    w = _w(rc, T)
    _, pf, posts, _ = learned.unrolled_forward(shape.hbm, shape.z, torch.from_numpy(llr),
                                               torch.from_numpy(cw), torch.from_numpy(w))
    code = ldpc.Code(shape.hbm, shape.z)
    x, b, wt = _cuda(llr, cw, w)
    post, rows, loss, loss_sum = code.train_forward(x, b, wt, 0.5)
    assert (post.cpu().numpy() == posts.numpy()).all()
    # inference applies the weights with fused updates (the oracle's learned
    # decoder); training rounds w m first (the weighted decoder)
    _, _, p_inf = code.decode_learned(x, wt, early_stop=False, want_post=True)
    _, _, p_ref = rc.decode_learned_f32(llr, w, max_iters=T, early_stop=False)
    assert (p_inf.cpu().numpy() == p_ref).all()
    _, _, p_w = rc.decode_layered_weighted_f32(llr, w, T, early_stop=False)
    assert (post[-1].cpu().numpy() == p_w).all()
    # loss: the float64 cross-entropy of the same posteriors
    want = learned.bce_posterior(posts.double(), torch.from_numpy(cw).double()).sum(dim=(0, 2))
    np.testing.assert_allclose(loss.cpu().numpy(), want.numpy(), rtol=1e-5)
    np.testing.assert_allclose(loss_sum.item(), 0.5 * want.sum().item(), rtol=1e-5)


def _agreeing_frames(shape, llr, cw, w):
    x = torch.from_numpy(llr)
    b = torch.from_numpy(cw)
    _, _, _, s32 = learned.unrolled_forward(shape.hbm, shape.z, x, b, torch.from_numpy(w))
    _, _, _, s64 = learned.unrolled_forward(shape.hbm, shape.z, x.double(), b,
                                            torch.from_numpy(w).double())
    return (s32 == s64).numpy()


def _rel_err(got, want):
    return np.abs(got - want).max() / np.abs(want).max()


@pytest.mark.parametrize("shape,T,frames", [(synth.wifi_n648_r12(), 8, 64),
                                            (synth.wifi_n1944_r56(), 6, 24),
                                            (synth.tiny_z3_code(), 5, 64)],
                         ids=["wifi648", "wifi1944", "tiny_z3"])
def test_backward_matches_reference_gradient(ldpc, shape, T, frames):
    rc, cw, llr = _batch(shape, frames)
    w = _w(rc, T)
    keep = _agreeing_frames(shape, llr, cw, w)
    assert keep.sum() >= frames * 0.9
    llr, cw = llr[keep], cw[keep]
    F = llr.shape[0]
    scale = 1.0 / (F * rc.n)
    _, _, gw_ref, gx_ref = learned.reference_gradient(shape.hbm, shape.z, llr, cw, w, scale)
    code = ldpc.Code(shape.hbm, shape.z)
    x, b, wt = _cuda(llr, cw, w)
    post, rows, _, _ = code.train_forward(x, b, wt, scale)
    gw, gx = code.train_backward(x, b, wt, post, rows, scale, want_llr_grad=True)
    assert _rel_err(gw.cpu().numpy(), gw_ref) < REL
    assert _rel_err(gx.cpu().numpy(), gx_ref) < REL
    # the reduction over frames is fixed-order: a second call is bit-identical
    gw2, _ = code.train_backward(x, b, wt, post, rows, scale)
    assert torch.equal(gw, gw2)


def test_backward_matches_central_differences(ldpc):
    """GPU weight gradient against float64 central differences (h = 1e-4) of
    the oracle's forward, on frames that cross no kink."""
    shape = synth.wifi_n648_r12()
    rc, cw, llr = _batch(shape, 16)
    T = 4
    w = _w(rc, T, seed=8)
    code = ldpc.Code(shape.hbm, shape.z)
    rng = np.random.default_rng(21)
    h = 1e-4
    checked = 0
    for _ in range(8):
        i = (int(rng.integers(T)), int(rng.integers(rc.nnz_blocks)))
        wd = w.astype(np.float64)
        outs = []
        for delta in (0.0, h, -h):
            ww = wd.copy()
            ww[i] += delta
            outs.append(learned.unrolled_forward(shape.hbm, shape.z,
                                                 torch.from_numpy(llr).double(),
                                                 torch.from_numpy(cw), torch.from_numpy(ww)))
        keep = ((outs[0][3] == outs[1][3]) & (outs[0][3] == outs[2][3])).numpy()
        keep &= _agreeing_frames(shape, llr, cw, w)
        if keep.sum() == 0:
            continue
        fd = ((outs[1][1] - outs[2][1]).numpy()[keep].sum()) / (2 * h)
        x, b, wt = _cuda(llr[keep], cw[keep], w)
        post, rows, _, _ = code.train_forward(x, b, wt)
        gw, _ = code.train_backward(x, b, wt, post, rows)
        g = gw[i].item()
        assert abs(g - fd) <= REL * max(abs(fd), 1e-2), (i, g, fd)
        checked += 1
    assert checked >= 4


def test_single_iteration_and_empty_batch(ldpc):
    shape = synth.tiny_z3_code()
    rc, cw, llr = _batch(shape, 10)
    w = _w(rc, 1)
    code = ldpc.Code(shape.hbm, shape.z)
    x, b, wt = _cuda(llr, cw, w)
    post, rows, loss, _ = code.train_forward(x, b, wt)
    assert rows.numel() == 0
    gw, gx = code.train_backward(x, b, wt, post, rows, want_llr_grad=True)
    _, _, gw_ref, gx_ref = learned.reference_gradient(shape.hbm, shape.z, llr, cw, w)
    assert _rel_err(gw.cpu().numpy(), gw_ref) < REL
    assert _rel_err(gx.cpu().numpy(), gx_ref) < REL
    # zero frames: zero gradient, no launch
    e = x[:0]
    post0, rows0, loss0, ls0 = code.train_forward(e, b[:0], wt, 1.0)
    gw0, _ = code.train_backward(e, b[:0], wt, post0, rows0)
    assert ls0.item() == 0.0 and (gw0 == 0).all()


def test_snr_sigma_and_per_frame_channel(ldpc):
    """Per-frame Eb/N0 draws and the per-frame-sigma channel equal the
    oracle's, bit for bit."""
    seed, f0, F, lo, hi, rate = 77, 1234, 20000, 1.0, 4.0, 0.5
    sig = ldpc.snr_sigma(seed, f0, F, lo, hi, rate).cpu().numpy()
    want = oracle.snr_sigma(seed, f0, F, lo, hi, rate)
    assert (sig.view(np.uint32) == want.view(np.uint32)).all()
    shape = synth.wifi_n648_r12()
    rc = oracle.RefCode(shape.hbm, shape.z)
    F = 300
    info = oracle.gen_info(seed, f0, F, rc.k)
    cw = rc.encode(info)
    got = ldpc.awgn_llr_frames(torch.from_numpy(cw).cuda(), f0, seed,
                               torch.from_numpy(want[:F].copy()).cuda()).cpu().numpy()
    ref = oracle.awgn_llr_frames(cw, f0, seed, want[:F])
    assert (got.view(np.uint32) == ref.view(np.uint32)).all()


def test_adam_step(ldpc):
    rng = np.random.default_rng(4)
    p = rng.standard_normal(1000).astype(np.float32)
    m = np.zeros(1000, np.float32)
    v = np.zeros(1000, np.float32)
    P, M, V = _cuda(p, m, v)
    pd, md, vd = p.astype(np.float64), m.astype(np.float64), v.astype(np.float64)
    for step in range(1, 6):
        g = rng.standard_normal(1000).astype(np.float32)
        ldpc.adam_step(P, torch.from_numpy(g).cuda(), M, V, step, 1e-2, 0.9, 0.999, 1e-8)
        md = 0.9 * md + 0.1 * g
        vd = 0.999 * vd + 0.001 * g.astype(np.float64) ** 2
        pd = pd - 1e-2 * (md / (1 - 0.9 ** step)) / (np.sqrt(vd / (1 - 0.999 ** step)) + 1e-8)
    np.testing.assert_allclose(P.cpu().numpy(), pd, rtol=0, atol=1e-5)


def test_autograd_function(ldpc):
    from paper_2306_12063_gb300 import train
    shape = synth.wifi_n648_r12()
    rc, cw, llr = _batch(shape, 20)
    code = ldpc.Code(shape.hbm, shape.z)
    x, b, wt = _cuda(llr, cw, _w(rc, 4))
    wt.requires_grad_(True)
    x.requires_grad_(True)
    loss = train.learned_loss(code, wt, x, b)
    (2.0 * loss).backward()
    post, rows, _, ls = code.train_forward(x.detach(), b, wt.detach(), 1.0 / (20 * rc.n))
    gw, gx = code.train_backward(x.detach(), b, wt.detach(), post, rows, 2.0 / (20 * rc.n),
                                 want_llr_grad=True)
    assert loss.item() == ls.item()
    assert torch.equal(wt.grad, gw) and torch.equal(x.grad, gx)


def test_short_training_lowers_loss_and_is_reproducible(ldpc):
    from paper_2306_12063_gb300 import train
    shape = synth.wifi_n648_r12()
    code = ldpc.Code(shape.hbm, shape.z)
    cfg = train.TrainConfig(T=8, steps=100, batch=1024, lr=1e-2)
    r1 = train.train_weights(code, cfg)
    r2 = train.train_weights(code, cfg)
    assert np.isfinite(r1.loss_history.cpu().numpy()).all()
    assert torch.equal(r1.weights, r2.weights)
    # held-out frames (another seed): the trained weights lower the loss
    rc, cw, llr = _batch(shape, 2048, seed=5)
    x, b = _cuda(llr, cw)
    w0 = torch.full_like(r1.weights, cfg.init)
    l0 = code.train_forward(x, b, w0, 1.0 / (2048 * rc.n))[3].item()
    l1 = code.train_forward(x, b, r1.weights, 1.0 / (2048 * rc.n))[3].item()
    assert l1 < 0.99 * l0, (l0, l1)
