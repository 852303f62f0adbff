"""Learned normalised min-sum on the GPU against the oracle (bit-exact), and
the learned-then-int8-fallback pipeline against the same steps done by the
oracle."""
import numpy as np
import pytest

import oracle
import synth

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")


@pytest.fixture(scope="module")
def ldpc():
    assert torch.cuda.is_available(), "GPU tests need a CUDA device"
    from paper_2306_12063_gb300 import _build
    _build.build()
    import paper_2306_12063_gb300 as m
    m.load()
    return m


def _inputs(shape, frames, ebn0, frame0=0):
    rc = oracle.RefCode(shape.hbm, shape.z)
    info = oracle.gen_info(1, frame0, frames, rc.k)
    llr = oracle.awgn_llr(rc.encode(info), frame0, 1, synth.ebn0_db_to_sigma(ebn0, rc.k / rc.n))
    return rc, info, llr


def _weights(rc, T, seed, lo=0.4, hi=1.0):
    rng = np.random.default_rng(seed)
    return rng.uniform(lo, hi, size=(T, rc.nnz_blocks)).astype(np.float32)


# long tables (T = 16, 17, 20): every iteration stages a new row
@pytest.mark.parametrize("shape,T,ebn0,frames", [(synth.wifi_n648_r12(), 8, 2.0, 333),
                                                 (synth.wifi_n1944_r56(), 6, 4.0, 257),
                                                 (synth.wimax_mixed_set()[-4], 8, 1.8, 41),
                                                 (synth.wifi_n648_r12(), 16, 1.5, 200),
                                                 (synth.wifi_n648_r12(), 17, 1.5, 200),
                                                 (synth.wifi_n1944_r56(), 20, 3.0, 120)],
                         ids=["wifi648", "wifi1944", "wimax2304", "wifi648_T16",
                              "wifi648_T17", "wifi1944_T20"])
def test_learned_bit_exact(ldpc, shape, T, ebn0, frames):
    rc, _, llr = _inputs(shape, frames, ebn0)
    w = _weights(rc, T, 5)
    wh, wi, wp = rc.decode_learned_f32(llr, w, max_iters=T, early_stop=True)
    code = ldpc.Code(shape.hbm, shape.z)
    gh, gi, gp = code.decode_learned(torch.from_numpy(llr).cuda(), torch.from_numpy(w).cuda(),
                                     early_stop=True, want_post=True)
    assert (gi.cpu().numpy() == wi).all()
    assert (gh.cpu().numpy().view(np.uint32) == wh).all()
    assert (gp.cpu().numpy() == wp).all()


@pytest.mark.parametrize("T,iters", [(1, 1), (1, 3), (2, 1), (3, 2), (2, 4), (5, 5)])
def test_learned_short_runs_bit_exact(ldpc, T, iters):
    """Runs of one to five iterations and tables of one to five rows: the
    weight rows streamed in ahead of each iteration (and the last row reused
    past the table) equal the oracle's decoder, with and without early stop."""
    shape = synth.wifi_n648_r12()
    rc, _, llr = _inputs(shape, 96, 2.5, frame0=7)
    w = _weights(rc, T, 23)
    code = ldpc.Code(shape.hbm, shape.z)
    for es in (False, True):
        wh, wi, wp = rc.decode_learned_f32(llr, w, max_iters=iters, early_stop=es)
        gh, gi, gp = code.decode_learned(torch.from_numpy(llr).cuda(), torch.from_numpy(w).cuda(),
                                         max_iters=iters, early_stop=es, want_post=True)
        assert (gi.cpu().numpy() == wi).all()
        assert (gh.cpu().numpy().view(np.uint32) == wh).all()
        assert (gp.cpu().numpy() == wp).all()


def test_learned_negative_and_mixed_weights(ldpc):
    """Weights of either sign (the sign multiplies the message sign)."""
    shape = synth.wifi_n648_r12()
    rc, _, llr = _inputs(shape, 64, 2.5)
    w = _weights(rc, 5, 9, lo=-0.3, hi=1.2)
    wh, wi, wp = rc.decode_learned_f32(llr, w, max_iters=5, early_stop=False)
    code = ldpc.Code(shape.hbm, shape.z)
    gh, gi, gp = code.decode_learned(torch.from_numpy(llr).cuda(), torch.from_numpy(w).cuda(),
                                     early_stop=False, want_post=True)
    assert (gp.cpu().numpy() == wp).all() and (gi.cpu().numpy() == wi).all()


@pytest.mark.parametrize("wval,alpha,normalise", [(0.5, 0.5, True), (1.0, 1.0, False)])
def test_learned_power_of_two_weights_equal_normalised(ldpc, wval, alpha, normalise):
    """Power-of-two weights make every product exact, so the fused learned
    updates equal the alpha decoder's."""
    shape = synth.wifi_n1944_r56()
    rc, _, llr = _inputs(shape, 200, 4.0)
    code = ldpc.Code(shape.hbm, shape.z)
    w = torch.full((8, rc.nnz_blocks), wval, dtype=torch.float32, device="cuda")
    x = torch.from_numpy(llr).cuda()
    a = code.decode_learned(x, w, early_stop=True, want_post=True)
    b = code.decode(x, max_iters=8, alpha=alpha, normalise=normalise, early_stop=True,
                    want_post=True)
    for u, v in zip(a, b):
        assert torch.equal(u, v)


def test_learned_dynamic_handout(ldpc, request):
    ldpc.set_grid_cap(1)
    request.addfinalizer(lambda: ldpc.set_grid_cap(0))
    shape = synth.wifi_n648_r12()
    rc, _, llr = _inputs(shape, 150, 1.5, frame0=77)
    w = _weights(rc, 8, 3)
    wh, wi, wp = rc.decode_learned_f32(llr, w, max_iters=8, early_stop=True)
    code = ldpc.Code(shape.hbm, shape.z)
    gh, gi, gp = code.decode_learned(torch.from_numpy(llr).cuda(), torch.from_numpy(w).cuda(),
                                     early_stop=True, want_post=True)
    assert (gi.cpu().numpy() == wi).all() and (gp.cpu().numpy() == wp).all()
    assert wi.min() < 4 and wi.max() == 8


@pytest.mark.parametrize("shape,T,ebn0", [(synth.wifi_n648_r12(), 4, 1.5),
                                          (synth.wifi_n1944_r56(), 3, 3.5)],
                         ids=["wifi648", "wifi1944"])
def test_learned_fallback_pipeline(ldpc, shape, T, ebn0):
    """Frames the learned decoder leaves with a nonzero syndrome are decoded
    again by int8 plain min-sum (20 iterations, (3m)>>2), exactly as the
    oracle does when it runs the same two steps."""
    frames = 301
    rc, _, llr = _inputs(shape, frames, ebn0)
    w = _weights(rc, T, 11, 0.6, 0.9)
    wh, wi, _ = rc.decode_learned_f32(llr, w, max_iters=T, early_stop=True, want_post=False)
    bits = oracle.unpack_hard(wh, rc.n)
    fail = np.array([rc.syndrome_weight(b) != 0 for b in bits])
    assert 0 < fail.sum() < frames
    q = oracle.quantize_i8(llr[fail], 4.0, 63)
    fh, fi, _, _ = rc.decode_layered_i8(q, 20, True, True, want_post=False)
    wh = wh.copy()
    wi = wi.copy()
    wh[fail] = fh
    wi[fail] = T + fi
    code = ldpc.Code(shape.hbm, shape.z)
    gh, gi, nfb = code.decode_learned_fallback(torch.from_numpy(llr).cuda(),
                                               torch.from_numpy(w).cuda(), 20)
    assert nfb == fail.sum()
    assert (gi.cpu().numpy() == wi).all()
    assert (gh.cpu().numpy().view(np.uint32) == wh).all()


def test_paired_frame_errors(ldpc):
    """2x2 table of paired frame outcomes against a host count from the
    unpacked hard decisions."""
    shape = synth.wifi_n648_r12()
    rc, info, llr = _inputs(shape, 2000, 1.6)
    code = ldpc.Code(shape.hbm, shape.z)
    x = torch.from_numpy(llr).cuda()
    ha, _, _ = code.decode(x, max_iters=3, early_stop=True)
    hb, _, _ = code.decode(x, max_iters=20, early_stop=True)
    cnt = code.paired_frame_errors(torch.from_numpy(info).cuda(), ha, hb).cpu().numpy()
    wa = (oracle.unpack_hard(ha.cpu().numpy().view(np.uint32), rc.n)[:, :rc.k] != info).any(1)
    wb = (oracle.unpack_hard(hb.cpu().numpy().view(np.uint32), rc.n)[:, :rc.k] != info).any(1)
    want = [(~wa & ~wb).sum(), (~wa & wb).sum(), (wa & ~wb).sum(), (wa & wb).sum()]
    assert cnt.tolist() == [int(v) for v in want]
    assert want[2] > 0 and want[3] > 0


# ------------------------------------------ past the weight table, give-up rule

@pytest.mark.parametrize("shape,T,ebn0,frames,stops", [
    (synth.wifi_n648_r12(), 8, 1.25, 401, ((4, 0.10), (10, 0.05))),
    (synth.wifi_n1944_r56(), 6, 3.0, 203, ((3, 0.12), (9, 0.04))),
    (synth.wimax_mixed_set()[-4], 8, 1.3, 37, ((5, 0.08), (0, 0.0))),
    (synth.wimax_mixed_set()[3 * 4 + 2], 6, 2.0, 120, ((2, 0.3), (7, 0.02)))],
    ids=["wifi648", "wifi1944", "wimax2304", "wimax36_r34"])
def test_learned_past_table_with_checkpoints_bit_exact(ldpc, shape, T, ebn0, frames, stops):
    """Iterations past the table repeat its last row; frames with too many
    unsatisfied checks at a checkpoint stop there: hard decisions, counts
    and posteriors equal the oracle's."""
    rc, _, llr = _inputs(shape, frames, ebn0, frame0=31)
    w = _weights(rc, T, 17, lo=0.5, hi=1.0)
    si = (stops[0][0], stops[1][0])
    sf = (stops[0][1], stops[1][1])
    wh, wi, wp = rc.decode_learned_f32(llr, w, max_iters=20, stop_iter=si, stop_frac=sf)
    code = ldpc.Code(shape.hbm, shape.z)
    gh, gi, gp = code.decode_learned(torch.from_numpy(llr).cuda(), torch.from_numpy(w).cuda(),
                                     early_stop=True, want_post=True, max_iters=20,
                                     stop_iter=si, stop_frac=sf)
    assert (gi.cpu().numpy() == wi).all()
    assert (gh.cpu().numpy().view(np.uint32) == wh).all()
    assert (gp.cpu().numpy() == wp).all()
    assert wi.max() > T   # some frames ran past the table


def test_learned_checkpoints_dynamic_handout(ldpc, request):
    ldpc.set_grid_cap(1)
    request.addfinalizer(lambda: ldpc.set_grid_cap(0))
    shape = synth.wifi_n648_r12()
    rc, _, llr = _inputs(shape, 160, 1.2, frame0=5)
    w = _weights(rc, 5, 3, lo=0.6, hi=0.95)
    wh, wi, _ = rc.decode_learned_f32(llr, w, max_iters=16, stop_iter=(3, 8),
                                      stop_frac=(0.1, 0.04), want_post=False)
    code = ldpc.Code(shape.hbm, shape.z)
    gh, gi, _ = code.decode_learned(torch.from_numpy(llr).cuda(), torch.from_numpy(w).cuda(),
                                    max_iters=16, stop_iter=(3, 8), stop_frac=(0.1, 0.04))
    assert (gi.cpu().numpy() == wi).all() and (gh.cpu().numpy().view(np.uint32) == wh).all()
    assert len(set(wi.tolist())) > 3


def test_learned_ex_argument_checks(ldpc):
    shape = synth.wifi_n648_r12()
    code = ldpc.Code(shape.hbm, shape.z)
    x = torch.zeros((4, code.n), dtype=torch.float32, device="cuda")
    w = torch.full((3, code.nnz_blocks), 0.75, dtype=torch.float32, device="cuda")
    with pytest.raises(ldpc.LdpcError):   # a checkpoint without early stop
        code.decode_learned(x, w, early_stop=False, max_iters=5, stop_iter=(2, 0),
                            stop_frac=(0.1, 0.0))
    with pytest.raises(ldpc.LdpcError):   # negative limit
        code.decode_learned(x, w, max_iters=5, stop_iter=(2, 0), stop_frac=(-0.1, 0.0))
    with pytest.raises(ldpc.LdpcError):
        code.decode_learned(x, w, max_iters=1001)
