"""Parity of the CUDA library with the CPU oracle, element by element on the
same seeded inputs (bit-exact for every integer output and, because both
sides round every FP32 operation the same way and never contract a
multiply-add, bit-exact for FP32 posteriors too)."""
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


def pack_i8(q: np.ndarray, clip: int = 63) -> np.ndarray:
    """int8[F][N] -> uint32[ceil(F/4)][N], byte b = frame 4g + b, pad +clip."""
    F, n = q.shape
    G = (F + 3) // 4
    pad = np.full((4 * G, n), clip, dtype=np.int8)
    pad[:F] = q
    b = pad.reshape(G, 4, n).astype(np.uint8).astype(np.uint32)
    return b[:, 0] | (b[:, 1] << 8) | (b[:, 2] << 16) | (b[:, 3] << 24)


def to_np(t):
    return t.detach().cpu().numpy()


SHAPES = {
    "wifi648": synth.wifi_n648_r12(),
    "wifi1944": synth.wifi_n1944_r56(),
    "eq7": synth.eq7_wimax_r34(),
    "z2": synth.tiny_z2_code(),
    "z3": synth.tiny_z3_code(),
    "rand_z1": synth.random_small_code(11, 4, 7, 1),
    "rand_z33": synth.random_small_code(12, 5, 12, 33),
    "rand_z65": synth.random_small_code(13, 6, 16, 65),
}
_mixed = synth.wimax_mixed_set()
SHAPES.update({"wimax96_r12": _mixed[-4], "wimax52_r23": _mixed[7 * 4 + 1],
               "wimax24_r56": _mixed[3]})


def oracle_inputs(shape, frames, frame0=0, ebn0=2.0, seed=1):
    rc = oracle.RefCode(shape.hbm, shape.z)
    info = oracle.gen_info(seed, frame0, frames, rc.k)
    cw = rc.encode(info)
    sigma = synth.ebn0_db_to_sigma(ebn0, rc.k / rc.n)
    llr = oracle.awgn_llr(cw, frame0, seed, sigma)
    return rc, info, cw, llr, sigma


# ---------------------------------------------------------------- generators

@pytest.mark.parametrize("k,frame0,frames", [(324, 0, 9), (1620, 77, 5), (1000, 2 ** 33, 3)])
def test_gen_info_bit_exact(ldpc, k, frame0, frames):
    got = to_np(ldpc.gen_info(1, frame0, frames, k))
    assert (got == oracle.gen_info(1, frame0, frames, k)).all()


@pytest.mark.parametrize("name", sorted(SHAPES))
def test_encode_bit_exact(ldpc, name):
    s = SHAPES[name]
    rc = oracle.RefCode(s.hbm, s.z)
    info = oracle.gen_info(3, 0, 37, rc.k)
    code = ldpc.Code(s.hbm, s.z)
    got = to_np(code.encode(torch.from_numpy(info).cuda()))
    assert (got == rc.encode(info)).all()


@pytest.mark.parametrize("n,frame0", [(648, 0), (1944, 12345), (1001, 5)])
def test_awgn_bit_exact(ldpc, n, frame0):
    rng = np.random.default_rng(n)
    cw = rng.integers(0, 2, size=(6, n), dtype=np.uint8)
    sigma = synth.ebn0_db_to_sigma(2.5, 0.5)
    want = oracle.awgn_llr(cw, frame0, 1, sigma)
    got = to_np(ldpc.awgn_llr(torch.from_numpy(cw).cuda(), frame0, 1, sigma))
    assert got.view(np.uint32).tolist() == want.view(np.uint32).tolist()


@pytest.mark.parametrize("frames", [1, 5, 8, 1001])
def test_quantize_pack_bit_exact(ldpc, frames):
    rng = np.random.default_rng(frames)
    llr = (rng.standard_normal((frames, 648)) * 12).astype(np.float32)
    llr[0, :6] = [0.125, 0.375, -0.125, -0.375, 100.0, -100.0]   # ties and clips
    want = pack_i8(oracle.quantize_i8(llr, 4.0, 63), 63)
    got = to_np(ldpc.quantize_pack_i8(torch.from_numpy(llr).cuda(), 4.0, 63)).view(np.uint32)
    assert (got == want).all()


# ---------------------------------------------------------------- decoders

def _decode_both(ldpc, shape, llr, dtype, max_iters, early_stop, normalise=True, alpha=0.75):
    rc = oracle.RefCode(shape.hbm, shape.z)
    code = ldpc.Code(shape.hbm, shape.z)
    F = llr.shape[0]
    if dtype == "f32":
        wh, wi, wp = rc.decode_layered_f32(llr, max_iters, alpha, normalise, early_stop)
        gh, gi, gp = code.decode(torch.from_numpy(llr).cuda(), dtype=ldpc.F32,
                                 max_iters=max_iters, alpha=alpha, normalise=normalise,
                                 early_stop=early_stop, want_post=True)
    else:
        q = oracle.quantize_i8(llr, 4.0, 63)
        wh, wi, wp, _ = rc.decode_layered_i8(q, max_iters, normalise, early_stop)
        words = torch.from_numpy(pack_i8(q).view(np.int32)).cuda()
        gh, gi, gp = code.decode(words, frames=F, dtype=ldpc.I8X4, max_iters=max_iters,
                                 normalise=normalise, early_stop=early_stop, want_post=True)
    code.sync()
    return (wh, wi, wp), (to_np(gh).view(np.uint32), to_np(gi), to_np(gp))


def _assert_same(want, got):
    wh, wi, wp = want
    gh, gi, gp = got
    assert (gi == wi).all(), np.nonzero(gi != wi)[0][:10]
    assert (gh == wh).all()
    assert (gp == wp).all()        # == treats +0 and -0 as equal


@pytest.mark.parametrize("dtype", ["f32", "i8"])
def test_decode_wifi648_fixed_10(ldpc, dtype):
    """The N=648 R=1/2 workload: 1000 frames at 2 dB, fixed 10 iterations."""
    s = SHAPES["wifi648"]
    _, _, _, llr, _ = oracle_inputs(s, 1000)
    _assert_same(*_decode_both(ldpc, s, llr, dtype, 10, False))


@pytest.mark.parametrize("dtype", ["f32", "i8"])
@pytest.mark.parametrize("ebn0", [3.5, 4.5])
def test_decode_wifi1944_early_stop(ldpc, dtype, ebn0):
    """N=1944 R=5/6, max 20 iterations with syndrome stop, ragged frame count."""
    s = SHAPES["wifi1944"]
    _, _, _, llr, _ = oracle_inputs(s, 1023, frame0=4096, ebn0=ebn0)
    want, got = _decode_both(ldpc, s, llr, dtype, 20, True)
    _assert_same(want, got)
    assert len(np.unique(want[1])) > 2     # frames stopped at different iterations


@pytest.mark.parametrize("name", ["z2", "z3", "rand_z1", "rand_z33", "rand_z65", "eq7",
                                  "wimax96_r12", "wimax52_r23", "wimax24_r56"])
@pytest.mark.parametrize("dtype", ["f32", "i8"])
def test_decode_shapes(ldpc, name, dtype):
    s = SHAPES[name]
    _, _, _, llr, _ = oracle_inputs(s, 13, ebn0=1.5)
    _assert_same(*_decode_both(ldpc, s, llr, dtype, 12, True))


@pytest.mark.parametrize("name", ["wifi648", "wifi1944", "wimax24_r56"])
@pytest.mark.parametrize("normalise", [True, False])
def test_i8_extreme_values(ldpc, name, normalise):
    """Raw int8 channel values heavy in 0, +-1 and +-127: exact zeros of
    Z_mn (whose sign the message rule never needs) and saturation on both
    sides, bit-exact against the oracle."""
    s = SHAPES[name]
    rc = oracle.RefCode(s.hbm, s.z)
    rng = np.random.default_rng(7)
    F = 61
    pick = rng.random((F, rc.n))
    q = rng.integers(-127, 128, (F, rc.n)).astype(np.int8)
    q[pick < 0.3] = 0
    q[(pick >= 0.3) & (pick < 0.4)] = 1
    q[(pick >= 0.4) & (pick < 0.5)] = -1
    q[(pick >= 0.5) & (pick < 0.6)] = 127
    q[(pick >= 0.6) & (pick < 0.7)] = -127
    wh, wi, wp, _ = rc.decode_layered_i8(q, 15, normalise, True)
    code = ldpc.Code(s.hbm, s.z)
    words = torch.from_numpy(pack_i8(q).view(np.int32)).cuda()
    gh, gi, gp = code.decode(words, frames=F, dtype=ldpc.I8X4, max_iters=15,
                             normalise=normalise, early_stop=True, want_post=True)
    code.sync()
    _assert_same((wh, wi, wp), (to_np(gh).view(np.uint32), to_np(gi), to_np(gp)))


@pytest.mark.parametrize("dtype", ["f32", "i8"])
def test_decode_plain_minsum(ldpc, dtype):
    s = SHAPES["wifi648"]
    _, _, _, llr, _ = oracle_inputs(s, 64, ebn0=2.5)
    _assert_same(*_decode_both(ldpc, s, llr, dtype, 8, True, normalise=False))


def test_worked_example_on_gpu(ldpc, golden_z2):
    s = SHAPES["z2"]
    code = ldpc.Code(s.hbm, s.z)
    llr = torch.tensor([golden_z2["llr"]], dtype=torch.float32, device="cuda")
    _, it, post = code.decode(llr, max_iters=1, normalise=False, want_post=True)
    assert to_np(post)[0].tolist() == golden_z2["alpha1_after_layer2"]
    _, _, post = code.decode(llr, max_iters=1, alpha=0.75, normalise=True, want_post=True)
    assert to_np(post)[0].tolist() == golden_z2["alpha075_after_layer2"]
    q = np.array([golden_z2["int8_llr"]], dtype=np.int8)
    words = torch.from_numpy(pack_i8(q).view(np.int32)).cuda()
    _, _, post = code.decode(words, frames=1, dtype=ldpc.I8X4, max_iters=1, want_post=True)
    assert to_np(post)[0].tolist() == golden_z2["int8_after_layer2"]


@pytest.mark.parametrize("dtype", ["f32", "i8"])
def test_unaligned_input_uses_plain_loads(ldpc, dtype):
    """A channel buffer that is not 16-byte aligned takes the plain-load
    path instead of the bulk copy; results must not change."""
    s = SHAPES["wifi648"]
    rc, _, _, llr, _ = oracle_inputs(s, 9)
    code = ldpc.Code(s.hbm, s.z)
    if dtype == "f32":
        buf = torch.empty(llr.size + 1, dtype=torch.float32, device="cuda")
        view = buf[1:].view(llr.shape)
        view.copy_(torch.from_numpy(llr))
        gh, gi, gp = code.decode(view, max_iters=10, early_stop=True, want_post=True)
        wh, wi, wp = rc.decode_layered_f32(llr, 10, 0.75, True, True)
    else:
        q = oracle.quantize_i8(llr)
        w = pack_i8(q).view(np.int32)
        buf = torch.empty(w.size + 1, dtype=torch.int32, device="cuda")
        view = buf[1:].view(w.shape)
        view.copy_(torch.from_numpy(w))
        gh, gi, gp = code.decode(view, frames=9, dtype=ldpc.I8X4, max_iters=10,
                                 early_stop=True, want_post=True)
        wh, wi, wp, _ = rc.decode_layered_i8(q, 10, True, True)
    _assert_same((wh, wi, wp), (to_np(gh).view(np.uint32), to_np(gi), to_np(gp)))


def test_zero_frames_is_noop(ldpc):
    s = SHAPES["wifi648"]
    code = ldpc.Code(s.hbm, s.z)
    llr = torch.zeros((0, s.n), dtype=torch.float32, device="cuda")
    h, i, _ = code.decode(llr)
    assert h.shape[0] == 0 and i.shape[0] == 0


@pytest.mark.parametrize("frames", [1, 2, 3, 6, 7])
def test_i8_partial_groups(ldpc, frames):
    """Frame counts that leave pad lanes in the last packed word."""
    s = SHAPES["wifi1944"]
    _, _, _, llr, _ = oracle_inputs(s, frames, ebn0=3.5)
    _assert_same(*_decode_both(ldpc, s, llr, "i8", 20, True))


@pytest.mark.parametrize("dtype", ["f32", "i8"])
@pytest.mark.parametrize("shape_name,frames", [("wifi648", 301), ("wifi1944", 150)])
def test_dynamic_frame_handout(ldpc, request, dtype, shape_name, frames):
    """One block (one warp) decodes every frame: finished frames
    are replaced through the work counter (per byte lane for int8), at low
    Eb/N0 so iteration counts vary widely."""
    ldpc.set_grid_cap(1)
    request.addfinalizer(lambda: ldpc.set_grid_cap(0))
    s = SHAPES[shape_name]
    ebn0 = {"wifi648": 1.5, "wifi1944": 3.5}[shape_name]
    _, _, _, llr, _ = oracle_inputs(s, frames, frame0=999, ebn0=ebn0)
    want, got = _decode_both(ldpc, s, llr, dtype, 15, True)
    _assert_same(want, got)
    assert want[1].min() < 5 and want[1].max() == 15


# ------------------------------------------------------- full-size sampled parity

@pytest.mark.parametrize("dtype", ["i8", "f32"])
def test_full_size_wifi1944_sampled(ldpc, dtype):
    """The benchmark's step: the three 262,144-frame N=1944 batches (3.5, 4.0,
    4.5 dB), generated on the GPU and decoded back to back by one call, as the
    benchmark times them; a sample of frames from every batch (its first and
    last frames among them) is regenerated and decoded independently by the
    oracle and must match bit for bit (channel LLRs, hard decisions,
    iteration counts)."""
    from paper_2306_12063_gb300.workload import make_batch
    s = SHAPES["wifi1944"]
    code = ldpc.Code(s.hbm, s.z)
    F = 262144
    ebn0 = (3.5, 4.0, 4.5)
    batches = [make_batch(code, F, b * F, eb, keep_cw=False) for b, eb in enumerate(ebn0)]
    if dtype == "i8":
        x = torch.cat([b.q for b in batches])
        hard, iters, _ = code.decode(x, frames=3 * F, dtype=ldpc.I8X4, max_iters=20,
                                     early_stop=True)
    else:
        x = torch.cat([b.llr for b in batches])
        hard, iters, _ = code.decode(x, dtype=ldpc.F32, max_iters=20, early_stop=True)
    del x
    code.sync()
    rng = np.random.default_rng(99)
    rc = oracle.RefCode(s.hbm, s.z)
    h_np, i_np = to_np(hard).view(np.uint32), to_np(iters)
    for bi, (b, eb) in enumerate(zip(batches, ebn0)):
        sample = np.unique(np.concatenate([[0, 1, 2, 3, F - 1], rng.integers(0, F, 14)]))
        sig = synth.ebn0_db_to_sigma(eb, rc.k / rc.n)
        llr_gpu = to_np(b.llr[torch.from_numpy(sample).cuda()])
        for row, f in enumerate(sample):
            g = bi * F + int(f)   # frame identity and its row in the step's outputs
            info = oracle.gen_info(1, g, 1, rc.k)
            cw = rc.encode(info)
            llr = oracle.awgn_llr(cw, g, 1, sig)
            assert (llr.view(np.uint32) == llr_gpu[row].view(np.uint32)).all()
            if dtype == "i8":
                wh, wi, _, _ = rc.decode_layered_i8(oracle.quantize_i8(llr), 20, True, True,
                                                    want_post=False)
            else:
                wh, wi, _ = rc.decode_layered_f32(llr, 20, 0.75, True, True, want_post=False)
            assert i_np[g] == wi[0], (g, i_np[g], wi[0])
            assert (h_np[g] == wh[0]).all()
    # properties that hold at any size
    assert i_np.min() >= 1 and i_np.max() <= 20
    info_all = torch.cat([b.info for b in batches])
    stats = to_np(code.frame_stats(info_all, hard, iters, 20))
    assert stats[3] == i_np.sum()
    assert stats[4:].sum() == 3 * F


def test_frame_stats_match_numpy(ldpc):
    s = SHAPES["wifi648"]
    rc, info, cw, llr, _ = oracle_inputs(s, 200, ebn0=1.0)
    code = ldpc.Code(s.hbm, s.z)
    wh, wi, _ = rc.decode_layered_f32(llr, 6, 0.75, True, True, want_post=False)
    bits = oracle.unpack_hard(wh, rc.n)
    errs = (bits[:, :rc.k] != info).sum(axis=1)
    syn0 = np.array([rc.syndrome_weight(b) == 0 for b in bits])
    got = to_np(code.frame_stats(torch.from_numpy(info).cuda(),
                                 torch.from_numpy(wh.view(np.int32)).cuda(),
                                 torch.from_numpy(wi).cuda(), 6))
    assert got[0] == errs.sum() and got[1] == (errs > 0).sum()
    assert got[2] == ((errs > 0) & syn0).sum()
    assert got[3] == wi.sum()
    assert (got[4:] == np.bincount(wi, minlength=7)).all()


@pytest.mark.parametrize("dtype", ["f32", "i8"])
@pytest.mark.parametrize("frames,chunk", [(1000, 128), (30, 128), (33, 128), (96, 128),
                                          (97, 128), (151, 128), (17, 4)])
def test_decode_host_pipeline(ldpc, dtype, frames, chunk):
    """End-to-end entry point on pinned host buffers equals the device call,
    with batches shorter than, equal to and just past the quarter-size first
    chunk, ragged last chunks and the smallest chunk."""
    s = SHAPES["wifi1944"]
    _, _, _, llr, _ = oracle_inputs(s, frames, ebn0=4.0)
    code = ldpc.Code(s.hbm, s.z)
    F = llr.shape[0]
    if dtype == "f32":
        src = torch.from_numpy(llr).pin_memory()
        dev = src.cuda()
        dt = ldpc.F32
    else:
        src = torch.from_numpy(pack_i8(oracle.quantize_i8(llr)).view(np.int32)).pin_memory()
        dev = src.cuda()
        dt = ldpc.I8X4
    h_hard = torch.empty((F, code.nwords), dtype=torch.int32).pin_memory()
    h_iters = torch.empty((F,), dtype=torch.int32).pin_memory()
    ws = torch.empty(code.host_workspace_bytes(dt, chunk), dtype=torch.uint8, device="cuda")
    code.decode_host(src, F, dt, h_hard, h_iters, ws, chunk, max_iters=20, early_stop=True)
    torch.cuda.synchronize()
    gh, gi, _ = code.decode(dev, frames=F, dtype=dt, max_iters=20, early_stop=True)
    assert (to_np(gi) == h_iters.numpy()).all()
    assert (to_np(gh) == h_hard.numpy()).all()
