"""The paper's variants on the GPU against the oracle, bit for bit: Section 5's
int16 wrap-around decoder and its quantiser, Section 3's bitmap encoder
(Alg. A1) and the flooding schedule (eq. 18-21)."""
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


def _llr(shape, frames, ebn0, seed=1):
    rc = oracle.RefCode(shape.hbm, shape.z)
    info = oracle.gen_info(seed, 0, frames, rc.k)
    cw = rc.encode(info)
    return rc, info, cw, oracle.awgn_llr(cw, 0, seed, synth.ebn0_db_to_sigma(ebn0, rc.k / rc.n))


def _pack(bits):
    bits = np.ascontiguousarray(bits, dtype=np.uint8)
    F, n = bits.shape
    return np.packbits(bits.reshape(F, n // 8, 8), axis=2, bitorder="little") \
             .reshape(F, n // 8).view(np.uint32)


def test_quantize_i16(ldpc):
    rng = np.random.default_rng(0)
    x = (rng.standard_normal(50000) * 40).astype(np.float32)
    x[:6] = [0.5 / 16, 1.5 / 16, -2.5 / 16, 1e9, -1e9, 0.0]
    for scale, qb in ((16.0, 10), (4.0, 8), (1.0, 14)):
        got = ldpc.quantize_i16(torch.from_numpy(x).cuda(), scale, qb).cpu().numpy()
        assert (got == oracle.quantize_i16(x, scale, qb)).all()


I16_CASES = [(synth.wifi_n648_r12(), 1.5, 10, False, True),
             (synth.wifi_n648_r12(), 2.5, 10, True, False),
             (synth.wifi_n1944_r56(), 3.5, 20, False, True),
             (synth.wimax_n2304_r56(), 3.0, 12, True, True),
             (synth.random_small_code(5, 7, 17, 45), 1.0, 15, False, True)]


@pytest.mark.parametrize("shape,ebn0,iters,norm,es", I16_CASES,
                         ids=["wifi648", "wifi648_norm", "wifi1944", "wimax2304_norm", "rand_z45"])
def test_int16_wrap_decoder_bit_exact(ldpc, shape, ebn0, iters, norm, es):
    rc, _, _, llr = _llr(shape, 129, ebn0)
    q = oracle.quantize_i16(llr, 16.0, 10)
    wh, wi, wp, _ = rc.decode_layered_i16w(q, iters, normalise=norm, early_stop=es)
    code = ldpc.Code(shape.hbm, shape.z)
    gh, gi, gp = code.decode(torch.from_numpy(q).cuda(), dtype=ldpc.I16W, max_iters=iters,
                             normalise=norm, early_stop=es, want_post=True)
    assert (gi.cpu().numpy() == wi).all()
    assert (gh.cpu().numpy().view(np.uint32) == wh).all()
    assert (gp.cpu().numpy() == wp).all()


def test_int16_one_frame_kernel_on_a_code_too_large_to_pack(ldpc):
    """A code whose packed two-frame row state (five words per check row)
    exceeds the device's shared memory per block runs the one-frame-per-warp
    int16 kernel (three words per row): mb = 31, nb = 32, Z = 384, the largest
    shape the library takes.  Bit-exact against the oracle like the packed
    kernel."""
    shape = synth.random_small_code(9, 31, 32, 384)
    n, m = 32 * 384, 31 * 384
    limit = torch.cuda.get_device_properties(0).shared_memory_per_block_optin
    assert 4 * (n + 32 + 5 * m) > limit >= 4 * (n + 32 + 3 * m)
    rc, _, _, llr = _llr(shape, 9, 14.0)   # rate 1/32: frames stop after 2-5 iterations
    q = oracle.quantize_i16(llr, 16.0, 10)
    for es in (True, False):
        wh, wi, wp, _ = rc.decode_layered_i16w(q, 6, normalise=True, early_stop=es)
        code = ldpc.Code(shape.hbm, shape.z)
        gh, gi, gp = code.decode(torch.from_numpy(q).cuda(), dtype=ldpc.I16W, max_iters=6,
                                 normalise=True, early_stop=es, want_post=True)
        assert (gi.cpu().numpy() == wi).all()
        assert (gh.cpu().numpy().view(np.uint32) == wh).all()
        assert (gp.cpu().numpy() == wp).all()


@pytest.mark.parametrize("shape,frames", [(synth.wifi_n648_r12(), 151),
                                          (synth.wifi_n1944_r56(), 77)])
def test_int16_lane_refills(ldpc, request, shape, frames):
    """Two frames per word, each 16-bit lane refilled on its own as its frame
    stops: one block decodes every frame, at low Eb/N0 so the iteration
    counts vary widely."""
    ldpc.set_grid_cap(1)
    request.addfinalizer(lambda: ldpc.set_grid_cap(0))
    rc, _, _, llr = _llr(shape, frames, 1.5 if shape.mb > 4 else 3.0)
    q = oracle.quantize_i16(llr, 16.0, 10)
    wh, wi, wp, _ = rc.decode_layered_i16w(q, 15, normalise=True, early_stop=True)
    code = ldpc.Code(shape.hbm, shape.z)
    gh, gi, gp = code.decode(torch.from_numpy(q).cuda(), dtype=ldpc.I16W, max_iters=15,
                             normalise=True, early_stop=True, want_post=True)
    assert (gi.cpu().numpy() == wi).all()
    assert (gh.cpu().numpy().view(np.uint32) == wh).all()
    assert (gp.cpu().numpy() == wp).all()
    assert len(set(wi.tolist())) > 5 and wi.max() == 15


def test_int16_wrap_overflow_cases(ldpc):
    """Inputs far beyond Q_B (up to the int16 limits): many wraps, including
    |-32768|; the GPU follows the oracle through every one."""
    from tests.conftest import load_golden
    g = load_golden("z2_int16_wrap.txt")
    sh = synth.tiny_z2_code()
    code = ldpc.Code(sh.hbm, sh.z)
    for key, want in (("llr", "after_iter1"), ("llr_b", "after_iter1_b")):
        x = torch.tensor([int(v) for v in g[key]], dtype=torch.int16).cuda()[None]
        _, _, post = code.decode(x, dtype=ldpc.I16W, max_iters=1, normalise=False,
                                 want_post=True)
        assert post[0].tolist() == [int(v) for v in g[want]]
    rng = np.random.default_rng(3)
    for shape in (synth.wifi_n648_r12(), synth.tiny_z3_code()):
        rc = oracle.RefCode(shape.hbm, shape.z)
        q = rng.integers(-32768, 32768, (64, rc.n)).astype(np.int16)
        q[0, :] = -32768
        q[1, ::3] = 32767
        for norm in (False, True):
            wh, wi, wp, ev = rc.decode_layered_i16w(q, 7, normalise=norm, early_stop=True)
            assert ev > 0
            c = ldpc.Code(shape.hbm, shape.z)
            gh, gi, gp = c.decode(torch.from_numpy(q).cuda(), dtype=ldpc.I16W, max_iters=7,
                                  normalise=norm, early_stop=True, want_post=True)
            assert (gi.cpu().numpy() == wi).all()
            assert (gh.cpu().numpy().view(np.uint32) == wh).all()
            assert (gp.cpu().numpy() == wp).all()


@pytest.mark.parametrize("z", [32, 64, 96])
def test_bitmap_encoder(ldpc, z):
    for sh in [s for s in synth.wimax_mixed_set() if s.z == z]:
        rc = oracle.RefCode(sh.hbm, sh.z)
        info = oracle.gen_info(4, 0, 301, rc.k)
        words = _pack(info)
        want = rc.encode_bitmap(words)
        code = ldpc.Code(sh.hbm, sh.z)
        got = code.encode_bitmap(torch.from_numpy(words.view(np.int32)).cuda())
        assert (got.cpu().numpy().view(np.uint32) == want).all()
        byte_cw = code.encode(torch.from_numpy(info).cuda()).cpu().numpy()
        assert (_pack(byte_cw) == want).all()


def test_bitmap_encoder_rejects_other_z(ldpc):
    sh = synth.wimax_mixed_set()[0]
    code = ldpc.Code(sh.hbm, sh.z)
    with pytest.raises(ldpc.LdpcError):
        code.encode_bitmap(torch.zeros((2, 9), dtype=torch.int32, device="cuda"))


@pytest.mark.parametrize("shape,ebn0,iters,norm,es",
                         [(synth.wifi_n648_r12(), 2.0, 10, True, False),
                          (synth.wifi_n648_r12(), 1.5, 20, False, True),
                          (synth.wifi_n1944_r56(), 4.0, 20, True, True),
                          (synth.tiny_z3_code(), 1.0, 8, True, True),
                          (synth.random_small_code(6, 5, 14, 41), 1.5, 12, False, False)],
                         ids=["wifi648", "wifi648_plain", "wifi1944", "tiny_z3", "rand_z41"])
def test_flooding_bit_exact(ldpc, shape, ebn0, iters, norm, es):
    rc, _, _, llr = _llr(shape, 97, ebn0)
    wh, wi, wp = rc.decode_flooding_f32(llr, iters, 0.75, norm, es)
    code = ldpc.Code(shape.hbm, shape.z)
    gh, gi, gp = code.decode_flooding(torch.from_numpy(llr).cuda(), iters, 0.75, norm, es,
                                      want_post=True)
    assert (gi.cpu().numpy() == wi).all()
    assert (gh.cpu().numpy().view(np.uint32) == wh).all()
    assert (gp.cpu().numpy() == wp).all()
