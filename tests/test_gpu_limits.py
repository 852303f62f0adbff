"""Edge cases on the GPU: the largest code shapes the kernels take (Z = 384,
a row of degree 27, slot class 27), codes whose shared-memory needs exceed
the device and must be refused cleanly, empty batches on every entry point,
and the failure path of the bounded waits (a wait that runs out is reported
by ldpc_sync and leaves the context usable)."""
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


def _max_code():
    """mb = 3, nb = 28, Z = 384: row 0 has all 25 info blocks, h_b and the
    first dual-diagonal block (degree 27, the largest the decoders take)."""
    rng = np.random.default_rng(11)
    mb, nb, z = 3, 28, 384
    kb = nb - mb
    h = -np.ones((mb, nb), dtype=np.int16)
    h[0, :kb] = rng.integers(0, z, kb)
    for i in (1, 2):
        cols = rng.choice(kb, 9, replace=False)
        h[i, cols] = rng.integers(0, z, 9)
    h[0, kb], h[1, kb], h[2, kb] = 5, 0, 5
    for t in range(mb - 1):
        h[t, kb + 1 + t] = 0
        h[t + 1, kb + 1 + t] = 0
    assert (h[0] >= 0).sum() == 27
    return synth.CodeShape("max_z384_deg27", h, z)


def test_largest_code_bit_exact(ldpc):
    shape = _max_code()
    rc = oracle.RefCode(shape.hbm, shape.z)
    assert rc.max_row_deg == 27
    info = oracle.gen_info(3, 0, 6, rc.k)
    cw = rc.encode(info)
    llr = oracle.awgn_llr(cw, 0, 3, synth.ebn0_db_to_sigma(2.5, rc.k / rc.n))
    code = ldpc.Code(shape.hbm, shape.z)
    assert code.max_row_deg == 27
    assert (code.encode(torch.from_numpy(info).cuda()).cpu().numpy() == cw).all()
    x = torch.from_numpy(llr).cuda()
    wh, wi, wp = rc.decode_layered_f32(llr, 12, 0.75, True, True)
    gh, gi, gp = code.decode(x, max_iters=12, early_stop=True, want_post=True)
    assert (gi.cpu().numpy() == wi).all() and (gp.cpu().numpy() == wp).all()
    assert (gh.cpu().numpy().view(np.uint32) == wh).all()
    q8 = oracle.quantize_i8(llr)
    wh, wi, wp, _ = rc.decode_layered_i8(q8, 12, True, True)
    gh, gi, gp = code.decode(ldpc.quantize_pack_i8(x), frames=6, dtype=ldpc.I8X4, max_iters=12,
                             early_stop=True, want_post=True)
    assert (gi.cpu().numpy() == wi).all() and (gp.cpu().numpy() == wp).all()
    q16 = oracle.quantize_i16(llr, 16.0, 10)
    wh, wi, wp, _ = rc.decode_layered_i16w(q16, 12, normalise=True, early_stop=True)
    gh, gi, gp = code.decode(torch.from_numpy(q16).cuda(), dtype=ldpc.I16W, max_iters=12,
                             normalise=True, early_stop=True, want_post=True)
    assert (gi.cpu().numpy() == wi).all() and (gp.cpu().numpy() == wp).all()
    w = np.random.default_rng(1).uniform(0.5, 1.0, (5, rc.nnz_blocks)).astype(np.float32)
    wh, wi, wp = rc.decode_learned_f32(llr, w, max_iters=5, early_stop=True)
    gh, gi, gp = code.decode_learned(x, torch.from_numpy(w).cuda(), early_stop=True,
                                     want_post=True)
    assert (gi.cpu().numpy() == wi).all() and (gp.cpu().numpy() == wp).all()


def test_oversized_shared_memory_is_refused(ldpc):
    """The flooding decoder and the training backward keep per-edge arrays in
    shared memory: on the largest code they do not fit and must return
    LDPC_ERR_UNSUPPORTED without launching."""
    shape = _max_code()
    code = ldpc.Code(shape.hbm, shape.z)
    x = torch.zeros((2, code.n), dtype=torch.float32, device="cuda")
    with pytest.raises(ldpc.LdpcError) as e:
        code.decode_flooding(x, 5)
    assert e.value.status == 6
    b = torch.zeros((2, code.n), dtype=torch.uint8, device="cuda")
    w = torch.full((3, code.nnz_blocks), 0.75, device="cuda")
    post, rows, _, _ = code.train_forward(x, b, w)
    with pytest.raises(ldpc.LdpcError) as e:
        code.train_backward(x, b, w, post, rows)
    assert e.value.status == 6
    code.sync()   # nothing was left running


def test_empty_batches(ldpc):
    shape = synth.wifi_n648_r12()
    code = ldpc.Code(shape.hbm, shape.z)
    x = torch.zeros((0, code.n), dtype=torch.float32, device="cuda")
    h, i, _ = code.decode(x, max_iters=5)
    assert h.shape[0] == 0 and i.shape[0] == 0
    h, i, _ = code.decode(torch.zeros((0, code.n), dtype=torch.int32, device="cuda"),
                          frames=0, dtype=ldpc.I8X4)
    h, i, _ = code.decode(torch.zeros((0, code.n), dtype=torch.int16, device="cuda"),
                          dtype=ldpc.I16W)
    h, i, _ = code.decode_flooding(x, 3)
    h, i, _ = code.decode_learned(x, torch.full((4, code.nnz_blocks), 0.8, device="cuda"))
    assert code.encode(torch.zeros((0, code.k), dtype=torch.uint8, device="cuda")).shape[0] == 0
    cs = ldpc.CodeSet([code])
    plan = ldpc.MixedPlan(cs, np.zeros(0, dtype=np.int32))
    hh, ii = plan.empty_outputs()
    plan.decode(torch.zeros(1, device="cuda"), ldpc.F32, out=(hh, ii, None))
    code.sync()


def test_bounded_wait_runs_out_and_is_reported(ldpc):
    """A wait whose bytes never arrive gives up after its poll limit, the
    kernel records it in the status word, ldpc_sync returns LDPC_ERR_TIMEOUT
    once (and clears it), and later work on the same context is correct."""
    shape = synth.wifi_n648_r12()
    rc = oracle.RefCode(shape.hbm, shape.z)
    code = ldpc.Code(shape.hbm, shape.z)
    code.check_bounded_wait(2048)
    with pytest.raises(ldpc.LdpcError) as e:
        code.sync(timeout_s=30.0)
    assert e.value.status == 5 and "wait" in str(e.value)
    code.sync()   # cleared
    info = oracle.gen_info(1, 0, 40, rc.k)
    llr = oracle.awgn_llr(rc.encode(info), 0, 1, synth.ebn0_db_to_sigma(2.0, 0.5))
    wh, wi, _ = rc.decode_layered_f32(llr, 10, 0.75, True, True, want_post=False)
    gh, gi, _ = code.decode(torch.from_numpy(llr).cuda(), max_iters=10, early_stop=True)
    code.sync()
    assert (gi.cpu().numpy() == wi).all()
    assert (gh.cpu().numpy().view(np.uint32) == wh).all()


def test_saturation_count_needs_the_debug_build(ldpc):
    """The release build keeps the int8 decoder free of counting work."""
    shape = synth.wifi_n648_r12()
    code = ldpc.Code(shape.hbm, shape.z)
    with pytest.raises(ldpc.LdpcError) as ei:
        code.saturation_count()
    assert ei.value.status == 6
