"""Mixed-code batches (one persistent launch per launch group) against the
oracle, frame by frame: every frame decoded by the mixed FP32 and int8
kernels must equal the oracle's decode of that frame with its own code
(hard decisions, iteration counts, posteriors), whatever the interleaving
of codes, the work-item sizes the autotuner picks, or the graph replay."""
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


def _shapes():
    full = synth.wimax_mixed_set()
    # rates 1/2 .. 5/6 at small, middle and the largest Z, plus the two Wi-Fi codes
    pick = [full[i] for i in (0, 1, 2, 3, 36, 37, 38, 39, 72, 73, 74, 75)]
    return pick + [synth.wifi_n648_r12(), synth.wifi_n1944_r56()]


def _setup(ldpc, shapes, frames, seed, ebn0=(1.5, 4.5)):
    """GPU batch of the plan, checked bit for bit against the same frames
    generated by the oracle; the oracle's own frames (info, LLRs in the
    plan's layout) are what the oracle decodes below."""
    from paper_2306_12063_gb300.workload import make_mixed_batch
    codes = [ldpc.Code(s.hbm, s.z) for s in shapes]
    cs = ldpc.CodeSet(codes)
    rng = np.random.default_rng(seed)
    cof = rng.integers(0, len(shapes), frames).astype(np.int32)
    plan = ldpc.MixedPlan(cs, cof)
    batch = make_mixed_batch(plan, ebn0)
    info, llr = oracle.mixed_frames(shapes, cof, ebn0)
    ref_llr = np.concatenate(llr)
    ref_info = np.concatenate(info)
    got = batch.llr.cpu().numpy()[:ref_llr.size]
    assert (got.view(np.uint32) == ref_llr.view(np.uint32)).all()
    assert (batch.info.cpu().numpy()[:ref_info.size] == ref_info).all()
    batch.ref_llr, batch.ref_info = ref_llr, ref_info
    return codes, cs, plan, batch


def _oracle_per_code(shapes, plan, llr_host, dtype, max_iters):
    """Oracle decode of every frame with its own code; returns per-frame
    (hard words, iters, post)."""
    out = {}
    for ci, s in enumerate(shapes):
        idx = np.nonzero(plan.code_of_frame == ci)[0]
        if idx.size == 0:
            continue
        rc = oracle.RefCode(s.hbm, s.z)
        x = np.stack([llr_host[plan.llr_off[f]:plan.llr_off[f] + rc.n] for f in idx])
        if dtype == "f32":
            h, it, p = rc.decode_layered_f32(x, max_iters, 0.75, True, True)
        else:
            h, it, p, _ = rc.decode_layered_i8(oracle.quantize_i8(x), max_iters, True, True)
        for j, f in enumerate(idx):
            out[int(f)] = (h[j], it[j], p[j])
    return out


def _check_frames(plan, ref, hard, iters, post):
    hard = hard.cpu().numpy().view(np.uint32)
    iters = iters.cpu().numpy()
    post = post.cpu().numpy()
    for f in range(plan.frames):
        h, it, p = ref[f]
        a, b = plan.hard_off[f], plan.hard_off[f + 1]
        assert iters[f] == it, f
        assert (hard[a:b] == h).all(), f
        assert (post[plan.llr_off[f]:plan.llr_off[f + 1]] == p).all(), f


@pytest.mark.parametrize("dtype", ["f32", "i8"])
def test_mixed_bit_exact_against_oracle(ldpc, dtype):
    shapes = _shapes()
    codes, cs, plan, batch = _setup(ldpc, shapes, 700, seed=4)
    assert plan.n_groups >= 4
    if dtype == "f32":
        d_in, dt = batch.llr, ldpc.F32
    else:
        d_in, dt = plan.quantize(batch.llr), ldpc.I8X4
    hard, iters, post = plan.decode(d_in, dt, max_iters=20, want_post=True)
    ref = _oracle_per_code(shapes, plan, batch.ref_llr, dtype, 20)
    _check_frames(plan, ref, hard, iters, post)
    # after autotuning (other work-item sizes and residency caps) still exact
    plan.autotune(d_in, dt, max_iters=20, reps=1)
    hard2, iters2, post2 = plan.decode(d_in, dt, max_iters=20, want_post=True)
    assert torch.equal(hard, hard2) and torch.equal(iters, iters2) and torch.equal(post, post2)


def test_mixed_unaligned_codes_and_single_code(ldpc):
    """Codes with N not a multiple of 4 (plain-load path) and a batch with one
    code only."""
    shapes = [synth.random_small_code(9, 5, 13, 3), synth.random_small_code(2, 4, 11, 7),
              synth.tiny_z3_code()]
    assert any(s.hbm.shape[1] * s.z % 4 for s in shapes)
    codes, cs, plan, batch = _setup(ldpc, shapes, 157, seed=8, ebn0=(0.5, 3.0))
    for dtype in ("f32", "i8"):
        d_in = batch.llr if dtype == "f32" else plan.quantize(batch.llr)
        dt = ldpc.F32 if dtype == "f32" else ldpc.I8X4
        hard, iters, post = plan.decode(d_in, dt, max_iters=12, want_post=True)
        ref = _oracle_per_code(shapes, plan, batch.ref_llr, dtype, 12)
        _check_frames(plan, ref, hard, iters, post)
    one = [synth.wimax_mixed_set()[40]]
    codes, cs, plan, batch = _setup(ldpc, one, 33, seed=2)
    hard, iters, post = plan.decode(batch.llr, ldpc.F32, max_iters=20, want_post=True)
    ref = _oracle_per_code(one, plan, batch.ref_llr, "f32", 20)
    _check_frames(plan, ref, hard, iters, post)


def test_mixed_stats_and_graph(ldpc):
    shapes = _shapes()
    codes, cs, plan, batch = _setup(ldpc, shapes, 900, seed=6, ebn0=(1.0, 3.0))
    q = plan.quantize(batch.llr)
    hard, iters, _ = plan.decode(q, ldpc.I8X4, max_iters=20)
    cnt, fe = plan.stats(batch.info, hard, iters, 20)
    # per-code frame errors from the unpacked hard decisions
    hw = hard.cpu().numpy().view(np.uint32)
    info = batch.ref_info
    want = np.zeros(len(shapes), dtype=np.int64)
    for f in range(plan.frames):
        c = codes[plan.code_of_frame[f]]
        bits = oracle.unpack_hard(hw[plan.hard_off[f]:plan.hard_off[f + 1]][None], c.n)[0]
        want[plan.code_of_frame[f]] += int((bits[:c.k] != info[plan.info_off[f]:
                                                               plan.info_off[f + 1]]).any())
    assert (fe.cpu().numpy() == want).all()
    assert cnt[1].item() == want.sum() > 0
    assert cnt[3].item() == int(iters.sum().item())
    # the captured step (quantise, decode groups, stats) replays the same results
    h2, i2 = plan.empty_outputs()
    q2 = torch.empty_like(q)
    c2 = torch.empty_like(cnt)
    f2 = torch.empty_like(fe)
    g = plan.graph(ldpc.I8X4, batch.llr, q2, h2, i2, batch.info, c2, f2, max_iters=20)
    for _ in range(2):
        g.launch()
        torch.cuda.synchronize()
        assert torch.equal(h2, hard) and torch.equal(i2, iters)
        assert torch.equal(c2, cnt) and torch.equal(f2, fe) and torch.equal(q2, q)


def test_mixed_learned_and_fallback(ldpc):
    """Learned decoding over a mixed batch (per-code weights, per-code T)
    equals the oracle's weighted decoder frame by frame; the fallback
    pipeline equals the oracle's two steps (learned, then int8 plain min-sum
    at 20 iterations on the frames whose syndrome is not zero)."""
    from paper_2306_12063_gb300.mixed_learned import decode_learned_fallback
    shapes = _shapes()
    codes, cs, plan, batch = _setup(ldpc, shapes, 600, seed=12, ebn0=(1.0, 3.5))
    rng = np.random.default_rng(2)
    Ts = [int(rng.integers(3, 9)) for _ in shapes]
    ws = [rng.uniform(0.5, 1.0, (T, c.nnz_blocks)).astype(np.float32) for T, c in zip(Ts, codes)]
    plan.set_weights([torch.from_numpy(w).cuda() for w in ws])
    hard, iters, post = plan.decode_learned(batch.llr, early_stop=True, want_post=True)
    fb_hard, fb_iters, nfb = decode_learned_fallback(plan, batch.llr)
    llr_h = batch.ref_llr
    hw, it, pw = hard.cpu().numpy().view(np.uint32), iters.cpu().numpy(), post.cpu().numpy()
    fhw, fit = fb_hard.cpu().numpy().view(np.uint32), fb_iters.cpu().numpy()
    bad_total = 0
    for ci, s in enumerate(shapes):
        idx = np.nonzero(plan.code_of_frame == ci)[0]
        if idx.size == 0:
            continue
        rc = oracle.RefCode(s.hbm, s.z)
        x = np.stack([llr_h[plan.llr_off[f]:plan.llr_off[f] + rc.n] for f in idx])
        h, i, p = rc.decode_learned_f32(x, ws[ci], max_iters=Ts[ci], early_stop=True)
        bits = oracle.unpack_hard(h, rc.n)
        bad = np.array([rc.syndrome_weight(b) != 0 for b in bits])
        bad_total += int(bad.sum())
        hq = h.copy()
        iq = i.copy()
        if bad.any():
            h8, i8, _, _ = rc.decode_layered_i8(oracle.quantize_i8(x[bad]), 20, True, True,
                                                want_post=False)
            hq[bad] = h8
            iq[bad] = Ts[ci] + i8
        for j, f in enumerate(idx):
            a, b = plan.hard_off[f], plan.hard_off[f + 1]
            assert it[f] == i[j] and (hw[a:b] == h[j]).all()
            assert (pw[plan.llr_off[f]:plan.llr_off[f + 1]] == p[j]).all()
            assert fit[f] == iq[j] and (fhw[a:b] == hq[j]).all()
    assert nfb == bad_total and 0 < nfb < plan.frames
    # per-frame flags and paired outcomes against host counts
    flags = plan.frame_flags(hard).cpu().numpy()
    assert flags.sum() == bad_total
    cnt = plan.paired_errors(batch.info, hard, fb_hard).cpu().numpy()
    info = batch.ref_info
    wa = np.zeros(plan.frames, bool)
    wb = np.zeros(plan.frames, bool)
    for f in range(plan.frames):
        c = codes[plan.code_of_frame[f]]
        a, b = plan.hard_off[f], plan.hard_off[f + 1]
        ref = info[plan.info_off[f]:plan.info_off[f + 1]]
        wa[f] = (oracle.unpack_hard(hw[a:b][None], c.n)[0][:c.k] != ref).any()
        wb[f] = (oracle.unpack_hard(fhw[a:b][None], c.n)[0][:c.k] != ref).any()
    assert cnt.tolist() == [int((~wa & ~wb).sum()), int((~wa & wb).sum()),
                            int((wa & ~wb).sum()), int((wa & wb).sum())]


def test_mixed_learned_past_table_with_checkpoints(ldpc):
    """The mixed learned launches with every code run up to 16 iterations
    (rows past T_c repeating the last) and two give-up checkpoints equal the
    oracle's decoder frame by frame.  Every third code has a 40-row table
    (a new row staged at every iteration), the others 3 to 8 rows."""
    shapes = _shapes()
    codes, cs, plan, batch = _setup(ldpc, shapes, 500, seed=21, ebn0=(1.0, 3.5))
    rng = np.random.default_rng(8)
    Ts = [40 if ci % 3 == 2 else int(rng.integers(3, 9)) for ci in range(len(shapes))]
    ws = [rng.uniform(0.55, 1.0, (T, c.nnz_blocks)).astype(np.float32) for T, c in zip(Ts, codes)]
    plan.set_weights([torch.from_numpy(w).cuda() for w in ws])
    si, sf = (4, 9), (0.1, 0.04)
    hard, iters, post = plan.decode_learned(batch.llr, want_post=True, max_iters=16,
                                            stop_iter=si, stop_frac=sf)
    llr_h = batch.ref_llr
    hw, it, pw = hard.cpu().numpy().view(np.uint32), iters.cpu().numpy(), post.cpu().numpy()
    stopped = 0
    for ci, s in enumerate(shapes):
        idx = np.nonzero(plan.code_of_frame == ci)[0]
        if idx.size == 0:
            continue
        rc = oracle.RefCode(s.hbm, s.z)
        x = np.stack([llr_h[plan.llr_off[f]:plan.llr_off[f] + rc.n] for f in idx])
        h, i, p = rc.decode_learned_f32(x, ws[ci], max_iters=16, stop_iter=si, stop_frac=sf)
        stopped += int(((i == 4) | (i == 9)).sum())
        for j, f in enumerate(idx):
            a, b = plan.hard_off[f], plan.hard_off[f + 1]
            assert it[f] == i[j] and (hw[a:b] == h[j]).all()
            assert (pw[plan.llr_off[f]:plan.llr_off[f + 1]] == p[j]).all()
    assert stopped > 0 and it.max() > min(Ts)
    # tuning the launches for the learned decoder changes the schedule only
    plan.autotune_learned(batch.llr, max_iters=16, stop_iter=si, stop_frac=sf, reps=1)
    h2, i2, p2 = plan.decode_learned(batch.llr, want_post=True, max_iters=16, stop_iter=si,
                                     stop_frac=sf)
    assert torch.equal(h2, hard) and torch.equal(i2, iters) and torch.equal(p2, post)


@pytest.mark.parametrize("wpf,fpb", [(2, 1), (3, 1), (1, 2), (3, 4), (2, 4)])
def test_mixed_f32_teams_bit_exact(ldpc, wpf, fpb):
    """Warps per frame and frames per block (the FP32 launch settings the
    autotuner searches) change the schedule only: plain FP32 and the learned
    decoder with checkpoints give the same outputs as one warp per frame."""
    shapes = _shapes()
    codes, cs, plan, batch = _setup(ldpc, shapes, 700, seed=31, ebn0=(1.0, 3.5))
    rng = np.random.default_rng(5)
    # 6-row and 40-row tables (the latter past every iteration run here)
    ws = [rng.uniform(0.55, 1.0, (40 if ci % 2 else 6, c.nnz_blocks)).astype(np.float32)
          for ci, c in enumerate(codes)]
    plan.set_weights([torch.from_numpy(w).cuda() for w in ws])
    kw = dict(max_iters=16, stop_iter=(4, 9), stop_frac=(0.1, 0.04))
    ref_f = plan.decode(batch.llr, ldpc.F32, max_iters=20, want_post=True)
    ref_l = plan.decode_learned(batch.llr, want_post=True, **kw)
    for gi in range(plan.n_groups):
        got = plan.group_launch(gi, ldpc.F32, warps_per_frame=wpf, frames_per_block=fpb,
                                frames_per_item=3)
        assert got["warps_per_frame"] == wpf and got["frames_per_block"] == fpb
    got_f = plan.decode(batch.llr, ldpc.F32, max_iters=20, want_post=True)
    got_l = plan.decode_learned(batch.llr, want_post=True, **kw)
    for a, b in zip(ref_f, got_f):
        assert torch.equal(a, b)
    for a, b in zip(ref_l, got_l):
        assert torch.equal(a, b)


def test_mixed_group_launch_argument_checks(ldpc):
    shapes = _shapes()[:3]
    codes = [ldpc.Code(s.hbm, s.z) for s in shapes]
    plan = ldpc.MixedPlan(ldpc.CodeSet(codes), np.arange(12, dtype=np.int32) % 3)
    with pytest.raises(ldpc.LdpcError):
        plan.group_launch(0, ldpc.F32, warps_per_frame=4)
    with pytest.raises(ldpc.LdpcError):
        plan.group_launch(0, ldpc.I8X4, warps_per_frame=2)
    with pytest.raises(ldpc.LdpcError):
        plan.group_launch(0, ldpc.F32, frames_per_block=5)
