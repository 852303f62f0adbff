"""Statistical sanity of the GPU decoders on the N=648, Z=27, R=1/2 code.

The paper's error-rate results use the standard 802.11 matrices, which are
not available, so the frame-error rates of the seeded stand-in codes are not
pinned to printed values.  What the paper's experiments do fix are trends,
checked here on 32,768 frames per point:

* FER falls as Eb/N0 rises (the waterfall of Section 6.1, Fig. 2): the 95 %
  Wilson intervals of neighbouring points 0.5 dB apart do not overlap;
* the mean iteration count with syndrome early stop falls as Eb/N0 rises
  (the trend of Tab. 4, 8.00 -> 6.36 over 1.0 -> 2.0 dB);
* the fixed-point decoder is no better than the float decoder (Section 6.1
  reports a fixed-point penalty of about 0.1 dB): on the same frames, the
  exact one-sided McNemar test does not find int8 better than FP32 at the
  1 % level, and the int8 FER lies no more than the intervals' width below
  the FP32 one.
"""
import numpy as np
import pytest

import synth

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")

EBN0 = (1.5, 2.0, 2.5)
FRAMES = 32768
MAX_ITERS = 20


@pytest.fixture(scope="module")
def ldpc():
    assert torch.cuda.is_available(), "GPU tests need a CUDA device"
    from paper_2306_12063_gb300 import _build
    _build.build()
    import paper_2306_12063_gb300 as m
    m.load()
    return m


@pytest.fixture(scope="module")
def curves(ldpc):
    from paper_2306_12063_gb300 import stats
    shape = synth.wifi_n648_r12()
    code = ldpc.Code(shape.hbm, shape.z)
    out = {}
    for b, eb in enumerate(EBN0):
        frame0 = b * FRAMES
        info = ldpc.gen_info(7, frame0, FRAMES, code.k)
        cw = code.encode(info)
        llr = ldpc.awgn_llr(cw, frame0, 7, synth.ebn0_db_to_sigma(eb, code.k / code.n))
        q = ldpc.quantize_pack_i8(llr)
        res = {}
        for name, kw in (("f32", dict(x=llr, dtype=ldpc.F32)),
                         ("i8", dict(x=q, dtype=ldpc.I8X4, frames=FRAMES))):
            x = kw.pop("x")
            h, it, _ = code.decode(x, max_iters=MAX_ITERS, alpha=0.75, normalise=True,
                                   early_stop=True, **kw)
            st = code.frame_stats(info, h, it, MAX_ITERS).cpu().numpy()
            res[name] = {"hard": h, "fe": int(st[1]), "fer": st[1] / FRAMES,
                         "ci": stats.wilson_interval(int(st[1]), FRAMES),
                         "mean_iters": st[3] / FRAMES}
        cnt = code.paired_frame_errors(info, res["i8"]["hard"], res["f32"]["hard"]).cpu().numpy()
        res["i8_vs_f32"] = stats.compare(cnt, FRAMES)
        out[eb] = res
    return out


@pytest.mark.parametrize("dtype", ["f32", "i8"])
def test_fer_falls_with_ebn0(curves, dtype):
    fers = [curves[eb][dtype]["fer"] for eb in EBN0]
    assert all(f > 0 for f in fers), f"need errors at every point to see a trend: {fers}"
    for lo, hi in zip(EBN0, EBN0[1:]):
        # the higher-Eb/N0 interval lies entirely below the lower-Eb/N0 one
        assert curves[hi][dtype]["ci"][1] < curves[lo][dtype]["ci"][0], (dtype, lo, hi, fers)


@pytest.mark.parametrize("dtype", ["f32", "i8"])
def test_mean_iterations_fall_with_ebn0(curves, dtype):
    its = [curves[eb][dtype]["mean_iters"] for eb in EBN0]
    assert all(a > b for a, b in zip(its, its[1:])), (dtype, its)
    assert all(1.0 <= x <= MAX_ITERS for x in its)


def test_fixed_point_is_no_better_than_float(curves):
    for eb in EBN0:
        c = curves[eb]["i8_vs_f32"]
        # one-sided McNemar for "FP32 fails more often than int8"
        from paper_2306_12063_gb300 import stats
        p_f32_worse = stats.mcnemar_one_sided(c["only_b_wrong"], c["only_a_wrong"])
        assert p_f32_worse >= 0.01, (eb, c)
        i8, f32 = curves[eb]["i8"], curves[eb]["f32"]
        width = (f32["ci"][1] - f32["ci"][0]) + (i8["ci"][1] - i8["ci"][0])
        assert i8["fer"] >= f32["fer"] - width, (eb, i8["fer"], f32["fer"])
