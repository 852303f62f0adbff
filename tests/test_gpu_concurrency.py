"""Host threads driving the library at once, each on its own stream with a
code of another size (the benchmark trains its 78 codes four at a time this
way): results equal those of the same calls made one after another."""
from concurrent.futures import ThreadPoolExecutor

import numpy as np
import pytest

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


def _work(ldpc, shape, seed, stream):
    """A few training steps and decodes of one code, all on `stream`."""
    from paper_2306_12063_gb300 import train
    with torch.cuda.stream(stream):
        code = ldpc.Code(shape.hbm, shape.z)
        cfg = train.TrainConfig(T=4, steps=6, batch=96, lr=2e-3, seed=seed)
        w = train.train_weights(code, cfg, stream=stream).weights
        info = ldpc.gen_info(seed, 0, 300, code.k, stream=stream)
        llr = ldpc.awgn_llr(code.encode(info, stream=stream), 0, seed,
                            synth.ebn0_db_to_sigma(2.0, code.k / code.n), stream=stream)
        out = []
        for _ in range(3):
            out.append(code.decode_learned(llr, w, max_iters=12, stop_iter=(3, 0),
                                           stop_frac=(0.1, 0.0), want_post=True, stream=stream))
            out.append(code.decode(llr, max_iters=12, early_stop=True, want_post=True,
                                   stream=stream))
        stream.synchronize()
        return [w.cpu()] + [t.cpu() for o in out for t in o if t is not None]


def test_threads_on_streams_match_one_after_another(ldpc):
    # same slot class (8), different sizes: the kernels' shared memory differs
    shapes = [synth.wifi_n648_r12(), synth.wimax_mixed_set()[-4], synth.wimax_mixed_set()[0],
              synth.wimax_mixed_set()[4 * 9]]
    streams = [torch.cuda.Stream() for _ in shapes]
    seq = [_work(ldpc, s, 40 + i, streams[i]) for i, s in enumerate(shapes)]
    for _ in range(2):
        with ThreadPoolExecutor(len(shapes)) as ex:
            par = list(ex.map(lambda i: _work(ldpc, shapes[i], 40 + i, streams[i]),
                              range(len(shapes))))
        for a, b in zip(seq, par):
            assert len(a) == len(b)
            for u, v in zip(a, b):
                assert torch.equal(u, v)
