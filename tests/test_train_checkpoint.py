"""Checkpoint and resume of learned-weight training: the file round trip on
the host, and on the GPU that stopping after a few steps, saving, loading
and resuming gives the weights and Adam state of one uninterrupted run bit
for bit (a step's batch depends on its index only, every kernel is
deterministic)."""
import numpy as np
import pytest

torch = pytest.importorskip("torch")


def test_checkpoint_round_trip(tmp_path):
    from paper_2306_12063_gb300.train import (TrainConfig, TrainResult, load_checkpoint,
                                              save_checkpoint)
    g = torch.Generator().manual_seed(3)
    cfg = TrainConfig(T=5, steps=40, batch=128, lr=2e-3, ebn0_db=(1.5, 3.5), seed=77)
    r = TrainResult(torch.rand((5, 31), generator=g), torch.rand(17, generator=g), cfg,
                    torch.rand((5, 31), generator=g), torch.rand((5, 31), generator=g), 17)
    path = str(tmp_path / "ckpt.pt")
    save_checkpoint(path, r)
    q = load_checkpoint(path)
    for a, b in ((r.weights, q.weights), (r.adam_m, q.adam_m), (r.adam_v, q.adam_v),
                 (r.loss_history, q.loss_history)):
        assert torch.equal(a, b)
    assert q.step == 17 and q.config == cfg


@pytest.mark.gpu
def test_resume_equals_uninterrupted():
    assert torch.cuda.is_available(), "GPU tests need a CUDA device"
    from paper_2306_12063_gb300 import _build
    _build.build()
    import synth
    import paper_2306_12063_gb300 as ldpc
    from paper_2306_12063_gb300.train import (TrainConfig, load_checkpoint, save_checkpoint,
                                              train_weights)
    ldpc.load()
    s = synth.wifi_n648_r12()
    code = ldpc.Code(s.hbm, s.z)
    cfg = TrainConfig(T=4, steps=6, batch=256, lr=5e-3)
    full = train_weights(code, cfg)
    part = train_weights(code, cfg, steps=3)
    assert part.step == 3
    import tempfile, os
    with tempfile.TemporaryDirectory() as d:
        path = os.path.join(d, "ckpt.pt")
        save_checkpoint(path, part)
        back = load_checkpoint(path, device="cuda")
    rest = train_weights(code, cfg, resume=back)
    torch.cuda.synchronize()
    assert rest.step == 6
    assert torch.equal(full.weights, rest.weights)
    assert torch.equal(full.adam_m, rest.adam_m) and torch.equal(full.adam_v, rest.adam_v)
    hist = torch.cat([part.loss_history, rest.loss_history])
    assert torch.equal(full.loss_history, hist)
    assert not torch.equal(full.weights, torch.full_like(full.weights, cfg.init))
