"""Training of learned normalised min-sum weights with the library's kernels.

The weights w[t][q] scale the eq. (23) message of iteration t on nonzero
block q of H_bm.  A training step draws a fresh batch from the library's own
generators (Philox info bits, the direct encoder of eq. (12)-(15), per-frame
Eb/N0 and the AWGN channel of eq. (16)-(17)), runs the unrolled decoder
forward with checkpoints, its hand-written backward and an Adam update; the
loss is the cross-entropy of every iteration's posterior bit probabilities,
averaged over frames and bits (summed over iterations).  Every step runs in
libldpc kernels; this module only allocates buffers and sequences calls.
"""
from __future__ import annotations

from dataclasses import dataclass, field
from typing import List, Optional, Tuple

import numpy as np

from . import Code, adam_step, awgn_llr_frames, gen_info, snr_sigma


def _torch():
    import torch
    return torch


def default_iterations(rate: float) -> int:
    """Unrolled depth: 8 iterations up to rate 2/3, 6 above."""
    return 8 if rate <= 2.0 / 3.0 + 1e-9 else 6


class LearnedMinSumLoss:
    """torch.autograd.Function: loss = loss_scale * sum over frames of the
    training loss, differentiable in the weights and the channel LLRs."""

    _fn = None

    @classmethod
    def apply(cls, weights, llr, bits, code: Code, loss_scale: float):
        if cls._fn is None:
            torch = _torch()

            class _Fn(torch.autograd.Function):
                @staticmethod
                def forward(ctx, w, x, b, code_, scale):
                    post, rows, _, loss_sum = code_.train_forward(x, b, w, scale)
                    ctx.save_for_backward(w, x, b, post, rows)
                    ctx.code = code_
                    ctx.scale = scale
                    return loss_sum.reshape(())

                @staticmethod
                def backward(ctx, g):
                    w, x, b, post, rows = ctx.saved_tensors
                    gw, gx = ctx.code.train_backward(x, b, w, post, rows,
                                                     ctx.scale * float(g),
                                                     want_llr_grad=ctx.needs_input_grad[1])
                    return gw, gx, None, None, None

            cls._fn = _Fn
        return cls._fn.apply(weights, llr, bits, code, loss_scale)


def learned_loss(code: Code, weights, llr, bits, loss_scale: Optional[float] = None):
    """Differentiable training loss (mean over frames and bits by default)."""
    if loss_scale is None:
        loss_scale = 1.0 / (llr.shape[0] * code.n)
    return LearnedMinSumLoss.apply(weights, llr, bits, code, float(loss_scale))


@dataclass
class TrainConfig:
    T: int = 8
    steps: int = 2000
    batch: int = 4096
    lr: float = 1e-3
    ebn0_db: Tuple[float, float] = (1.0, 4.0)
    seed: int = 1000          # info and noise seed of the training frames
    init: float = 0.75
    beta1: float = 0.9
    beta2: float = 0.999
    eps: float = 1e-8


@dataclass
class TrainResult:
    weights: object                       # float32[T][nnz_blocks] on the GPU
    loss_history: object                  # float32[steps] on the GPU (this run's steps)
    config: TrainConfig = field(default_factory=TrainConfig)
    adam_m: object = None                 # Adam first and second moments
    adam_v: object = None
    step: int = 0                         # Adam steps taken in total


def train_weights(code: Code, cfg: TrainConfig = TrainConfig(), weights=None,
                  stream=None, resume: Optional[TrainResult] = None,
                  steps: Optional[int] = None) -> TrainResult:
    """Adam on the learned weights; batch b of step s holds frames
    s * batch .. (s + 1) * batch - 1 of the training streams.  `resume`
    continues from a result (or a loaded checkpoint): its weights, Adam
    moments and step count; since a step's batch depends on its index only
    and every kernel is deterministic, stopping and resuming gives the same
    weights bit for bit as one uninterrupted run.  `steps` (default
    cfg.steps) ends the run early, counted from the first step."""
    torch = _torch()
    dev = code.device
    B, T, E = cfg.batch, cfg.T, code.nnz_blocks
    s0 = 0
    if resume is not None:
        weights = resume.weights.to(dev).clone()
        m = resume.adam_m.to(dev).clone()
        v = resume.adam_v.to(dev).clone()
        s0 = int(resume.step)
        if tuple(weights.shape) != (T, E):
            raise ValueError(f"checkpoint weights {tuple(weights.shape)} do not fit T={T}, "
                             f"{E} blocks")
    else:
        if weights is None:
            weights = torch.full((T, E), float(cfg.init), dtype=torch.float32, device=dev)
        m = torch.zeros_like(weights)
        v = torch.zeros_like(weights)
    s1 = cfg.steps if steps is None else min(cfg.steps, int(steps))
    info = torch.empty((B, code.k), dtype=torch.uint8, device=dev)
    cw = torch.empty((B, code.n), dtype=torch.uint8, device=dev)
    sigma = torch.empty((B,), dtype=torch.float32, device=dev)
    llr = torch.empty((B, code.n), dtype=torch.float32, device=dev)
    post = torch.empty((T, B, code.n), dtype=torch.float32, device=dev)
    rows = torch.empty((max(T - 1, 0), B, code.m, 4), dtype=torch.int32, device=dev)
    loss = torch.empty((B,), dtype=torch.float32, device=dev)
    hist = torch.empty((max(s1 - s0, 0),), dtype=torch.float32, device=dev)
    gw = torch.empty((T, E), dtype=torch.float32, device=dev)
    ws = torch.empty(max(code.train_workspace_bytes(B, T), 1), dtype=torch.uint8, device=dev)
    rate = code.k / code.n
    scale = 1.0 / (B * code.n)
    for s in range(s0, s1):
        f0 = s * B
        gen_info(cfg.seed, f0, B, code.k, device=dev, out=info, stream=stream)
        code.encode(info, out=cw, stream=stream)
        snr_sigma(cfg.seed, f0, B, cfg.ebn0_db[0], cfg.ebn0_db[1], rate, device=dev,
                  out=sigma, stream=stream)
        awgn_llr_frames(cw, f0, cfg.seed, sigma, out=llr, stream=stream)
        code.train_forward(llr, cw, weights, scale,
                           out=(post, rows, loss, hist[s - s0:s - s0 + 1]), stream=stream)
        code.train_backward(llr, cw, weights, post, rows, scale, workspace=ws, out=(gw, None),
                            stream=stream)
        adam_step(weights, gw, m, v, s + 1, cfg.lr, cfg.beta1, cfg.beta2, cfg.eps, stream=stream)
    return TrainResult(weights, hist, cfg, m, v, max(s1, s0))


def operating_range(code: Code, lo: float = 1.5, hi: float = 4.5, step: float = 0.25,
                    frames: int = 4096, fer_max: float = 0.5, max_iters: int = 20,
                    alpha: float = 0.75, seed: int = 7, stream=None) -> Tuple[float, float]:
    """Eb/N0 training range of a code where plain min-sum decodes it (a
    reading of the training recipe for codes of many rates): the lowest
    step b = lo, lo + step, ... whose centre b + step / 2 gives a frame-error
    rate of at most fer_max for plain FP32 layered min-sum (alpha, max_iters
    iterations, early stop) on `frames` calibration frames of their own seed,
    and the range [b, max(b + 1, hi)] dB.  Every decode and count runs in the
    library's kernels."""
    from . import awgn_llr
    dev = code.device
    rate = code.k / code.n
    info = gen_info(seed, 0, frames, code.k, device=dev, stream=stream)
    cw = code.encode(info, stream=stream)
    b = lo
    nsteps = int(round((hi - lo) / step))
    for i in range(nsteps):
        b = lo + i * step
        # unit-energy BPSK: sigma^2 = 1 / (2 R 10^(Eb/N0 / 10))
        sigma = (1.0 / (2.0 * rate * 10.0 ** ((b + step / 2) / 10.0))) ** 0.5
        llr = awgn_llr(cw, 0, seed + 1 + i, sigma, stream=stream)
        h, it, _ = code.decode(llr, max_iters=max_iters, alpha=alpha, early_stop=True,
                               stream=stream)
        st = code.frame_stats(info, h, it, max_iters, stream=stream)
        if float(st[1].item()) / frames <= fer_max:
            break
    return float(b), float(max(b + 1.0, hi))


def save_checkpoint(path: str, result: TrainResult) -> None:
    """Weights, Adam moments, step count, loss history and configuration as
    one torch file (tensors moved to the host)."""
    torch = _torch()
    torch.save({"weights": result.weights.detach().cpu(),
                "adam_m": result.adam_m.detach().cpu(),
                "adam_v": result.adam_v.detach().cpu(),
                "step": int(result.step),
                "loss_history": result.loss_history.detach().cpu(),
                "config": dict(result.config.__dict__)}, path)


def load_checkpoint(path: str, device="cpu") -> TrainResult:
    """A TrainResult from save_checkpoint, its tensors on `device`; pass it
    as `resume` to continue training."""
    torch = _torch()
    d = torch.load(path, map_location="cpu", weights_only=True)
    cfg = d["config"]
    cfg["ebn0_db"] = tuple(cfg["ebn0_db"])
    return TrainResult(d["weights"].to(device), d["loss_history"].to(device), TrainConfig(**cfg),
                       d["adam_m"].to(device), d["adam_v"].to(device), int(d["step"]))
