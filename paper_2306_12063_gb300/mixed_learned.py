"""Learned normalised min-sum over mixed-code batches, with the int8 plain
min-sum fallback for the frames the learned decoder leaves with a nonzero
syndrome.

The fallback pipeline: one learned launch set over the whole batch, the
per-frame syndrome flags, then (host) a plan for the failed frames only,
their LLR rows moved into it, the int8 quantiser and plain decoder on that
plan, and the results moved back (iteration count T_c plus the fallback's).
Every step runs in libldpc kernels; the host only reads the flags and builds
the small plan.
"""
from __future__ import annotations

import numpy as np

from . import I8X4, MixedPlan, train


def train_codeset_weights(codes, cfg_for, device=None):
    """Per-code learned weights: train.train_weights on each code with the
    configuration cfg_for(code) (T = 8 up to rate 2/3, 6 above by default)."""
    out = []
    for code in codes:
        out.append(train.train_weights(code, cfg_for(code)).weights)
    return out


def decode_learned_fallback(plan: MixedPlan, llr, fallback_iters: int = 20,
                            quant_scale: float = 4.0, quant_clip: int = 63, out=None):
    """Returns (hard, iters, number of fallback frames)."""
    import torch
    hard, iters = out if out is not None else plan.empty_outputs()
    plan.decode_learned(llr, early_stop=True, out=(hard, iters, None))
    bad = plan.frame_flags(hard)
    idx = np.nonzero(bad.cpu().numpy())[0].astype(np.int64)   # waits for the learned pass
    nf = int(idx.size)
    if nf:
        sub = MixedPlan(plan.codeset, plan.code_of_frame[idx])
        d_idx = torch.from_numpy(idx).to(llr.device)
        sub_llr = torch.empty((max(sub.llr_elems, 1),), dtype=torch.float32, device=llr.device)
        plan.move_frames(sub, d_idx, 0, llr, sub_llr)
        q = sub.quantize(sub_llr, quant_scale, quant_clip)
        sh, si, _ = sub.decode(q, I8X4, max_iters=fallback_iters, normalise=True,
                               early_stop=True)
        plan.move_frames(sub, d_idx, 1, hard, sh)
        plan.move_frames(sub, d_idx, 2, iters, si)
    return hard, iters, nf
