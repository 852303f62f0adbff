"""Synthetic decode workloads generated on the GPU by the library's own
kernels: Philox info bits -> direct encoder (Section 2) -> BPSK/AWGN channel
LLRs (eq. 16-17) -> int8 quantisation packed four frames per word."""
from __future__ import annotations

from dataclasses import dataclass

import synth

from . import Code, awgn_llr, awgn_llr_frames, gen_info, quantize_pack_i8, snr_sigma


@dataclass
class Batch:
    info: object      # uint8[F][K]
    cw: object        # uint8[F][N]
    llr: object       # float32[F][N]
    q: object         # int32[ceil(F/4)][N], four int8 frames per word
    frame0: int
    ebn0_db: float
    sigma: float


def make_batch(code: Code, frames: int, frame0: int, ebn0_db: float, seed: int = 1,
               quant_scale: float = 4.0, quant_clip: int = 63, keep_cw: bool = True,
               stream=None) -> Batch:
    """Frames frame0 .. frame0+frames-1 of the seeded stream at one Eb/N0."""
    sigma = synth.ebn0_db_to_sigma(ebn0_db, code.k / code.n)
    info = gen_info(seed, frame0, frames, code.k, device=code.device, stream=stream)
    cw = code.encode(info, stream=stream)
    llr = awgn_llr(cw, frame0, seed, sigma, stream=stream)
    q = quantize_pack_i8(llr, quant_scale, quant_clip, stream=stream)
    if not keep_cw:
        cw = None
    return Batch(info, cw, llr, q, frame0, ebn0_db, sigma)


@dataclass
class MixedBatch:
    info: object      # uint8[info_elems], frame f at plan.info_off[f]
    llr: object       # float32[llr_elems], frame f at plan.llr_off[f]


def mixed_frame_id(code_index: int, j: int) -> int:
    """Frame identity of the j-th frame of code `code_index` in a mixed batch
    (the counter of its info bits, noise and Eb/N0 draws; synth's rule)."""
    return synth.mixed_frame_id(code_index, j)


def make_mixed_batch(plan, ebn0_db=(1.5, 4.5), seed: int = 1, frame_base: int = 0,
                     stream=None) -> MixedBatch:
    """Every frame of the plan: info bits, direct encoding, Eb/N0 uniform in
    [lo, hi) dB per frame and the AWGN channel, generated per code by the
    library's kernels and placed in the plan layout by ldpc_mixed_scatter.
    The j-th frame of code c has identity mixed_frame_id(c, frame_base + j)
    (ranks of a sharded batch pass their first global frame, so no two ranks
    draw the same frame)."""
    import numpy as np
    import torch
    codes = plan.codeset.codes
    dev = codes[0].device
    info = torch.empty((max(plan.info_elems, 1),), dtype=torch.uint8, device=dev)
    llr = torch.empty((max(plan.llr_elems, 1),), dtype=torch.float32, device=dev)
    counts = np.bincount(plan.code_of_frame, minlength=len(codes))
    for ci, code in enumerate(codes):
        F = int(counts[ci])
        if F == 0:
            continue
        f0 = mixed_frame_id(ci, frame_base)
        inf_c = gen_info(seed, f0, F, code.k, device=dev, stream=stream)
        cw = code.encode(inf_c, stream=stream)
        sig = snr_sigma(seed, f0, F, ebn0_db[0], ebn0_db[1], code.k / code.n, device=dev,
                        stream=stream)
        llr_c = awgn_llr_frames(cw, f0, seed, sig, stream=stream)
        plan.scatter(ci, 1, inf_c, info, stream=stream)
        plan.scatter(ci, 0, llr_c, llr, stream=stream)
    return MixedBatch(info, llr)
