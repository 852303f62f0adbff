"""Synthetic decode workloads generated on the GPU by the library's own
kernels: Philox info bits -> direct encoder (Section 2) -> BPSK/AWGN channel
LLRs (eq. 16-17) -> int8 quantisation packed four frames per word."""
from __future__ import annotations

from dataclasses import dataclass

import synth

from . import Code, awgn_llr, gen_info, quantize_pack_i8


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
