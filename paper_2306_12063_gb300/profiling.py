"""Small, reproducible cases that launch each decoder-family kernel exactly
once (after generating its inputs), for a kernel profiler's name filter:

    python -m paper_2306_12063_gb300.profiling

1. learned FP32 decoder (`decode_f32_kernel<8, true>`), N=648, 65,536 frames,
   T = 8, weights 0.8, Eb/N0 uniform in [1.5, 4.5) dB;
2. mixed int8 and FP32 decoders (`mixed_i8_kernel`, `mixed_f32_kernel`) on
   the four R=3/4 WiMAX-shaped codes with Z = 84..96 (one launch group),
   65,536 frames;
3. Section 5 int16 wrap-around decoder (`decode_i16w_kernel`), N=1944,
   65,536 frames at 4.0 dB;
4. flooding FP32 decoder (`decode_flooding_kernel`), N=648, 16,384 frames,
   10 iterations;
5. Alg. A1 bitmap encoder (`encode_bitmap_kernel`), N=2304 R=5/6, 262,144
   frames;
6. one training step (`train_forward_kernel`, `train_backward_kernel`),
   N=648, batch 4,096, T = 8.

Every input is generated on the GPU by the library's own kernels first
(those kernels are not among the names above).
"""
from __future__ import annotations

import numpy as np


def main():
    import torch

    import synth
    from . import F32, I8X4, I16W, Code, CodeSet, MixedPlan, awgn_llr, awgn_llr_frames
    from . import gen_info, load, quantize_i16, snr_sigma
    from .workload import make_mixed_batch

    load()
    dev = "cuda"
    # 1. learned decoder
    s648 = synth.wifi_n648_r12()
    c648 = Code(s648.hbm, s648.z)
    F = 65536
    info = gen_info(1, 0, F, c648.k)
    cw = c648.encode(info)
    sig = snr_sigma(1, 0, F, 1.5, 4.5, 0.5)
    llr648 = awgn_llr_frames(cw, 0, 1, sig)
    w = torch.full((8, c648.nnz_blocks), 0.8, dtype=torch.float32, device=dev)
    torch.cuda.synchronize()
    c648.decode_learned(llr648, w, early_stop=True)
    torch.cuda.synchronize()
    # 2. mixed batch, one launch group
    shapes = [s for s in synth.wimax_mixed_set() if s.mb == 6 and s.z >= 84]
    codes = [Code(s.hbm, s.z) for s in shapes]
    cs = CodeSet(codes)
    cof = (np.arange(F) % len(shapes)).astype(np.int32)
    plan = MixedPlan(cs, cof)
    batch = make_mixed_batch(plan, (1.5, 4.5), seed=1)
    q = plan.quantize(batch.llr)
    torch.cuda.synchronize()
    plan.decode(q, I8X4, max_iters=20)
    plan.decode(batch.llr, F32, max_iters=20)
    torch.cuda.synchronize()
    # 3. int16 wrap-around decoder
    s1944 = synth.wifi_n1944_r56()
    c1944 = Code(s1944.hbm, s1944.z)
    info = gen_info(1, 0, F, c1944.k)
    cw = c1944.encode(info)
    llr = awgn_llr(cw, 0, 1, synth.ebn0_db_to_sigma(4.0, c1944.k / c1944.n))
    q16 = quantize_i16(llr, 16.0, 10)
    torch.cuda.synchronize()
    c1944.decode(q16, dtype=I16W, max_iters=20, normalise=True, early_stop=True)
    torch.cuda.synchronize()
    # 4. flooding decoder
    c648.decode_flooding(llr648[:16384], 10, 0.75, True, False)
    torch.cuda.synchronize()
    # 5. bitmap encoder
    s2304 = synth.wimax_n2304_r56()
    c2304 = Code(s2304.hbm, s2304.z)
    Fe = 262144
    words = torch.randint(-2**31, 2**31 - 1, (Fe, c2304.k // 32), dtype=torch.int32,
                          device=dev)
    torch.cuda.synchronize()
    c2304.encode_bitmap(words)
    torch.cuda.synchronize()
    # 6. one training step
    from .train import TrainConfig, train_weights
    train_weights(c648, TrainConfig(T=8, steps=1, batch=4096))
    torch.cuda.synchronize()
    print("profiling cases done")


if __name__ == "__main__":
    main()
