"""Throughput benchmark: layered min-sum decoding of the N=1944, Z=81, R=5/6
Wi-Fi-6-shaped code on GB300.

One step = decoding the whole workload once: three batches of 262,144
frames at Eb/N0 = 3.5, 4.0 and 4.5 dB, int8 packed four frames per word,
max 20 iterations with syndrome early stop, the three batches back to back
in one buffer and decoded by one call (one persistent launch, so the ragged
end of a launch, where warps finishing their last frames leave SMs idle,
comes once per step instead of once per batch).  Inputs are generated on the
GPU (Philox info bits, direct encoder, AWGN, quantiser) before timing and
stay resident in HBM (the 1.5 GB of packed LLRs exceed the 129 MB L2, so no
flush is needed between steps).  The FP32 decoder is timed on the same
frames and reported beside it.

Prints one JSON line (rank 0).  With --impl reference it times the CPU
oracle on a bounded sample of the same workload instead.
"""
from __future__ import annotations

import argparse
import hashlib
import json
import os
import re
import statistics
import subprocess
import sys
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

import synth  # noqa: E402

EBN0 = (3.5, 4.0, 4.5)
MAX_ITERS = 20
WORKLOAD = ("wifi6-shaped N=1944 Z=81 R=5/6 (seeded 4x24 base matrix, seed 2), "
            "3 x 262144 frames at Eb/N0 3.5/4.0/4.5 dB, max 20 iterations, early stop, "
            "the three batches decoded by one call per step")
METRIC = "info Gbit/s at matched FER, learned-NMS vs plain min-sum; % roofline"
METRIC_BASIS = ("value: info Gbit/s of the plain int8 layered min-sum decoder on the batched "
                "N=1944 workload (fp32: the same frames in FP32, the like-for-like figure "
                "against the paper's float decoder); % roofline: roofline.frac; learned-NMS "
                "against plain min-sum at matched FER: learned_vs_plain (summary of the "
                "learned_scale and learned objects)")
# Algorithmic operations per edge per iteration (per frame, or per packed
# word of four frames), the scope table's count: pass 1 = 9 (old message
# rebuilt by a select and a sign, subtract, |.|, two compare/select pairs for
# the two minima and the argmin, sign xor); pass 2 = 3 (select, sign, add);
# syndrome = 1 (xor).  Shared-memory accesses are not counted.  Per row per
# iteration: two scalings, the sign extraction and the state store (4).
OPS_PER_EDGE = 13
OPS_PER_ROW = 4
SMS = 152
LANES_PER_SM = 128


def _dist():
    ws = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return ws, rank, local


class ClockSampler:
    """nvidia-smi samples of SM clock and throttle reasons during a region."""
    FIELDS = ("clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, device_index: int):
        self.dev = device_index
        self.proc = None

    def __enter__(self):
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", f"--query-gpu={self.FIELDS}", "--format=csv,noheader,nounits",
                 "-lms", "100", "-i", str(self.dev)],
                stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
        except OSError:
            self.proc = None
        return self

    def __exit__(self, *exc):
        self.out = ""
        if self.proc is not None:
            self.proc.terminate()
            try:
                self.out, _ = self.proc.communicate(timeout=5)
            except subprocess.TimeoutExpired:
                self.proc.kill()
                self.out, _ = self.proc.communicate()

    def summary(self):
        rows = []
        for line in (self.out or "").strip().splitlines():
            parts = [p.strip() for p in line.split(",")]
            if len(parts) < 8:
                continue
            try:
                rows.append((float(parts[0]), float(parts[1]), parts[4:8]))
            except ValueError:
                continue
        if not rows:
            return None
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        reasons = sorted({names[i] for _, _, fl in rows for i, v in enumerate(fl)
                          if v.lower() == "active"})
        return {"sm_mhz": statistics.median(r[0] for r in rows),
                "sm_max_mhz": max(r[1] for r in rows), "reasons": reasons,
                "samples": len(rows)}


_TOKENS = re.compile(r'"(?:\\.|[^"\\])*"|\'(?:\\.|[^\'\\])*\'|//[^\n]*|/\*.*?\*/|\s+', re.S)


def code_text(src: str) -> str:
    """C/CUDA source without comments, whitespace runs folded to one space."""
    def keep(m):
        t = m.group(0)
        if t.startswith("//") or t.startswith("/*"):
            return " "
        return " " if t.isspace() else t
    return re.sub(r"\s+", " ", _TOKENS.sub(keep, src)).strip()


def kernel_source_digest() -> str:
    """sha256 (first 16 hex digits) of the decoder kernel sources' code (comments
    and layout do not count, so a profile stays valid across comment edits)."""
    h = hashlib.sha256()
    for name in ("ldpc_decode.cu", "ldpc_decode_dev.cuh", "ldpc_internal.cuh"):
        with open(os.path.join(ROOT, "paper_2306_12063_gb300", "csrc", name)) as fh:
            h.update(code_text(fh.read()).encode())
    return h.hexdigest()[:16]


def _profile_traffic(kernel_tag: str):
    """DRAM bytes per launch from the committed ncu summary, if it was taken
    on the current kernel source (its hash is recorded beside the number)."""
    path = os.path.join(ROOT, "profiles", f"{kernel_tag}.md")
    try:
        txt = open(path).read()
        digest = kernel_source_digest()
    except OSError:
        return None
    m = re.search(r"source_sha256_16:\s*([0-9a-f]{16})", txt)
    t = re.search(r"traffic_bytes_per_launch:\s*([0-9.e+]+)", txt)
    if not m or not t or m.group(1) != digest:
        return None
    return float(t.group(1))


def _alg_ops(code_e: int, code_m: int, iters_sum: int, words: bool) -> float:
    ops = iters_sum * (OPS_PER_EDGE * code_e + OPS_PER_ROW * code_m)
    return ops / 4.0 if words else float(ops)


# --------------------------------------------------------------------------- oracle

def run_oracle_sample(frames: int, ebn0: float, threads: int, dtype: str = "i8"):
    """Oracle (as it stands) on `frames` frames of the 4.0 dB batch, decoded on
    a thread pool in blocks of 10 frames per task (ctypes releases the GIL).
    Returns (info bits decoded, seconds)."""
    import oracle
    from concurrent.futures import ThreadPoolExecutor
    shape = synth.wifi_n1944_r56()
    rc = oracle.RefCode(shape.hbm, shape.z)
    sigma = synth.ebn0_db_to_sigma(ebn0, rc.k / rc.n)
    frame0 = EBN0.index(ebn0) * 262144
    blocks = [(f, min(10, frames - f)) for f in range(0, frames, 10)]

    def gen(b):
        f, n = b
        info = oracle.gen_info(1, frame0 + f, n, rc.k)
        llr = oracle.awgn_llr(rc.encode(info), frame0 + f, 1, sigma)
        return oracle.quantize_i8(llr) if dtype == "i8" else llr

    with ThreadPoolExecutor(threads) as ex:
        inputs = list(ex.map(gen, blocks))

    def dec(x):
        if dtype == "i8":
            return rc.decode_layered_i8(x, MAX_ITERS, True, True, want_post=False)[1]
        return rc.decode_layered_f32(x, MAX_ITERS, 0.75, True, True, want_post=False)[1]

    t0 = time.perf_counter()
    with ThreadPoolExecutor(threads) as ex:
        list(ex.map(dec, inputs))
    dt = time.perf_counter() - t0
    return frames * rc.k, dt


LEARNED_EBN0 = (1.5, 4.5)
LEARNED_WORKLOAD = ("wifi6-shaped N=648 Z=27 R=1/2 (seeded 12x24 base matrix, seed 0), "
                    "frames with Eb/N0 uniform in [1.5, 4.5) dB per frame")


def learned_leg(args, ldpc, torch, dev, stream, barrier, rank, ws, pg):
    """Learned normalised min-sum (weights trained at start-up with the
    library's training kernels, untimed) against plain layered min-sum at 20
    iterations, decoding the same frames; FER compared with McNemar's test."""
    from paper_2306_12063_gb300 import stats, train
    from paper_2306_12063_gb300.shard import reduce_counters

    shape = synth.wifi_n648_r12()
    code = ldpc.Code(shape.hbm, shape.z, device=dev)
    rate = code.k / code.n
    T = train.default_iterations(rate)
    cfg = train.TrainConfig(T=T)
    t0 = time.time()
    tr = train.train_weights(code, cfg)
    torch.cuda.synchronize()
    train_s = time.time() - t0
    hist = tr.loss_history.cpu().numpy()
    w = tr.weights
    F = args.learned_frames
    frame0 = rank * F
    info = ldpc.gen_info(1, frame0, F, code.k, device=dev)
    cw = code.encode(info)
    sig = ldpc.snr_sigma(1, frame0, F, LEARNED_EBN0[0], LEARNED_EBN0[1], rate, device=dev)
    llr = ldpc.awgn_llr_frames(cw, frame0, 1, sig)
    del cw
    q = ldpc.quantize_pack_i8(llr)
    wsfb = torch.empty(code.learned_workspace_bytes(F), dtype=torch.uint8, device=dev)

    def out():
        return (torch.empty((F, code.nwords), dtype=torch.int32, device=dev),
                torch.empty((F,), dtype=torch.int32, device=dev), None)

    names = ("plain_i8_20", "plain_f32_20", "learned", "learned_fallback", "learned_gated",
             "learned_20", "ablation_const_gated")
    outs = {k: out() for k in names}
    fb_frames = [0]
    w_const = torch.full_like(w, 0.75)
    gate = dict(max_iters=MAX_ITERS, stop_iter=GATE_ITERS, stop_frac=GATE_FRACS)

    def run(name):
        o = outs[name]
        if name == "plain_i8_20":
            code.decode(q, frames=F, dtype=ldpc.I8X4, max_iters=MAX_ITERS, early_stop=True, out=o)
        elif name == "plain_f32_20":
            code.decode(llr, dtype=ldpc.F32, max_iters=MAX_ITERS, alpha=0.75, early_stop=True,
                        out=o)
        elif name == "learned":
            code.decode_learned(llr, w, early_stop=True, out=o)
        elif name == "learned_gated":
            code.decode_learned(llr, w, out=o, **gate)
        elif name == "learned_20":
            code.decode_learned(llr, w, out=o, max_iters=MAX_ITERS)
        elif name == "ablation_const_gated":
            code.decode_learned(llr, w_const, out=o, **gate)
        else:
            _, _, fb_frames[0] = code.decode_learned_fallback(llr, w, MAX_ITERS, workspace=wsfb,
                                                              out=(o[0], o[1]))

    steps = max(1, args.steps // 2)
    res = {}
    for name in outs:
        for _ in range(args.warmup):
            run(name)
        barrier()
        a = torch.cuda.Event(enable_timing=True)
        b = torch.cuda.Event(enable_timing=True)
        a.record(stream)
        for _ in range(steps):
            run(name)
        b.record(stream)
        torch.cuda.synchronize()
        barrier()
        ms = a.elapsed_time(b) / steps
        if pg is not None:
            tt = torch.tensor([ms], device=dev)
            pg.all_reduce(tt, op=pg.ReduceOp.MAX)
            ms = float(tt.item())
        mi = T + MAX_ITERS if name == "learned_fallback" else (T if name == "learned" else MAX_ITERS)
        st = reduce_counters(code.frame_stats(info, outs[name][0], outs[name][1], mi).cpu().numpy())
        nf = F * ws
        res[name] = {"value": nf * code.k / (ms * 1e-3) / 1e9, "unit": "Gbit/s", "ms": ms,
                     "fer": float(st[1]) / nf, "wilson95": stats.wilson_interval(int(st[1]), nf),
                     "mean_iters": float(st[3]) / nf}
    res["learned_fallback"]["fallback_frames"] = int(
        reduce_counters(np.array([fb_frames[0]], dtype=np.int64))[0])
    comps = {}
    for plain in ("plain_i8_20", "plain_f32_20"):
        for lrn in names[2:]:
            cnt = reduce_counters(code.paired_frame_errors(info, outs[lrn][0],
                                                           outs[plain][0]).cpu().numpy())
            c = stats.compare(cnt, F * ws)
            c["speedup"] = res[lrn]["value"] / res[plain]["value"]
            comps[f"{lrn}_vs_{plain}"] = c
    wstat = {str(t + 1): {"mean": float(w[t].mean()), "min": float(w[t].min()),
                          "max": float(w[t].max())} for t in range(w.shape[0])}
    return {"workload": LEARNED_WORKLOAD, "frames": F * ws, "T": T,
            "decoders": res, "comparisons": comps, "weights_per_iteration": wstat,
            "decoder_notes": {"learned_gated": f"up to {MAX_ITERS} iterations (rows past T "
                                               "repeat the last), give-up checkpoints "
                                               f"{list(zip(GATE_ITERS, GATE_FRACS))}",
                              "learned_20": f"up to {MAX_ITERS} iterations, no checkpoints",
                              "ablation_const_gated": "learned_gated with every weight 0.75"},
            "matched_fer_test": "exact one-sided McNemar on paired frame outcomes; matched = "
                                "learned not worse at the 5 % level",
            "training": {"steps": cfg.steps, "batch": cfg.batch, "lr": cfg.lr,
                         "ebn0_db": list(cfg.ebn0_db), "init": cfg.init, "seconds": train_s,
                         "loss_first_100": float(hist[:100].mean()),
                         "loss_last_100": float(hist[-100:].mean()),
                         "kernels": "ldpc_learned_train_forward/backward, ldpc_adam_step"}}


MIXED_WORKLOAD = ("WiMAX-shaped mixed set: 76 codes, N = 24 Z for Z = 24..96 step 4, rates "
                  "1/2, 2/3, 3/4, 5/6 (seed 3); frames interleaved at random over the codes "
                  "(seed 3), Eb/N0 uniform in [1.5, 4.5) dB per frame, max 20 iterations, "
                  "early stop")


def mixed_leg(args, ldpc, torch, dev, stream, barrier, rank, ws, pg):
    """Mixed-size batch: one persistent launch per launch group (autotuned,
    captured in a CUDA graph with the quantiser and the error counting),
    against the same frames decoded by one single-code launch per code."""
    from paper_2306_12063_gb300.shard import reduce_counters
    from paper_2306_12063_gb300.workload import make_mixed_batch, mixed_frame_id

    shapes = synth.wimax_mixed_set()
    codes = [ldpc.Code(s.hbm, s.z, device=dev) for s in shapes]
    cs = ldpc.CodeSet(codes)
    F = args.mixed_frames
    from paper_2306_12063_gb300.shard import mixed_shard
    first, cof = mixed_shard(synth.mixed_frame_assignment(len(shapes), F * ws, seed=3)[0], rank,
                             ws)
    plan = ldpc.MixedPlan(cs, cof)
    batch = make_mixed_batch(plan, LEARNED_EBN0, seed=1, frame_base=first)
    q = plan.quantize(batch.llr)
    hard, iters = plan.empty_outputs()
    info_bits = int(plan.info_elems)
    edges_iter = np.array([int((s.hbm >= 0).sum()) * s.z for s in shapes], dtype=np.int64)
    res = {"workload": MIXED_WORKLOAD, "frames": F * ws, "codes": len(shapes),
           "launch_groups": plan.n_groups}
    steps = max(1, args.steps // 2)

    def time_fn(fn):
        for _ in range(args.warmup):
            fn()
        barrier()
        a = torch.cuda.Event(enable_timing=True)
        b = torch.cuda.Event(enable_timing=True)
        a.record(stream)
        for _ in range(steps):
            fn()
        b.record(stream)
        torch.cuda.synchronize()
        barrier()
        ms = a.elapsed_time(b) / steps
        if pg is not None:
            tt = torch.tensor([ms], device=dev)
            pg.all_reduce(tt, op=pg.ReduceOp.MAX)
            ms = float(tt.item())
        return ms

    # per-code reference layout: each code's frames contiguous (single-code kernels)
    counts = np.bincount(cof, minlength=len(shapes))
    per_code = []
    for ci, code in enumerate(codes):
        if counts[ci] == 0:
            continue
        f0 = mixed_frame_id(ci, first)
        inf_c = ldpc.gen_info(1, f0, int(counts[ci]), code.k, device=dev)
        cw = code.encode(inf_c)
        sig = ldpc.snr_sigma(1, f0, int(counts[ci]), LEARNED_EBN0[0], LEARNED_EBN0[1],
                             code.k / code.n, device=dev)
        llr_c = ldpc.awgn_llr_frames(cw, f0, 1, sig)
        per_code.append((code, llr_c, ldpc.quantize_pack_i8(llr_c), int(counts[ci])))
    del cw

    for name, dt, d_in in (("int8", ldpc.I8X4, q), ("fp32", ldpc.F32, batch.llr)):
        t0 = time.time()
        plan.autotune(d_in, dt, max_iters=MAX_ITERS, reps=3, out=(hard, iters))
        groups = plan.autotune(d_in, dt, max_iters=MAX_ITERS, reps=3, out=(hard, iters))
        tune_s = time.time() - t0
        direct_ms = time_fn(lambda: plan.decode(d_in, dt, max_iters=MAX_ITERS,
                                                out=(hard, iters, None)))
        cnt = torch.empty((5 + MAX_ITERS,), dtype=torch.int64, device=dev)
        fe = torch.empty((len(shapes),), dtype=torch.int64, device=dev)
        qg = torch.empty_like(q)
        g = plan.graph(dt, batch.llr, qg if dt == ldpc.I8X4 else None, hard, iters, batch.info,
                       cnt, fe, max_iters=MAX_ITERS)
        graph_ms = time_fn(lambda: g.launch())
        st = reduce_counters(cnt.cpu().numpy())

        def same_contents_direct():
            # the graph's contents launched one by one on the stream
            if dt == ldpc.I8X4:
                plan.quantize(batch.llr, out=qg)
            plan.decode(qg if dt == ldpc.I8X4 else batch.llr, dt, max_iters=MAX_ITERS,
                        out=(hard, iters, None))
            plan.stats(batch.info, hard, iters, MAX_ITERS)

        same_ms = time_fn(same_contents_direct)

        def per_code_step():
            for code, llr_c, q_c, n_c in per_code:
                if dt == ldpc.I8X4:
                    code.decode(q_c, frames=n_c, dtype=dt, max_iters=MAX_ITERS, early_stop=True)
                else:
                    code.decode(llr_c, dtype=dt, max_iters=MAX_ITERS, early_stop=True)

        pc_ms = time_fn(per_code_step)
        nf = F * ws
        it_sum = float(st[3])
        # algorithmic operations of the decode (as for the single-code leg)
        it_host = iters.cpu().numpy().astype(np.int64)
        ops = float(((OPS_PER_EDGE * edges_iter[cof] + OPS_PER_ROW *
                      np.array([s.hbm.shape[0] * s.z for s in shapes])[cof]) * it_host).sum())
        if dt == ldpc.I8X4:
            ops /= 4.0
        res[name] = {"value": info_bits * ws / (direct_ms * 1e-3) / 1e9, "unit": "Gbit/s",
                     "ms": direct_ms,
                     "graph_step": {"value": info_bits * ws / (graph_ms * 1e-3) / 1e9,
                                    "ms": graph_ms,
                                    "contents": ("quantise + " if dt == ldpc.I8X4 else "")
                                    + f"{plan.n_groups} decode launches + error counting",
                                    "same_contents_direct": {
                                        "value": info_bits * ws / (same_ms * 1e-3) / 1e9,
                                        "ms": same_ms}},
                     "per_code_launches": {"value": info_bits * ws / (pc_ms * 1e-3) / 1e9,
                                           "ms": pc_ms, "launches": len(per_code)},
                     "alg_tops": ops / (direct_ms * 1e-3) / 1e12,
                     "alg_frac": ops / (direct_ms * 1e-3) / (SMS * LANES_PER_SM * 2070e6),
                     "alg_unit": ("word-operations (four frames)" if dt == ldpc.I8X4
                                  else "operations (one frame)") + " per second; alg_frac "
                                 f"against {SMS} SMs x {LANES_PER_SM} lanes x 2070 MHz",
                     "fer": float(st[1]) / nf, "mean_iters": it_sum / nf,
                     "autotune_seconds": tune_s, "groups": groups,
                     "serial_groups": plan.serial()[name]}
    return res


SCALE_WORKLOAD = ("learned vs plain at scale: the 76 WiMAX-shaped codes plus the N=648 and "
                  "N=1944 Wi-Fi-shaped codes, frames interleaved at random over the 78 codes "
                  "(seed 3), Eb/N0 uniform in [1.5, 4.5) dB per frame")


def _frame_errors_mixed(ldpc, torch, plan, codes, info, hard):
    """Per-frame info-bit error flags of a mixed batch (bool[frames] on the
    GPU), from the plan layout: analysis of the decoded frames, untimed."""
    dev = hard.device
    err = torch.zeros(plan.frames, dtype=torch.bool, device=dev)
    cof = plan.code_of_frame
    shifts = torch.arange(32, device=dev, dtype=torch.int32)
    for ci, code in enumerate(codes):
        idx = np.nonzero(cof == ci)[0]
        if idx.size == 0:
            continue
        nw = (code.k + 31) // 32
        hw = torch.from_numpy(plan.hard_off[idx]).to(dev)[:, None] + torch.arange(nw, device=dev)
        bits = ((hard[hw].unsqueeze(-1) >> shifts) & 1).reshape(idx.size, -1)[:, :code.k]
        io = torch.from_numpy(plan.info_off[idx]).to(dev)[:, None] + torch.arange(code.k,
                                                                                  device=dev)
        err[torch.from_numpy(idx).to(dev)] = (bits.to(torch.uint8) != info[io]).any(dim=1)
    return err


def _mixed_ebn0(ldpc, torch, plan, codes, first, lo_hi):
    """Per-frame Eb/N0 (dB) of a mixed batch, regenerated with the batch's own
    draws (ldpc_snr_sigma is deterministic in the frame identity)."""
    from paper_2306_12063_gb300.workload import mixed_frame_id
    eb = np.zeros(plan.frames, dtype=np.float64)
    cof = plan.code_of_frame
    for ci, code in enumerate(codes):
        idx = np.nonzero(cof == ci)[0]
        if idx.size == 0:
            continue
        rate = code.k / code.n
        sig = ldpc.snr_sigma(1, mixed_frame_id(ci, first), int(idx.size), lo_hi[0], lo_hi[1], rate,
                             device=codes[0].device).double().cpu().numpy()
        eb[idx] = 10.0 * np.log10(1.0 / (2.0 * rate * sig * sig))
    return eb


EBN0_BINS = (1.5, 2.0, 2.5, 3.0, 3.5, 4.0, 4.5)


def _per_bin(err_np, eb, iters_np):
    out = []
    for lo, hi in zip(EBN0_BINS, EBN0_BINS[1:]):
        m = (eb >= lo) & (eb < hi)
        n = int(m.sum())
        out.append({"ebn0_db": [lo, hi], "frames": n,
                    "fer": float(err_np[m].mean()) if n else None,
                    "mean_iters": float(iters_np[m].mean()) if n else None})
    return out


# Give-up checkpoints of the learned pipeline: at iteration 4 a frame with
# more than 10 % of its checks unsatisfied stops, at iteration 10 one with
# more than 5 %; frames are otherwise decoded up to 20 iterations.
GATE_ITERS = (4, 10)
GATE_FRACS = (0.10, 0.05)


def learned_scale_leg(args, ldpc, torch, dev, stream, barrier, rank, ws, pg):
    """Learned normalised min-sum at scale (per-code weights) against plain
    min-sum at 20 iterations on the same mixed batch.  Decoders, all timed:
    plain int8 / FP32 at 20 iterations; the learned decoder at T_c
    iterations and with its int8 fallback (the recipe's pipeline); and the
    learned pipeline run up to 20 iterations with the give-up checkpoints,
    with weights trained over each code's operating range.  Ablation on the
    same frames: the same pipeline with constant 0.75 weights (plain FP32
    min-sum plus the checkpoints) and with weights trained on the recipe's
    common [1, 4] dB.  FER per Eb/N0 bin, McNemar against plain, the
    weights' statistics per iteration, and the oracle's decode of a subset."""
    from paper_2306_12063_gb300 import stats, train
    from paper_2306_12063_gb300.mixed_learned import decode_learned_fallback
    from paper_2306_12063_gb300.shard import mixed_shard, reduce_counters
    from paper_2306_12063_gb300.workload import make_mixed_batch

    shapes = synth.wimax_mixed_set() + [synth.wifi_n648_r12(), synth.wifi_n1944_r56()]
    codes = [ldpc.Code(s.hbm, s.z, device=dev) for s in shapes]
    cs = ldpc.CodeSet(codes)
    F = args.scale_frames
    first, cof = mixed_shard(synth.mixed_frame_assignment(len(shapes), F * ws, seed=3)[0], rank,
                             ws)
    plan = ldpc.MixedPlan(cs, cof)
    batch = make_mixed_batch(plan, LEARNED_EBN0, seed=1, frame_base=first)
    counts = np.bincount(cof, minlength=len(shapes))
    # per-code training on the library's own generators (bounded budget)
    t0 = time.time()
    # the codes train independently (and deterministically), four at a time
    # on their own streams: one code's small batches leave the GPU mostly idle
    from concurrent.futures import ThreadPoolExecutor
    streams = [torch.cuda.Stream(device=dev) for _ in range(4)]

    def train_code(ci):
        if counts[ci] == 0:
            return None, None, None
        code = codes[ci]
        s = streams[ci % len(streams)]
        with torch.cuda.stream(s):
            T = train.default_iterations(code.k / code.n)
            rng_c = train.operating_range(code, LEARNED_EBN0[0], LEARNED_EBN0[1], stream=s)
            base = dict(T=T, steps=args.scale_train_steps, batch=1024, lr=2e-3, seed=1000 + ci)
            wr = train.train_weights(code, train.TrainConfig(ebn0_db=rng_c, **base), stream=s)
            wc = train.train_weights(code, train.TrainConfig(**base), stream=s)
            s.synchronize()
            return rng_c, wr.weights, wc.weights

    with ThreadPoolExecutor(len(streams)) as ex:
        trained = list(ex.map(train_code, range(len(codes))))
    ranges = [t[0] for t in trained]
    w_range = [t[1] for t in trained]
    w_recipe = [t[2] for t in trained]
    w_const = [None if w is None else torch.full_like(w, 0.75) for w in w_range]
    torch.cuda.synchronize()
    train_s = time.time() - t0
    q = plan.quantize(batch.llr)
    names = ("plain_i8_20", "plain_f32_20", "learned", "learned_fallback", "learned_gated",
             "ablation_const_gated", "ablation_recipe_gated", "ablation_range_20")
    outs = {k: plan.empty_outputs() for k in names}
    plan.autotune(q, ldpc.I8X4, max_iters=MAX_ITERS, reps=2, out=outs["plain_i8_20"])
    plan.autotune(batch.llr, ldpc.F32, max_iters=MAX_ITERS, reps=2, out=outs["plain_f32_20"])
    fbn = [0]
    gate = dict(max_iters=MAX_ITERS, stop_iter=GATE_ITERS, stop_frac=GATE_FRACS)
    weights_of = {"learned": w_range, "learned_fallback": w_range, "learned_gated": w_range,
                  "ablation_const_gated": w_const, "ablation_recipe_gated": w_recipe,
                  "ablation_range_20": w_range}

    def run(name):
        o = outs[name]
        if name == "plain_i8_20":
            plan.decode(q, ldpc.I8X4, max_iters=MAX_ITERS, out=(o[0], o[1], None))
        elif name == "plain_f32_20":
            plan.decode(batch.llr, ldpc.F32, max_iters=MAX_ITERS, out=(o[0], o[1], None))
        elif name == "learned":
            plan.decode_learned(batch.llr, early_stop=True, out=(o[0], o[1], None))
        elif name == "learned_fallback":
            _, _, fbn[0] = decode_learned_fallback(plan, batch.llr, MAX_ITERS, out=o)
        elif name == "ablation_range_20":
            plan.decode_learned(batch.llr, out=(o[0], o[1], None), max_iters=MAX_ITERS)
        else:
            plan.decode_learned(batch.llr, out=(o[0], o[1], None), **gate)


    steps = max(1, args.steps // 4)
    res = {}
    info_bits = plan.info_elems * ws
    nf = F * ws
    eb = _mixed_ebn0(ldpc, torch, plan, codes, first, LEARNED_EBN0)
    errs = {}
    tuned = {}
    for name in names:
        if name in weights_of:
            plan.set_weights(weights_of[name])   # outside the timed region
        if name == "learned":
            # the learned launches share the FP32 items and caps: tune them on
            # the gated learned decoder (plain FP32-20 was timed with its own)
            t1 = time.time()
            plan.autotune_learned(batch.llr, reps=2, out=outs["learned_gated"], **gate)
            tuned = {"seconds": time.time() - t1, "groups": plan.groups()}
        for _ in range(2):
            run(name)
        barrier()
        a = torch.cuda.Event(enable_timing=True)
        b = torch.cuda.Event(enable_timing=True)
        a.record(stream)
        for _ in range(steps):
            run(name)
        b.record(stream)
        torch.cuda.synchronize()
        barrier()
        ms = a.elapsed_time(b) / steps
        if pg is not None:
            tt = torch.tensor([ms], device=dev)
            pg.all_reduce(tt, op=pg.ReduceOp.MAX)
            ms = float(tt.item())
        mi = 28 if name == "learned_fallback" else MAX_ITERS
        cnt, _ = plan.stats(batch.info, outs[name][0], outs[name][1], mi, per_code=False)
        st = reduce_counters(cnt.cpu().numpy())
        e = _frame_errors_mixed(ldpc, torch, plan, codes, batch.info, outs[name][0])
        errs[name] = e
        res[name] = {"value": info_bits / (ms * 1e-3) / 1e9, "unit": "Gbit/s", "ms": ms,
                     "fer": float(st[1]) / nf, "wilson95": stats.wilson_interval(int(st[1]), nf),
                     "mean_iters": float(st[3]) / nf,
                     "per_ebn0_bin": _per_bin(e.cpu().numpy(), eb,
                                              outs[name][1].cpu().numpy())}
    plan.set_weights(w_range)
    res["learned_fallback"]["fallback_frames"] = int(
        reduce_counters(np.array([fbn[0]], dtype=np.int64))[0])
    comps = {}
    for plain in ("plain_i8_20", "plain_f32_20"):
        for lrn in names[2:]:
            cnt = reduce_counters(plan.paired_errors(batch.info, outs[lrn][0],
                                                     outs[plain][0]).cpu().numpy())
            c = stats.compare(cnt, nf)
            c["speedup"] = res[lrn]["value"] / res[plain]["value"]
            comps[f"{lrn}_vs_{plain}"] = c
    wstat = {}
    Tmax = max(w.shape[0] for w in w_range if w is not None)
    for t in range(Tmax):
        rows = torch.cat([w[t] for w in w_range if w is not None and w.shape[0] > t])
        wstat[str(t + 1)] = {"mean": float(rows.mean()), "min": float(rows.min()),
                             "max": float(rows.max())}
    lo_c = [r[0] for r in ranges if r is not None]
    out = {"workload": SCALE_WORKLOAD, "frames": nf, "codes": len(shapes),
           "decoders": res, "comparisons": comps,
           "decoder_notes": {
               "learned": "operating-range weights, T_c iterations (8 up to rate 2/3, else 6)",
               "learned_fallback": "learned, then int8 plain min-sum (20 iterations) on "
                                   "the frames with a nonzero syndrome",
               "learned_gated": f"operating-range weights, up to {MAX_ITERS} iterations "
                                "(rows past T_c repeat the last), give-up checkpoints "
                                f"{list(zip(GATE_ITERS, GATE_FRACS))} (iteration, "
                                "unsatisfied-check fraction of M)",
               "ablation_const_gated": "the learned_gated pipeline with every weight 0.75 "
                                       "(plain FP32 min-sum plus the checkpoints)",
               "ablation_recipe_gated": "the learned_gated pipeline with weights trained on "
                                        "the recipe's common [1, 4] dB",
               "ablation_range_20": "operating-range weights, up to 20 iterations, no "
                                    "checkpoints"},
           "weights_per_iteration": wstat, "learned_autotune": tuned,
           "training": {"per_code": {"steps": args.scale_train_steps, "batch": 1024, "lr": 2e-3,
                                     "T": "8 (R <= 2/3), 6 (R > 2/3)",
                                     "operating_range": "[b, max(b + 1, 4.5)] dB, b the lowest "
                                     "0.25 dB step from 1.5 where plain FP32-20 FER <= 0.5 on "
                                     "4,096 calibration frames",
                                     "recipe_range_db": [1.0, 4.0]},
                        "range_lower_db": {"min": min(lo_c), "max": max(lo_c),
                                           "mean": float(np.mean(lo_c))},
                        "codes_trained": int((counts > 0).sum()), "seconds": train_s}}
    if rank == 0 and args.scale_oracle_frames > 0:
        out["oracle_subset"] = _oracle_learned_subset(plan, shapes, w_range, batch,
                                                      outs["learned_gated"],
                                                      args.scale_oracle_frames, first)
    return out


def _oracle_learned_subset(plan, shapes, weights, batch, gated_out, nsub, frame_base):
    """The oracle's gated learned decode (up to 20 iterations, the give-up
    checkpoints) of the first nsub frames (thread pool over codes), on frames
    the oracle generates itself from the batch's definition (frame j of code
    c at identity c * 2^32 + frame_base + j); the learned weights, the
    decoder's parameters, are the ones the GPU trained.  Reports how many of
    those frames' LLRs equal the GPU batch's, the oracle's FER and how many
    hard decisions and iteration counts equal the GPU's."""
    import oracle
    from concurrent.futures import ThreadPoolExecutor
    nsub = min(nsub, plan.frames)
    cof = plan.code_of_frame[:nsub]
    info_l, llr_l = oracle.mixed_frames(shapes, cof, LEARNED_EBN0, seed=1,
                                        frame_base=frame_base)
    llr = np.concatenate(llr_l)
    info = np.concatenate(info_l)
    gpu_llr = batch.llr[:int(plan.llr_off[nsub])].cpu().numpy()
    inputs_equal = sum(int((gpu_llr[plan.llr_off[f]:plan.llr_off[f + 1]].view(np.uint32) ==
                            llr_l[f].view(np.uint32)).all()) for f in range(nsub))
    gpu_h = gated_out[0][:int(plan.hard_off[nsub])].cpu().numpy().view(np.uint32)
    gpu_i = gated_out[1][:nsub].cpu().numpy()

    def one(ci):
        idx = np.nonzero(cof == ci)[0]
        if idx.size == 0:
            return 0, 0, 0
        s = shapes[ci]
        rc = oracle.RefCode(s.hbm, s.z)
        w = weights[ci].cpu().numpy()
        x = np.stack([llr[plan.llr_off[f]:plan.llr_off[f] + rc.n] for f in idx])
        h, it, _ = rc.decode_learned_f32(x, w, max_iters=MAX_ITERS, stop_iter=GATE_ITERS,
                                         stop_frac=GATE_FRACS, want_post=False)
        bits = oracle.unpack_hard(h, rc.n)
        fe = 0
        same = 0
        for j, f in enumerate(idx):
            ref = info[plan.info_off[f]:plan.info_off[f + 1]]
            fe += int((bits[j][:rc.k] != ref).any())
            same += int((gpu_h[plan.hard_off[f]:plan.hard_off[f + 1]] == h[j]).all() and
                        gpu_i[f] == it[j])
        return idx.size, fe, same

    t0 = time.time()
    with ThreadPoolExecutor(os.cpu_count() or 1) as ex:
        parts = list(ex.map(one, range(len(shapes))))
    n = sum(p[0] for p in parts)
    fe = sum(p[1] for p in parts)
    same = sum(p[2] for p in parts)
    return {"decoder": "learned_gated", "frames": n, "fer": fe / max(n, 1),
            "frames_equal_to_gpu": same, "inputs_equal_to_gpu": inputs_equal,
            "seconds": time.time() - t0}


# Tab. 5 of the paper (data-bit throughput, WiMAX N=2304 R=5/6, fixed 10
# iterations, blocks of 10 codewords per thread): the best float and the best
# fixed-point (int16, Q_B = 10) rows, both on the 16-core AMD Ryzen 9 5950X.
PAPER_TAB5 = {"float_32_threads_mtx_mbps": 37.76, "fixed_32_threads_mtx_mbps": 43.95,
              "hardware": "AMD Ryzen 9 5950X (16 cores / 32 threads), MATLAB R2022a MEX"}


def paper_protocol_leg(args, ldpc, torch, dev, stream, barrier, pg):
    """The paper's throughput protocol (Section 6.2): WiMAX-shaped N=2304
    R=5/6, a fixed 10 iterations without early stop, plain min-sum (eq. 23):
    FP32, the paper's int16 wrap-around fixed point, and the int8 decoder;
    plus the oracle's int16 decoder on the host cores under the same protocol."""
    sh = synth.wimax_n2304_r56()
    code = ldpc.Code(sh.hbm, sh.z, device=dev)
    F = args.paper_frames
    info = ldpc.gen_info(1, 0, F, code.k, device=dev)
    cw = code.encode(info)
    llr = ldpc.awgn_llr(cw, 0, 1, synth.ebn0_db_to_sigma(3.0, code.k / code.n))
    del cw
    q16 = ldpc.quantize_i16(llr, 16.0, 10)
    q8 = ldpc.quantize_pack_i8(llr)
    hard = torch.empty((F, code.nwords), dtype=torch.int32, device=dev)
    iters = torch.empty((F,), dtype=torch.int32, device=dev)
    steps = max(1, args.steps // 2)

    def time_fn(fn):
        for _ in range(args.warmup):
            fn()
        barrier()
        a = torch.cuda.Event(enable_timing=True)
        b = torch.cuda.Event(enable_timing=True)
        a.record(stream)
        for _ in range(steps):
            fn()
        b.record(stream)
        torch.cuda.synchronize()
        barrier()
        ms = a.elapsed_time(b) / steps
        if pg is not None:
            tt = torch.tensor([ms], device=dev)
            pg.all_reduce(tt, op=pg.ReduceOp.MAX)
            ms = float(tt.item())
        return ms

    out = {"workload": f"WiMAX-shaped N=2304 R=5/6 (seed 3), {F} frames at 3.0 dB, fixed 10 "
                       "iterations, no early stop, plain min-sum (eq. 23)",
           "paper_tab5": PAPER_TAB5}
    cases = (("fp32", ldpc.F32, llr, {}), ("int16_wrap", ldpc.I16W, q16, {}),
             ("int8", ldpc.I8X4, q8, {"frames": F}))
    for name, dt, x, kw in cases:
        ms = time_fn(lambda: code.decode(x, dtype=dt, max_iters=10, normalise=False,
                                         early_stop=False, out=(hard, iters, None), **kw))
        g = F * code.k / (ms * 1e-3) / 1e9
        out[name] = {"value": g, "unit": "Gbit/s", "ms": ms,
                     "vs_paper_best_fixed": g * 1e3 / PAPER_TAB5["fixed_32_threads_mtx_mbps"]}
    # the oracle (plain C, one thread per task of 10 codewords) on the host
    import oracle
    from concurrent.futures import ThreadPoolExecutor
    rc = oracle.RefCode(sh.hbm, sh.z)
    nsmp = min(args.paper_oracle_frames, F)
    # the same first frames, generated by the oracle itself (untimed)
    sig = synth.ebn0_db_to_sigma(3.0, rc.k / rc.n)
    x16 = oracle.quantize_i16(oracle.awgn_llr(rc.encode(oracle.gen_info(1, 0, nsmp, rc.k)), 0, 1,
                                              sig), 16.0, 10)
    same = int((x16 == q16[:nsmp].cpu().numpy()).all())
    blocks = [x16[i:i + 10] for i in range(0, nsmp, 10)]
    threads = os.cpu_count() or 1

    def dec(b):
        return rc.decode_layered_i16w(b, 10, normalise=False, early_stop=False,
                                      want_post=False)[1]

    t0 = time.perf_counter()
    with ThreadPoolExecutor(threads) as ex:
        list(ex.map(dec, blocks))
    secs = time.perf_counter() - t0
    out["oracle_int16_host"] = {"value": nsmp * rc.k / secs / 1e9, "unit": "Gbit/s",
                                "cores": threads, "frames": nsmp, "seconds": secs,
                                "inputs_equal_to_gpu": bool(same)}
    return out


def variants_leg(args, ldpc, torch, dev, stream, barrier, code, batch, pg):
    """The paper's variants timed on the same inputs as the main decoders:
    Section 5's int16 wrap-around decoder and the flooding schedule on the
    4.0 dB batch of the N=1944 workload, and the Alg. A1 bitmap encoder
    against the byte encoder on the Z=96, R=5/6 WiMAX-shaped code."""
    steps = max(1, args.steps // 2)

    def time_fn(fn):
        for _ in range(args.warmup):
            fn()
        barrier()
        a = torch.cuda.Event(enable_timing=True)
        b = torch.cuda.Event(enable_timing=True)
        a.record(stream)
        for _ in range(steps):
            fn()
        b.record(stream)
        torch.cuda.synchronize()
        barrier()
        ms = a.elapsed_time(b) / steps
        if pg is not None:
            tt = torch.tensor([ms], device=dev)
            pg.all_reduce(tt, op=pg.ReduceOp.MAX)
            ms = float(tt.item())
        return ms

    F = batch.info.shape[0]
    bits = F * code.k
    out = {"workload": "N=1944 R=5/6 batch at 4.0 dB (" + str(F) + " frames), max 20 iterations, "
                       "early stop; encoder: WiMAX-shaped N=2304 R=5/6 (Z=96), " + str(F) +
                       " frames"}
    q16 = ldpc.quantize_i16(batch.llr, 16.0, 10)
    hard = torch.empty((F, code.nwords), dtype=torch.int32, device=dev)
    iters = torch.empty((F,), dtype=torch.int32, device=dev)
    ms = time_fn(lambda: code.decode(q16, dtype=ldpc.I16W, max_iters=MAX_ITERS, normalise=True,
                                     early_stop=True, out=(hard, iters, None)))
    st = code.frame_stats(batch.info, hard, iters, MAX_ITERS).cpu().numpy()
    out["int16_wrap"] = {"value": bits / (ms * 1e-3) / 1e9, "unit": "Gbit/s", "ms": ms,
                         "fer": float(st[1]) / F, "mean_iters": float(st[3]) / F,
                         "quantiser": "rint(clamp(16 LLR, +-1023)), Q_B = 10",
                         "normalise": "(3m)>>2"}
    fl = {}

    def flood():
        fl["r"] = code.decode_flooding(batch.llr, MAX_ITERS, 0.75, True, True)

    ms = time_fn(flood)
    fh, fi, _ = fl["r"]
    st = code.frame_stats(batch.info, fh, fi, MAX_ITERS).cpu().numpy()
    out["flooding_f32"] = {"value": bits / (ms * 1e-3) / 1e9, "unit": "Gbit/s", "ms": ms,
                           "fer": float(st[1]) / F, "mean_iters": float(st[3]) / F}
    sh = synth.wimax_n2304_r56()
    ec = ldpc.Code(sh.hbm, sh.z, device=dev)
    info = ldpc.gen_info(5, 0, F, ec.k, device=dev)
    words = torch.from_numpy(np.packbits(info.cpu().numpy().reshape(F, ec.k // 8, 8), axis=2,
                                         bitorder="little").reshape(F, ec.k // 8)
                             .view(np.int32)).to(dev)
    cwb = torch.empty((F, ec.n // 32), dtype=torch.int32, device=dev)
    cw = torch.empty((F, ec.n), dtype=torch.uint8, device=dev)
    ms_b = time_fn(lambda: ec.encode_bitmap(words, out=cwb))
    ms_y = time_fn(lambda: ec.encode(info, out=cw))
    out["encoder_bitmap"] = {"value": F * ec.k / (ms_b * 1e-3) / 1e9, "unit": "Gbit/s",
                             "ms": ms_b, "hbm_gbs": F * (ec.k + ec.n) / 8 / (ms_b * 1e-3) / 1e9}
    out["encoder_bytes"] = {"value": F * ec.k / (ms_y * 1e-3) / 1e9, "unit": "Gbit/s",
                            "ms": ms_y, "hbm_gbs": F * (ec.k + ec.n) / (ms_y * 1e-3) / 1e9}
    return out


def reference_arm(args):
    ws, rank, _ = _dist()
    if rank != 0:
        return
    threads = os.cpu_count() or 1
    frames = args.ref_frames
    for _ in range(args.warmup):
        run_oracle_sample(min(frames, 200), 4.0, threads)
    bits = 0
    secs = 0.0
    for _ in range(args.steps):
        b, s = run_oracle_sample(frames, 4.0, threads)
        bits += b
        secs += s
    gbps = bits / secs / 1e9
    sample = (f"{frames} frames of the 4.0 dB batch per step, int8, max 20 iterations, "
              f"early stop, {threads} threads in blocks of 10 frames")
    line = {"impl": "reference", "metric": METRIC, "value": gbps, "unit": "Gbit/s",
            "n_gpus": args.gpus, "steps": args.steps, "warmup": args.warmup,
            "ms_per_step": 1e3 * secs / max(args.steps, 1), "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "int8", "data": "synthetic",
            "config": {"workload": WORKLOAD},
            "cpu_baseline": {"value": gbps, "unit": "Gbit/s", "cores": threads,
                             "kind": "oracle", "sample": sample},
            "e2e": {"value": gbps, "unit": "Gbit/s", "h2d_bytes_per_step": 0,
                    "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)


# --------------------------------------------------------------------------- profiling

def profile_cases():
    """Small, reproducible cases that launch each decoder-family kernel exactly
    once (after generating its inputs), for a kernel profiler's name filter
    (``python bench.py --profile-cases``):

    1. learned FP32 decoder (`decode_f32_kernel<8, true>`), N=648, 65,536 frames,
       T = 8, weights 0.8, Eb/N0 uniform in [1.5, 4.5) dB, a fixed 8
       iterations; then the plain FP32 decoder (`decode_f32_kernel<8, false>`)
       on the same frames, also a fixed 8 iterations (the two launches' counts
       compare per frame-iteration);
    2. mixed int8 and FP32 decoders (`mixed_i8_kernel`, `mixed_f32_kernel`) on
       the four R=3/4 WiMAX-shaped codes with Z = 84..96 (one launch group),
       65,536 frames;
    3. Section 5 int16 wrap-around decoder (`decode_i16x2_kernel`, two frames
       per word), N=1944, 65,536 frames at 4.0 dB;
    4. flooding FP32 decoder (`decode_flooding_kernel`), N=648, 16,384 frames,
       10 iterations;
    5. Alg. A1 bitmap encoder (`encode_bitmap_kernel`), N=2304 R=5/6, 262,144
       frames;
    6. one training step (`train_forward_kernel`, `train_backward_kernel`),
       N=648, batch 4,096, T = 8.

    Every input is generated on the GPU by the library's own kernels first
    (those kernels are not among the names above).
    """
    import torch

    import synth
    from paper_2306_12063_gb300 import (F32, I8X4, I16W, Code, CodeSet, MixedPlan, awgn_llr,
                                        awgn_llr_frames, gen_info, load, quantize_i16,
                                        snr_sigma, _build)
    from paper_2306_12063_gb300.workload import make_mixed_batch

    _build.build()
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
    c648.decode_learned(llr648, w, early_stop=False)
    c648.decode(llr648, max_iters=8, early_stop=False)
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
    from paper_2306_12063_gb300.train import TrainConfig, train_weights
    train_weights(c648, TrainConfig(T=8, steps=1, batch=4096))
    torch.cuda.synchronize()
    print("profiling cases done")


# --------------------------------------------------------------------------- GPU arm

def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=10)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--frames", type=int, default=262144, help="frames per Eb/N0 batch")
    ap.add_argument("--ref-frames", type=int, default=32768,
                    help="frames per step of the CPU reference arm")
    ap.add_argument("--cpu-baseline-frames", type=int, default=262144,
                    help="frames of the CPU-baseline sample (the whole 4.0 dB batch)")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-e2e", action="store_true")
    ap.add_argument("--no-fp32", action="store_true")
    ap.add_argument("--no-learned", action="store_true")
    ap.add_argument("--learned-frames", type=int, default=262144)
    ap.add_argument("--no-mixed", action="store_true")
    ap.add_argument("--no-variants", action="store_true")
    ap.add_argument("--no-scale", action="store_true")
    ap.add_argument("--no-paper", action="store_true")
    ap.add_argument("--paper-frames", type=int, default=262144)
    ap.add_argument("--paper-oracle-frames", type=int, default=40000)
    ap.add_argument("--e2e-chunk", type=int, default=131072,
                    help="frames per chunk of the end-to-end host pipeline")
    ap.add_argument("--scale-frames", type=int, default=1048576)
    ap.add_argument("--scale-train-steps", type=int, default=300)
    ap.add_argument("--scale-oracle-frames", type=int, default=10000)
    ap.add_argument("--mixed-frames", type=int, default=65536)
    ap.add_argument("--profile-cases", action="store_true",
                    help="launch each decoder-family kernel once on a small case (for ncu)")
    args = ap.parse_args()
    if args.profile_cases:
        return profile_cases()
    if args.warmup < 3:
        args.warmup = 3
    if args.impl == "reference":
        return reference_arm(args)

    ws, rank, local = _dist()
    import torch
    import paper_2306_12063_gb300 as ldpc
    from paper_2306_12063_gb300 import _build
    from paper_2306_12063_gb300.shard import frame_offset, reduce_counters
    from paper_2306_12063_gb300.workload import make_batch

    assert torch.cuda.is_available(), "bench.py needs a GPU"
    torch.cuda.set_device(local)
    if rank == 0:
        _build.build()   # the other ranks wait at the barrier below, then load it
    pg = None
    if ws > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl")
        pg = dist
        dist.barrier()
    ldpc.load()

    shape = synth.wifi_n1944_r56()
    code = ldpc.Code(shape.hbm, shape.z, device=f"cuda:{local}")
    E = sum(int((shape.hbm[i] >= 0).sum()) for i in range(shape.mb)) * shape.z
    F = args.frames
    assert F % 4 == 0   # batch b's packed words start at row b F / 4 of q_all
    dev = torch.device("cuda", local)
    nall = len(EBN0) * F
    q_all = torch.empty((nall // 4, code.n), dtype=torch.int32, device=dev)
    llr_all = None if args.no_fp32 else torch.empty((nall, code.n), dtype=torch.float32,
                                                    device=dev)
    batches = []
    for b, eb in enumerate(EBN0):
        frame0 = frame_offset(rank, b, F, len(EBN0))
        bt = make_batch(code, F, frame0, eb, keep_cw=False)
        # the batch's rows move into the step's buffers; bt keeps views
        q_all[b * F // 4:(b + 1) * F // 4] = bt.q
        bt.q = q_all[b * F // 4:(b + 1) * F // 4]
        if llr_all is not None:
            llr_all[b * F:(b + 1) * F] = bt.llr
            bt.llr = llr_all[b * F:(b + 1) * F]
        else:
            bt.llr = None
        batches.append(bt)
    torch.cuda.synchronize()
    hard_all = torch.empty((nall, code.nwords), dtype=torch.int32, device=dev)
    iters_all = torch.empty((nall,), dtype=torch.int32, device=dev)
    outs = [(hard_all[b * F:(b + 1) * F], iters_all[b * F:(b + 1) * F], None)
            for b in range(len(EBN0))]
    stream = torch.cuda.current_stream()

    def barrier():
        torch.cuda.synchronize()
        if pg is not None:
            pg.barrier()
        torch.cuda.synchronize()

    def step(dtype, events=None):
        # the three batches in one call: one launch
        if events is not None:
            events[0].record(stream)
        if dtype == ldpc.I8X4:
            code.decode(q_all, frames=nall, dtype=ldpc.I8X4, max_iters=MAX_ITERS,
                        early_stop=True, out=(hard_all, iters_all, None))
        else:
            code.decode(llr_all, dtype=ldpc.F32, max_iters=MAX_ITERS, early_stop=True,
                        out=(hard_all, iters_all, None))
        if events is not None:
            events[1].record(stream)

    def timed(dtype, steps):
        for _ in range(args.warmup):
            step(dtype)
        barrier()
        ev = [[torch.cuda.Event(enable_timing=True) for _ in range(2)] for _ in range(steps)]
        t0 = torch.cuda.Event(enable_timing=True)
        t1 = torch.cuda.Event(enable_timing=True)
        with ClockSampler(local) as clk:
            t0.record(stream)
            for s in range(steps):
                step(dtype, ev[s])
            t1.record(stream)
            torch.cuda.synchronize()
        barrier()
        total_ms = t0.elapsed_time(t1)
        kern_ms = [e[0].elapsed_time(e[1]) for e in ev]
        if pg is not None:
            tt = torch.tensor([total_ms], device=dev)
            pg.all_reduce(tt, op=pg.ReduceOp.MAX)
            total_ms = float(tt.item())
        iters_sum = int(iters_all.sum().item())
        return total_ms, kern_ms, iters_sum, clk.summary()

    res = {}
    i8_ms, i8_kern, i8_iters, i8_clk = timed(ldpc.I8X4, args.steps)
    bits_per_step = len(EBN0) * F * code.k * ws
    value = bits_per_step * args.steps / (i8_ms * 1e-3) / 1e9

    # FER / iteration statistics of the last decode (not timed)
    fer = {}
    for i, (eb, bt) in enumerate(zip(EBN0, batches)):
        st = code.frame_stats(bt.info, outs[i][0], outs[i][1], MAX_ITERS).cpu().numpy()
        st = reduce_counters(st)          # summed over ranks (each decodes its own frames)
        nf = F * ws
        fer[str(eb)] = {"fer": float(st[1]) / nf, "ber": float(st[0]) / (nf * code.k),
                        "undetected_frames": int(st[2]), "mean_iters": float(st[3]) / nf,
                        "iters_hist": [int(x) for x in st[4:]]}

    clk = i8_clk or {}
    mhz = clk.get("sm_mhz") or 2070.0
    peak_tops = SMS * LANES_PER_SM * mhz * 1e6 / 1e12
    launch_s = (sum(i8_kern) / len(i8_kern)) * 1e-3
    ops_per_launch = _alg_ops(E, code.m, i8_iters, True)   # one launch per step
    ach_tops = ops_per_launch / launch_s / 1e12
    roofline = {"bound": "alu", "achieved": ach_tops, "peak": peak_tops, "unit": "Tops/s",
                "frac": ach_tops / peak_tops,
                "traffic": _profile_traffic("ldpc_decode_i8_wifi1944"),
                "kernel": "decode_i8_kernel<20, 19> (int8, four frames per word; 19 edge slots, the code's largest row degree)",
                "peak_basis": f"{SMS} SMs x {LANES_PER_SM} lanes x {mhz:.0f} MHz "
                              "(median SM clock sampled during the timed region)",
                "hbm_gbs": ((nall // 4) * code.n * 4 + nall * (code.nwords * 4 + 4))
                           / launch_s / 1e9,
                "hbm_frac_of_measured": None}
    try:
        peaks = json.load(open(os.path.join(ROOT, "MEASURED_PEAKS.json")))
        roofline["hbm_frac_of_measured"] = roofline["hbm_gbs"] / float(peaks["hbm_gbs"])
    except (OSError, KeyError, ValueError):
        pass

    if not args.no_fp32:
        f_steps = max(1, args.steps // 2)
        f_ms, f_kern, f_iters, f_clk = timed(ldpc.F32, f_steps)
        f_launch = (sum(f_kern) / len(f_kern)) * 1e-3
        f_ops = _alg_ops(E, code.m, f_iters, False)
        f_mhz = (f_clk or {}).get("sm_mhz") or mhz
        f_peak = SMS * LANES_PER_SM * f_mhz * 1e6 / 1e12
        res["fp32"] = {"value": bits_per_step * f_steps / (f_ms * 1e-3) / 1e9,
                       "unit": "Gbit/s", "steps": f_steps, "ms_per_step": f_ms / f_steps,
                       "roofline": {"bound": "alu", "achieved": f_ops / f_launch / 1e12,
                                    "peak": f_peak, "unit": "Tops/s",
                                    "frac": f_ops / f_launch / 1e12 / f_peak,
                                    "traffic": _profile_traffic("ldpc_decode_f32_wifi1944")},
                       "mean_iters": f_iters / (len(EBN0) * F)}

    e2e = None
    if not args.no_e2e:
        # the step's packed words in one pinned buffer: one pipelined call per
        # step
        host_q = [q_all.cpu().pin_memory()]
        h_hard = [torch.empty((nall, code.nwords), dtype=torch.int32).pin_memory()]
        h_iters = [torch.empty((nall,), dtype=torch.int32).pin_memory()]
        chunk = args.e2e_chunk
        wsb = torch.empty(code.host_workspace_bytes(ldpc.I8X4, chunk), dtype=torch.uint8,
                          device=dev)

        def e2e_step():
            code.decode_host(host_q[0], nall, ldpc.I8X4, h_hard[0], h_iters[0], wsb, chunk,
                             max_iters=MAX_ITERS, early_stop=True)

        for _ in range(args.warmup):
            e2e_step()
        a = torch.cuda.Event(enable_timing=True)
        b_ = torch.cuda.Event(enable_timing=True)
        e_steps = max(1, args.steps // 2)
        # three timed windows of e_steps steps each; the line reports the
        # median window (the host link is shared with the machine's other
        # GPUs, and a transient there can slow one window) and all three
        windows = []
        for _ in range(3):
            barrier()
            a.record(stream)
            for _ in range(e_steps):
                e2e_step()
            b_.record(stream)
            torch.cuda.synchronize()
            barrier()
            w_ms = a.elapsed_time(b_)
            if pg is not None:
                tt = torch.tensor([w_ms], device=dev)
                pg.all_reduce(tt, op=pg.ReduceOp.MAX)
                w_ms = float(tt.item())
            windows.append(w_ms)
        e_ms = statistics.median(windows)
        # the box's pinned host-to-device copy rate, beside the number: the
        # host link is shared with the machine's other GPUs
        probe = host_q[0].view(-1)[: (256 << 20) // 4]
        probe_d = torch.empty_like(probe, device=dev)
        probe_d.copy_(probe, non_blocking=True)
        a.record(stream)
        for _ in range(3):
            probe_d.copy_(probe, non_blocking=True)
        b_.record(stream)
        torch.cuda.synchronize()
        h2d_gbs = 3 * probe.numel() * 4 / (a.elapsed_time(b_) * 1e-3) / 1e9
        del probe_d
        e2e = {"value": bits_per_step * e_steps / (e_ms * 1e-3) / 1e9, "unit": "Gbit/s",
               "windows": [bits_per_step * e_steps / (w * 1e-3) / 1e9 for w in windows],
               "statistic": f"median of 3 timed windows of {e_steps} steps",
               "h2d_copy_gbs": h2d_gbs,
               "h2d_bytes_per_step": sum(int(h.numel()) * 4 for h in host_q),
               "d2h_bytes_per_step": sum(int(h.numel()) * 4 for h in h_hard) +
               sum(int(h.numel()) * 4 for h in h_iters),
               "steps": e_steps, "chunk_frames": chunk,
               "api": "ldpc_decode_host (pinned host buffers, copies inside the timed region)"}

    if not args.no_learned:
        res["learned"] = learned_leg(args, ldpc, torch, dev, stream, barrier, rank, ws, pg)
    if not args.no_mixed:
        res["mixed"] = mixed_leg(args, ldpc, torch, dev, stream, barrier, rank, ws, pg)
    if not args.no_scale:
        res["learned_scale"] = learned_scale_leg(args, ldpc, torch, dev, stream, barrier, rank,
                                                 ws, pg)
    if not args.no_paper:
        res["paper_protocol"] = paper_protocol_leg(args, ldpc, torch, dev, stream, barrier, pg)
    if not args.no_variants and not args.no_fp32:
        res["variants"] = variants_leg(args, ldpc, torch, dev, stream, barrier, code, batches[1],
                                       pg)

    cpu = None
    if rank == 0 and ws == 1 and not args.no_cpu_baseline:
        threads = os.cpu_count() or 1
        nf = args.cpu_baseline_frames
        bits, secs = run_oracle_sample(nf, 4.0, threads)
        n1 = max(10, nf // 16)
        bits1, secs1 = run_oracle_sample(n1, 4.0, 1)
        cpu = {"value": bits / secs / 1e9, "unit": "Gbit/s", "cores": threads,
               "kind": "oracle", "seconds": secs,
               "sample": f"{nf} frames of the 4.0 dB batch, int8, max 20 "
                         f"iterations, early stop, {threads} threads, blocks of 10 frames",
               "single_thread": {"value": bits1 / secs1 / 1e9, "unit": "Gbit/s",
                                 "frames": n1, "seconds": secs1}}

    if rank == 0:
        line = {"metric": METRIC, "metric_basis": METRIC_BASIS, "value": value,
                "unit": "Gbit/s", "n_gpus": ws,
                "steps": args.steps, "warmup": args.warmup,
                "ms_per_step": i8_ms / args.steps, "higher_is_better": True,
                "scaling": "weak", "vs_baseline": None, "dtype": "int8", "data": "synthetic",
                "config": {"workload": WORKLOAD, "frames_per_step_per_gpu": len(EBN0) * F,
                           "decoder": "int8 packed 4 frames/word, normalisation (3m)>>2",
                           "parallelism": f"frames sharded over {ws} GPU(s), no collective",
                           "launches_per_step": 1,
                           "l2": "inputs larger than L2 (1.5 GB of packed LLRs per step)"},
                "roofline": roofline, "cpu_baseline": cpu, "e2e": e2e,
                "gpu_launches": args.steps, "clocks": i8_clk,
                "mean_iters": i8_iters / (len(EBN0) * F), "fer": fer}
        line.update(res)
        lvp = {}
        for key, leg in (("mixed_78_codes", "learned_scale"), ("n648", "learned")):
            if leg not in res:
                continue
            L = res[leg]
            dec = L["decoders"]
            c32 = L["comparisons"]["learned_gated_vs_plain_f32_20"]
            c8 = L["comparisons"]["learned_gated_vs_plain_i8_20"]
            lvp[key] = {"workload": L["workload"], "learned_decoder": "learned_gated",
                        "value": dec["learned_gated"]["value"],
                        "plain_f32_20": dec["plain_f32_20"]["value"],
                        "ratio_vs_plain_f32_20": c32["speedup"], "matched_f32": c32["matched"],
                        "mcnemar_p_learned_worse_f32": c32["mcnemar_p_a_worse"],
                        "fer": dec["learned_gated"]["fer"],
                        "fer_plain_f32_20": dec["plain_f32_20"]["fer"],
                        "plain_i8_20": dec["plain_i8_20"]["value"],
                        "ratio_vs_plain_i8_20": c8["speedup"], "matched_i8": c8["matched"],
                        "fer_plain_i8_20": dec["plain_i8_20"]["fer"]}
        if lvp:
            line["learned_vs_plain"] = lvp
        print(json.dumps(line), flush=True)
    if pg is not None:
        pg.destroy_process_group()


if __name__ == "__main__":
    main()
