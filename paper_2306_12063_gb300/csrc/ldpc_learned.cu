// Learned (neural) normalised min-sum decoding with a plain min-sum fallback.
//
// The paper decodes with plain min-sum (Section 4, eq. 23).  Here the layered
// decoder of ldpc_decode.cu runs T iterations with one trained weight per
// iteration and nonzero block of H_bm scaling the messages; frames whose hard
// decisions still violate a parity check (Section 4, step 4) are then decoded
// again from their channel LLRs by the int8 plain min-sum decoder, and their
// outputs replace the learned ones.
#include <algorithm>

#include "ldpc_internal.cuh"

namespace ldpc {

constexpr unsigned kFull32 = 0xFFFFFFFFu;

// One warp per frame: the parity checks of its hard decisions (eq. 21); a
// frame with any unsatisfied check is appended to `list`.
__global__ void failed_frames_kernel(DevCode c, const uint32_t *__restrict__ hard, int64_t frames,
                                     int32_t *__restrict__ list, unsigned *__restrict__ count) {
    const int lane = threadIdx.x & 31;
    const int64_t warps = static_cast<int64_t>(gridDim.x) * (blockDim.x >> 5);
    for (int64_t f = (blockIdx.x * static_cast<int64_t>(blockDim.x) + threadIdx.x) >> 5;
         f < frames; f += warps) {
        const uint32_t *h = hard + f * c.nwords;
        uint32_t bad = 0;
        for (int l = 0; l < c.mb; ++l) {
            const int d = __ldg(c.rowinfo + l) & 255;
            for (int t = 0; t < c.rpl; ++t) {
                if (lane + 32 * t >= c.z) continue;
                uint32_t par = 0;
                for (int e = 0; e < d; ++e) {
                    const int slot = c.dslots - d + e;
                    const int v = c.voff[((l * c.rpl + t) * c.dslots + slot) * 32 + lane] >> 2;
                    par ^= (h[v >> 5] >> (v & 31)) & 1u;
                }
                bad |= par;
            }
        }
        if (__any_sync(kFull32, bad) && lane == 0) list[atomicAdd(count, 1u)] = static_cast<int32_t>(f);
    }
}

// Packs the listed frames' LLRs as int8, four frames per word, like
// ldpc_quantize_pack_i8: q = rint(clamp(scale * llr, -clip, clip)).
__global__ void gather_quantize_kernel(const float *__restrict__ llr, int n,
                                       const int32_t *__restrict__ list, int64_t cnt, float scale,
                                       int clip, uint32_t *__restrict__ q) {
    const int64_t groups = (cnt + 3) / 4;
    const float fc = static_cast<float>(clip);
    for (int64_t t = blockIdx.x * static_cast<int64_t>(blockDim.x) + threadIdx.x;
         t < groups * n; t += static_cast<int64_t>(gridDim.x) * blockDim.x) {
        const int64_t g = t / n;
        const int p = static_cast<int>(t - g * n);
        uint32_t word = 0;
#pragma unroll
        for (int b = 0; b < 4; ++b) {
            int v = clip;
            if (4 * g + b < cnt) {
                const int64_t f = list[4 * g + b];
                float x = __fmul_rn(scale, llr[f * n + p]);
                x = fminf(fmaxf(x, -fc), fc);
                v = __float2int_rn(x);
            }
            word |= (static_cast<uint32_t>(v) & 0xFFu) << (8 * b);
        }
        q[t] = word;
    }
}

// Writes the fallback outputs back to the listed frames; their iteration
// count becomes T plus the fallback's.
__global__ void scatter_kernel(const int32_t *__restrict__ list, int64_t cnt, int nwords,
                               const uint32_t *__restrict__ hard_fb,
                               const int32_t *__restrict__ iters_fb, int T,
                               uint32_t *__restrict__ hard, int32_t *__restrict__ iters) {
    for (int64_t t = blockIdx.x * static_cast<int64_t>(blockDim.x) + threadIdx.x;
         t < cnt * nwords; t += static_cast<int64_t>(gridDim.x) * blockDim.x) {
        const int64_t i = t / nwords;
        const int w = static_cast<int>(t - i * nwords);
        const int64_t f = list[i];
        hard[f * nwords + w] = hard_fb[t];
        if (w == 0) iters[f] = T + iters_fb[i];
    }
}

static int grid_for(int64_t work, int threads) {
    int dev = 0, sms = 148;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    const int64_t want = (work + threads - 1) / threads;
    return static_cast<int>(std::min<int64_t>(std::max<int64_t>(want, 1), 32LL * sms));
}

static size_t a256(size_t x) { return (x + 255) & ~static_cast<size_t>(255); }

struct FallbackSpace {
    unsigned *count;
    int32_t *list;
    uint32_t *q;
    uint32_t *hard;
    int32_t *iters;
    size_t bytes;
};

static FallbackSpace fallback_space(const Code &c, int64_t frames, void *base) {
    FallbackSpace s;
    char *p = static_cast<char *>(base);
    size_t off = 0;
    auto take = [&](size_t b) {
        char *r = p ? p + off : nullptr;
        off += a256(b);
        return r;
    };
    const int nw = (c.n + 31) / 32;
    s.count = reinterpret_cast<unsigned *>(take(sizeof(unsigned)));
    s.list = reinterpret_cast<int32_t *>(take(sizeof(int32_t) * frames));
    s.q = reinterpret_cast<uint32_t *>(take(sizeof(uint32_t) * ((frames + 3) / 4) * c.n));
    s.hard = reinterpret_cast<uint32_t *>(take(sizeof(uint32_t) * frames * nw));
    s.iters = reinterpret_cast<int32_t *>(take(sizeof(int32_t) * frames));
    s.bytes = off;
    return s;
}

size_t learned_fallback_workspace(const Code &c, int64_t frames) {
    return fallback_space(c, frames, nullptr).bytes;
}

ldpc_status learned_fallback(const Code &c, const float *d_llr, int64_t frames,
                             const DecodeParams &learned, const DecodeParams &fb, float scale,
                             int clip, uint32_t *d_hard, int32_t *d_iters, int64_t *h_count,
                             void *d_ws, cudaStream_t s) {
    ldpc_status st = launch_decode_learned(c, d_llr, frames, learned, d_hard, d_iters, nullptr, s);
    if (st) return st;
    FallbackSpace w = fallback_space(c, frames, d_ws);
    cudaError_t e = cudaMemsetAsync(w.count, 0, sizeof(unsigned), s);
    if (e != cudaSuccess) return cuda_fail(e, "cudaMemsetAsync fallback count");
    failed_frames_kernel<<<grid_for(frames * 32, 256), 256, 0, s>>>(dev_view(c), d_hard, frames,
                                                                    w.list, w.count);
    if ((e = cudaGetLastError()) != cudaSuccess) return cuda_fail(e, "failed_frames_kernel");
    unsigned cnt = 0;
    e = cudaMemcpyAsync(&cnt, w.count, sizeof(unsigned), cudaMemcpyDeviceToHost, s);
    if (e == cudaSuccess) e = cudaStreamSynchronize(s);
    if (e != cudaSuccess) return cuda_fail(e, "reading the fallback count");
    if (h_count) *h_count = cnt;
    if (cnt == 0) return LDPC_OK;
    const int64_t n = cnt;
    gather_quantize_kernel<<<grid_for(((n + 3) / 4) * c.n, 256), 256, 0, s>>>(
        d_llr, c.n, w.list, n, scale, clip, w.q);
    if ((e = cudaGetLastError()) != cudaSuccess) return cuda_fail(e, "gather_quantize_kernel");
    st = launch_decode(c, LDPC_I8X4, w.q, n, fb, w.hard, w.iters, nullptr, s);
    if (st) return st;
    const int nw = (c.n + 31) / 32;
    scatter_kernel<<<grid_for(n * nw, 256), 256, 0, s>>>(w.list, n, nw, w.hard, w.iters,
                                                         learned.max_iters, d_hard, d_iters);
    if ((e = cudaGetLastError()) != cudaSuccess) return cuda_fail(e, "scatter_kernel");
    return LDPC_OK;
}

static ldpc_status learned_params(const ldpc_code *code, int64_t frames, const float *d_weights,
                                  int T, int early_stop, DecodeParams *p, const char *who) {
    if (!code) return fail(LDPC_ERR_INVALID_ARG, std::string(who) + ": code is NULL");
    if (frames < 0) return fail(LDPC_ERR_INVALID_ARG, std::string(who) + ": frames < 0");
    if (T < 1 || T > kMaxIters)
        return fail(LDPC_ERR_INVALID_ARG, std::string(who) + ": T must be in [1, 1000]");
    if (early_stop != 0 && early_stop != 1)
        return fail(LDPC_ERR_INVALID_ARG, std::string(who) + ": early_stop must be 0 or 1");
    if (frames && !d_weights)
        return fail(LDPC_ERR_INVALID_ARG, std::string(who) + ": weights are NULL");
    if (code->c.max_deg > kMaxRowDeg)
        return fail(LDPC_ERR_UNSUPPORTED, std::string(who) + ": row degree above 27");
    p->max_iters = T;
    p->alpha = 1.0f;
    p->normalise = 0;
    p->early_stop = early_stop;
    p->weights = d_weights;
    p->n_edges = code->c.n_edges;
    return LDPC_OK;
}

ldpc_status learned_run_params(const ldpc_learned_params *lp, DecodeParams *dp, const char *who) {
    if (!lp) return fail(LDPC_ERR_INVALID_ARG, std::string(who) + ": run limits are NULL");
    if (lp->max_iters < 0 || lp->max_iters > kMaxIters)
        return fail(LDPC_ERR_INVALID_ARG, std::string(who) + ": max_iters outside 0..1000");
    if (lp->early_stop != 0 && lp->early_stop != 1)
        return fail(LDPC_ERR_INVALID_ARG, std::string(who) + ": early_stop must be 0 or 1");
    for (int j = 0; j < 2; ++j) {
        if (lp->stop_iter[j] < 0 || lp->stop_iter[j] > kMaxIters)
            return fail(LDPC_ERR_INVALID_ARG, std::string(who) + ": stop_iter outside 0..1000");
        if (lp->stop_iter[j] && (!lp->early_stop || !(lp->stop_frac[j] >= 0.0f) ||
                                 !(lp->stop_frac[j] <= 1e6f)))
            return fail(LDPC_ERR_INVALID_ARG,
                        std::string(who) + ": a checkpoint needs early_stop and stop_frac >= 0");
    }
    dp->max_iters = lp->max_iters;
    dp->alpha = 1.0f;
    dp->normalise = 0;
    dp->early_stop = lp->early_stop;
    for (int j = 0; j < 2; ++j) {
        dp->stop_iter[j] = lp->stop_iter[j];
        dp->stop_frac[j] = lp->stop_iter[j] ? lp->stop_frac[j] : 0.0f;
    }
    return LDPC_OK;
}

}  // namespace ldpc

using namespace ldpc;

extern "C" {

ldpc_status ldpc_decode_learned_minsum_ex(const ldpc_code *code, const float *d_llr,
                                          int64_t frames, const float *d_weights, int T,
                                          const ldpc_learned_params *lp, uint32_t *d_hard,
                                          int32_t *d_iters, float *d_post, cudaStream_t stream) {
    const char *who = "ldpc_decode_learned_minsum_ex";
    DecodeParams p;
    ldpc_status st = learned_params(code, frames, d_weights, T, 0, &p, who);
    if (st) return st;
    st = learned_run_params(lp, &p, who);
    if (st) return st;
    p.weights = d_weights;
    p.n_edges = code->c.n_edges;
    p.weight_iters = T;
    if (p.max_iters == 0) p.max_iters = T;
    if (frames == 0) return LDPC_OK;
    if (!d_llr || !d_hard || !d_iters)
        return fail(LDPC_ERR_INVALID_ARG, std::string(who) + ": NULL buffer");
    cudaError_t e = cudaSetDevice(code->c.device);
    if (e != cudaSuccess) return cuda_fail(e, "cudaSetDevice");
    return launch_decode_learned(code->c, d_llr, frames, p, d_hard, d_iters, d_post, stream);
}

ldpc_status ldpc_decode_learned_minsum(const ldpc_code *code, const float *d_llr, int64_t frames,
                                       const float *d_weights, int T, int early_stop,
                                       uint32_t *d_hard, int32_t *d_iters, float *d_post,
                                       cudaStream_t stream) {
    DecodeParams p;
    ldpc_status st = learned_params(code, frames, d_weights, T, early_stop, &p,
                                    "ldpc_decode_learned_minsum");
    if (st) return st;
    if (frames == 0) return LDPC_OK;
    if (!d_llr || !d_hard || !d_iters)
        return fail(LDPC_ERR_INVALID_ARG, "ldpc_decode_learned_minsum: NULL buffer");
    cudaError_t e = cudaSetDevice(code->c.device);
    if (e != cudaSuccess) return cuda_fail(e, "cudaSetDevice");
    return launch_decode_learned(code->c, d_llr, frames, p, d_hard, d_iters, d_post, stream);
}

size_t ldpc_learned_fallback_workspace_bytes(const ldpc_code *code, int64_t frames) {
    if (!code || frames < 0) return 0;
    return learned_fallback_workspace(code->c, frames);
}

ldpc_status ldpc_decode_learned_fallback(const ldpc_code *code, const float *d_llr,
                                         int64_t frames, const float *d_weights, int T,
                                         const ldpc_decode_params *fallback, float quant_scale,
                                         int quant_clip, uint32_t *d_hard, int32_t *d_iters,
                                         int64_t *h_fallback_frames, void *d_workspace,
                                         size_t workspace_bytes, cudaStream_t stream) {
    const char *who = "ldpc_decode_learned_fallback";
    DecodeParams p;
    ldpc_status st = learned_params(code, frames, d_weights, T, 1, &p, who);
    if (st) return st;
    if (!fallback) return fail(LDPC_ERR_INVALID_ARG, std::string(who) + ": fallback is NULL");
    if (fallback->max_iters < 1 || fallback->max_iters > kMaxIters ||
        (fallback->normalise != 0 && fallback->normalise != 1) ||
        (fallback->early_stop != 0 && fallback->early_stop != 1))
        return fail(LDPC_ERR_INVALID_ARG, std::string(who) + ": bad fallback parameters");
    if (fallback->normalise && fallback->alpha != 0.75f)
        return fail(LDPC_ERR_UNSUPPORTED,
                    std::string(who) + ": the int8 fallback scales by (3m)>>2 (alpha 0.75)");
    if (quant_clip < 0 || quant_clip > 127 || !(quant_scale == quant_scale))
        return fail(LDPC_ERR_INVALID_ARG, std::string(who) + ": bad quantiser parameters");
    if (h_fallback_frames) *h_fallback_frames = 0;
    if (frames == 0) return LDPC_OK;
    if (!d_llr || !d_hard || !d_iters || !d_workspace)
        return fail(LDPC_ERR_INVALID_ARG, std::string(who) + ": NULL buffer");
    if (workspace_bytes < learned_fallback_workspace(code->c, frames))
        return fail(LDPC_ERR_INVALID_ARG, std::string(who) + ": workspace too small");
    cudaError_t e = cudaSetDevice(code->c.device);
    if (e != cudaSuccess) return cuda_fail(e, "cudaSetDevice");
    DecodeParams fb;
    fb.max_iters = fallback->max_iters;
    fb.alpha = fallback->normalise ? fallback->alpha : 1.0f;
    fb.normalise = fallback->normalise;
    fb.early_stop = fallback->early_stop;
    return learned_fallback(code->c, d_llr, frames, p, fb, quant_scale, quant_clip, d_hard,
                            d_iters, h_fallback_frames, d_workspace, stream);
}

}  // extern "C"
