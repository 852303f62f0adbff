// Input generation and evaluation kernels of libldpc: synthetic info bits,
// the direct encoder (arXiv 2306.12063, Section 2, eq. 8-15), BPSK/AWGN
// channel LLRs (eq. 16-17), fixed-point quantisation with four-frame packing,
// and error counting (the evaluation of Section 6.1).
#include <algorithm>

#include "ldpc_decode_dev.cuh"

namespace ldpc {

// ---------------------------------------------------------------------------
// Philox4x32-10 (Salmon, Moraes, Dror & Shaw, SC'11): ten rounds, each with
// two 32x32 -> 64-bit products; the key advances by the Weyl increments
// between rounds.
// ---------------------------------------------------------------------------
__device__ __forceinline__ uint4 philox4x32_10(uint4 ctr, uint2 key) {
#pragma unroll
    for (int round = 0; round < 10; ++round) {
        if (round > 0) {
            key.x += 0x9E3779B9u;
            key.y += 0xBB67AE85u;
        }
        const uint32_t lo0 = 0xD2511F53u * ctr.x, hi0 = __umulhi(0xD2511F53u, ctr.x);
        const uint32_t lo1 = 0xCD9E8D57u * ctr.z, hi1 = __umulhi(0xCD9E8D57u, ctr.z);
        ctr = make_uint4(hi1 ^ ctr.y ^ key.x, lo1, hi0 ^ ctr.w ^ key.y, lo0);
    }
    return ctr;
}

__global__ void gen_info_kernel(uint64_t seed, int64_t frame0, int64_t frames, int k,
                                uint8_t *__restrict__ info) {
    const int calls = (k + 127) / 128;
    const int64_t total = frames * calls;
    const uint2 key = make_uint2(static_cast<uint32_t>(seed),
                                 static_cast<uint32_t>(seed >> 32) ^ 0x494E464Fu);
    for (int64_t t = blockIdx.x * static_cast<int64_t>(blockDim.x) + threadIdx.x; t < total;
         t += static_cast<int64_t>(gridDim.x) * blockDim.x) {
        const int64_t i = t / calls;
        const int c = static_cast<int>(t - i * calls);
        const uint64_t f = static_cast<uint64_t>(frame0 + i);
        const uint4 w = philox4x32_10(
            make_uint4(static_cast<uint32_t>(c), static_cast<uint32_t>(f),
                       static_cast<uint32_t>(f >> 32), 0u),
            key);
        const uint32_t ws[4] = {w.x, w.y, w.z, w.w};
        uint8_t *out = info + i * k;
        const int b0 = c * 128;
        const int nb = min(128, k - b0);
        for (int b = 0; b < nb; ++b) out[b0 + b] = (ws[b >> 5] >> (b & 31)) & 1u;
    }
}

// ---------------------------------------------------------------------------
// Direct encoder, one warp per frame.  Shared memory per warp: the info bits
// u (K bytes), S_i for every block row (Mb Z bytes, eq. 15) and v_0 (Z).
// ---------------------------------------------------------------------------
constexpr int kEncWarps = 4;

__global__ void __launch_bounds__(kEncWarps * 32)
    encode_kernel(DevCode c, const uint8_t *__restrict__ info, uint8_t *__restrict__ cw,
                  int64_t frames, int warp_bytes) {
    extern __shared__ __align__(16) uint8_t esm[];
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    uint8_t *u = esm + warp * warp_bytes;
    uint8_t *S = u + c.k;
    uint8_t *v0 = S + c.mb * c.z;
    const int z = c.z, kb = c.kb, nb = c.nb;
    for (int64_t f = blockIdx.x * static_cast<int64_t>(kEncWarps) + warp; f < frames;
         f += static_cast<int64_t>(gridDim.x) * kEncWarps) {
        const uint8_t *src = info + f * c.k;
        uint8_t *dst = cw + f * c.n;
        for (int t = lane; t < c.k; t += 32) {     // systematic part, eq. (1)
            const uint8_t b = src[t] & 1u;
            u[t] = b;
            dst[t] = b;
        }
        __syncwarp();
        // eq. (15): S_i[r] = sum_j u_j[(r + H(i,j)) mod Z] over the info columns
        for (int q = lane; q < c.mb * z; q += 32) {
            const int i = q / z, r = q - i * z;
            uint32_t acc = 0;
            for (int j = 0; j < kb; ++j) {
                const int s = c.hbm[i * nb + j];
                if (s < 0) continue;
                int p = r + s;
                p = p >= z ? p - z : p;
                acc ^= u[j * z + p];
            }
            S[q] = static_cast<uint8_t>(acc);
        }
        __syncwarp();
        // eq. (12): v_0 = P^{-1}_{H(y,Kb)} sum_i S_i, i.e. v_0[r] = T[(r - b) mod Z]
        const int b = c.hbm[c.y * nb + kb];
        for (int r = lane; r < z; r += 32) {
            int p = r - b;
            p = p < 0 ? p + z : p;
            uint32_t t = 0;
            for (int i = 0; i < c.mb; ++i) t ^= S[i * z + p];
            v0[r] = static_cast<uint8_t>(t);
            dst[c.k + r] = static_cast<uint8_t>(t);
        }
        __syncwarp();
        // eq. (13)-(14): v_1 = P_{H(0,Kb)} v_0 + S_0; v_{i+1} = v_i + P_{H(i,Kb)} v_0 + S_i
        for (int r = lane; r < z; r += 32) {
            uint32_t v = 0;
            for (int i = 0; i < c.mb - 1; ++i) {
                const int s = c.hbm[i * nb + kb];
                uint32_t pv = 0;
                if (s >= 0) {
                    int p = r + s;
                    p = p >= z ? p - z : p;
                    pv = v0[p];
                }
                v = (i == 0 ? 0u : v) ^ pv ^ S[i * z + r];
                dst[c.k + (i + 1) * z + r] = static_cast<uint8_t>(v);
            }
        }
        __syncwarp();
    }
}

// ---------------------------------------------------------------------------
// Channel.  The Gaussian numbers come from Box-Muller (1958) on Philox words.
// ln and sin/cos are evaluated here from their series with one correctly
// rounded float operation per step, so every machine that follows the same
// steps gets the same bits.
// ---------------------------------------------------------------------------

// ln u for a positive normal float: u = m 2^e with m in [sqrt(1/2), sqrt(2)),
// ln m = 2 atanh(t), t = (m - 1)/(m + 1), odd series through t^11.
__device__ __forceinline__ float series_lnf(float u) {
    const uint32_t bits = __float_as_uint(u);
    int e = static_cast<int>((bits >> 23) & 0xFFu) - 127;
    uint32_t mbits = (bits & 0x007FFFFFu) | 0x3F800000u;
    if (mbits > 0x3FB504F3u) {   // m > sqrt(2): halve it
        mbits -= 0x00800000u;
        e += 1;
    }
    const float m = __uint_as_float(mbits);
    const float t = __fdiv_rn(__fsub_rn(m, 1.0f), __fadd_rn(m, 1.0f));
    const float t2 = __fmul_rn(t, t);
    float s = 0x1.745d18p-4f;                                  // 1/11
    s = __fadd_rn(__fmul_rn(s, t2), 0x1.c71c72p-4f);           // 1/9
    s = __fadd_rn(__fmul_rn(s, t2), 0x1.24924ap-3f);           // 1/7
    s = __fadd_rn(__fmul_rn(s, t2), 0x1.99999ap-3f);           // 1/5
    s = __fadd_rn(__fmul_rn(s, t2), 0x1.555556p-2f);           // 1/3
    s = __fadd_rn(__fmul_rn(s, t2), 1.0f);
    const float lnm = __fmul_rn(__fmul_rn(2.0f, t), s);
    return __fadd_rn(__fmul_rn(static_cast<float>(e), 0x1.62e430p-1f), lnm);   // + e ln 2
}

// sin and cos of 2 pi k / 2^24: exact split into a quadrant and a remainder,
// remainder reflected into [0, pi/4], Taylor series of sin (to x^11) and cos
// (to x^12) in the reduced angle.
__device__ __forceinline__ void series_sincos_turn(uint32_t k24, float *s_out, float *c_out) {
    const uint32_t q = (k24 >> 22) & 3u;
    const uint32_t rem = k24 & 0x3FFFFFu;
    const bool swap = rem > 0x200000u;
    const uint32_t red = swap ? 0x400000u - rem : rem;
    const float phi = __fmul_rn(static_cast<float>(red), 0x1.921fb6p-22f);   // pi / 2^23
    const float x = __fmul_rn(phi, phi);
    float ps = -0x1.ae6456p-26f;
    ps = __fadd_rn(__fmul_rn(ps, x), 0x1.71de3ap-19f);
    ps = __fadd_rn(__fmul_rn(ps, x), -0x1.a01a02p-13f);
    ps = __fadd_rn(__fmul_rn(ps, x), 0x1.111112p-7f);
    ps = __fadd_rn(__fmul_rn(ps, x), -0x1.555556p-3f);
    ps = __fadd_rn(__fmul_rn(ps, x), 1.0f);
    const float sinp = __fmul_rn(phi, ps);
    float pc = 0x1.1eed8ep-29f;
    pc = __fadd_rn(__fmul_rn(pc, x), -0x1.27e4fcp-22f);
    pc = __fadd_rn(__fmul_rn(pc, x), 0x1.a01a02p-16f);
    pc = __fadd_rn(__fmul_rn(pc, x), -0x1.6c16c2p-10f);
    pc = __fadd_rn(__fmul_rn(pc, x), 0x1.555556p-5f);
    pc = __fadd_rn(__fmul_rn(pc, x), -0.5f);
    pc = __fadd_rn(__fmul_rn(pc, x), 1.0f);
    const float ct = swap ? sinp : pc;
    const float st = swap ? pc : sinp;
    float cs, sn;
    switch (q) {
        case 0: cs = ct; sn = st; break;
        case 1: cs = -st; sn = ct; break;
        case 2: cs = -ct; sn = -st; break;
        default: cs = st; sn = -ct; break;
    }
    *s_out = sn;
    *c_out = cs;
}

__device__ __forceinline__ void box_muller(uint32_t w0, uint32_t w1, float *g0, float *g1) {
    const float u1 = __fmul_rn(static_cast<float>((w0 >> 8) + 1u), 0x1p-24f);
    const float r = __fsqrt_rn(__fmul_rn(-2.0f, series_lnf(u1)));
    float s, co;
    series_sincos_turn(w1 >> 8, &s, &co);
    *g0 = __fmul_rn(r, co);
    *g1 = __fmul_rn(r, s);
}

// sigmas == NULL: every frame uses (sigma, scale); otherwise frame i uses
// sigma = sigmas[i] and scale = 2 / sigma^2 (eq. 17), each operation rounded
// once.
__global__ void awgn_kernel(const uint8_t *__restrict__ cw, int64_t frame0, int64_t frames,
                            int n, uint64_t seed, float sigma, float scale,
                            const float *__restrict__ sigmas, float *__restrict__ llr) {
    const int calls = (n + 3) / 4;
    const int64_t total = frames * calls;
    const uint2 key = make_uint2(static_cast<uint32_t>(seed),
                                 static_cast<uint32_t>(seed >> 32) ^ 0x4E4F4953u);
    for (int64_t t = blockIdx.x * static_cast<int64_t>(blockDim.x) + threadIdx.x; t < total;
         t += static_cast<int64_t>(gridDim.x) * blockDim.x) {
        const int64_t i = t / calls;
        const int c = static_cast<int>(t - i * calls);
        const uint64_t f = static_cast<uint64_t>(frame0 + i);
        const uint4 w = philox4x32_10(
            make_uint4(static_cast<uint32_t>(c), static_cast<uint32_t>(f),
                       static_cast<uint32_t>(f >> 32), 0u),
            key);
        float sg = sigma, sc = scale;
        if (sigmas) {
            sg = sigmas[i];
            sc = __fdiv_rn(2.0f, __fmul_rn(sg, sg));
        }
        float g[4];
        box_muller(w.x, w.y, &g[0], &g[1]);
        box_muller(w.z, w.w, &g[2], &g[3]);
#pragma unroll
        for (int j = 0; j < 4; ++j) {
            const int p = 4 * c + j;
            if (p < n) {
                // eq. (16): x -> 1 - 2x plus noise; eq. (17): llr = 2 y / sigma^2
                const float x = (cw[i * n + p] & 1u) ? -1.0f : 1.0f;
                const float y = __fadd_rn(x, __fmul_rn(sg, g[j]));
                llr[i * n + p] = __fmul_rn(y, sc);
            }
        }
    }
}

// Per-frame noise level for training batches: Eb/N0 of frame f uniform in
// [lo, hi) dB from the top 24 bits of word 0 of Philox4x32-10 at counter
// {0, f mod 2^32, f / 2^32, 0} under key {seed mod 2^32,
// (seed / 2^32) ^ 0x534E5253}, u = (bits + 1/2) 2^-24; then
// sigma^2 = 1 / (2 R 10^(Eb/N0 / 10)) (the BPSK Eb/N0 to noise variance
// relation), evaluated in double precision with every operation rounded on
// its own (no fused multiply-add) and rounded to float.
__global__ void snr_sigma_kernel(uint64_t seed, int64_t frame0, int64_t frames, double lo,
                                 double hi, double rate, float *__restrict__ sigma) {
    const uint2 key = make_uint2(static_cast<uint32_t>(seed),
                                 static_cast<uint32_t>(seed >> 32) ^ 0x534E5253u);
    for (int64_t i = blockIdx.x * static_cast<int64_t>(blockDim.x) + threadIdx.x; i < frames;
         i += static_cast<int64_t>(gridDim.x) * blockDim.x) {
        const uint64_t f = static_cast<uint64_t>(frame0 + i);
        const uint4 w = philox4x32_10(
            make_uint4(0u, static_cast<uint32_t>(f), static_cast<uint32_t>(f >> 32), 0u), key);
        const double u = (static_cast<double>(w.x >> 8) + 0.5) * 0x1p-24;
        const double ebn0 = __dadd_rn(lo, __dmul_rn(__dsub_rn(hi, lo), u));
        const double p = pow(10.0, __ddiv_rn(ebn0, 10.0));
        sigma[i] = static_cast<float>(__dsqrt_rn(__ddiv_rn(1.0, __dmul_rn(__dmul_rn(2.0, rate), p))));
    }
}

// q = rint(clamp(scale * llr, -clip, clip)), four frames per word.
__global__ void quantize_kernel(const float *__restrict__ llr, uint32_t *__restrict__ q,
                                int64_t frames, int n, float scale, int clip) {
    const int64_t groups = (frames + 3) / 4;
    const int64_t total = groups * n;
    const float fc = static_cast<float>(clip);
    for (int64_t t = blockIdx.x * static_cast<int64_t>(blockDim.x) + threadIdx.x; t < total;
         t += static_cast<int64_t>(gridDim.x) * blockDim.x) {
        const int64_t g = t / n;
        const int p = static_cast<int>(t - g * n);
        uint32_t word = 0;
#pragma unroll
        for (int b = 0; b < 4; ++b) {
            const int64_t f = 4 * g + b;
            const uint32_t v = f < frames ? quantize_one(llr[f * n + p], scale, fc)
                                          : static_cast<uint32_t>(clip);
            word |= v << (8 * b);
        }
        q[t] = word;
    }
}

// Error counts: one warp per frame.
__global__ void stats_kernel(DevCode c, const uint8_t *__restrict__ info,
                             const uint32_t *__restrict__ hard,
                             const int32_t *__restrict__ iters, int64_t frames, int max_iters,
                             unsigned long long *__restrict__ cnt) {
    const int lane = threadIdx.x & 31;
    const int64_t warps = static_cast<int64_t>(gridDim.x) * (blockDim.x >> 5);
    for (int64_t f = (blockIdx.x * static_cast<int64_t>(blockDim.x) + threadIdx.x) >> 5;
         f < frames; f += warps) {
        bool syn_ok;
        const unsigned long long errs =
            frame_outcome(c, info + f * c.k, hard + f * c.nwords, lane, &syn_ok);
        if (lane == 0) count_frame(cnt, errs, syn_ok, iters[f], max_iters);
    }
}

// Paired frame outcomes of two decoders on the same frames: cnt[2 a + b]
// counts the frames where decoder A is wrong (a = 1) or right (a = 0) and
// decoder B likewise; "wrong" = any info bit differs.  One warp per frame.
__global__ void paired_kernel(int k, int nwords, const uint8_t *__restrict__ info,
                              const uint32_t *__restrict__ ha, const uint32_t *__restrict__ hb,
                              int64_t frames, unsigned long long *__restrict__ cnt) {
    const int lane = threadIdx.x & 31;
    const int64_t warps = static_cast<int64_t>(gridDim.x) * (blockDim.x >> 5);
    for (int64_t f = (blockIdx.x * static_cast<int64_t>(blockDim.x) + threadIdx.x) >> 5;
         f < frames; f += warps) {
        const uint8_t *in = info + f * k;
        uint32_t ea = 0, eb = 0;
        for (int t = lane; t < k; t += 32) {
            const uint32_t x = in[t] & 1u;
            ea |= ((ha[f * nwords + (t >> 5)] >> (t & 31)) & 1u) ^ x;
            eb |= ((hb[f * nwords + (t >> 5)] >> (t & 31)) & 1u) ^ x;
        }
        const bool wa = __any_sync(0xFFFFFFFFu, ea), wb = __any_sync(0xFFFFFFFFu, eb);
        if (lane == 0) atomicAdd(&cnt[2 * (wa ? 1 : 0) + (wb ? 1 : 0)], 1ull);
    }
}

// Failure-path check of the decoders' bounded wait: one warp waits on a
// bulk-copy barrier that expects bytes no copy will deliver, gives up after
// `polls` polls, records the timeout in the status word and exits.
__global__ void wait_check_kernel(int *status, uint32_t polls) {
    __shared__ uint64_t bar;
    const int lane = threadIdx.x & 31;
    if (lane == 0) {
        mbar_init(&bar, 1);
        fence_mbar_init();
    }
    __syncwarp();
    if (lane == 0) mbar_arrive_expect_tx(&bar, 16u);   // 16 bytes that never come
    const bool ok = mbar_wait_bounded(&bar, 0u, polls);
    if (!__all_sync(0xFFFFFFFFu, ok) && lane == 0) atomicOr(status, kStatusCopyTimeout);
}

static int grid_for(int64_t work, int threads) {
    int dev = 0, sms = 148;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    const int64_t want = (work + threads - 1) / threads;
    return static_cast<int>(std::min<int64_t>(std::max<int64_t>(want, 1), 32LL * sms));
}

ldpc_status launch_gen_info(uint64_t seed, int64_t frame0, int64_t frames, int k,
                            uint8_t *d_info, cudaStream_t s) {
    const int64_t work = frames * ((k + 127) / 128);
    gen_info_kernel<<<grid_for(work, 256), 256, 0, s>>>(seed, frame0, frames, k, d_info);
    cudaError_t e = cudaGetLastError();
    return e == cudaSuccess ? LDPC_OK : cuda_fail(e, "gen_info_kernel");
}

ldpc_status launch_encode(const Code &c, const uint8_t *d_info, uint8_t *d_code,
                          int64_t frames, cudaStream_t s) {
    const int warp_bytes = (c.k + c.mb * c.z + c.z + 15) & ~15;
    const int smem = kEncWarps * warp_bytes;
    cudaError_t e = allow_dynamic_smem(reinterpret_cast<const void *>(encode_kernel));
    if (e != cudaSuccess) return cuda_fail(e, "encode_kernel attribute");
    int dev = 0, sms = 148;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    const int64_t want = (frames + kEncWarps - 1) / kEncWarps;
    const int grid = static_cast<int>(std::min<int64_t>(want, 16LL * sms));
    encode_kernel<<<grid, kEncWarps * 32, smem, s>>>(dev_view(c), d_info, d_code, frames,
                                                     warp_bytes);
    e = cudaGetLastError();
    return e == cudaSuccess ? LDPC_OK : cuda_fail(e, "encode_kernel");
}

ldpc_status launch_awgn(const uint8_t *d_code, int64_t frame0, int64_t frames, int n,
                        uint64_t seed, float sigma, float scale, float *d_llr,
                        cudaStream_t s) {
    const int64_t work = frames * ((n + 3) / 4);
    awgn_kernel<<<grid_for(work, 256), 256, 0, s>>>(d_code, frame0, frames, n, seed, sigma,
                                                    scale, nullptr, d_llr);
    cudaError_t e = cudaGetLastError();
    return e == cudaSuccess ? LDPC_OK : cuda_fail(e, "awgn_kernel");
}

ldpc_status launch_awgn_frames(const uint8_t *d_code, int64_t frame0, int64_t frames, int n,
                               uint64_t seed, const float *d_sigma, float *d_llr,
                               cudaStream_t s) {
    const int64_t work = frames * ((n + 3) / 4);
    awgn_kernel<<<grid_for(work, 256), 256, 0, s>>>(d_code, frame0, frames, n, seed, 0.0f, 0.0f,
                                                    d_sigma, d_llr);
    cudaError_t e = cudaGetLastError();
    return e == cudaSuccess ? LDPC_OK : cuda_fail(e, "awgn_kernel");
}

ldpc_status launch_snr_sigma(uint64_t seed, int64_t frame0, int64_t frames, double lo,
                             double hi, double rate, float *d_sigma, cudaStream_t s) {
    snr_sigma_kernel<<<grid_for(frames, 256), 256, 0, s>>>(seed, frame0, frames, lo, hi, rate,
                                                           d_sigma);
    cudaError_t e = cudaGetLastError();
    return e == cudaSuccess ? LDPC_OK : cuda_fail(e, "snr_sigma_kernel");
}

ldpc_status launch_quantize(const float *d_llr, uint32_t *d_q, int64_t frames, int n,
                            float scale, int clip, cudaStream_t s) {
    const int64_t work = ((frames + 3) / 4) * n;
    quantize_kernel<<<grid_for(work, 256), 256, 0, s>>>(d_llr, d_q, frames, n, scale, clip);
    cudaError_t e = cudaGetLastError();
    return e == cudaSuccess ? LDPC_OK : cuda_fail(e, "quantize_kernel");
}

ldpc_status launch_stats(const Code &c, const uint8_t *d_info, const uint32_t *d_hard,
                         const int32_t *d_iters, int64_t frames, int max_iters,
                         int64_t *d_counters, cudaStream_t s) {
    cudaError_t e = cudaMemsetAsync(d_counters, 0, sizeof(int64_t) * (5 + max_iters), s);
    if (e != cudaSuccess) return cuda_fail(e, "cudaMemsetAsync counters");
    if (frames == 0) return LDPC_OK;
    stats_kernel<<<grid_for(frames * 32, 256), 256, 0, s>>>(
        dev_view(c), d_info, d_hard, d_iters, frames, max_iters,
        reinterpret_cast<unsigned long long *>(d_counters));
    e = cudaGetLastError();
    return e == cudaSuccess ? LDPC_OK : cuda_fail(e, "stats_kernel");
}

ldpc_status launch_paired(const Code &c, const uint8_t *d_info, const uint32_t *d_hard_a,
                          const uint32_t *d_hard_b, int64_t frames, int64_t *d_counts,
                          cudaStream_t s) {
    cudaError_t e = cudaMemsetAsync(d_counts, 0, sizeof(int64_t) * 4, s);
    if (e != cudaSuccess) return cuda_fail(e, "cudaMemsetAsync counters");
    if (frames == 0) return LDPC_OK;
    paired_kernel<<<grid_for(frames * 32, 256), 256, 0, s>>>(
        c.k, (c.n + 31) / 32, d_info, d_hard_a, d_hard_b, frames,
        reinterpret_cast<unsigned long long *>(d_counts));
    e = cudaGetLastError();
    return e == cudaSuccess ? LDPC_OK : cuda_fail(e, "paired_kernel");
}

ldpc_status launch_wait_check(const Code &c, uint32_t polls, cudaStream_t s) {
    wait_check_kernel<<<1, 32, 0, s>>>(c.d_status, polls);
    cudaError_t e = cudaGetLastError();
    return e == cudaSuccess ? LDPC_OK : cuda_fail(e, "wait_check_kernel");
}

}  // namespace ldpc
