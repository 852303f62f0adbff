// The paper's own variants of the path, beside the GB300 decoders:
//   * Section 5's fixed-point decoder: int16 values with Q_B-bit channel
//     samples and native wrap-around arithmetic (no saturation);
//   * Section 3's bitmap encoder (Alg. A1 word/bit rotation), Z a multiple
//     of 32;
//   * Section 4's flooding schedule (eq. 18-21) in FP32.
// Each uses one warp per frame, the code's tables and the shared device
// helpers of the layered decoders.
#include <algorithm>
#include <string>

#include "ldpc_decode_dev.cuh"

namespace ldpc {
namespace {

// x reduced modulo 2^16 into [-32768, 32767].
__device__ __forceinline__ int wrap16(int x) {
    return static_cast<int>(static_cast<unsigned>(x) << 16) >> 16;
}

// ---------------------------------------------------------------------------
// int16 wrap-around layered decoder.  Posteriors as sign-extended int16 in
// 32-bit shared words (the FP32 offset table applies unchanged); row state
// [m1, m2, meta] as in the FP32 kernel with scaled magnitudes.  The dummy
// posterior of unused slots is +32767 and those slots' old message is
// forced to 0, so their |Z_mn| = 32767 never lowers a minimum.
// ---------------------------------------------------------------------------
template <int DMAX>
__device__ __forceinline__ void layer_i16w(const DevCode &c, int layer, uint32_t *Zs,
                                           uint32_t *rows, int lane, bool norm) {
    const uint32_t ri = __ldg(c.rowinfo + layer);
    const int d = ri & 255;
    const int start = DMAX - d;
    for (int t = 0; t < c.rpl; ++t) {
        const int r = lane + 32 * t;
        if (r >= c.z) break;
        uint32_t *rs = rows + (layer * c.z + r) * 3;
        const int m1 = static_cast<int>(rs[0]), m2 = static_cast<int>(rs[1]);
        const uint32_t meta = rs[2];
        const int idx = static_cast<int>(meta >> 27);
        const uint16_t *vrow = c.voff + (layer * c.rpl + t) * (DMAX * 32) + lane;
        uint32_t off[DMAX];
        int Q[DMAX], A[DMAX];
#pragma unroll
        for (int i = 0; i < DMAX; ++i) off[i] = edge_off(c, vrow + i * 32);
        int mn1 = 0x7FFFFFFF, mn2 = 0x7FFFFFFF;
        uint32_t sx = 0;
#pragma unroll
        for (int i = 0; i < DMAX; ++i) {
            const int z = static_cast<int>(lds_u32(Zs, off[i]));
            const int M = (idx == i) ? m2 : m1;
            const bool neg = (meta >> (DMAX - 1 - i)) & 1u;
            int lo = neg ? wrap16(-M) : M;
            lo = i < start ? 0 : lo;
            const int q = wrap16(z - lo);                    // eq. (22)
            const int a = wrap16(q < 0 ? -q : q);            // |Z_mn| in 16 bits
            Q[i] = q;
            A[i] = a;
            mn2 = max(mn1, min(mn2, a));
            mn1 = min(mn1, a);
            sx ^= q < 0 ? 1u : 0u;
        }
        const int n1 = norm ? wrap16((3 * mn1) >> 2) : mn1;   // eq. (23) magnitudes
        const int n2 = norm ? wrap16((3 * mn2) >> 2) : mn2;
        uint32_t nsg = 0;
        int id = 0;
#pragma unroll
        for (int i = 0; i < DMAX; ++i) {
            const bool at_min = A[i] == mn1;
            id = at_min ? i : id;
            const int Mi = at_min ? n2 : n1;
            const uint32_t sg = sx ^ (Q[i] < 0 ? 1u : 0u);
            const int L = sg ? wrap16(-Mi) : Mi;
            if (i >= start)
                sts_u32(Zs, off[i], static_cast<uint32_t>(wrap16(Q[i] + L)));   // eq. (20)
            nsg = (nsg << 1) | sg;
        }
        rs[0] = static_cast<uint32_t>(n1);
        rs[1] = static_cast<uint32_t>(n2);
        rs[2] = nsg | (static_cast<uint32_t>(id) << 27);
    }
}

// True when every check holds; the scan ends at the first failing layer.
template <int DMAX>
__device__ __forceinline__ bool syndrome_ok_int(const DevCode &c, const uint32_t *Zs, int lane) {
    for (int l = 0; l < c.mb; ++l) {
        uint32_t bad = 0;
        for (int t = 0; t < c.rpl; ++t) {
            if (lane + 32 * t >= c.z) break;
            const uint16_t *vrow = c.voff + (l * c.rpl + t) * (DMAX * 32) + lane;
            uint32_t par = 0;
#pragma unroll
            for (int i = 0; i < DMAX; ++i)
                par ^= static_cast<int>(lds_u32(Zs, edge_off(c, vrow + i * 32))) <= 0 ? 1u : 0u;
            bad |= par;
        }
        if (__any_sync(0xFFFFFFFFu, bad)) return false;
    }
    return true;
}

template <int DMAX>
__global__ void __launch_bounds__(32)
    decode_i16w_kernel(DevCode c, const int16_t *__restrict__ llr, int64_t frames,
                       DecodeParams p, uint32_t *__restrict__ hard, int32_t *__restrict__ iters,
                       int16_t *__restrict__ post, unsigned long long *work) {
    extern __shared__ __align__(16) uint32_t smem[];
    const int lane = threadIdx.x & 31;
    uint32_t *Zs = smem;
    uint32_t *rows = Zs + posterior_words(c.n);
    const bool norm = p.normalise != 0;
    Zs[c.n + lane] = 32767u;   // dummy posterior
    __syncwarp();
    int64_t f = blockIdx.x;
    while (f < frames) {
        const int16_t *src = llr + f * c.n;
        for (int i = lane; i < c.n; i += 32) Zs[i] = static_cast<uint32_t>(static_cast<int>(src[i]));
        for (int i = lane; i < c.m * 3; i += 32) rows[i] = 0u;
        __syncwarp();
        int done = p.max_iters;
        for (int k = 1; k <= p.max_iters; ++k) {
            for (int l = 0; l < c.mb; ++l) {
                layer_i16w<DMAX>(c, l, Zs, rows, lane, norm);
                __syncwarp();
            }
            if (p.early_stop && syndrome_ok_int<DMAX>(c, Zs, lane)) {
                done = k;
                break;
            }
        }
        uint32_t *h = hard + f * c.nwords;
        for (int wb = 0; wb < c.nwords; wb += 32) {
            uint32_t mine = 0;
            for (int i = 0; i < 32 && wb + i < c.nwords; ++i) {
                const int n = (wb + i) * 32 + lane;
                const bool b = n < c.n && static_cast<int>(Zs[n]) <= 0;
                const uint32_t bal = __ballot_sync(0xFFFFFFFFu, b);
                if (lane == i) mine = bal;
            }
            if (wb + lane < c.nwords) h[wb + lane] = mine;
        }
        if (lane == 0) iters[f] = done;
        if (post)
            for (int n = lane; n < c.n; n += 32)
                post[f * c.n + n] = static_cast<int16_t>(static_cast<int>(Zs[n]));
        __syncwarp();
        f = next_work(work, gridDim.x, lane);
    }
}

// ---------------------------------------------------------------------------
// The same decoder with two frames per 32-bit word, one per 16-bit lane
// (frame 2g in bits 0-15, 2g + 1 in bits 16-31): the wrap-around additions
// are single packed add-max instructions (a + b per lane modulo 2^16, then
// the max with -32768, which keeps it), and |x|, the minima and the masks
// act on both frames at once.  Row state per check row, five words:
// [N1, N2, IDX] with a frame per lane (scaled minima, argmin slot) and
// [SGA, SGB], the message signs of each frame at bit DMAX - 1 - i for slot
// i.  The results are those of layer_i16w, lane by lane.
// ---------------------------------------------------------------------------
constexpr int kRowWordsI16x2 = 5;

// a + b per 16-bit lane, modulo 2^16
__device__ __forceinline__ uint32_t wadd16x2(uint32_t a, uint32_t b) {
    return __viaddmax_s16x2(a, b, 0x80008000u);
}
// -a per 16-bit lane, modulo 2^16 (-(-32768) stays -32768)
__device__ __forceinline__ uint32_t wneg16x2(uint32_t a) { return wadd16x2(~a, 0x00010001u); }
__device__ __forceinline__ uint32_t smin16x2(uint32_t a, uint32_t b) {
    uint32_t r;
    asm("min.s16x2 %0, %1, %2;" : "=r"(r) : "r"(a), "r"(b));
    return r;
}
__device__ __forceinline__ uint32_t smax16x2(uint32_t a, uint32_t b) {
    uint32_t r;
    asm("max.s16x2 %0, %1, %2;" : "=r"(r) : "r"(a), "r"(b));
    return r;
}
__device__ __forceinline__ uint32_t umin16x2(uint32_t a, uint32_t b) {
    uint32_t r;
    asm("min.u16x2 %0, %1, %2;" : "=r"(r) : "r"(a), "r"(b));
    return r;
}
// 0xFFFF in each lane whose bit 15 is set (prmt sign replication)
__device__ __forceinline__ uint32_t lane_sign_mask(uint32_t x) { return prmt(x, 0u, 0xBB99u); }
// 0xFFFF in each lane where a == b
__device__ __forceinline__ uint32_t lane_eq_mask(uint32_t a, uint32_t b, uint32_t one) {
    const uint32_t t = umin16x2(a ^ b, 0x00010001u) ^ 0x00010001u;   // 1 where equal
    return imad(t, 0xFFFFu * one, 0u);
}
// floor(3 m / 4) per lane, wrapped (the (3m) >> 2 of layer_i16w)
__device__ __forceinline__ uint32_t scale34_16x2(uint32_t m) {
    const int lo = static_cast<int16_t>(m & 0xFFFFu), hi = static_cast<int16_t>(m >> 16);
    return (static_cast<uint32_t>(wrap16((3 * lo) >> 2)) & 0xFFFFu) |
           (static_cast<uint32_t>(wrap16((3 * hi) >> 2)) << 16);
}

template <int DMAX>
__device__ __forceinline__ void layer_i16x2(const DevCode &c, int layer, uint32_t *Zs,
                                            uint32_t *rows, int lane, bool norm) {
    const uint32_t ri = __ldg(c.rowinfo + layer);
    const int d = ri & 255;
    const int start = DMAX - d;
    const uint32_t one = opaque_one(c.z);
    for (int t = 0; t < c.rpl; ++t) {
        const int r = lane + 32 * t;
        if (r >= c.z) break;
        uint32_t *rs = rows + (layer * c.z + r) * kRowWordsI16x2;
        const uint32_t N1 = rs[0], N2 = rs[1], IDX = rs[2], SGA = rs[3], SGB = rs[4];
        const uint32_t G1 = wneg16x2(N1), G2 = wneg16x2(N2);   // -N per lane
        const uint16_t *vrow = c.voff + (layer * c.rpl + t) * (DMAX * 32) + lane;
        uint32_t off[DMAX], Q[DMAX], A[DMAX];
#pragma unroll
        for (int i = 0; i < DMAX; ++i) off[i] = edge_off(c, vrow + i * 32);
        uint32_t mn1 = 0x7FFF7FFFu, mn2 = 0x7FFF7FFFu, sx = 0;
#pragma unroll
        for (int i = 0; i < DMAX; ++i) {
            const uint32_t z = lds_u32(Zs, off[i]);
            // 0xFFFF where slot i is not the lane's argmin: (IDX ^ i) + 0x7FFF
            // has bit 15 set (no carry between lanes: IDX <= 26)
            const uint32_t nq = lane_sign_mask(imad(IDX ^ (0x00010001u * i), one, 0x7FFF7FFFu));
            // 0xFFFF where the old message of slot i is negative
            const int b = DMAX - 1 - i;
            const uint32_t sm = prmt(SGA << (31 - b), SGB << (31 - b), 0xFFBBu);
            // -L_old per lane: M for a negative message, -M for a positive one;
            // 0 for the leading unused slots
            uint32_t g = bsel(bsel(G2, G1, nq), bsel(N2, N1, nq), sm);
            g = i < start ? 0u : g;
            const uint32_t q = wadd16x2(z, g);                 // eq. (22)
            // |Z_mn| in 16 bits: max(-q, q) with -q = ~q + 1 wrapped, the
            // add and the max in one instruction
            const uint32_t a = __viaddmax_s16x2(~q, 0x00010001u, q);
            Q[i] = q;
            A[i] = a;
            mn2 = smax16x2(mn1, smin16x2(mn2, a));
            mn1 = smin16x2(mn1, a);
            sx ^= q;
        }
        const uint32_t n1 = norm ? scale34_16x2(mn1) : mn1;   // eq. (23) magnitudes
        const uint32_t n2 = norm ? scale34_16x2(mn2) : mn2;
        const uint32_t h1 = wneg16x2(n1), h2 = wneg16x2(n2);
        uint32_t nsa = 0, nsb = 0, id = 0;
#pragma unroll
        for (int i = 0; i < DMAX; ++i) {
            const uint32_t at_min = lane_eq_mask(A[i], mn1, one);
            id = bsel(id, 0x00010001u * i, at_min);
            const uint32_t sg = lane_sign_mask(sx ^ Q[i]);   // message sign per lane
            const uint32_t L = bsel(bsel(n1, n2, at_min), bsel(h1, h2, at_min), sg);
            if (i >= start) sts_u32(Zs, off[i], wadd16x2(Q[i], L));   // eq. (20)
            nsa = __funnelshift_l(sg << 16, nsa, 1);
            nsb = __funnelshift_l(sg, nsb, 1);
        }
        rs[0] = n1;
        rs[1] = n2;
        rs[2] = id;
        rs[3] = nsa;
        rs[4] = nsb;
    }
}

// Bit 15 (frame of lane 0) and bit 31 (lane 1) set where a check fails, for
// the lanes of `need` (bit 15 / 31 of each lane decoding a frame; the others'
// bits are unspecified); the scan ends once all of them have failed.
template <int DMAX>
__device__ __forceinline__ uint32_t syndrome_bad_i16x2(const DevCode &c, const uint32_t *Zs,
                                                       int lane, uint32_t need) {
    uint32_t bad = 0;
    for (int l = 0; l < c.mb; ++l) {
        for (int t = 0; t < c.rpl; ++t) {
            if (lane + 32 * t >= c.z) break;
            const uint16_t *vrow = c.voff + (l * c.rpl + t) * (DMAX * 32) + lane;
            uint32_t par = 0;
#pragma unroll
            for (int i = 0; i < DMAX; ++i) {
                const uint32_t v = lds_u32(Zs, edge_off(c, vrow + i * 32));
                par ^= v | wadd16x2(v, 0xFFFFFFFFu);   // bit 15 / 31 set iff Z <= 0
            }
            bad |= par;
        }
        const uint32_t all = __reduce_or_sync(0xFFFFFFFFu, bad & 0x80008000u);
        if ((all & need) == need) return all;
    }
    return __reduce_or_sync(0xFFFFFFFFu, bad & 0x80008000u);
}

// Lane `half` (0 or 1) of the packed posteriors, sign-extended.
__device__ __forceinline__ int lane16(uint32_t w, int half) {
    return static_cast<int16_t>((w >> (16 * half)) & 0xFFFFu);
}

template <int DMAX>
__global__ void __launch_bounds__(32)
    decode_i16x2_kernel(DevCode c, const int16_t *__restrict__ llr, int64_t frames,
                        DecodeParams p, uint32_t *__restrict__ hard, int32_t *__restrict__ iters,
                        int16_t *__restrict__ post, unsigned long long *work) {
    extern __shared__ __align__(16) uint32_t smem[];
    const int lane = threadIdx.x & 31;
    uint32_t *Zs = smem;
    uint32_t *rows = Zs + posterior_words(c.n);
    const bool norm = p.normalise != 0;
    const int64_t g0 = blockIdx.x;
    if (2 * g0 >= frames) return;
    int64_t fr[2];
    int kb[2];
    for (int b = 0; b < 2; ++b) {
        fr[b] = 2 * g0 + b < frames ? 2 * g0 + b : -1;
        kb[b] = 0;
    }
    // a lane without a frame holds +1023 (the all-zero codeword, which stops
    // after one iteration)
    for (int i = lane; i < c.n; i += 32) {
        const uint32_t lo = fr[0] >= 0 ? static_cast<uint16_t>(llr[fr[0] * c.n + i]) : 1023u;
        const uint32_t hi = fr[1] >= 0 ? static_cast<uint16_t>(llr[fr[1] * c.n + i]) : 1023u;
        Zs[i] = lo | (hi << 16);
    }
    for (int i = lane; i < c.m * kRowWordsI16x2; i += 32) rows[i] = 0u;
    Zs[c.n + lane] = 0x7FFF7FFFu;   // dummy posterior +32767 in both lanes
    __syncwarp();
    const int64_t dyn_base = 2 * static_cast<int64_t>(gridDim.x);
    int64_t pend = next_work(work, dyn_base, lane);
    if (pend < frames) prefetch_l2(llr + pend * c.n, 2u * static_cast<uint32_t>(c.n), lane);
    for (;;) {
        if (fr[0] < 0 && fr[1] < 0) break;
        for (int l = 0; l < c.mb; ++l) {
            layer_i16x2<DMAX>(c, l, Zs, rows, lane, norm);
            __syncwarp();
        }
        const uint32_t need = (fr[0] >= 0 ? 0x8000u : 0u) | (fr[1] >= 0 ? 0x80000000u : 0u);
        const uint32_t bad =
            p.early_stop ? syndrome_bad_i16x2<DMAX>(c, Zs, lane, need) : 0x80008000u;
        for (int b = 0; b < 2; ++b) {
            if (fr[b] < 0) continue;
            kb[b] += 1;
            const bool ok = !((bad >> (16 * b + 15)) & 1u);
            if (!ok && kb[b] < p.max_iters) continue;
            // frame finished: outputs, then the next frame into this lane
            uint32_t *h = hard + fr[b] * c.nwords;
            for (int wb = 0; wb < c.nwords; wb += 32) {
                uint32_t mine = 0;
                for (int i = 0; i < 32 && wb + i < c.nwords; ++i) {
                    const int n = (wb + i) * 32 + lane;
                    const bool hb = n < c.n && lane16(Zs[n], b) <= 0;
                    const uint32_t bal = __ballot_sync(0xFFFFFFFFu, hb);
                    if (lane == i) mine = bal;
                }
                if (wb + lane < c.nwords) h[wb + lane] = mine;
            }
            if (lane == 0) iters[fr[b]] = kb[b];
            if (post)
                for (int n = lane; n < c.n; n += 32)
                    post[fr[b] * c.n + n] = static_cast<int16_t>(lane16(Zs[n], b));
            const int64_t nf = pend;
            if (nf >= frames) {
                fr[b] = -1;
                continue;
            }
            pend = next_work(work, dyn_base, lane);
            if (pend < frames) prefetch_l2(llr + pend * c.n, 2u * static_cast<uint32_t>(c.n), lane);
            fr[b] = nf;
            kb[b] = 0;
            const uint32_t keep = b ? 0x0000FFFFu : 0xFFFF0000u;
            __syncwarp();
            for (int i = lane; i < c.n; i += 32) {
                const uint32_t v = static_cast<uint16_t>(llr[nf * c.n + i]);
                Zs[i] = (Zs[i] & keep) | (v << (16 * b));
            }
            // zero minima make every old message of the lane zero
            for (int r = lane; r < c.m; r += 32) {
                uint32_t *rs = rows + r * kRowWordsI16x2;
                rs[0] &= keep;
                rs[1] &= keep;
            }
            __syncwarp();
        }
    }
}

__global__ void quantize_i16_kernel(const float *__restrict__ llr, int16_t *__restrict__ q,
                                    int64_t count, float scale, float lim) {
    for (int64_t i = blockIdx.x * static_cast<int64_t>(blockDim.x) + threadIdx.x; i < count;
         i += static_cast<int64_t>(gridDim.x) * blockDim.x) {
        float x = __fmul_rn(scale, llr[i]);
        x = fminf(fmaxf(x, -lim), lim);
        q[i] = static_cast<int16_t>(__float2int_rn(x));
    }
}

// ---------------------------------------------------------------------------
// Bitmap encoder, one warp per frame; blocks of zw = Z / 32 words.  Shared
// memory per warp: u (Kb zw words), S_i (Mb zw), the sum of the S_i and v_0
// (zw each).
// ---------------------------------------------------------------------------
constexpr int kBitmapWarps = 4;

// Word w of P_s applied to the packed block b (Alg. A1's split of s into
// whole words and bits).
__device__ __forceinline__ uint32_t rot_word(const uint32_t *b, int zw, int s, int w) {
    const int sw = s >> 5, sb = s & 31;
    int i0 = w + sw;
    i0 = i0 >= zw ? i0 - zw : i0;
    int i1 = i0 + 1;
    i1 = i1 >= zw ? i1 - zw : i1;
    const uint32_t lo = b[i0];
    return sb ? (lo >> sb) | (b[i1] << (32 - sb)) : lo;
}

__global__ void __launch_bounds__(kBitmapWarps * 32)
    encode_bitmap_kernel(DevCode c, const uint32_t *__restrict__ info, uint32_t *__restrict__ cw,
                         int64_t frames, int warp_words) {
    extern __shared__ __align__(16) uint32_t bsm[];
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int zw = c.z >> 5, kb = c.kb, nb = c.nb, mb = c.mb;
    uint32_t *u = bsm + warp * warp_words;
    uint32_t *S = u + kb * zw;
    uint32_t *sum = S + mb * zw;
    uint32_t *v0 = sum + zw;
    for (int64_t f = blockIdx.x * static_cast<int64_t>(kBitmapWarps) + warp; f < frames;
         f += static_cast<int64_t>(gridDim.x) * kBitmapWarps) {
        const uint32_t *src = info + f * (kb * zw);
        uint32_t *dst = cw + f * (nb * zw);
        for (int w = lane; w < kb * zw; w += 32) {      // systematic part
            const uint32_t x = src[w];
            u[w] = x;
            dst[w] = x;
        }
        __syncwarp();
        for (int q = lane; q < mb * zw; q += 32) {      // eq. (15)
            const int i = q / zw, w = q - i * zw;
            uint32_t acc = 0;
            for (int j = 0; j < kb; ++j) {
                const int s = c.hbm[i * nb + j];
                if (s >= 0) acc ^= rot_word(u + j * zw, zw, s, w);
            }
            S[q] = acc;
        }
        __syncwarp();
        for (int w = lane; w < zw; w += 32) {
            uint32_t t = 0;
            for (int i = 0; i < mb; ++i) t ^= S[i * zw + w];
            sum[w] = t;
        }
        __syncwarp();
        const int b = c.hbm[c.y * nb + kb];             // eq. (12): v_0 = P_b^{-1} sum
        const int binv = b == 0 ? 0 : c.z - b;
        for (int w = lane; w < zw; w += 32) {
            const uint32_t x = rot_word(sum, zw, binv, w);
            v0[w] = x;
            dst[kb * zw + w] = x;
        }
        __syncwarp();
        for (int w = lane; w < zw; w += 32) {           // eq. (13)-(14)
            uint32_t v = 0;
            for (int i = 0; i < mb - 1; ++i) {
                const int s = c.hbm[i * nb + kb];
                const uint32_t pv = s >= 0 ? rot_word(v0, zw, s, w) : 0u;
                v = (i == 0 ? 0u : v) ^ pv ^ S[i * zw + w];
                dst[(kb + 1 + i) * zw + w] = v;
            }
        }
        __syncwarp();
    }
}

// ---------------------------------------------------------------------------
// Flooding min-sum, FP32, one warp per frame.  Shared memory: channel LLRs
// Z^(0) [N], posteriors [N + dummy], messages L and the new messages
// [E = nnz(H)] each, indexed (block edge) Z + row.  The sums of eq. (19)
// and (20) run over a variable's checks in increasing index, i.e. over the
// block column's nonzero blocks in increasing block row.
// ---------------------------------------------------------------------------
template <int DMAX>
__global__ void __launch_bounds__(32)
    decode_flooding_kernel(DevCode c, const float *__restrict__ llr, int64_t frames,
                           DecodeParams p, uint32_t *__restrict__ hard,
                           int32_t *__restrict__ iters, float *__restrict__ post,
                           unsigned long long *work) {
    extern __shared__ __align__(16) uint32_t smem[];
    const int lane = threadIdx.x & 31;
    const int n = c.n, z = c.z, E = c.n_edges * c.z;
    float *Z0 = reinterpret_cast<float *>(smem);
    uint32_t *Zn = smem + ((n + 3) & ~3);
    float *La = reinterpret_cast<float *>(Zn + posterior_words(n));
    float *Lb = La + E;
    Zn[n + lane] = 0x7F800000u;   // dummy posterior for the syndrome table
    __syncwarp();
    const float alpha = p.normalise ? p.alpha : 1.0f;
    int64_t f = blockIdx.x;
    while (f < frames) {
        for (int i = lane; i < n; i += 32) {
            const float x = llr[f * n + i];
            Z0[i] = x;
            Zn[i] = __float_as_uint(x);
        }
        for (int i = lane; i < E; i += 32) La[i] = 0.0f;
        __syncwarp();
        float *L = La, *Lnew = Lb;
        int done = p.max_iters;
        for (int k = 1; k <= p.max_iters; ++k) {
            // check update from the previous iteration's messages
            for (int l = 0; l < c.mb; ++l) {
                const uint32_t ri = __ldg(c.rowinfo + l);
                const int d = ri & 255, e0 = static_cast<int>(ri >> 8);
                for (int r = lane; r < z; r += 32) {
                    float Q[DMAX];
                    float mn1 = __int_as_float(0x7F800000), mn2 = mn1;
                    uint32_t sx = 0;
#pragma unroll
                    for (int i = 0; i < DMAX; ++i) {
                        if (i < d) {
                            const uint32_t ed = __ldg(c.edges + e0 + i);
                            const int j = static_cast<int>(ed >> 16);
                            int cl = r + static_cast<int>(ed & 0xFFFFu);
                            cl = cl >= z ? cl - z : cl;           // local column of the edge
                            float s = Z0[j * z + cl];               // eq. (19)
                            for (int q = __ldg(c.coloff + j); q < __ldg(c.coloff + j + 1); ++q) {
                                const uint32_t ce = __ldg(c.colent + q);
                                if (static_cast<int>(ce >> 20) == l) continue;   // this check
                                int rr = cl - static_cast<int>(ce & 0x1FFu);
                                rr = rr < 0 ? rr + z : rr;
                                s = __fadd_rn(s, L[static_cast<int>((ce >> 9) & 0x7FFu) * z + rr]);
                            }
                            Q[i] = s;
                            const float a = fabsf(s);
                            mn2 = fmaxf(mn1, fminf(mn2, a));
                            mn1 = fminf(mn1, a);
                            sx ^= __float_as_uint(s);
                        }
                    }
                    const uint32_t S = sx & 0x80000000u;
#pragma unroll
                    for (int i = 0; i < DMAX; ++i) {
                        if (i < d) {
                            const float mag = fabsf(Q[i]) == mn1 ? mn2 : mn1;   // eq. (18)
                            const float m = __uint_as_float(__float_as_uint(mag) |
                                                            (S ^ (__float_as_uint(Q[i]) &
                                                                  0x80000000u)));
                            Lnew[(e0 + i) * z + r] = p.normalise ? __fmul_rn(alpha, m) : m;
                        }
                    }
                }
            }
            __syncwarp();
            float *tmp = L;
            L = Lnew;
            Lnew = tmp;
            // posteriors, eq. (20)
            for (int v = lane; v < n; v += 32) {
                const int j = v / z, cl = v - j * z;
                float s = Z0[v];
                for (int q = __ldg(c.coloff + j); q < __ldg(c.coloff + j + 1); ++q) {
                    const uint32_t ce = __ldg(c.colent + q);
                    int rr = cl - static_cast<int>(ce & 0x1FFu);
                    rr = rr < 0 ? rr + z : rr;
                    s = __fadd_rn(s, L[static_cast<int>((ce >> 9) & 0x7FFu) * z + rr]);
                }
                Zn[v] = __float_as_uint(s);
            }
            __syncwarp();
            if (p.early_stop && syndrome_ok_f32<DMAX>(c, Zn, lane)) {
                done = k;
                break;
            }
        }
        write_frame_f32_to(c, Zn, done, hard + f * c.nwords, iters + f,
                           post ? post + f * n : nullptr, lane);
        __syncwarp();
        f = next_work(work, gridDim.x, lane);
    }
}

int sm_count(int device) {
    int sms = 148;
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, device);
    return sms;
}

int smem_optin(int device) {
    int v = 48 * 1024;
    cudaDeviceGetAttribute(&v, cudaDevAttrMaxSharedMemoryPerBlockOptin, device);
    return v;
}

template <int DMAX>
ldpc_status launch_i16w_t(const Code &c, const int16_t *llr, int64_t frames,
                          const DecodeParams &p, uint32_t *hard, int32_t *iters, int16_t *post,
                          cudaStream_t s) {
    // two frames per word when the packed row state fits, else one per warp
    const int smem2 = 4 * (posterior_words(c.n) + c.m * kRowWordsI16x2);
    if (smem2 <= smem_optin(c.device)) {
        const void *kern = reinterpret_cast<const void *>(decode_i16x2_kernel<DMAX>);
        cudaError_t e = allow_dynamic_smem(kern);
        if (e != cudaSuccess) return cuda_fail(e, "decode (int16) attribute");
        int per_sm = 0;
        e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kern, 32, smem2);
        if (e != cudaSuccess) return cuda_fail(e, "decode (int16) occupancy");
        const int64_t units = (frames + 1) / 2;
        const int grid = static_cast<int>(std::min<int64_t>(
            units, grid_cap(static_cast<int64_t>(std::max(per_sm, 1)) * sm_count(c.device))));
        unsigned long long *work = work_slot(c, s);
        if (!work) return LDPC_ERR_CUDA;
        decode_i16x2_kernel<DMAX><<<grid, 32, smem2, s>>>(dev_view(c), llr, frames, p, hard,
                                                          iters, post, work);
        e = cudaGetLastError();
        return e == cudaSuccess ? LDPC_OK : cuda_fail(e, "decode (int16) launch");
    }
    const int smem = 4 * (posterior_words(c.n) + c.m * 3);
    if (smem > smem_optin(c.device))
        return fail(LDPC_ERR_UNSUPPORTED, "decode (int16): code too large for shared memory");
    const void *kern = reinterpret_cast<const void *>(decode_i16w_kernel<DMAX>);
    cudaError_t e = allow_dynamic_smem(reinterpret_cast<const void *>(kern));
    if (e != cudaSuccess) return cuda_fail(e, "decode (int16) attribute");
    int per_sm = 0;
    e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kern, 32, smem);
    if (e != cudaSuccess) return cuda_fail(e, "decode (int16) occupancy");
    const int grid = static_cast<int>(
        std::min<int64_t>(frames, static_cast<int64_t>(std::max(per_sm, 1)) * sm_count(c.device)));
    unsigned long long *work = work_slot(c, s);
    if (!work) return LDPC_ERR_CUDA;
    decode_i16w_kernel<DMAX><<<grid, 32, smem, s>>>(dev_view(c), llr, frames, p, hard, iters,
                                                    post, work);
    e = cudaGetLastError();
    return e == cudaSuccess ? LDPC_OK : cuda_fail(e, "decode (int16) launch");
}

template <int DMAX>
ldpc_status launch_flooding_t(const Code &c, const float *llr, int64_t frames,
                              const DecodeParams &p, uint32_t *hard, int32_t *iters, float *post,
                              cudaStream_t s) {
    const size_t words =
        ((c.n + 3) & ~3) + posterior_words(c.n) + 2 * static_cast<size_t>(c.n_edges) * c.z;
    const size_t smem = 4 * words;
    if (smem > static_cast<size_t>(smem_optin(c.device)))
        return fail(LDPC_ERR_UNSUPPORTED, "flooding decode: code too large for shared memory");
    const void *kern = reinterpret_cast<const void *>(decode_flooding_kernel<DMAX>);
    cudaError_t e = allow_dynamic_smem(reinterpret_cast<const void *>(kern));
    if (e != cudaSuccess) return cuda_fail(e, "flooding attribute");
    int per_sm = 0;
    e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kern, 32, smem);
    if (e != cudaSuccess) return cuda_fail(e, "flooding occupancy");
    const int grid = static_cast<int>(
        std::min<int64_t>(frames, static_cast<int64_t>(std::max(per_sm, 1)) * sm_count(c.device)));
    unsigned long long *work = work_slot(c, s);
    if (!work) return LDPC_ERR_CUDA;
    decode_flooding_kernel<DMAX><<<grid, 32, smem, s>>>(dev_view(c), llr, frames, p, hard, iters,
                                                        post, work);
    e = cudaGetLastError();
    return e == cudaSuccess ? LDPC_OK : cuda_fail(e, "flooding launch");
}

}  // namespace

ldpc_status launch_decode_i16w(const Code &c, const int16_t *d_llr, int64_t frames,
                               const DecodeParams &p, uint32_t *d_hard, int32_t *d_iters,
                               int16_t *d_post, cudaStream_t s) {
    switch (c.dslots) {
#define LDPC_I16_CASE(D) \
    case D: return launch_i16w_t<D>(c, d_llr, frames, p, d_hard, d_iters, d_post, s);
        LDPC_SLOT_CLASSES(LDPC_I16_CASE)
#undef LDPC_I16_CASE
        default: return fail(LDPC_ERR_UNSUPPORTED, "decode (int16): row degree above 27");
    }
}

}  // namespace ldpc

using namespace ldpc;

extern "C" {

ldpc_status ldpc_quantize_i16(const float *d_llr, int16_t *d_q, int64_t count, float scale,
                              int qb, cudaStream_t stream) {
    if (count < 0 || qb < 1 || qb > 14 || !(scale == scale))
        return fail(LDPC_ERR_INVALID_ARG, "ldpc_quantize_i16: bad count, qb or scale");
    if (count == 0) return LDPC_OK;
    if (!d_llr || !d_q) return fail(LDPC_ERR_INVALID_ARG, "ldpc_quantize_i16: NULL buffer");
    int dev = 0;
    cudaGetDevice(&dev);
    const int64_t blocks = std::min<int64_t>((count + 255) / 256, 16LL * sm_count(dev));
    quantize_i16_kernel<<<static_cast<unsigned>(blocks), 256, 0, stream>>>(
        d_llr, d_q, count, scale, static_cast<float>((1 << qb) - 1));
    cudaError_t e = cudaGetLastError();
    return e == cudaSuccess ? LDPC_OK : cuda_fail(e, "quantize_i16_kernel");
}

ldpc_status ldpc_encode_bitmap(const ldpc_code *code, const uint32_t *d_info, uint32_t *d_code,
                               int64_t frames, cudaStream_t stream) {
    if (!code) return fail(LDPC_ERR_INVALID_ARG, "ldpc_encode_bitmap: code is NULL");
    if (frames < 0) return fail(LDPC_ERR_INVALID_ARG, "ldpc_encode_bitmap: frames < 0");
    const Code &c = code->c;
    if (c.z % 32)
        return fail(LDPC_ERR_UNSUPPORTED, "ldpc_encode_bitmap: Z must be a multiple of 32");
    if (frames == 0) return LDPC_OK;
    if (!d_info || !d_code) return fail(LDPC_ERR_INVALID_ARG, "ldpc_encode_bitmap: NULL buffer");
    cudaError_t e = cudaSetDevice(c.device);
    if (e != cudaSuccess) return cuda_fail(e, "cudaSetDevice");
    const int zw = c.z / 32;
    const int warp_words = (c.kb + c.mb + 2) * zw;
    const int smem = kBitmapWarps * warp_words * 4;
    e = allow_dynamic_smem(reinterpret_cast<const void *>(encode_bitmap_kernel));
    if (e != cudaSuccess) return cuda_fail(e, "encode_bitmap attribute");
    const int64_t blocks =
        std::min<int64_t>((frames + kBitmapWarps - 1) / kBitmapWarps, 32LL * sm_count(c.device));
    encode_bitmap_kernel<<<static_cast<unsigned>(blocks), kBitmapWarps * 32, smem, stream>>>(
        dev_view(c), d_info, d_code, frames, warp_words);
    e = cudaGetLastError();
    return e == cudaSuccess ? LDPC_OK : cuda_fail(e, "encode_bitmap_kernel");
}

ldpc_status ldpc_decode_flooding_minsum(const ldpc_code *code, const float *d_llr,
                                        int64_t frames, const ldpc_decode_params *params,
                                        uint32_t *d_hard, int32_t *d_iters, float *d_post,
                                        cudaStream_t stream) {
    static const char *kWhat = "ldpc_decode_flooding_minsum";
    if (!code || !params) return fail(LDPC_ERR_INVALID_ARG, std::string(kWhat) + ": NULL code or params");
    if (frames < 0 || params->max_iters < 1 || params->max_iters > kMaxIters ||
        (params->normalise != 0 && params->normalise != 1) ||
        (params->early_stop != 0 && params->early_stop != 1) ||
        (params->normalise && !(params->alpha == params->alpha)))
        return fail(LDPC_ERR_INVALID_ARG, std::string(kWhat) + ": bad frames or parameters");
    const Code &c = code->c;
    if (!c.dslots) return fail(LDPC_ERR_UNSUPPORTED, std::string(kWhat) + ": row degree above 27");
    if (frames == 0) return LDPC_OK;
    if (!d_llr || !d_hard || !d_iters)
        return fail(LDPC_ERR_INVALID_ARG, std::string(kWhat) + ": NULL buffer");
    cudaError_t e = cudaSetDevice(c.device);
    if (e != cudaSuccess) return cuda_fail(e, "cudaSetDevice");
    DecodeParams p;
    p.max_iters = params->max_iters;
    p.alpha = params->normalise ? params->alpha : 1.0f;
    p.normalise = params->normalise;
    p.early_stop = params->early_stop;
    switch (c.dslots) {
#define LDPC_FLOOD_CASE(D) \
    case D: return launch_flooding_t<D>(c, d_llr, frames, p, d_hard, d_iters, d_post, stream);
        LDPC_SLOT_CLASSES(LDPC_FLOOD_CASE)
#undef LDPC_FLOOD_CASE
        default: return fail(LDPC_ERR_UNSUPPORTED, std::string(kWhat) + ": row degree");
    }
}

}  // extern "C"
