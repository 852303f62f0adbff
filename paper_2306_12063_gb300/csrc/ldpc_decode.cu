// Layered single-scan min-sum decoders of libldpc (arXiv 2306.12063,
// Section 4: eq. 20, 22, 23 under the layered schedule; Section 5 for the
// fixed-point variant, here 8-bit saturating).
//
// Mapping: one warp decodes one frame (FP32) or one group of four frames
// packed one byte each in a 32-bit word (int8).  The warp keeps the whole
// posterior vector Z_n and the compressed check messages of every row in
// shared memory for all iterations; the channel LLRs are brought in by one
// 1-D bulk copy (TMA engine) per frame.  Lane l handles rows l, l+32, ... of
// the current layer; the Z rows of a layer touch disjoint variables, so a
// layer needs no synchronisation beyond a __syncwarp before the next one.
// The per-lane variable of each edge, j Z + (r + s) mod Z (the cyclic shift
// of the circulant as an index rotation), comes precomputed from a small
// table built with the code.
#include <algorithm>

#include "ldpc_internal.cuh"

namespace ldpc {

constexpr uint32_t kFull = 0xFFFFFFFFu;
constexpr uint32_t kWaitLimit = 1u << 22;   // polls of a bulk-copy barrier

// Row state words in shared memory (per check row):
//   FP32:  [m1, m2, meta, -]; meta bits 0..26 = sign of L_mn on edge e
//          (1 = negative), bits 27..31 = argmin edge.  m1, m2 already scaled.
//   int8:  [M1, M2, IDX, SG0, SG1, SG2, SG3, -]; one byte per frame: scaled
//          magnitudes, argmin edge; SGk byte b bit u = sign of L_mn of frame
//          b on edge 8k + u.
constexpr int kRowWordsF32 = 4;
constexpr int kRowWordsI8 = 8;

__device__ __forceinline__ uint32_t lds_u32(const uint32_t *base, uint32_t byte_off) {
    return *reinterpret_cast<const uint32_t *>(reinterpret_cast<const char *>(base) + byte_off);
}
__device__ __forceinline__ void sts_u32(uint32_t *base, uint32_t byte_off, uint32_t v) {
    *reinterpret_cast<uint32_t *>(reinterpret_cast<char *>(base) + byte_off) = v;
}

// ---------------------------------------------------------------------------
// FP32 layer: eq. (22) Z_mn = Z_n - L_mn, eq. (23) new L_mn from the minimum
// and second minimum of |Z_mn| and the product of signs, eq. (20) written in
// its single-scan form Z_n = Z_mn + L_mn.  Every float operation is an
// explicitly rounded intrinsic so no multiply-add is ever contracted.
// ---------------------------------------------------------------------------
template <int D>
__device__ __forceinline__ void layer_f32(const DevCode &c, int layer, int e0, uint32_t *Zs,
                                          uint32_t *rows, int lane, bool norm, float alpha) {
    const int stride = c.rpl * 32;
    for (int t = 0; t < c.rpl; ++t) {
        const int r = lane + 32 * t;
        if (r >= c.z) break;
        uint4 *rs = reinterpret_cast<uint4 *>(rows + (layer * c.z + r) * kRowWordsF32);
        const uint4 st = *rs;
        const float m1 = __uint_as_float(st.x), m2 = __uint_as_float(st.y);
        const uint32_t meta = st.z;
        const int idx = static_cast<int>(meta >> 27);
        const uint16_t *vo = c.voff + (e0 * c.rpl + t) * 32 + lane;
        uint32_t off[D];
        float Q[D];
        float mn1 = __int_as_float(0x7F800000), mn2 = mn1;
        int id = 0;
        uint32_t sx = 0;
#pragma unroll
        for (int e = 0; e < D; ++e) {
            off[e] = __ldg(vo + e * stride);
            const float zv = __uint_as_float(lds_u32(Zs, off[e]));
            const float mag = (e == idx) ? m2 : m1;
            const float L = __uint_as_float(__float_as_uint(mag) |
                                            ((meta << (31 - e)) & 0x80000000u));
            const float q = __fsub_rn(zv, L);
            Q[e] = q;
            const float a = fabsf(q);
            mn2 = fminf(mn2, fmaxf(mn1, a));
            id = (a < mn1) ? e : id;
            mn1 = fminf(mn1, a);
            sx ^= __float_as_uint(q);
        }
        const float n1 = norm ? __fmul_rn(alpha, mn1) : mn1;
        const float n2 = norm ? __fmul_rn(alpha, mn2) : mn2;
        const uint32_t S = sx & 0x80000000u;
        const uint32_t s1 = __float_as_uint(n1) | S, s2 = __float_as_uint(n2) | S;
        uint32_t nsg = 0;
#pragma unroll
        for (int e = 0; e < D; ++e) {
            const uint32_t ms = (e == id) ? s2 : s1;
            const uint32_t L = ms ^ (__float_as_uint(Q[e]) & 0x80000000u);
            sts_u32(Zs, off[e], __float_as_uint(__fadd_rn(Q[e], __uint_as_float(L))));
            nsg |= (L >> 31) << e;
        }
        *rs = make_uint4(__float_as_uint(n1), __float_as_uint(n2),
                         nsg | (static_cast<uint32_t>(id) << 27), 0u);
    }
}

// ---------------------------------------------------------------------------
// int8 layer, four frames per word.  Z_mn and Z_n saturate to [-127, 127];
// messages are (3 m) >> 2 when normalising.  Byte-parallel arithmetic uses
// the CUDA SIMD intrinsics (saturating add/sub, min/max, compares).
// ---------------------------------------------------------------------------
__device__ __forceinline__ uint32_t scale34(uint32_t m) {
    // per byte floor(3 m / 4) = m - ceil(m / 4), m <= 127 (no carries cross bytes)
    return m - (((m + 0x03030303u) >> 2) & 0x3F3F3F3Fu);
}

template <int D>
__device__ __forceinline__ void layer_i8(const DevCode &c, int layer, int e0, uint32_t *Zs,
                                         uint32_t *rows, int lane, bool norm) {
    constexpr int K = (D + 7) / 8;
    const int stride = c.rpl * 32;
    for (int t = 0; t < c.rpl; ++t) {
        const int r = lane + 32 * t;
        if (r >= c.z) break;
        uint32_t *rs = rows + (layer * c.z + r) * kRowWordsI8;
        const uint4 st0 = reinterpret_cast<const uint4 *>(rs)[0];
        const uint4 st1 = reinterpret_cast<const uint4 *>(rs)[1];
        const uint32_t M1 = st0.x, M2 = st0.y, IDX = st0.z;
        const uint32_t SG[4] = {st0.w, st1.x, st1.y, st1.z};
        const uint16_t *vo = c.voff + (e0 * c.rpl + t) * 32 + lane;
        uint32_t off[D], Q[D];
        uint32_t mn1 = 0xFFFFFFFFu, mn2 = 0xFFFFFFFFu, id = 0, sx = 0;
#pragma unroll
        for (int e = 0; e < D; ++e) {
            const uint32_t E = 0x01010101u * static_cast<uint32_t>(e);
            off[e] = __ldg(vo + e * stride);
            const uint32_t zv = lds_u32(Zs, off[e]);
            const uint32_t sm = msb_bytes_to_mask(SG[e >> 3] << (7 - (e & 7)));
            const uint32_t mag = bsel(M1, M2, __vcmpeq4(IDX, E));
            const uint32_t L = bsel(mag, __vneg4(mag), sm);
            const uint32_t q = __vmaxs4(__vsubss4(zv, L), 0x81818181u);
            Q[e] = q;
            const uint32_t a = __vabsss4(q);
            const uint32_t lt = __vcmpltu4(a, mn1);
            mn2 = __vminu4(mn2, __vmaxu4(mn1, a));
            id = bsel(id, E, lt);
            mn1 = __vminu4(mn1, a);
            sx ^= q;
        }
        const uint32_t n1 = norm ? scale34(mn1) : mn1;
        const uint32_t n2 = norm ? scale34(mn2) : mn2;
        const uint32_t S = sx & 0x80808080u;
        uint32_t nsg[4] = {0u, 0u, 0u, 0u};
#pragma unroll
        for (int e = 0; e < D; ++e) {
            const uint32_t E = 0x01010101u * static_cast<uint32_t>(e);
            const uint32_t neg = (Q[e] ^ S) & 0x80808080u;      // S xor sgn(Z_mn)
            const uint32_t mag = bsel(n1, n2, __vcmpeq4(id, E));
            const uint32_t L = bsel(mag, __vneg4(mag), msb_bytes_to_mask(neg));
            const uint32_t zn = __vmaxs4(__vaddss4(Q[e], L), 0x81818181u);
            sts_u32(Zs, off[e], zn);
            nsg[e >> 3] |= neg >> (7 - (e & 7));
        }
        reinterpret_cast<uint4 *>(rs)[0] = make_uint4(n1, n2, id, nsg[0]);
        reinterpret_cast<uint4 *>(rs)[1] = make_uint4(nsg[1], K > 2 ? nsg[2] : 0u,
                                                      K > 3 ? nsg[3] : 0u, 0u);
    }
}

#define LDPC_DEG_CASES(X) \
    X(2) X(3) X(4) X(5) X(6) X(7) X(8) X(9) X(10) X(11) X(12) X(13) X(14) X(15) \
    X(16) X(17) X(18) X(19) X(20) X(21) X(22) X(23) X(24) X(25) X(26) X(27)

__device__ __forceinline__ void run_layer_f32(const DevCode &c, int layer, uint32_t *Zs,
                                           uint32_t *rows, int lane, bool norm, float alpha) {
    const uint32_t ri = __ldg(c.rowinfo + layer);
    const int d = ri & 255, e0 = static_cast<int>(ri >> 8);
    switch (d) {
#define X(D) \
    case D: layer_f32<D>(c, layer, e0, Zs, rows, lane, norm, alpha); break;
        LDPC_DEG_CASES(X)
#undef X
        default: break;
    }
}

__device__ __forceinline__ void run_layer_i8(const DevCode &c, int layer, uint32_t *Zs,
                                          uint32_t *rows, int lane, bool norm) {
    const uint32_t ri = __ldg(c.rowinfo + layer);
    const int d = ri & 255, e0 = static_cast<int>(ri >> 8);
    switch (d) {
#define X(D) \
    case D: layer_i8<D>(c, layer, e0, Zs, rows, lane, norm); break;
        LDPC_DEG_CASES(X)
#undef X
        default: break;
    }
}

// ---------------------------------------------------------------------------
// Hard decision (eq. 21) and syndrome test after a full iteration.
// ---------------------------------------------------------------------------
// FP32: true when every check is satisfied (warp-uniform).
__device__ __forceinline__ bool syndrome_ok_f32(const DevCode &c, const uint32_t *Zs, int lane) {
    uint32_t bad = 0;
    for (int l = 0; l < c.mb; ++l) {
        const uint32_t ri = __ldg(c.rowinfo + l);
        const int d = ri & 255, e0 = static_cast<int>(ri >> 8);
        for (int t = 0; t < c.rpl; ++t) {
            if (lane + 32 * t >= c.z) break;
            const uint16_t *vo = c.voff + (e0 * c.rpl + t) * 32 + lane;
            uint32_t par = 0;
            for (int e = 0; e < d; ++e) {
                const float zv = __uint_as_float(lds_u32(Zs, __ldg(vo + e * c.rpl * 32)));
                par ^= (zv > 0.0f) ? 0u : 1u;
            }
            bad |= par;
        }
    }
    return !__any_sync(kFull, bad);
}

// int8: per byte, bit 7 set where the posterior is <= 0 (values in [-127, 127]).
__device__ __forceinline__ uint32_t hard_bytes(uint32_t z) {
    const uint32_t t = (z & 0x7F7F7F7Fu) + 0x7F7F7F7Fu;   // bit 7: low 7 bits nonzero
    return (z | ~t) & 0x80808080u;
}

// int8: bit 7 of byte b set when frame b has an unsatisfied check.
__device__ __forceinline__ uint32_t syndrome_bad_i8(const DevCode &c, const uint32_t *Zs, int lane) {
    uint32_t bad = 0;
    for (int l = 0; l < c.mb; ++l) {
        const uint32_t ri = __ldg(c.rowinfo + l);
        const int d = ri & 255, e0 = static_cast<int>(ri >> 8);
        for (int t = 0; t < c.rpl; ++t) {
            if (lane + 32 * t >= c.z) break;
            const uint16_t *vo = c.voff + (e0 * c.rpl + t) * 32 + lane;
            uint32_t par = 0;
            for (int e = 0; e < d; ++e) par ^= hard_bytes(lds_u32(Zs, __ldg(vo + e * c.rpl * 32)));
            bad |= par;
        }
    }
    return __reduce_or_sync(kFull, bad);
}

// ---------------------------------------------------------------------------
// Output of one frame: packed hard decisions, iteration count, posteriors.
// ---------------------------------------------------------------------------
__device__ __forceinline__ void write_frame_f32(const DevCode &c, const uint32_t *Zs, int64_t f, int it,
                                uint32_t *hard, int32_t *iters, float *post, int lane) {
    uint32_t *h = hard + f * c.nwords;
    for (int wb = 0; wb < c.nwords; wb += 32) {
        uint32_t mine = 0;
        for (int i = 0; i < 32 && wb + i < c.nwords; ++i) {
            const int n = (wb + i) * 32 + lane;
            const bool b = n < c.n && !(__uint_as_float(Zs[n]) > 0.0f);
            const uint32_t bal = __ballot_sync(kFull, b);
            if (lane == i) mine = bal;
        }
        if (wb + lane < c.nwords) h[wb + lane] = mine;
    }
    if (lane == 0) iters[f] = it;
    if (post) {
        float *p = post + f * c.n;
        for (int n = lane; n < c.n; n += 32) p[n] = __uint_as_float(Zs[n]);
    }
}

__device__ __forceinline__ void write_frame_i8(const DevCode &c, const uint32_t *Zs, int64_t f, int byte,
                               int it, uint32_t *hard, int32_t *iters, int8_t *post, int lane) {
    uint32_t *h = hard + f * c.nwords;
    const int sh = 8 * byte + 7;
    for (int wb = 0; wb < c.nwords; wb += 32) {
        uint32_t mine = 0;
        for (int i = 0; i < 32 && wb + i < c.nwords; ++i) {
            const int n = (wb + i) * 32 + lane;
            const bool b = n < c.n && ((hard_bytes(Zs[n]) >> sh) & 1u);
            const uint32_t bal = __ballot_sync(kFull, b);
            if (lane == i) mine = bal;
        }
        if (wb + lane < c.nwords) h[wb + lane] = mine;
    }
    if (lane == 0) iters[f] = it;
    if (post) {
        int8_t *p = post + f * c.n;
        for (int n = lane; n < c.n; n += 32)
            p[n] = static_cast<int8_t>((Zs[n] >> (8 * byte)) & 0xFFu);
    }
}

// ---------------------------------------------------------------------------
// Decoder kernel.  Shared memory: [W mbarriers (8 B each, padded to 16 B
// multiples)][W per-warp regions]; a region holds Z_n (N words, 16-byte
// aligned, the bulk-copy target) then the row state of all M rows.
// ---------------------------------------------------------------------------
template <bool I8>
__global__ void __launch_bounds__(128)
    decode_kernel(DevCode c, const uint32_t *__restrict__ llr, int64_t frames, DecodeParams p,
                  uint32_t *__restrict__ hard, int32_t *__restrict__ iters, void *post,
                  int region_words, int use_bulk) {
    extern __shared__ __align__(16) uint32_t smem[];
    const int W = blockDim.x >> 5;
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    uint64_t *bar = reinterpret_cast<uint64_t *>(smem) + warp;
    const int bar_words = ((2 * W) + 3) & ~3;
    uint32_t *Zs = smem + bar_words + warp * region_words;
    const int zwords = (c.n + 3) & ~3;
    uint32_t *rows = Zs + zwords;
    constexpr int RW = I8 ? kRowWordsI8 : kRowWordsF32;
    const bool norm = p.normalise != 0;

    if (use_bulk) {
        if (lane == 0) {
            mbar_init(bar, 1);
            fence_mbar_init();
        }
        __syncwarp();
    }
    uint32_t phase = 0;
    const int64_t units = I8 ? (frames + 3) / 4 : frames;
    for (int64_t u = blockIdx.x * static_cast<int64_t>(W) + warp; u < units;
         u += static_cast<int64_t>(gridDim.x) * W) {
        const uint32_t *src = llr + u * c.n;
        // ---- stage the channel LLRs in (Z_n^(0)) and clear the messages ----
        if (use_bulk) {
            fence_proxy_async_smem();
            __syncwarp();
            if (lane == 0) {
                mbar_arrive_expect_tx(bar, static_cast<uint32_t>(c.n) * 4u);
                bulk_copy_g2s(Zs, src, static_cast<uint32_t>(c.n) * 4u, bar);
            }
        } else {
            for (int i = lane; i < c.n; i += 32) Zs[i] = __ldg(src + i);
        }
        for (int i = lane; i < c.m * RW; i += 32) rows[i] = 0u;   // every L_mn = 0
        if (use_bulk) {
            const bool ok = mbar_wait_bounded(bar, phase, kWaitLimit);
            if (!__all_sync(kFull, ok)) {   // the whole warp gives up together
                if (lane == 0) atomicOr(c.status, kStatusCopyTimeout);
                mbar_wait_bounded(bar, phase, kWaitLimit);   // let the copy land
                return;
            }
            phase ^= 1u;
        }
        __syncwarp();

        if (!I8) {
            int done = p.max_iters;
            for (int k = 1; k <= p.max_iters; ++k) {
                for (int l = 0; l < c.mb; ++l) {
                    run_layer_f32(c, l, Zs, rows, lane, norm, p.alpha);
                    __syncwarp();
                }
                if (p.early_stop && syndrome_ok_f32(c, Zs, lane)) {
                    done = k;
                    break;
                }
            }
            write_frame_f32(c, Zs, u, done, hard, iters, static_cast<float *>(post), lane);
        } else {
            // frames of this group still running: bit 7 of byte b for frame 4u+b
            uint32_t pending = 0;
            for (int b = 0; b < 4; ++b)
                if (4 * u + b < frames) pending |= 0x80u << (8 * b);
            for (int k = 1; k <= p.max_iters && pending; ++k) {
                for (int l = 0; l < c.mb; ++l) {
                    run_layer_i8(c, l, Zs, rows, lane, norm);
                    __syncwarp();
                }
                if (p.early_stop) {
                    const uint32_t fin = pending & ~syndrome_bad_i8(c, Zs, lane);
                    for (int b = 0; b < 4; ++b)
                        if ((fin >> (8 * b + 7)) & 1u)
                            write_frame_i8(c, Zs, 4 * u + b, b, k, hard, iters,
                                           static_cast<int8_t *>(post), lane);
                    pending &= ~fin;
                }
            }
            for (int b = 0; b < 4; ++b)
                if ((pending >> (8 * b + 7)) & 1u)
                    write_frame_i8(c, Zs, 4 * u + b, b, p.max_iters, hard, iters,
                                   static_cast<int8_t *>(post), lane);
        }
        __syncwarp();
    }
}

ldpc_status launch_decode(const Code &c, ldpc_dtype dtype, const void *d_llr, int64_t frames,
                          const DecodeParams &p, uint32_t *d_hard, int32_t *d_iters,
                          void *d_post, cudaStream_t s) {
    const bool i8 = dtype == LDPC_I8X4;
    const int rw = i8 ? kRowWordsI8 : kRowWordsF32;
    const int region_words = (((c.n + 3) & ~3) + c.m * rw + 3) & ~3;
    int dev = 0, sms = 148, max_optin = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    cudaDeviceGetAttribute(&max_optin, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev);
    int W = 4;
    auto smem_for = [&](int w) { return (((2 * w) + 3) & ~3) * 4 + w * region_words * 4; };
    while (W > 1 && smem_for(W) > max_optin) --W;
    const int smem = smem_for(W);
    if (smem > max_optin)
        return fail(LDPC_ERR_UNSUPPORTED, "decode: code too large for shared memory");
    const bool aligned = (reinterpret_cast<uintptr_t>(d_llr) & 15u) == 0 && (c.n % 4) == 0;
    const int use_bulk = aligned ? 1 : 0;
    auto kern = i8 ? decode_kernel<true> : decode_kernel<false>;
    cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, smem);
    if (e != cudaSuccess) return cuda_fail(e, "decode_kernel attribute");
    int per_sm = 0;
    e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kern, W * 32, smem);
    if (e != cudaSuccess) return cuda_fail(e, "decode occupancy");
    per_sm = std::max(per_sm, 1);
    const int64_t units = i8 ? (frames + 3) / 4 : frames;
    const int64_t want = (units + W - 1) / W;
    const int grid = static_cast<int>(std::min<int64_t>(want, static_cast<int64_t>(per_sm) * sms));
    kern<<<grid, W * 32, smem, s>>>(dev_view(c), static_cast<const uint32_t *>(d_llr), frames, p,
                                    d_hard, d_iters, d_post, region_words, use_bulk);
    e = cudaGetLastError();
    return e == cudaSuccess ? LDPC_OK : cuda_fail(e, "decode_kernel");
}

}  // namespace ldpc
