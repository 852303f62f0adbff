// Layered single-scan min-sum decoders of libldpc (arXiv 2306.12063,
// Section 4: eq. 20, 22, 23 under the layered schedule; Section 5 for the
// fixed-point variant, here 8-bit saturating).
//
// Mapping.  One warp decodes one frame (FP32) or four frames at once, one per
// byte of a 32-bit word (int8).  The warp keeps the posteriors Z_n of its
// frames and the compressed check messages of every row in shared memory for
// all iterations.  Lane l handles rows l, l+32, ... of the current layer; the
// Z rows of a layer touch disjoint variables, so a layer needs only a
// __syncwarp before the next one.  The variable of each edge,
// j Z + (r + s) mod Z (the circulant's cyclic shift as an index rotation),
// comes from a per-lane offset table built with the code.
//
// Each kernel is built for a slot class DMAX (8, 12, ..., 27 edge slots per
// row, the smallest that holds the code's largest row degree) and runs every
// row as straight-line code over all DMAX slots; a row of degree d fills the
// last d slots and the leading ones read a dummy posterior (one word per
// lane after Z_n) that cannot change the row.  Per-edge state (the argmin,
// the sign bits) is indexed by slot.
//
// Scheduling.  Frames are handed out by an atomic counter, so a warp whose
// frame stops early takes the next one.  In the int8 kernel each byte lane
// is refilled on its own: when one of the four frames in a word passes its
// parity check (or reaches max_iters) its outputs are written and the next
// frame is loaded into that byte while the other three keep iterating.
#include <algorithm>
#include <atomic>

#include "ldpc_decode_dev.cuh"

namespace ldpc {

// Cap on the persistent grid of the single-code decoders (0: none), set by
// ldpc_test_set_grid_cap.
static std::atomic<int> g_grid_cap{0};

// `cap` lowered to the testing cap, if one is set.

int64_t grid_cap(int64_t cap) {
    const int v = g_grid_cap.load(std::memory_order_relaxed);
    return v > 0 ? std::min<int64_t>(cap, v) : cap;
}

// ---------------------------------------------------------------------------
// Kernels, one warp per block.  Shared memory: [mbarrier (16 B)][Z_n: N
// words, 16-byte aligned, the bulk-copy target, then 32 dummy words][row
// state of all M rows].
// With a single warp the posterior array sits at a fixed shared address, so
// every access is one load or store at the table offset.
// ---------------------------------------------------------------------------
template <int DMAX, bool WT = false, int DM = DMAX>
__global__ void __launch_bounds__(32)
    decode_f32_kernel(DevCode c, const uint32_t *__restrict__ llr, int64_t frames, DecodeParams p,
                      uint32_t *__restrict__ hard, int32_t *__restrict__ iters,
                      float *__restrict__ post, unsigned long long *work, int region_words,
                      int use_bulk) {
    extern __shared__ __align__(16) uint32_t smem[];
    constexpr int W = 1;   // one warp per block: Z_n sits at a fixed shared address
    const int warp = 0, lane = threadIdx.x & 31;
    uint64_t *bar = reinterpret_cast<uint64_t *>(smem);
    uint32_t *Zs = smem + 4;
    uint32_t *rows = Zs + posterior_words(c.n);   // Z_n words, then the per-lane dummy words
    // learned weights, [kWeightBuffers][mb][wpad(DMAX)], 16-byte aligned
    float *wbuf = reinterpret_cast<float *>(rows + ((c.m * kRowWordsF32 + 3) & ~3));
    Zs[c.n + lane] = 0x7F800000u;   // dummy posterior +inf for unused edge slots
    if (use_bulk) {
        if (lane == 0) {
            mbar_init(bar, 1);
            fence_mbar_init();
        }
    }
    __syncwarp();
    uint32_t phase = 0;
    const int64_t nwarps = static_cast<int64_t>(gridDim.x) * W;
    // the first frame static, the rest from the counter, each drawn one frame
    // ahead so that its LLRs are pulled into L2 while this one decodes
    int64_t f = blockIdx.x * static_cast<int64_t>(W) + warp;
    int64_t pend = f < frames ? next_work(work, nwarps, lane) : frames;
    while (f < frames) {
        if (pend < frames) prefetch_l2(llr + pend * c.n, 4u * static_cast<uint32_t>(c.n), lane);
        const int done = decode_one_f32<DMAX, WT, DM>(c, Zs, rows, wbuf, llr + f * c.n,
                                                      use_bulk != 0, bar, phase, p, lane);
        if (!done) return;
        write_frame_f32(c, Zs, f, done, hard, iters, post, lane);
        __syncwarp();
        f = pend;
        if (f < frames) pend = next_work(work, nwarps, lane);
    }
}

template <int DMAX, int DM = DMAX>
__global__ void __launch_bounds__(32)
    decode_i8_kernel(DevCode c, const uint32_t *__restrict__ llr, int64_t frames, DecodeParams p,
                     uint32_t *__restrict__ hard, int32_t *__restrict__ iters,
                     int8_t *__restrict__ post, unsigned long long *work, int region_words,
                     int use_bulk) {
    extern __shared__ __align__(16) uint32_t smem[];
    constexpr int W = 1;   // one warp per block: Z_n sits at a fixed shared address
    const int warp = 0, lane = threadIdx.x & 31;
    uint64_t *bar = reinterpret_cast<uint64_t *>(smem);
    uint32_t *Zs = smem + 4;
    uint32_t *rows = Zs + posterior_words(c.n);   // Z_n words, then the per-lane dummy words
    const bool norm = p.normalise != 0;
    const int64_t nwarps = static_cast<int64_t>(gridDim.x) * W;
    const int64_t g0 = blockIdx.x * static_cast<int64_t>(W) + warp;
    if (4 * g0 >= frames) return;

    // Initial fill: this warp's own group of four frames in one bulk copy.
    int64_t fr[4];
    int kb[4];
    for (int b = 0; b < 4; ++b) {
        fr[b] = (4 * g0 + b < frames) ? 4 * g0 + b : -1;
        kb[b] = 0;
    }
    {
        const uint32_t *src = llr + g0 * c.n;
        if (use_bulk) {
            if (lane == 0) {
                mbar_init(bar, 1);
                fence_mbar_init();
            }
            __syncwarp();
            uint32_t phase = 0;
            if (!stage_bulk(c, Zs, src, bar, phase, lane)) return;
            for (int i = lane; i < c.n; i += 32) Zs[i] = to_offset127(Zs[i]);
        } else {
            for (int i = lane; i < c.n; i += 32) Zs[i] = to_offset127(__ldg(src + i));
        }
        for (int i = lane; i < c.m * row_words_i8(DMAX); i += 32) rows[i] = 0u;
        Zs[c.n + lane] = kDummyI8;   // dummy posterior +127 for unused edge slots
        __syncwarp();
    }
    const int64_t dyn_base = 4 * nwarps;   // frames beyond the initial groups
    // the next refill's frame, drawn one refill ahead so that its packed row
    // is pulled into L2 while the word keeps iterating
    int64_t pend = next_work(work, dyn_base, lane);
    if (pend < frames) prefetch_l2(llr + (pend >> 2) * c.n, 4u * static_cast<uint32_t>(c.n), lane);
    for (;;) {
        bool any = false;
        for (int b = 0; b < 4; ++b) any |= fr[b] >= 0;
        if (!any) break;
        uint32_t live = 0;   // byte lanes decoding a frame (debug saturation count)
#ifdef LDPC_DEBUG
        for (int b = 0; b < 4; ++b) live |= fr[b] >= 0 ? 0xFFu << (8 * b) : 0u;
#endif
        for (int l = 0; l < c.mb; ++l) {
            layer_i8_any<DMAX, DM>(c, l, Zs, rows, lane, norm, live);
            __syncwarp();
        }
        uint32_t need = 0;   // bit 7 of every byte lane decoding a frame
        for (int b = 0; b < 4; ++b) need |= fr[b] >= 0 ? 0x80u << (8 * b) : 0u;
        const uint32_t bad =
            p.early_stop ? syndrome_bad_i8<DMAX, DM>(c, Zs, lane, need) : 0x80808080u;
        for (int b = 0; b < 4; ++b) {
            if (fr[b] < 0) continue;
            kb[b] += 1;
            const bool ok = !((bad >> (8 * b + 7)) & 1u);
            if (!ok && kb[b] < p.max_iters) continue;
            // frame finished at this iteration: outputs now, then refill the byte
            write_frame_i8(c, Zs, fr[b], b, kb[b], hard, iters, post, lane);
            const int64_t nf = pend;
            if (nf >= frames) {
                fr[b] = -1;
                continue;
            }
            pend = next_work(work, dyn_base, lane);
            if (pend < frames)
                prefetch_l2(llr + (pend >> 2) * c.n, 4u * static_cast<uint32_t>(c.n), lane);
            fr[b] = nf;
            kb[b] = 0;
            const uint32_t *src = llr + (nf >> 2) * c.n;
            const uint32_t sel = (0x3210u & ~(0xFu << (4 * b))) |
                                 (static_cast<uint32_t>(4 + (nf & 3)) << (4 * b));
            __syncwarp();
            // eight loads in flight per lane (sixteen cost more than they hide)
#pragma unroll 8
            for (int i = lane; i < c.n; i += 32)
                Zs[i] = prmt(Zs[i], to_offset127(__ldg(src + i)), sel);
            const uint32_t keep = ~(0xFFu << (8 * b));
            clear_row_minima_i8<DMAX>(rows, c.m, keep, lane);
            __syncwarp();
        }
    }
}

template <int DMAX, int DM>
static ldpc_status launch_decode_t(const Code &c, bool i8, const void *d_llr, int64_t frames,
                                   const DecodeParams &p, uint32_t *d_hard, int32_t *d_iters,
                                   void *d_post, cudaStream_t s) {
    const int rw = i8 ? row_words_i8(DMAX) : kRowWordsF32;
    const int region_words = (posterior_words(c.n) + c.m * rw + 3) & ~3;
    int dev = 0, sms = 148, max_optin = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    cudaDeviceGetAttribute(&max_optin, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev);
    const int smem = 16 + region_words * 4;
    if (smem > max_optin)
        return fail(LDPC_ERR_UNSUPPORTED, "decode: code too large for shared memory");
    const bool aligned = (reinterpret_cast<uintptr_t>(d_llr) & 15u) == 0 && (c.n % 4) == 0;
    const int use_bulk = aligned ? 1 : 0;
    const void *kern = i8 ? reinterpret_cast<const void *>(decode_i8_kernel<DMAX, DM>)
                          : reinterpret_cast<const void *>(decode_f32_kernel<DMAX, false, DM>);
    cudaError_t e = allow_dynamic_smem(reinterpret_cast<const void *>(kern));
    if (e != cudaSuccess) return cuda_fail(e, "decode kernel attribute");
    int per_sm = 0;
    e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kern, 32, smem);
    if (e != cudaSuccess) return cuda_fail(e, "decode occupancy");
    per_sm = std::max(per_sm, 1);
    const int64_t units = i8 ? (frames + 3) / 4 : frames;
    const int64_t cap = grid_cap(static_cast<int64_t>(per_sm) * sms);
    const int grid = static_cast<int>(std::min<int64_t>(units, cap));
    unsigned long long *work = work_slot(c, s);
    if (!work) return LDPC_ERR_CUDA;
    const DevCode dc = dev_view(c);
    const uint32_t *in = static_cast<const uint32_t *>(d_llr);
    if (i8)
        decode_i8_kernel<DMAX, DM><<<grid, 32, smem, s>>>(dc, in, frames, p, d_hard, d_iters,
                                                          static_cast<int8_t *>(d_post), work,
                                                          region_words, use_bulk);
    else
        decode_f32_kernel<DMAX, false, DM><<<grid, 32, smem, s>>>(
            dc, in, frames, p, d_hard, d_iters, static_cast<float *>(d_post), work,
            region_words, use_bulk);
    e = cudaGetLastError();
    return e == cudaSuccess ? LDPC_OK : cuda_fail(e, "decode kernel launch");
}

ldpc_status launch_decode(const Code &c, ldpc_dtype dtype, const void *d_llr, int64_t frames,
                          const DecodeParams &p, uint32_t *d_hard, int32_t *d_iters,
                          void *d_post, cudaStream_t s) {
    const bool i8 = dtype == LDPC_I8X4;
    // the instance fitted to the code's largest row degree (see small_slots)
    const int dm = c.max_deg >= c.dslots - 3 ? c.max_deg : c.dslots;
    switch (c.dslots * 32 + dm) {
#define L(D, M)          \
    case D * 32 + M:     \
        return launch_decode_t<D, M>(c, i8, d_llr, frames, p, d_hard, d_iters, d_post, s);
        LDPC_FITTED_SLOTS(L)
#undef L
        default: return fail(LDPC_ERR_UNSUPPORTED, "decode: no kernel for this row degree");
    }
}

template <int DMAX>
static ldpc_status launch_learned_t(const Code &c, const float *d_llr, int64_t frames,
                                   const DecodeParams &p, uint32_t *d_hard, int32_t *d_iters,
                                   float *d_post, cudaStream_t s) {
    const int region_words = (posterior_words(c.n) + c.m * kRowWordsF32 + 3) & ~3;
    const int smem = 16 + (region_words + kWeightBuffers * c.mb * wpad(DMAX)) * 4;
    int dev = 0, sms = 148, max_optin = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    cudaDeviceGetAttribute(&max_optin, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev);
    if (smem > max_optin)
        return fail(LDPC_ERR_UNSUPPORTED, "decode: code too large for shared memory");
    const bool aligned = (reinterpret_cast<uintptr_t>(d_llr) & 15u) == 0 && (c.n % 4) == 0;
    const void *kern = reinterpret_cast<const void *>(decode_f32_kernel<DMAX, true>);
    cudaError_t e = allow_dynamic_smem(reinterpret_cast<const void *>(kern));
    if (e != cudaSuccess) return cuda_fail(e, "decode kernel attribute");
    int per_sm = 0;
    e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kern, 32, smem);
    if (e != cudaSuccess) return cuda_fail(e, "decode occupancy");
    per_sm = std::max(per_sm, 1);
    const int64_t cap = grid_cap(static_cast<int64_t>(per_sm) * sms);
    const int grid = static_cast<int>(std::min<int64_t>(frames, cap));
    unsigned long long *work = work_slot(c, s);
    if (!work) return LDPC_ERR_CUDA;
    decode_f32_kernel<DMAX, true><<<grid, 32, smem, s>>>(
        dev_view(c), reinterpret_cast<const uint32_t *>(d_llr), frames, p, d_hard, d_iters,
        d_post, work, region_words, aligned ? 1 : 0);
    e = cudaGetLastError();
    return e == cudaSuccess ? LDPC_OK : cuda_fail(e, "learned decode kernel launch");
}

ldpc_status launch_decode_learned(const Code &c, const float *d_llr, int64_t frames,
                                  const DecodeParams &p, uint32_t *d_hard, int32_t *d_iters,
                                  float *d_post, cudaStream_t s) {
    switch (c.dslots) {
#define L(D) \
    case D: return launch_learned_t<D>(c, d_llr, frames, p, d_hard, d_iters, d_post, s);
        LDPC_SLOT_CLASSES(L)
#undef L
        default: return fail(LDPC_ERR_UNSUPPORTED, "decode: no kernel for this row degree");
    }
}

// Launch on a kernel-side code view whose tables, status word and work
// counter are supplied by the caller (the entry point that allocates
// nothing keeps them in a static device array).
template <int DMAX>
static ldpc_status launch_decode_view_t(const DevCode &dc, bool i8, const void *d_llr,
                                        int64_t frames, const DecodeParams &p, uint32_t *d_hard,
                                        int32_t *d_iters, void *d_post,
                                        unsigned long long *work, cudaStream_t s) {
    const int rw = i8 ? row_words_i8(DMAX) : kRowWordsF32;
    const int region_words = (posterior_words(dc.n) + dc.m * rw + 3) & ~3;
    int dev = 0, sms = 148, max_optin = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    cudaDeviceGetAttribute(&max_optin, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev);
    const int smem = 16 + region_words * 4;
    if (smem > max_optin)
        return fail(LDPC_ERR_UNSUPPORTED, "decode: code too large for shared memory");
    const bool aligned = (reinterpret_cast<uintptr_t>(d_llr) & 15u) == 0 && (dc.n % 4) == 0;
    const void *kern = i8 ? reinterpret_cast<const void *>(decode_i8_kernel<DMAX>)
                          : reinterpret_cast<const void *>(decode_f32_kernel<DMAX>);
    cudaError_t e = allow_dynamic_smem(reinterpret_cast<const void *>(kern));
    if (e != cudaSuccess) return cuda_fail(e, "decode kernel attribute");
    int per_sm = 0;
    e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kern, 32, smem);
    if (e != cudaSuccess) return cuda_fail(e, "decode occupancy");
    per_sm = std::max(per_sm, 1);
    const int64_t units = i8 ? (frames + 3) / 4 : frames;
    const int grid =
        static_cast<int>(std::min<int64_t>(units, static_cast<int64_t>(per_sm) * sms));
    const uint32_t *in = static_cast<const uint32_t *>(d_llr);
    if (i8)
        decode_i8_kernel<DMAX><<<grid, 32, smem, s>>>(dc, in, frames, p, d_hard, d_iters,
                                                      static_cast<int8_t *>(d_post), work,
                                                      region_words, aligned ? 1 : 0);
    else
        decode_f32_kernel<DMAX><<<grid, 32, smem, s>>>(dc, in, frames, p, d_hard, d_iters,
                                                       static_cast<float *>(d_post), work,
                                                       region_words, aligned ? 1 : 0);
    e = cudaGetLastError();
    return e == cudaSuccess ? LDPC_OK : cuda_fail(e, "decode kernel launch");
}

ldpc_status launch_decode_view(const DevCode &dc, ldpc_dtype dtype, const void *d_llr,
                               int64_t frames, const DecodeParams &p, uint32_t *d_hard,
                               int32_t *d_iters, void *d_post, unsigned long long *work,
                               cudaStream_t s) {
    const bool i8 = dtype == LDPC_I8X4;
    switch (dc.dslots) {
#define L(D)                                                                                 \
    case D:                                                                                  \
        return launch_decode_view_t<D>(dc, i8, d_llr, frames, p, d_hard, d_iters, d_post,  \
                                       work, s);
        LDPC_SLOT_CLASSES(L)
#undef L
        default: return fail(LDPC_ERR_UNSUPPORTED, "decode: no kernel for this row degree");
    }
}

}  // namespace ldpc

extern "C" ldpc_status ldpc_test_set_grid_cap(int blocks) {
    if (blocks < 0)
        return ldpc::fail(LDPC_ERR_INVALID_ARG, "ldpc_test_set_grid_cap: negative cap");
    ldpc::g_grid_cap.store(blocks, std::memory_order_relaxed);
    return LDPC_OK;
}
