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
// A row's edges are processed by one fully unrolled sequence of kMaxRowDeg
// slots entered at slot kMaxRowDeg - d (a computed jump), so every degree
// shares one copy of the code; per-edge state (the argmin, the sign bits)
// is indexed by slot.
//
// Scheduling.  Frames are handed out by an atomic counter, so a warp whose
// frame stops early takes the next one.  In the int8 kernel each byte lane
// is refilled on its own: when one of the four frames in a word passes its
// parity check (or reaches max_iters) its outputs are written and the next
// frame is loaded into that byte while the other three keep iterating.
#include <algorithm>
#include <cstdlib>

#include "ldpc_internal.cuh"

namespace ldpc {

constexpr uint32_t kFull = 0xFFFFFFFFu;
constexpr uint32_t kWaitLimit = 1u << 22;   // polls of a bulk-copy barrier
constexpr int DMAX = kMaxRowDeg;

// Row state words in shared memory (per check row):
//   FP32: [m1, m2, meta, -]; m1, m2 scaled magnitudes; meta bits 0..26 hold
//         the sign of L_mn for slot i at bit DMAX-1-i, bits 27..31 the argmin
//         slot.
//   int8: [M1, M2, IDX, SG0, SG1, SG2, SG3, -], one byte per frame: scaled
//         magnitudes and argmin slot; SGk byte b bit u = sign of L_mn of frame
//         b for slot 8k + u.
constexpr int kRowWordsF32 = 4;
constexpr int kRowWordsI8 = 8;

__device__ __forceinline__ uint32_t lds_u32(const uint32_t *base, uint32_t byte_off) {
    return *reinterpret_cast<const uint32_t *>(reinterpret_cast<const char *>(base) + byte_off);
}
__device__ __forceinline__ void sts_u32(uint32_t *base, uint32_t byte_off, uint32_t v) {
    *reinterpret_cast<uint32_t *>(reinterpret_cast<char *>(base) + byte_off) = v;
}

// Fixed-width bit helpers (single instructions).
__device__ __forceinline__ uint32_t prmt(uint32_t a, uint32_t b, uint32_t sel) {
    uint32_t r;
    asm("prmt.b32 %0, %1, %2, %3;" : "=r"(r) : "r"(a), "r"(b), "r"(sel));
    return r;
}
__device__ __forceinline__ uint32_t clamp_u16x2(uint32_t x, uint32_t lo, uint32_t hi) {
    uint32_t r;
    asm("max.u16x2 %0, %1, %2;" : "=r"(r) : "r"(x), "r"(lo));
    asm("min.u16x2 %0, %0, %1;" : "+r"(r) : "r"(hi));
    return r;
}
// Bytes 0, 2 (resp. 1, 3) of x zero-extended into two 16-bit lanes.
__device__ __forceinline__ uint32_t lanes_even(uint32_t x) { return prmt(x, 0u, 0x4240u); }
__device__ __forceinline__ uint32_t lanes_odd(uint32_t x) { return prmt(x, 0u, 0x4341u); }
// Low bytes of the lanes of e (frames 0, 2) and o (frames 1, 3) back into one word.
__device__ __forceinline__ uint32_t lanes_join(uint32_t e, uint32_t o) { return prmt(e, o, 0x6240u); }
// Per byte: 0xFF where a < b, for a, b <= 127.
__device__ __forceinline__ uint32_t lt_mask7(uint32_t a, uint32_t b) {
    return msb_bytes_to_mask(b + 0x7F7F7F7Fu - a);
}
// Per byte: 0xFF where x != 0, for x <= 128.
__device__ __forceinline__ uint32_t nonzero_mask(uint32_t x) {
    return msb_bytes_to_mask(x + 0x7F7F7F7Fu);
}
// Per byte floor(3 m / 4) = m - ceil(m / 4), m <= 127 (no carry crosses bytes).
__device__ __forceinline__ uint32_t scale34(uint32_t m) {
    return m - (((m + 0x03030303u) >> 2) & 0x3F3F3F3Fu);
}

#define LDPC_SLOTS(X)                                                                       \
    X(0) X(1) X(2) X(3) X(4) X(5) X(6) X(7) X(8) X(9) X(10) X(11) X(12) X(13) X(14) X(15) \
    X(16) X(17) X(18) X(19) X(20) X(21) X(22) X(23) X(24) X(25) X(26)
static_assert(DMAX == 27, "slot list must match kMaxRowDeg");

// ---------------------------------------------------------------------------
// FP32 layer: eq. (22) Z_mn = Z_n - L_mn; eq. (23) new L_mn from the
// smallest and second smallest |Z_mn| and the product of signs; eq. (20) in
// single-scan form Z_n = Z_mn + L_mn.  Each float operation is an explicitly
// rounded intrinsic, so no multiply-add is ever contracted.
// ---------------------------------------------------------------------------
__device__ __forceinline__ void layer_f32(const DevCode &c, int layer, uint32_t *Zs,
                                          uint32_t *rows, int lane, bool norm, float alpha) {
    const uint32_t ri = __ldg(c.rowinfo + layer);
    const int d = ri & 255, e0 = static_cast<int>(ri >> 8);
    const int start = DMAX - d;
    const int stride = c.rpl * 32;
    for (int t = 0; t < c.rpl; ++t) {
        const int r = lane + 32 * t;
        if (r >= c.z) break;
        uint4 *rs = reinterpret_cast<uint4 *>(rows + (layer * c.z + r) * kRowWordsF32);
        const uint4 st = *rs;
        const float m1 = __uint_as_float(st.x), m2 = __uint_as_float(st.y);
        const uint32_t meta = st.z;
        const int idx = static_cast<int>(meta >> 27);
        const int vb = (e0 * c.rpl + t) * 32 + lane - start * stride;   // slot i: vb + i * stride
        uint32_t off[DMAX];
        float Q[DMAX];
        float mn1 = __int_as_float(0x7F800000), mn2 = mn1;
        int id = 0;
        uint32_t sx = 0;
        switch (start) {
#define P1(i)                                                                                \
    case i: {                                                                                \
        off[i] = __ldg(c.voff + vb + (i) * stride);                                                   \
        const float zv = __uint_as_float(lds_u32(Zs, off[i]));                               \
        const float mag = (idx == (i)) ? m2 : m1;                                            \
        const float L = __uint_as_float(__float_as_uint(mag) |                               \
                                        ((meta << ((i) + 32 - DMAX)) & 0x80000000u));        \
        const float q = __fsub_rn(zv, L);                                                    \
        Q[i] = q;                                                                            \
        const float a = fabsf(q);                                                            \
        mn2 = fminf(mn2, fmaxf(mn1, a));                                                     \
        id = (a < mn1) ? (i) : id;                                                           \
        mn1 = fminf(mn1, a);                                                                 \
        sx ^= __float_as_uint(q);                                                            \
    }
            LDPC_SLOTS(P1)
#undef P1
            default: break;
        }
        const float n1 = norm ? __fmul_rn(alpha, mn1) : mn1;
        const float n2 = norm ? __fmul_rn(alpha, mn2) : mn2;
        const uint32_t S = sx & 0x80000000u;
        const uint32_t s1 = __float_as_uint(n1) | S, s2 = __float_as_uint(n2) | S;
        uint32_t nsg = 0;
        switch (start) {
#define P2(i)                                                                                \
    case i: {                                                                                \
        const uint32_t ms = (id == (i)) ? s2 : s1;                                           \
        const uint32_t L = ms ^ (__float_as_uint(Q[i]) & 0x80000000u);                      \
        sts_u32(Zs, off[i], __float_as_uint(__fadd_rn(Q[i], __uint_as_float(L))));           \
        nsg = __funnelshift_l(L, nsg, 1);                                                    \
    }
            LDPC_SLOTS(P2)
#undef P2
            default: break;
        }
        *rs = make_uint4(__float_as_uint(n1), __float_as_uint(n2),
                         nsg | (static_cast<uint32_t>(id) << 27), 0u);
    }
}

// FP32 hard decision (eq. 21) and syndrome: true when every check holds.
__device__ __forceinline__ bool syndrome_ok_f32(const DevCode &c, const uint32_t *Zs, int lane) {
    uint32_t bad = 0;
    const int stride = c.rpl * 32;
    for (int l = 0; l < c.mb; ++l) {
        const uint32_t ri = __ldg(c.rowinfo + l);
        const int d = ri & 255, e0 = static_cast<int>(ri >> 8);
        const int start = DMAX - d;
        for (int t = 0; t < c.rpl; ++t) {
            if (lane + 32 * t >= c.z) break;
            const int vb = (e0 * c.rpl + t) * 32 + lane - start * stride;   // slot i: vb + i * stride
            uint32_t par = 0;
            switch (start) {
#define SY(i) \
    case i: par ^= (__uint_as_float(lds_u32(Zs, __ldg(c.voff + vb + (i) * stride))) > 0.0f) ? 0u : 1u;
                LDPC_SLOTS(SY)
#undef SY
                default: break;
            }
            bad |= par;
        }
    }
    return !__any_sync(kFull, bad);
}

// ---------------------------------------------------------------------------
// int8 layer, four frames per word.  Posteriors are held in shared memory in
// offset form (Z + 128, one byte per frame, 1..255).  The check side works on
// two's-complement bytes: |Z_mn|, the running minimum and second minimum,
// the argmin slot and the sign parity, with byte-wise compare masks built by
// prmt's sign replication.  The saturating additions Z_mn = Z_n - L_mn and
// Z_n = Z_mn + L_mn run on two 16-bit lanes per word (frames 0, 2 and 1, 3)
// holding non-negative biased values, clamped with packed u16 min/max.
// ---------------------------------------------------------------------------
__device__ __forceinline__ void layer_i8(const DevCode &c, int layer, uint32_t *Zs, uint32_t *rows,
                                         int lane, bool norm) {
    const uint32_t ri = __ldg(c.rowinfo + layer);
    const int d = ri & 255, e0 = static_cast<int>(ri >> 8);
    const int start = DMAX - d;
    const int stride = c.rpl * 32;
    for (int t = 0; t < c.rpl; ++t) {
        const int r = lane + 32 * t;
        if (r >= c.z) break;
        uint32_t *rs = rows + (layer * c.z + r) * kRowWordsI8;
        const uint4 st0 = reinterpret_cast<const uint4 *>(rs)[0];
        const uint4 st1 = reinterpret_cast<const uint4 *>(rs)[1];
        const uint32_t IDX = st0.z;
        const uint32_t SG[4] = {st0.w, st1.x, st1.y, st1.z};
        // offset-128 bytes of -L_old for the four (sign, magnitude) cases
        const uint32_t P1c = 0x80808080u - st0.x, P2c = 0x80808080u - st0.y;   // L > 0
        const uint32_t N1c = 0x80808080u | st0.x, N2c = 0x80808080u | st0.y;   // L < 0
        const int vb = (e0 * c.rpl + t) * 32 + lane - start * stride;   // slot i: vb + i * stride
        uint32_t off[DMAX], Q[DMAX];
        uint32_t mn1 = 0x7F7F7F7Fu, mn2 = 0x7F7F7F7Fu, id = 0, sx = 0;
        switch (start) {
#define I1(i)                                                                                \
    case i: {                                                                                \
        off[i] = __ldg(c.voff + vb + (i) * stride);                                                   \
        const uint32_t u = lds_u32(Zs, off[i]);                                              \
        const uint32_t sm = msb_bytes_to_mask(SG[(i) >> 3] << (7 - ((i) & 7)));              \
        const uint32_t nq = nonzero_mask(IDX ^ (0x01010101u * (i)));                         \
        const uint32_t nl = bsel(bsel(P2c, P1c, nq), bsel(N2c, N1c, nq), sm);                \
        const uint32_t qe = clamp_u16x2(lanes_even(u) + lanes_even(nl), 0x00810081u,         \
                                        0x017F017Fu);                                        \
        const uint32_t qo = clamp_u16x2(lanes_odd(u) + lanes_odd(nl), 0x00810081u,           \
                                        0x017F017Fu);                                        \
        const uint32_t q = lanes_join(qe, qo);                                               \
        Q[i] = q;                                                                            \
        const uint32_t sq = msb_bytes_to_mask(q);                                            \
        const uint32_t a = (q ^ sq) + (sq & 0x01010101u);                                    \
        const uint32_t lt = lt_mask7(a, mn1);                                                \
        const uint32_t tmax = bsel(a, mn1, lt);                                              \
        mn1 = bsel(mn1, a, lt);                                                              \
        id = bsel(id, 0x01010101u * (i), lt);                                                \
        mn2 = bsel(mn2, tmax, lt_mask7(tmax, mn2));                                          \
        sx ^= q;                                                                             \
    }
            LDPC_SLOTS(I1)
#undef I1
            default: break;
        }
        const uint32_t n1 = norm ? scale34(mn1) : mn1;
        const uint32_t n2 = norm ? scale34(mn2) : mn2;
        const uint32_t S = sx & 0x80808080u;
        // offset-128 bytes of L_new for the four (sign, magnitude) cases
        const uint32_t Lp1 = 0x80808080u | n1, Lp2 = 0x80808080u | n2;       // L > 0
        const uint32_t Ln1 = 0x80808080u - n1, Ln2 = 0x80808080u - n2;       // L < 0
        uint32_t nsg[4] = {0u, 0u, 0u, 0u};
        switch (start) {
#define I2(i)                                                                                \
    case i: {                                                                                \
        const uint32_t q = Q[i];                                                             \
        const uint32_t neg = (q ^ S) & 0x80808080u;                                          \
        const uint32_t nq = nonzero_mask(id ^ (0x01010101u * (i)));                          \
        const uint32_t y = bsel(bsel(Lp2, Lp1, nq), bsel(Ln2, Ln1, nq), msb_bytes_to_mask(neg)); \
        const uint32_t x = q ^ 0x80808080u;                                                  \
        const uint32_t ze = clamp_u16x2(lanes_even(x) + lanes_even(y) + 0x00800080u,         \
                                        0x01010101u, 0x01FF01FFu);                           \
        const uint32_t zo = clamp_u16x2(lanes_odd(x) + lanes_odd(y) + 0x00800080u,           \
                                        0x01010101u, 0x01FF01FFu);                           \
        sts_u32(Zs, off[i], lanes_join(ze, zo));                                             \
        nsg[(i) >> 3] |= neg >> (7 - ((i) & 7));                                             \
    }
            LDPC_SLOTS(I2)
#undef I2
            default: break;
        }
        reinterpret_cast<uint4 *>(rs)[0] = make_uint4(n1, n2, id, nsg[0]);
        reinterpret_cast<uint4 *>(rs)[1] = make_uint4(nsg[1], nsg[2], nsg[3], 0u);
    }
}

// int8 hard decision per byte: bit 7 set where Z <= 0, i.e. offset value <= 128.
__device__ __forceinline__ uint32_t hard_bytes_off(uint32_t u) {
    return ~(u - 0x01010101u) & 0x80808080u;   // u >= 1: no borrow crosses bytes
}

// int8 syndrome: bit 7 of byte b set when frame b has an unsatisfied check.
__device__ __forceinline__ uint32_t syndrome_bad_i8(const DevCode &c, const uint32_t *Zs,
                                                    int lane) {
    uint32_t bad = 0;
    const int stride = c.rpl * 32;
    for (int l = 0; l < c.mb; ++l) {
        const uint32_t ri = __ldg(c.rowinfo + l);
        const int d = ri & 255, e0 = static_cast<int>(ri >> 8);
        const int start = DMAX - d;
        for (int t = 0; t < c.rpl; ++t) {
            if (lane + 32 * t >= c.z) break;
            const int vb = (e0 * c.rpl + t) * 32 + lane - start * stride;   // slot i: vb + i * stride
            uint32_t par = 0;
            switch (start) {
#define SY(i) \
    case i: par ^= hard_bytes_off(lds_u32(Zs, __ldg(c.voff + vb + (i) * stride)));
                LDPC_SLOTS(SY)
#undef SY
                default: break;
            }
            bad |= par;
        }
    }
    return __reduce_or_sync(kFull, bad);
}

// ---------------------------------------------------------------------------
// Outputs of one frame: packed hard decisions, iteration count, posteriors.
// ---------------------------------------------------------------------------
__device__ __forceinline__ void write_frame_f32(const DevCode &c, const uint32_t *Zs, int64_t f,
                                                int it, uint32_t *hard, int32_t *iters,
                                                float *post, int lane) {
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

__device__ __forceinline__ void write_frame_i8(const DevCode &c, const uint32_t *Zs, int64_t f,
                                               int byte, int it, uint32_t *hard, int32_t *iters,
                                               int8_t *post, int lane) {
    uint32_t *h = hard + f * c.nwords;
    const int sh = 8 * byte + 7;
    for (int wb = 0; wb < c.nwords; wb += 32) {
        uint32_t mine = 0;
        for (int i = 0; i < 32 && wb + i < c.nwords; ++i) {
            const int n = (wb + i) * 32 + lane;
            const bool b = n < c.n && ((hard_bytes_off(Zs[n]) >> sh) & 1u);
            const uint32_t bal = __ballot_sync(kFull, b);
            if (lane == i) mine = bal;
        }
        if (wb + lane < c.nwords) h[wb + lane] = mine;
    }
    if (lane == 0) iters[f] = it;
    if (post) {
        int8_t *p = post + f * c.n;
        for (int n = lane; n < c.n; n += 32)
            p[n] = static_cast<int8_t>(((Zs[n] >> (8 * byte)) & 0xFFu) ^ 0x80u);
    }
}

// ---------------------------------------------------------------------------
// Stage-in helpers.
// ---------------------------------------------------------------------------
// Bulk copy of n words from global to Zs, bounded wait.  Returns false (whole
// warp) if the copy did not complete in time; the status word records it.
__device__ __forceinline__ bool stage_bulk(const DevCode &c, uint32_t *Zs, const uint32_t *src,
                                           uint64_t *bar, uint32_t &phase, int lane) {
    fence_proxy_async_smem();
    __syncwarp();
    if (lane == 0) {
        mbar_arrive_expect_tx(bar, static_cast<uint32_t>(c.n) * 4u);
        bulk_copy_g2s(Zs, src, static_cast<uint32_t>(c.n) * 4u, bar);
    }
    const bool ok = mbar_wait_bounded(bar, phase, kWaitLimit);
    if (!__all_sync(kFull, ok)) {
        if (lane == 0) atomicOr(c.status, kStatusCopyTimeout);
        mbar_wait_bounded(bar, phase, kWaitLimit);   // let the copy land before leaving
        return false;
    }
    phase ^= 1u;
    return true;
}

__device__ __forceinline__ int64_t next_work(unsigned long long *ctr, int64_t base, int lane) {
    unsigned long long v = 0;
    if (lane == 0) v = atomicAdd(ctr, 1ull);
    v = __shfl_sync(kFull, v, 0);
    return base + static_cast<int64_t>(v);
}

// ---------------------------------------------------------------------------
// Kernels.  Shared memory: [W mbarriers (padded to 16 B)][W per-warp regions];
// a region holds Z_n (N words, 16-byte aligned: the bulk-copy target) and then
// the row state of all M rows.
// ---------------------------------------------------------------------------
__global__ void __launch_bounds__(128)
    decode_f32_kernel(DevCode c, const uint32_t *__restrict__ llr, int64_t frames, DecodeParams p,
                      uint32_t *__restrict__ hard, int32_t *__restrict__ iters,
                      float *__restrict__ post, unsigned long long *work, int region_words,
                      int use_bulk) {
    extern __shared__ __align__(16) uint32_t smem[];
    const int W = blockDim.x >> 5;
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    uint64_t *bar = reinterpret_cast<uint64_t *>(smem) + warp;
    uint32_t *Zs = smem + (((2 * W) + 3) & ~3) + warp * region_words;
    uint32_t *rows = Zs + ((c.n + 3) & ~3);
    const bool norm = p.normalise != 0;
    if (use_bulk) {
        if (lane == 0) {
            mbar_init(bar, 1);
            fence_mbar_init();
        }
        __syncwarp();
    }
    uint32_t phase = 0;
    const int64_t nwarps = static_cast<int64_t>(gridDim.x) * W;
    int64_t f = blockIdx.x * static_cast<int64_t>(W) + warp;   // first frame static,
    while (f < frames) {                                       // the rest from the counter
        const uint32_t *src = llr + f * c.n;
        if (use_bulk) {
            if (!stage_bulk(c, Zs, src, bar, phase, lane)) return;
        } else {
            for (int i = lane; i < c.n; i += 32) Zs[i] = __ldg(src + i);
        }
        for (int i = lane; i < c.m * kRowWordsF32; i += 32) rows[i] = 0u;   // all L_mn = 0
        __syncwarp();
        int done = p.max_iters;
        for (int k = 1; k <= p.max_iters; ++k) {
            for (int l = 0; l < c.mb; ++l) {
                layer_f32(c, l, Zs, rows, lane, norm, p.alpha);
                __syncwarp();
            }
            if (p.early_stop && syndrome_ok_f32(c, Zs, lane)) {
                done = k;
                break;
            }
        }
        write_frame_f32(c, Zs, f, done, hard, iters, post, lane);
        __syncwarp();
        f = next_work(work, nwarps, lane);
    }
}

__global__ void __launch_bounds__(128)
    decode_i8_kernel(DevCode c, const uint32_t *__restrict__ llr, int64_t frames, DecodeParams p,
                     uint32_t *__restrict__ hard, int32_t *__restrict__ iters,
                     int8_t *__restrict__ post, unsigned long long *work, int region_words,
                     int use_bulk) {
    extern __shared__ __align__(16) uint32_t smem[];
    const int W = blockDim.x >> 5;
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    uint64_t *bar = reinterpret_cast<uint64_t *>(smem) + warp;
    uint32_t *Zs = smem + (((2 * W) + 3) & ~3) + warp * region_words;
    uint32_t *rows = Zs + ((c.n + 3) & ~3);
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
            for (int i = lane; i < c.n; i += 32) Zs[i] ^= 0x80808080u;   // to offset form
        } else {
            for (int i = lane; i < c.n; i += 32) Zs[i] = __ldg(src + i) ^ 0x80808080u;
        }
        for (int i = lane; i < c.m * kRowWordsI8; i += 32) rows[i] = 0u;
        __syncwarp();
    }
    const int64_t dyn_base = 4 * nwarps;   // frames beyond the initial groups
    for (;;) {
        bool any = false;
        for (int b = 0; b < 4; ++b) any |= fr[b] >= 0;
        if (!any) break;
        for (int l = 0; l < c.mb; ++l) {
            layer_i8(c, l, Zs, rows, lane, norm);
            __syncwarp();
        }
        const uint32_t bad = p.early_stop ? syndrome_bad_i8(c, Zs, lane) : 0x80808080u;
        for (int b = 0; b < 4; ++b) {
            if (fr[b] < 0) continue;
            kb[b] += 1;
            const bool ok = !((bad >> (8 * b + 7)) & 1u);
            if (!ok && kb[b] < p.max_iters) continue;
            // frame finished at this iteration: outputs now, then refill the byte
            write_frame_i8(c, Zs, fr[b], b, kb[b], hard, iters, post, lane);
            const int64_t nf = next_work(work, dyn_base, lane);
            if (nf >= frames) {
                fr[b] = -1;
                continue;
            }
            fr[b] = nf;
            kb[b] = 0;
            const uint32_t *src = llr + (nf >> 2) * c.n;
            const uint32_t sel = (0x3210u & ~(0xFu << (4 * b))) |
                                 (static_cast<uint32_t>(4 + (nf & 3)) << (4 * b));
            __syncwarp();
            for (int i = lane; i < c.n; i += 32)
                Zs[i] = prmt(Zs[i], __ldg(src + i) ^ 0x80808080u, sel);
            const uint32_t keep = ~(0xFFu << (8 * b));
            for (int i = lane; i < c.m * kRowWordsI8; i += 32) rows[i] &= keep;
            __syncwarp();
        }
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
    const void *kern = i8 ? reinterpret_cast<const void *>(decode_i8_kernel)
                          : reinterpret_cast<const void *>(decode_f32_kernel);
    cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, smem);
    if (e != cudaSuccess) return cuda_fail(e, "decode kernel attribute");
    int per_sm = 0;
    e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kern, W * 32, smem);
    if (e != cudaSuccess) return cuda_fail(e, "decode occupancy");
    per_sm = std::max(per_sm, 1);
    const int64_t units = i8 ? (frames + 3) / 4 : frames;
    const int64_t want = (units + W - 1) / W;
    int64_t cap = static_cast<int64_t>(per_sm) * sms;
    // LDPC_DECODE_MAX_BLOCKS caps the persistent grid (for tests of the
    // dynamic frame hand-out on small batches).
    if (const char *env = std::getenv("LDPC_DECODE_MAX_BLOCKS")) {
        const long v = std::strtol(env, nullptr, 10);
        if (v > 0) cap = std::min<int64_t>(cap, v);
    }
    const int grid = static_cast<int>(std::min<int64_t>(want, cap));
    unsigned long long *work = work_slot(c, s);
    if (!work) return LDPC_ERR_CUDA;
    const DevCode dc = dev_view(c);
    const uint32_t *in = static_cast<const uint32_t *>(d_llr);
    if (i8)
        decode_i8_kernel<<<grid, W * 32, smem, s>>>(dc, in, frames, p, d_hard, d_iters,
                                                    static_cast<int8_t *>(d_post), work,
                                                    region_words, use_bulk);
    else
        decode_f32_kernel<<<grid, W * 32, smem, s>>>(dc, in, frames, p, d_hard, d_iters,
                                                     static_cast<float *>(d_post), work,
                                                     region_words, use_bulk);
    e = cudaGetLastError();
    return e == cudaSuccess ? LDPC_OK : cuda_fail(e, "decode kernel launch");
}

}  // namespace ldpc
