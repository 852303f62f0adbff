// Device-side building blocks of the layered min-sum decoders (shared by
// the single-code kernels in ldpc_decode.cu and the mixed-code kernels in
// ldpc_mixed.cu): row processing for FP32 and packed int8, hard decisions
// and syndrome, frame outputs, bulk-copy stage-in and work hand-out.
#pragma once

#include "ldpc_internal.cuh"

namespace ldpc {


constexpr uint32_t kFull = 0xFFFFFFFFu;
constexpr uint32_t kWaitLimit = 1u << 22;   // polls of a bulk-copy barrier

// Row state words in shared memory (per check row):
//   FP32: [m1, m2, meta]; m1, m2 scaled magnitudes; meta bits 0..26 hold the
//         sign of L_mn for slot i at bit DMAX-1-i, bits 27..31 the argmin slot.
//   int8: [M1, M2, IDX, SG0 .. SG(k-1)] (padded to an even count), one byte
//         per frame: scaled magnitudes and argmin slot; SGk byte b bit u =
//         sign of L_mn of frame b for slot 8k + u.
constexpr int kRowWordsF32 = 3;
__host__ __device__ constexpr int sign_words(int dmax) { return (dmax + 7) / 8; }
__host__ __device__ constexpr int row_words_i8(int dmax) { return (3 + sign_words(dmax) + 1) & ~1; }

__device__ __forceinline__ uint32_t lds_u32(const uint32_t *base, uint32_t byte_off) {
    return *reinterpret_cast<const uint32_t *>(reinterpret_cast<const char *>(base) + byte_off);
}
__device__ __forceinline__ void sts_u32(uint32_t *base, uint32_t byte_off, uint32_t v) {
    *reinterpret_cast<uint32_t *>(reinterpret_cast<char *>(base) + byte_off) = v;
}

// Byte offset of an edge's posterior, read from the offset table at p.
// Debug builds (-DLDPC_DEBUG, the stand-in for a memory checker) check it
// against the posterior region (N words and the per-lane dummy words, word
// aligned): an offset outside is recorded in the status word, which
// ldpc_sync reports, and replaced by the first dummy word, so the access
// stays in bounds.
__device__ __forceinline__ uint32_t edge_off(const DevCode &c, const uint16_t *p) {
    uint32_t o = __ldg(p);
#ifdef LDPC_DEBUG
    if (o >= 4u * static_cast<uint32_t>(c.n + kDummyWords) || (o & 3u)) {
        atomicOr(c.status, kStatusBadOffset);
        o = 4u * static_cast<uint32_t>(c.n);
    }
#else
    (void)c;
#endif
    return o;
}

// Fixed-width bit helpers (single instructions).
__device__ __forceinline__ uint32_t prmt(uint32_t a, uint32_t b, uint32_t sel) {
    uint32_t r;
    asm("prmt.b32 %0, %1, %2, %3;" : "=r"(r) : "r"(a), "r"(b), "r"(sel));
    return r;
}
// int8 posteriors in shared memory are offset bytes Z + 127 (0..254): bit 7
// is set exactly where Z >= 1, so it is the complement of the hard decision
// (eq. 21).  Channel bytes (two's complement, -127..127) convert per byte
// without borrows: (q xor 128) - 1.
constexpr uint32_t kDummyI8 = 0xFEFEFEFEu;   // +127
__device__ __forceinline__ uint32_t to_offset127(uint32_t q) {
    return (q ^ 0x80808080u) - 0x01010101u;
}
// Byte lanes of x as two 16-bit lanes: bytes 0, 2 (frames 0, 2) or bytes
// 1, 3 (frames 1, 3), zero-extended (offset-form posteriors, 0..254) or
// sign-extended (two's-complement messages, -127..127).
__device__ __forceinline__ uint32_t lanes_even(uint32_t x) { return prmt(x, 0u, 0x4240u); }
__device__ __forceinline__ uint32_t lanes_odd(uint32_t x) { return prmt(x, 0u, 0x4341u); }
__device__ __forceinline__ uint32_t lanes_even_sx(uint32_t x) { return prmt(x, 0u, 0xA280u); }
__device__ __forceinline__ uint32_t lanes_odd_sx(uint32_t x) { return prmt(x, 0u, 0xB391u); }
// min(max(a + b, 0), 254) on two signed 16-bit lanes (|a + b| < 32768),
// as the add-min-relu intrinsic max(min(a + b, 254), 0) (the same value for
// every input, since 0 <= 254).
__device__ __forceinline__ uint32_t add_clamp_off16x2(uint32_t a, uint32_t b) {
    return __viaddmin_s16x2_relu(a, b, 0x00FE00FEu);
}
// 0xFF per byte where bit 7 of the low byte of a lane is set, lanes of e
// holding frames 0, 2 and lanes of o frames 1, 3: back in frame-byte order.
__device__ __forceinline__ uint32_t msb_lanes_to_mask(uint32_t e, uint32_t o) {
    return prmt(e, o, 0xEAC8u);
}
// Integer constants that the compiler cannot see through, so that the
// products and sums below stay multiply-adds (the FMA pipe) instead of being
// strength-reduced to shifts, adds and logic on the ALU pipe, which bounds
// the int8 decoder.  z >= 1 for every code, so the result is 1.
__device__ __forceinline__ uint32_t opaque_one(int z) {
    uint32_t r;
    asm("{\n\t.reg .u32 t;\n\tshr.u32 t, %1, 31;\n\txor.b32 %0, t, 1;\n\t}" : "=r"(r) : "r"(z));
    return r;
}
// a * b + c as one multiply-add (b opaque).
__device__ __forceinline__ uint32_t imad(uint32_t a, uint32_t b, uint32_t c) {
    uint32_t r;
    asm("mad.lo.u32 %0, %1, %2, %3;" : "=r"(r) : "r"(a), "r"(b), "r"(c));
    return r;
}
// Per byte floor(3 m / 4) = m - ceil(m / 4), m <= 127 (no carry crosses bytes).
__device__ __forceinline__ uint32_t scale34(uint32_t m) {
    return m - (((m + 0x03030303u) >> 2) & 0x3F3F3F3Fu);
}


// ---------------------------------------------------------------------------
// Row processing.  Every row runs all DMAX edge slots of its instance as
// straight-line code (so the compiler can interleave the slots freely); a
// layer of degree d uses slots DMAX-d .. DMAX-1 and the leading slots of
// lane l read a dummy posterior (word N + l of the posterior array) whose
// value leaves the row's minimum, second minimum, sign parity and syndrome
// unchanged.  Every slot stores (a per-slot store predicate costs an ALU
// instruction per slot): the FP32 dummy keeps its value under the store,
// the int8 one is reset once per row.  DS is the kernel's slot class (the
// offset-table and row-state layout); DMAX <= DS the slots this instance
// processes.
// ---------------------------------------------------------------------------

// FP32 layer: eq. (22) Z_mn = Z_n - L_mn; eq. (23) new L_mn from the
// smallest and second smallest |Z_mn| and the product of signs; eq. (20) in
// single-scan form Z_n = Z_mn + L_mn.  Each float operation is an explicitly
// rounded intrinsic, so no multiply-add is ever contracted.  The dummy
// posterior is +inf: |Z_mn| = +inf is never a minimum and its sign is +.
//
// WT (learned normalised min-sum): the message of edge q in iteration k is
// w[k-1][q] times the unscaled min-sum message m, q numbering the nonzero
// blocks of H_bm row by row.  The row state then keeps the unscaled minima
// and the message signs before weighting.  wprev / wcur point at this
// layer's weights of the previous and the current iteration, staged in
// shared memory in slot order (wpad(DMAX) floats per layer, 16-byte
// aligned, zero in the leading unused slots).  The posterior updates
// Z_mn = Z_n - w' m_old and Z_n = Z_mn + w m are each one fused
// multiply-add (one rounding), so the learned row costs what the plain one
// does.
__host__ __device__ constexpr int wpad(int dmax) { return (dmax + 3) & ~3; }

// t0, tstep: the row slots t = t0, t0 + tstep, ... of the layer this warp
// processes (a team of tstep warps shares a frame's rows; 0, 1 for one warp).
template <int DS, int DMAX, bool WT = false>
__device__ __forceinline__ void layer_f32(const DevCode &c, int layer, int d, uint32_t *Zs,
                                          uint32_t *rows, int lane, bool norm, float alpha,
                                          const float *wprev = nullptr,
                                          const float *wcur = nullptr, int t0 = 0,
                                          int tstep = 1) {
    (void)d;   // leading unused slots run like the others (see the store below)
    float wp[WT ? wpad(DMAX) : 1], wc[WT ? wpad(DMAX) : 1];
    if (WT) {
        // this layer's slots are the last DMAX of the DS staged ones
        const float4 *p4 = reinterpret_cast<const float4 *>(wprev + (DS - DMAX));
        const float4 *c4 = reinterpret_cast<const float4 *>(wcur + (DS - DMAX));
#pragma unroll
        for (int j = 0; j < wpad(DMAX) / 4; ++j) {
            const float4 a = p4[j], b = c4[j];
            wp[WT ? 4 * j : 0] = a.x; wp[WT ? 4 * j + 1 : 0] = a.y;
            wp[WT ? 4 * j + 2 : 0] = a.z; wp[WT ? 4 * j + 3 : 0] = a.w;
            wc[WT ? 4 * j : 0] = b.x; wc[WT ? 4 * j + 1 : 0] = b.y;
            wc[WT ? 4 * j + 2 : 0] = b.z; wc[WT ? 4 * j + 3 : 0] = b.w;
        }
    }
    for (int t = t0; t < c.rpl; t += tstep) {
        const int r = lane + 32 * t;
        if (r >= c.z) break;
        uint32_t *rs = rows + (layer * c.z + r) * kRowWordsF32;
        const float m1 = __uint_as_float(rs[0]), m2 = __uint_as_float(rs[1]);
        const uint32_t meta = rs[2];
        const int idx = static_cast<int>(meta >> 27);
        const uint16_t *vrow = c.voff + (layer * c.rpl + t) * (DS * 32) + (DS - DMAX) * 32 + lane;
        uint32_t off[DMAX];
        float Q[DMAX];
#pragma unroll
        for (int i = 0; i < DMAX; ++i) off[i] = edge_off(c, vrow + i * 32);
#pragma unroll
        for (int i = 0; i < DMAX; ++i) Q[i] = __uint_as_float(lds_u32(Zs, off[i]));
        float mn1 = __int_as_float(0x7F800000), mn2 = mn1;
        uint32_t sx = 0;
#pragma unroll
        for (int i = 0; i < DMAX; ++i) {
            const float mag = (idx == i) ? m2 : m1;
            // slot i's sign bit moved to bit 31 (a multiply, so it may issue
            // on the FMA pipe)
            const uint32_t sbit = (meta * (1u << (i + 32 - DMAX))) & 0x80000000u;
            const float Lu = __uint_as_float(__float_as_uint(mag) | sbit);
            // learned weights: Z - w' m_old rounded once (fused)
            const float q = WT ? __fmaf_rn(-wp[WT ? i : 0], Lu, Q[i]) : __fsub_rn(Q[i], Lu);
            Q[i] = q;
            sx ^= __float_as_uint(q);
        }
        // smallest and second smallest |Z_mn|, two slots at a time: the
        // pair's min x and max y merge with (mn1, mn2) as mn1 = min(mn1, x),
        // mn2 = min(max(mn1, x), mn2, y), the 3-way min on the bit patterns
        // (non-negative floats order as unsigned integers)
#pragma unroll
        for (int i = 0; i + 1 < DMAX; i += 2) {
            const float a = fabsf(Q[i]), b = fabsf(Q[i + 1]);
            const float x = fminf(a, b), y = fmaxf(a, b);
            const float hi = fmaxf(mn1, x);
            mn1 = fminf(mn1, x);
            mn2 = __uint_as_float(
                __vimin3_u32(__float_as_uint(hi), __float_as_uint(mn2), __float_as_uint(y)));
        }
        if (DMAX & 1) {
            const float a = fabsf(Q[DMAX - 1]);
            mn2 = fmaxf(mn1, fminf(mn2, a));
            mn1 = fminf(mn1, a);
        }
        const float n1 = (norm && !WT) ? __fmul_rn(alpha, mn1) : mn1;
        const float n2 = (norm && !WT) ? __fmul_rn(alpha, mn2) : mn2;
        const uint32_t S = sx & 0x80000000u;
        const uint32_t s1 = __float_as_uint(n1) | S, s2 = __float_as_uint(n2) | S;
        uint32_t nsg = 0;
        int id = 0;
        // an edge whose |Z_mn| equals the minimum gets the second minimum (on
        // ties both minima are equal, so any such edge may be the argmin)
#pragma unroll
        for (int i = 0; i < DMAX; ++i) {
            const bool at_min = fabsf(Q[i]) == mn1;
            const uint32_t ms = at_min ? s2 : s1;
            id = at_min ? i : id;
            const uint32_t L = ms ^ (__float_as_uint(Q[i]) & 0x80000000u);
            // unconditional: a leading unused slot stores +inf + L = +inf back
            // into the dummy posterior (learned: weight 0 there); learned
            // weights: Z_mn + w m rounded once (fused)
            const float zn = WT ? __fmaf_rn(wc[WT ? i : 0], __uint_as_float(L), Q[i])
                                : __fadd_rn(Q[i], __uint_as_float(L));
            sts_u32(Zs, off[i], __float_as_uint(zn));
            nsg = __funnelshift_l(L, nsg, 1);
        }
        rs[0] = __float_as_uint(n1);
        rs[1] = __float_as_uint(n2);
        rs[2] = nsg | (static_cast<uint32_t>(id) << 27);
    }
}

// Slots processed for a layer of degree d in a kernel built for DS slots: the
// DS - 4 instance serves the layers that fit it (fewer padding slots), the
// full instance the others.  Both read the same offset table (a row's real
// edges occupy its last d slots) and keep their own row-state layout, since
// a layer is always processed by the same instance.
template <int DS>
__host__ __device__ constexpr int sub_slots() { return DS >= 12 ? DS - 4 : (DS == 8 ? 4 : DS); }
// Kernels fitted to a code: DM (<= DS) is the number of slots of the large
// instance, the code's largest row degree when that lies in DS - 3 .. DS,
// so rows run no padding slots beyond the code's own degrees; DM = DS is the
// class-wide instance.  The small instance has min(DS - 4, DM) slots.
template <int DS, int DM>
__host__ __device__ constexpr int small_slots() { return sub_slots<DS>() < DM ? sub_slots<DS>() : DM; }
template <int DS, int DM = DS>
__device__ __forceinline__ bool use_sub(int d) {
    return small_slots<DS, DM>() < DM && d <= small_slots<DS, DM>();
}
// The int8 row body is about twice the FP32 one; two large instances that
// alternate from layer to layer no longer fit the instruction cache, so the
// int8 kernels split only the small slot classes.
template <int DS, int DM = DS>
__device__ __forceinline__ bool use_sub_i8(int d) { return DS <= 12 && use_sub<DS, DM>(d); }

// FP32 hard decision (eq. 21) and parity of row slot t of layer l: bit 31
// set when the check is unsatisfied.
template <int DS, int DMAX>
__device__ __forceinline__ uint32_t syndrome_row_f32(const DevCode &c, const uint32_t *Zs, int l,
                                                     int t, int lane) {
    const uint16_t *vrow = c.voff + (l * c.rpl + t) * (DS * 32) + (DS - DMAX) * 32 + lane;
    uint32_t off[DMAX];
#pragma unroll
    for (int i = 0; i < DMAX; ++i) off[i] = edge_off(c, vrow + i * 32);
    uint32_t par = 0;
#pragma unroll
    for (int i = 0; i < DMAX; ++i) {
        const uint32_t u = lds_u32(Zs, off[i]);
        par ^= (u - 1u) | u;   // bit 31 set iff Z <= 0 (negatives, -0 and +0)
    }
    return par;
}

// FP32 hard decision (eq. 21) and syndrome over the rows of one layer.
template <int DS, int DMAX>
__device__ __forceinline__ uint32_t syndrome_rows_f32(const DevCode &c, const uint32_t *Zs, int l,
                                                      int lane) {
    uint32_t bad = 0;
    for (int t = 0; t < c.rpl; ++t) {
        if (lane + 32 * t >= c.z) break;
        bad |= syndrome_row_f32<DS, DMAX>(c, Zs, l, t, lane);
    }
    return bad;
}

// Unsatisfied checks of the hard decisions (eq. 21), warp-uniform.
template <int DS, int DM = DS>
__device__ __forceinline__ int syndrome_count_f32(const DevCode &c, const uint32_t *Zs,
                                                  int lane) {
    uint32_t cnt = 0;
    for (int l = 0; l < c.mb; ++l) {
        const int d = __ldg(c.rowinfo + l) & 255;
        if (use_sub<DS, DM>(d)) {
            for (int t = 0; t < c.rpl; ++t)
                if (lane + 32 * t < c.z)
                    cnt += syndrome_row_f32<DS, small_slots<DS, DM>()>(c, Zs, l, t, lane) >> 31;
        } else {
            for (int t = 0; t < c.rpl; ++t)
                if (lane + 32 * t < c.z)
                    cnt += syndrome_row_f32<DS, DM>(c, Zs, l, t, lane) >> 31;
        }
    }
    return static_cast<int>(__reduce_add_sync(kFull, cnt));
}

// True when every check holds.  The scan ends at the first layer with an
// unsatisfied check: a frame that has not converged usually fails in the
// first layer it looks at, so only the iteration that ends a frame pays
// for a full pass over the edges.
template <int DS, int DM = DS>
__device__ __forceinline__ bool syndrome_ok_f32(const DevCode &c, const uint32_t *Zs, int lane) {
    for (int l = 0; l < c.mb; ++l) {
        const int d = __ldg(c.rowinfo + l) & 255;
        const uint32_t bad = use_sub<DS, DM>(d)
                                 ? syndrome_rows_f32<DS, small_slots<DS, DM>()>(c, Zs, l, lane)
                                 : syndrome_rows_f32<DS, DM>(c, Zs, l, lane);
        if (__any_sync(kFull, bad >> 31)) return false;
    }
    return true;
}

// One FP32 layer through the instance that fits it.  Learned weights are
// staged with 16-byte loads at slot DS - DMAX of each layer, so the learned
// kernels use only instances whose slot count differs from DS by a multiple
// of four.
template <int DS, bool WT = false, int DM = DS>
__device__ __forceinline__ void layer_f32_any(const DevCode &c, int layer, uint32_t *Zs,
                                              uint32_t *rows, int lane, bool norm, float alpha,
                                              const float *wprev = nullptr,
                                              const float *wcur = nullptr, int t0 = 0,
                                              int tstep = 1) {
    static_assert(!WT || ((DS - DM) % 4 == 0 && (DS - small_slots<DS, DM>()) % 4 == 0),
                  "learned weights need 16-byte aligned slot offsets");
    const int d = __ldg(c.rowinfo + layer) & 255;
    if (use_sub<DS, DM>(d))
        layer_f32<DS, small_slots<DS, DM>(), WT>(c, layer, d, Zs, rows, lane, norm, alpha, wprev,
                                                 wcur, t0, tstep);
    else
        layer_f32<DS, DM, WT>(c, layer, d, Zs, rows, lane, norm, alpha, wprev, wcur, t0, tstep);
}

// ---------------------------------------------------------------------------
// int8 layer, four frames per word.  Posteriors live in shared memory in
// offset form (Z + 127, one byte per frame, values 0..254) and so does Z_mn
// inside the row; messages are two's-complement bytes.  The saturating
// additions Z_mn = Z_n - L_mn and Z_n = Z_mn + L_mn run on two 16-bit lanes
// per word (frames 0, 2 and 1, 3): the zero-extended offset value plus the
// sign-extended message, clamped to 0..254 with packed s16 add-max and min,
// is the result in offset form again; the two lane words are joined back
// into bytes with one multiply-add.  The check side works byte-wise:
// |Z_mn| = |x - 127| (one absolute-difference instruction), the running
// minimum and second minimum against compare masks from prmt's sign
// replication, the sign parity by XOR of bit 7 (set for Z_mn >= 1: a zero
// Z_mn counts as negative, which changes no message, since it makes the
// minimum 0 and its own message takes the other edges' signs only).  The
// minima are kept biased by 127 per byte so that each compare is one
// multiply-add; the argmin test of pass 2 likewise.  This moves a third of
// the row's integer work from the ALU pipe, which bounds the kernel, to the
// FMA pipe.  The dummy posterior is
// +127 and the leading slots' stored message sign is kept negative, so
// their Z_mn clamps to +127: never below a minimum.  Their stores change the
// lane's dummy word, which the lane sets back to +127 after the row.
// ---------------------------------------------------------------------------
// Debug builds count the clamps the saturating additions take (eq. 22 and
// eq. 20 results outside [-127, 127]) on the real edges of the byte lanes
// set in `live` (0xFF per lane decoding a frame) into c.sat, the count the
// oracle reports; release builds ignore `live`.
#ifdef LDPC_DEBUG
__device__ __forceinline__ uint32_t clamps_taken(uint32_t off_bytes_lo, uint32_t off_bytes_hi,
                                                 uint32_t add, uint32_t live) {
    // off_bytes_*: per frame b the offset-form value (0..254), frames 0, 2 in
    // the 16-bit lanes of _lo and 1, 3 of _hi; add: two's-complement bytes
    uint32_t n = 0;
#pragma unroll
    for (int b = 0; b < 4; ++b) {
        if (!((live >> (8 * b)) & 0xFFu)) continue;
        const uint32_t w = (b & 1) ? off_bytes_hi : off_bytes_lo;
        const int v = static_cast<int>((w >> (16 * (b >> 1))) & 0xFFFFu);
        const int a = static_cast<int>(static_cast<int8_t>((add >> (8 * b)) & 0xFFu));
        n += (v + a < 0 || v + a > 254) ? 1u : 0u;
    }
    return n;
}
#endif

template <int DS, int DMAX>
__device__ __forceinline__ void layer_i8(const DevCode &c, int layer, int d, uint32_t *Zs,
                                         uint32_t *rows, int lane, bool norm,
                                         uint32_t live = 0u) {
    (void)live;
#ifdef LDPC_DEBUG
    uint32_t nsat = 0;
#endif
    constexpr int SGW = sign_words(DMAX);
    constexpr uint32_t kB = 0x7F7F7F7Fu;   // bias of the running minima
    const int start = DMAX - d;
    const uint32_t one = opaque_one(c.z), m_one = 0u - one, k256 = one << 8;
    // sign bits forced on for the leading (unused) slots, per sign word
    uint32_t pad[SGW];
#pragma unroll
    for (int k = 0; k < SGW; ++k) {
        const int nb = min(max(start - 8 * k, 0), 8);
        pad[k] = ((1u << nb) - 1u) * 0x01010101u;
    }
    for (int t = 0; t < c.rpl; ++t) {
        const int r = lane + 32 * t;
        if (r >= c.z) break;
        uint32_t *rs = rows + (layer * c.z + r) * row_words_i8(DS);
        const uint32_t M1 = rs[0], M2 = rs[1], IDX = rs[2];
        uint32_t SG[SGW];
#pragma unroll
        for (int k = 0; k < SGW; ++k) SG[k] = rs[3 + k];
        // bytes of -L_old for the four (sign, magnitude) cases
        const uint32_t G1 = (0x80808080u - M1) ^ 0x80808080u;   // L > 0: -M
        const uint32_t G2 = (0x80808080u - M2) ^ 0x80808080u;
        const uint16_t *vrow = c.voff + (layer * c.rpl + t) * (DS * 32) + (DS - DMAX) * 32 + lane;
        uint32_t off[DMAX], QE[DMAX], QO[DMAX], A[DMAX];
#pragma unroll
        for (int i = 0; i < DMAX; ++i) off[i] = edge_off(c, vrow + i * 32);
#pragma unroll
        for (int i = 0; i < DMAX; ++i) QE[i] = lds_u32(Zs, off[i]);
        uint32_t mk1 = kB + 0x7F7F7F7Fu, mk2 = kB + 0x7F7F7F7Fu, sx = 0;
#pragma unroll
        for (int i = 0; i < DMAX; ++i) {
            const uint32_t u = QE[i];
            const uint32_t sm = msb_bytes_to_mask(SG[i >> 3] << (7 - (i & 7)));   // L_old < 0
            // 0xFF where slot i is not the argmin: (IDX ^ i) + 127 has bit 7 set
            const uint32_t nq = msb_bytes_to_mask(imad(IDX ^ (0x01010101u * i), one, kB));
            const uint32_t g = bsel(bsel(G2, G1, nq), bsel(M2, M1, nq), sm);      // -L_old
#ifdef LDPC_DEBUG
            if (i >= start) nsat += clamps_taken(lanes_even(u), lanes_odd(u), g, live);
#endif
            // eq. (22): (Z + 127) - L_old, clamped to Z_mn + 127 in 0..254
            const uint32_t qe = add_clamp_off16x2(lanes_even(u), lanes_even_sx(g));
            const uint32_t qo = add_clamp_off16x2(lanes_odd(u), lanes_odd_sx(g));
            QE[i] = qe;
            QO[i] = qo;
            const uint32_t x = imad(qo, k256, qe);                   // offset bytes of Z_mn
            const uint32_t a = __vabsdiffu4(x, 0x7F7F7F7Fu);         // |Z_mn|
            A[i] = a;
            // a < min: bit 7 of (min + 127) - a, no borrow across bytes
            const uint32_t lt1 = msb_bytes_to_mask(imad(a, m_one, mk1));
            const uint32_t lt2 = msb_bytes_to_mask(imad(a, m_one, mk2));
            const uint32_t ak = imad(a, one, kB);
            mk2 = bsel(bsel(mk2, ak, lt2), mk1, lt1);
            mk1 = bsel(mk1, ak, lt1);
            sx ^= x;
        }
        const uint32_t mn1 = mk1 - kB, mn2 = mk2 - kB;
        const uint32_t n1 = norm ? scale34(mn1) : mn1;
        const uint32_t n2 = norm ? scale34(mn2) : mn2;
        // parity of the Z_mn <= 0: offset bytes have bit 7 set for
        // Z_mn >= 1, so flip once per slot
        const uint32_t P = msb_bytes_to_mask(sx ^ ((DMAX & 1) ? 0x80808080u : 0u));
        // bytes of L_new by the sign of Z_mn (eq. 23): the message is
        // negative where Z_mn >= 1 xor the parity is odd
        const uint32_t h1 = (0x80808080u - n1) ^ 0x80808080u, h2 = (0x80808080u - n2) ^ 0x80808080u;
        const uint32_t Yp1 = bsel(n1, h1, P), Yp2 = bsel(n2, h2, P);   // Z_mn >= 1
        const uint32_t Yn1 = bsel(h1, n1, P), Yn2 = bsel(h2, n2, P);   // Z_mn <= 0
        const uint32_t mn1p = mn1 + 0x80808080u;
        uint32_t zsg[SGW];
#pragma unroll
        for (int k = 0; k < SGW; ++k) zsg[k] = 0u;
        uint32_t id = 0;
#pragma unroll
        for (int i = 0; i < DMAX; ++i) {
            const uint32_t pos = msb_lanes_to_mask(QE[i], QO[i]);   // 0xFF: Z_mn >= 1
            // |Z_mn| >= min, so min + 128 - |Z_mn| lies in [1, 128] and equals
            // 128 exactly at the minimum: that edge gets the second minimum (on
            // ties both minima are equal, so any such edge may be the argmin)
            const uint32_t at_min = msb_bytes_to_mask(imad(A[i], m_one, mn1p));
            id = bsel(id, 0x01010101u * i, at_min);
            const uint32_t y = bsel(bsel(Yn1, Yn2, at_min), bsel(Yp1, Yp2, at_min), pos);
#ifdef LDPC_DEBUG
            if (i >= start) nsat += clamps_taken(QE[i], QO[i], y, live);
#endif
            // eq. (20): (Z_mn + 127) + L_new, clamped to Z + 127 in 0..254
            const uint32_t ze = add_clamp_off16x2(QE[i], lanes_even_sx(y));
            const uint32_t zo = add_clamp_off16x2(QO[i], lanes_odd_sx(y));
            sts_u32(Zs, off[i], imad(zo, k256, ze));
            zsg[i >> 3] |= pos & ((1u << (i & 7)) * 0x01010101u);
        }
        // the leading unused slots stored into this lane's dummy posterior
        // (word N + lane): back to +127 before the lane's next row reads it
        Zs[c.n + lane] = kDummyI8;
        rs[0] = n1;
        rs[1] = n2;
        rs[2] = id;
        // message sign = not (Z_mn >= 1 xor parity); leading slots negative
#pragma unroll
        for (int k = 0; k < SGW; ++k) rs[3 + k] = ~(zsg[k] ^ P) | pad[k];
    }
#ifdef LDPC_DEBUG
    if (nsat && c.sat) atomicAdd(c.sat, static_cast<unsigned long long>(nsat));
#endif
}

// A refilled byte lane must start with every message zero: clearing its
// byte of the two stored minima does that (eq. 23 magnitudes 0 give L = 0
// whatever the argmin and sign bits still hold), at a third of the stores
// of clearing the whole row state.
template <int DS>
__device__ __forceinline__ void clear_row_minima_i8(uint32_t *rows, int m, uint32_t keep,
                                                    int lane) {
    static_assert(row_words_i8(DS) % 2 == 0, "rows start 8-byte aligned");
    for (int r = lane; r < m; r += 32) {
        uint2 *q = reinterpret_cast<uint2 *>(rows + r * row_words_i8(DS));   // 8-byte aligned
        uint2 v = *q;
        v.x &= keep;
        v.y &= keep;
        *q = v;
    }
}

// int8 hard decision per byte: bit 7 set where Z <= 0, i.e. offset value <= 127.
__device__ __forceinline__ uint32_t hard_bytes_off(uint32_t u) { return ~u & 0x80808080u; }

// int8 syndrome over the rows of one layer: bit 7 of byte b set when frame b
// has an unsatisfied check there.
template <int DS, int DMAX>
__device__ __forceinline__ uint32_t syndrome_rows_i8(const DevCode &c, const uint32_t *Zs, int l,
                                                     int lane) {
    uint32_t bad = 0;
    for (int t = 0; t < c.rpl; ++t) {
        if (lane + 32 * t >= c.z) break;
        const uint16_t *vrow = c.voff + (l * c.rpl + t) * (DS * 32) + (DS - DMAX) * 32 + lane;
        uint32_t off[DMAX];
#pragma unroll
        for (int i = 0; i < DMAX; ++i) off[i] = edge_off(c, vrow + i * 32);
        // bit 7 of u is set iff Z >= 1, so each of the DMAX terms (the dummy
        // +127 ones included) flips the parity of the hard decisions
        uint32_t par = (DMAX & 1) ? 0x80808080u : 0u;
#pragma unroll
        for (int i = 0; i < DMAX; ++i)
            par ^= lds_u32(Zs, off[i]);
        bad |= par;
    }
    return bad;
}

// int8 syndrome: bit 7 of byte b set when frame b has an unsatisfied check,
// for the byte lanes of `need` (bit 7 of each byte lane decoding a frame);
// the other lanes' bits are unspecified.  The scan ends once every lane of
// `need` has an unsatisfied check.
template <int DS, int DM = DS>
__device__ __forceinline__ uint32_t syndrome_bad_i8(const DevCode &c, const uint32_t *Zs,
                                                    int lane, uint32_t need = 0x80808080u) {
    uint32_t bad = 0;
    for (int l = 0; l < c.mb; ++l) {
        const int d = __ldg(c.rowinfo + l) & 255;
        bad |= use_sub_i8<DS, DM>(d)
                   ? syndrome_rows_i8<DS, small_slots<DS, DM>()>(c, Zs, l, lane)
                   : syndrome_rows_i8<DS, DM>(c, Zs, l, lane);
        const uint32_t all = __reduce_or_sync(kFull, bad & 0x80808080u);
        if ((all & need) == need) return all;
    }
    return __reduce_or_sync(kFull, bad & 0x80808080u);
}

// One int8 layer through the instance that fits it.
template <int DS, int DM = DS>
__device__ __forceinline__ void layer_i8_any(const DevCode &c, int layer, uint32_t *Zs,
                                             uint32_t *rows, int lane, bool norm,
                                             uint32_t live = 0u) {
    const int d = __ldg(c.rowinfo + layer) & 255;
    if (use_sub_i8<DS, DM>(d))
        layer_i8<DS, small_slots<DS, DM>()>(c, layer, d, Zs, rows, lane, norm, live);
    else
        layer_i8<DS, DM>(c, layer, d, Zs, rows, lane, norm, live);
}

// ---------------------------------------------------------------------------
// Outputs of one frame: packed hard decisions, iteration count, posteriors.
// ---------------------------------------------------------------------------
// h: the frame's ceil(N/32) hard-decision words; it_out: its iteration
// count; p: its N posteriors or NULL.
__device__ __forceinline__ void write_frame_f32_to(const DevCode &c, const uint32_t *Zs, int it,
                                                   uint32_t *h, int32_t *it_out, float *p,
                                                   int lane) {
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
    if (lane == 0) *it_out = it;
    if (p)
        for (int n = lane; n < c.n; n += 32) p[n] = __uint_as_float(Zs[n]);
}

__device__ __forceinline__ void write_frame_f32(const DevCode &c, const uint32_t *Zs, int64_t f,
                                                int it, uint32_t *hard, int32_t *iters,
                                                float *post, int lane) {
    write_frame_f32_to(c, Zs, it, hard + f * c.nwords, iters + f, post ? post + f * c.n : nullptr,
                       lane);
}

// Outputs of byte lane `byte` (one frame of the packed word).
__device__ __forceinline__ void write_frame_i8_to(const DevCode &c, const uint32_t *Zs, int byte,
                                                  int it, uint32_t *h, int32_t *it_out,
                                                  int8_t *p, int lane) {
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
    if (lane == 0) *it_out = it;
    if (p)
        for (int n = lane; n < c.n; n += 32)
            p[n] = static_cast<int8_t>((((Zs[n] >> (8 * byte)) & 0xFFu) + 1u) ^ 0x80u);
}

__device__ __forceinline__ void write_frame_i8(const DevCode &c, const uint32_t *Zs, int64_t f,
                                               int byte, int it, uint32_t *hard, int32_t *iters,
                                               int8_t *post, int lane) {
    write_frame_i8_to(c, Zs, byte, it, hard + f * c.nwords, iters + f,
                      post ? post + f * c.n : nullptr, lane);
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

// Pulls `bytes` bytes at p into L2 ahead of their use (one prefetch per
// 128-byte line, spread over the lanes; no data is returned).
__device__ __forceinline__ void prefetch_l2(const void *p, uint32_t bytes, int lane) {
    const char *c = static_cast<const char *>(p);
    for (uint32_t o = static_cast<uint32_t>(lane) * 128u; o < bytes; o += 32u * 128u)
        asm volatile("prefetch.L2 [%0];" ::"l"(c + o));
}

__device__ __forceinline__ int64_t next_work(unsigned long long *ctr, int64_t base, int lane) {
    unsigned long long v = 0;
    if (lane == 0) v = atomicAdd(ctr, 1ull);
    v = __shfl_sync(kFull, v, 0);
    return base + static_cast<int64_t>(v);
}

// ---------------------------------------------------------------------------
// Learned weights in shared memory: three rows of mb * wpad(DMAX) floats in
// slot order; iteration k reads row buffer k % 3 (weights of iteration k,
// table row min(k, T) - 1) and, for the old messages, buffer (k - 1) % 3
// (iteration 1 its own).  The row of iteration k + 1 is copied in
// asynchronously while iteration k runs, into the buffer iteration k - 2
// used; after iteration T + 2 all three buffers hold the last row and the
// copies stop.
// ---------------------------------------------------------------------------
constexpr int kWeightBuffers = 3;

// Issue the copies of iteration k's weights into buf (one commit group per
// thread; unused slots get 0), threads tid = 0 .. nthr-1.
template <int WP>
__device__ __forceinline__ void stage_weights_async(const DevCode &c, const DecodeParams &p,
                                                    int wT, int k, float *buf, int tid,
                                                    int nthr) {
    const float *wk = p.weights + static_cast<size_t>(min(k, wT) - 1) * p.n_edges;
    for (int i = tid; i < c.mb * WP; i += nthr) {
        const int g = __ldg(c.wgather + i);
        if (g >= 0)
            cp_async4(buf + i, wk + g);
        else
            buf[i] = 0.0f;
    }
    cp_async_commit();
}

// Before iteration k: issue iteration k + 1's weights when it needs a new
// row, then wait for iteration k's (the caller synchronises the threads).
template <int WP>
__device__ __forceinline__ void weights_for_iteration(const DevCode &c, const DecodeParams &p,
                                                      int wT, int k, float *wbuf, int tid,
                                                      int nthr) {
    const int j = k + 1;
    if (j <= p.max_iters && j <= wT + 2) {
        stage_weights_async<WP>(c, p, wT, j, wbuf + (j % kWeightBuffers) * c.mb * WP, tid, nthr);
        cp_async_wait<1>();
    } else {
        cp_async_wait<0>();
    }
}

// ---------------------------------------------------------------------------
// One FP32 frame: stage its LLRs (src, N words) into Zs, clear the messages,
// run the layered iterations (eq. 22, 23, 20) with the syndrome stop after
// each full iteration (eq. 21, Section 4 step 4).  Returns the iteration
// count, or 0 if the bulk copy timed out (the status word records it).
// Learned weights (WT) stream into wbuf (kWeightBuffers rows) as above.
// ---------------------------------------------------------------------------
template <int DMAX, bool WT, int DM = DMAX>
__device__ __forceinline__ int decode_one_f32(const DevCode &c, uint32_t *Zs, uint32_t *rows,
                                              float *wbuf, const uint32_t *src, bool use_bulk,
                                              uint64_t *bar, uint32_t &phase,
                                              const DecodeParams &p, int lane) {
    if (use_bulk) {
        if (!stage_bulk(c, Zs, src, bar, phase, lane)) return 0;
    } else {
        for (int i = lane; i < c.n; i += 32) Zs[i] = __ldg(src + i);
    }
    for (int i = lane; i < c.m * kRowWordsF32; i += 32) rows[i] = 0u;   // all L_mn = 0
    const bool norm = p.normalise != 0;
    const int wT = p.weight_iters > 0 ? p.weight_iters : p.max_iters;
    const bool checkpoints = p.early_stop && (p.stop_iter[0] | p.stop_iter[1]) != 0;
    // give-up limits, floor(stop_frac * M) with the product rounded in FP32
    const int lim0 = static_cast<int>(floorf(__fmul_rn(p.stop_frac[0], static_cast<float>(c.m))));
    const int lim1 = static_cast<int>(floorf(__fmul_rn(p.stop_frac[1], static_cast<float>(c.m))));
    constexpr int WP = wpad(DMAX);
    if (WT) stage_weights_async<WP>(c, p, wT, 1, wbuf + c.mb * WP, lane, 32);
    __syncwarp();
    for (int k = 1; k <= p.max_iters; ++k) {
        const float *wcur = wbuf + (k % kWeightBuffers) * c.mb * WP;
        const float *wprev = k > 1 ? wbuf + ((k - 1) % kWeightBuffers) * c.mb * WP : wcur;
        if (WT) {
            weights_for_iteration<WP>(c, p, wT, k, wbuf, lane, 32);
            __syncwarp();
        }
        for (int l = 0; l < c.mb; ++l) {
            layer_f32_any<DMAX, WT, DM>(c, l, Zs, rows, lane, norm, p.alpha, wprev + l * WP,
                                    wcur + l * WP);
            __syncwarp();
        }
        bool stop = false;
        if (checkpoints && (k == p.stop_iter[0] || k == p.stop_iter[1])) {
            // a give-up checkpoint: count the unsatisfied checks; none ends
            // the frame (eq. 21), too many ends it too
            const int u = syndrome_count_f32<DMAX, DM>(c, Zs, lane);
            stop = u == 0 || (k == p.stop_iter[0] && u > lim0) || (k == p.stop_iter[1] && u > lim1);
        } else if (p.early_stop) {
            stop = syndrome_ok_f32<DMAX, DM>(c, Zs, lane);
        }
        if (stop) {
            if (WT) cp_async_wait<0>();   // the next iteration's copies land before reuse
            return k;
        }
    }
    return p.max_iters;
}

// ---------------------------------------------------------------------------
// Teams: tstep warps decoding one FP32 frame together, warp wi taking the row
// slots t = wi, wi + tstep, ... of every layer, with a named barrier between
// layers.  Every decision (copy timeout, stop, the next work item) goes
// through the team's shared words tw[] so that all warps of a team take the
// same path and meet at every barrier.  tw[0]: copy-timeout flag; tw[1 + w]:
// warp w's syndrome result; tw[4..5]: the next work item.
// ---------------------------------------------------------------------------
__device__ __forceinline__ void team_sync(int id, int nw) {
    if (nw == 1)
        __syncwarp();
    else
        asm volatile("bar.sync %0, %1;" ::"r"(id), "r"(nw * 32) : "memory");
}

// This warp's part of the syndrome: 1 when one of its rows fails (the scan
// ends at the first layer where one does), 0 otherwise; or (count) the
// number of its failing rows.
template <int DS, int DM>
__device__ __forceinline__ uint32_t syndrome_part_f32(const DevCode &c, const uint32_t *Zs, int lane,
                                                      int t0, int tstep, bool count) {
    uint32_t acc = 0;
    for (int l = 0; l < c.mb; ++l) {
        const int d = __ldg(c.rowinfo + l) & 255;
        for (int t = t0; t < c.rpl; t += tstep) {
            if (lane + 32 * t >= c.z) break;
            const uint32_t par = use_sub<DS, DM>(d)
                                     ? syndrome_row_f32<DS, small_slots<DS, DM>()>(c, Zs, l, t, lane)
                                     : syndrome_row_f32<DS, DM>(c, Zs, l, t, lane);
            acc = count ? acc + (par >> 31) : (acc | par);
        }
        if (!count && __any_sync(kFull, acc >> 31)) return 1u;
    }
    return count ? __reduce_add_sync(kFull, acc) : 0u;
}

// decode_one_f32 for a team of tstep warps (wi: this warp's index in it).
template <int DMAX, bool WT>
__device__ __forceinline__ int decode_one_f32_team(const DevCode &c, uint32_t *Zs, uint32_t *rows,
                                                   float *wbuf, const uint32_t *src,
                                                   bool use_bulk, uint64_t *bar, uint32_t &phase,
                                                   const DecodeParams &p, int lane, int wi,
                                                   int tstep, int bar_id, volatile int *tw) {
    const int tid = wi * 32 + lane, nthr = tstep * 32;
    fence_proxy_async_smem();
    if (tid == 0) tw[0] = 0;
    team_sync(bar_id, tstep);   // the previous frame's reads of Zs are done
    if (use_bulk) {
        if (tid == 0) {
            mbar_arrive_expect_tx(bar, static_cast<uint32_t>(c.n) * 4u);
            bulk_copy_g2s(Zs, src, static_cast<uint32_t>(c.n) * 4u, bar);
        }
        const bool ok = mbar_wait_bounded(bar, phase, kWaitLimit);
        if (!__all_sync(kFull, ok)) {
            if (lane == 0) {
                atomicOr(c.status, kStatusCopyTimeout);
                tw[0] = 1;
            }
            mbar_wait_bounded(bar, phase, kWaitLimit);   // let the copy land
        }
        team_sync(bar_id, tstep);
        if (tw[0]) return 0;
        phase ^= 1u;
    } else {
        for (int i = tid; i < c.n; i += nthr) Zs[i] = __ldg(src + i);
    }
    for (int i = tid; i < c.m * kRowWordsF32; i += nthr) rows[i] = 0u;   // all L_mn = 0
    const bool norm = p.normalise != 0;
    const int wT = p.weight_iters > 0 ? p.weight_iters : p.max_iters;
    const bool checkpoints = p.early_stop && (p.stop_iter[0] | p.stop_iter[1]) != 0;
    const int lim0 = static_cast<int>(floorf(__fmul_rn(p.stop_frac[0], static_cast<float>(c.m))));
    const int lim1 = static_cast<int>(floorf(__fmul_rn(p.stop_frac[1], static_cast<float>(c.m))));
    constexpr int WP = wpad(DMAX);
    if (WT) stage_weights_async<WP>(c, p, wT, 1, wbuf + c.mb * WP, tid, nthr);
    team_sync(bar_id, tstep);
    for (int k = 1; k <= p.max_iters; ++k) {
        const float *wcur = wbuf + (k % kWeightBuffers) * c.mb * WP;
        const float *wprev = k > 1 ? wbuf + ((k - 1) % kWeightBuffers) * c.mb * WP : wcur;
        if (WT) {
            weights_for_iteration<WP>(c, p, wT, k, wbuf, tid, nthr);
            team_sync(bar_id, tstep);
        }
        for (int l = 0; l < c.mb; ++l) {
            layer_f32_any<DMAX, WT>(c, l, Zs, rows, lane, norm, p.alpha, wprev + l * WP,
                                    wcur + l * WP, wi, tstep);
            team_sync(bar_id, tstep);
        }
        if (p.early_stop) {
            const bool count = checkpoints && (k == p.stop_iter[0] || k == p.stop_iter[1]);
            const uint32_t part = syndrome_part_f32<DMAX, DMAX>(c, Zs, lane, wi, tstep, count);
            if (lane == 0) tw[1 + wi] = static_cast<int>(part);
            team_sync(bar_id, tstep);
            int u = 0;
            for (int w = 0; w < tstep; ++w) u += tw[1 + w];
            if (u == 0 || (count && ((k == p.stop_iter[0] && u > lim0) ||
                                     (k == p.stop_iter[1] && u > lim1)))) {
                if (WT) cp_async_wait<0>();   // the next iteration's copies land before reuse
                return k;
            }
        }
    }
    return p.max_iters;
}

// ---------------------------------------------------------------------------
// Evaluation of one decoded frame (Section 6.1 error counting): the number of
// info bits (the first K hard decisions) that differ from the sent ones, and
// whether the hard decisions satisfy every check (eq. 21 termination test),
// both warp-uniform.
// ---------------------------------------------------------------------------
// True (warp-uniform) when the packed hard decisions h satisfy every check.
__device__ __forceinline__ bool hard_syndrome_ok(const DevCode &c, const uint32_t *h, int lane) {
    uint32_t bad = 0;
    for (int l = 0; l < c.mb; ++l) {
        const int d = c.rowinfo[l] & 255;
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
    return !__any_sync(kFull, bad);
}

__device__ __forceinline__ unsigned long long frame_outcome(const DevCode &c, const uint8_t *in,
                                                            const uint32_t *h, int lane,
                                                            bool *syn_ok) {
    unsigned long long errs = 0;
    for (int t = lane; t < c.k; t += 32) errs += ((h[t >> 5] >> (t & 31)) & 1u) ^ (in[t] & 1u);
    for (int o = 16; o; o >>= 1) errs += __shfl_xor_sync(kFull, errs, o);
    *syn_ok = hard_syndrome_ok(c, h, lane);
    return errs;
}

// Counter layout of ldpc_frame_stats: [0] bit errors, [1] frame errors,
// [2] undetected frame errors, [3] iteration sum, [4 + t] frames ending at t.
__device__ __forceinline__ void count_frame(unsigned long long *cnt, unsigned long long errs,
                                            bool syn_ok, int it, int max_iters) {
    if (errs) {
        atomicAdd(&cnt[0], errs);
        atomicAdd(&cnt[1], 1ull);
        if (syn_ok) atomicAdd(&cnt[2], 1ull);
    }
    atomicAdd(&cnt[3], static_cast<unsigned long long>(it));
    if (it >= 0 && it <= max_iters) atomicAdd(&cnt[4 + it], 1ull);
}

// Fixed-point channel value of one LLR (Section 5, 8 bits):
// rint(clamp(scale * llr, -clip, clip)), round half to even.
__device__ __forceinline__ uint32_t quantize_one(float llr, float scale, float fc) {
    float x = __fmul_rn(scale, llr);
    x = fminf(fmaxf(x, -fc), fc);
    return static_cast<uint32_t>(__float2int_rn(x)) & 0xFFu;
}

}  // namespace ldpc
