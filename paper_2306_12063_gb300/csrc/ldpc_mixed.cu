// Mixed-code batches: frames of many codes (different Z and rate) decoded
// together, the workload of a receiver that serves several links at once.
// The paper decodes one code at a time (its MEX interface takes one base
// matrix per call); this is the batched form of the same decoders.
//
// A code set holds the kernel-side descriptors of its codes in device
// memory.  A plan fixes a batch's frame-to-code assignment: buffers hold the
// frames back to back in the caller's order (per-frame offsets), while the
// decoders walk an internal order that groups frames by code, each code's
// range padded to a multiple of four (int8 words hold four frames of one
// code).  Codes are partitioned into launch groups that share a kernel
// instance (the slot class of the row degree) and a shared-memory size
// (within a factor of two); each group is one persistent launch whose warps
// pull work items -- a run of consecutive frames of one code -- from the
// group's atomic counter, largest codes first.  The groups' launches run
// concurrently on forked streams.  The frames per work item and the number
// of resident blocks per group are picked by an autotuner that times the
// batch itself.
#include <algorithm>
#include <cstring>
#include <mutex>
#include <numeric>
#include <string>
#include <vector>

#include "ldpc_decode_dev.cuh"

namespace ldpc {

struct MixedItem {
    int code;             // index in the code set
    int count;            // frames (internal indices start .. start + count - 1)
    long long start;
};

namespace {

// One FP32 launch: work items of the group's codes, one frame at a time.
// WT: learned normalised min-sum with code c's weights wptr[c], a table of
// wT[c] rows (streamed into buffers after the row state); each code runs
// p.max_iters iterations when that is set, else wT[c], rows past the table
// repeating its last one.
template <int DMAX, bool WT = false>
__global__ void __launch_bounds__(32)
    mixed_f32_kernel(const DevCode *__restrict__ codes, const MixedItem *__restrict__ items,
                     int n_items, const long long *__restrict__ uframe,
                     const long long *__restrict__ llr_off, const long long *__restrict__ hard_off,
                     const float *__restrict__ llr, DecodeParams p, uint32_t *__restrict__ hard,
                     int32_t *__restrict__ iters, float *__restrict__ post,
                     unsigned long long *work, int use_bulk, const float *const *wptr,
                     const int *wT) {
    extern __shared__ __align__(16) uint32_t smem[];
    const int lane = threadIdx.x & 31;
    uint64_t *bar = reinterpret_cast<uint64_t *>(smem);
    uint32_t *Zs = smem + 4;
    if (use_bulk && lane == 0) {
        mbar_init(bar, 1);
        fence_mbar_init();
    }
    __syncwarp();
    uint32_t phase = 0;
    int64_t it = blockIdx.x;
    while (it < n_items) {
        const MixedItem item = items[it];
        const DevCode c = codes[item.code];
        uint32_t *rows = Zs + posterior_words(c.n);
        float *wbuf = reinterpret_cast<float *>(rows + ((c.m * 3 + 3) & ~3));
        DecodeParams pc = p;
        if (WT) {
            pc.weights = wptr[item.code];
            pc.weight_iters = wT[item.code];
            pc.max_iters = p.max_iters > 0 ? p.max_iters : wT[item.code];
            pc.n_edges = c.n_edges;
        }
        Zs[c.n + lane] = 0x7F800000u;   // dummy posterior of unused edge slots
        __syncwarp();
        for (long long i = item.start; i < item.start + item.count; ++i) {
            const long long uf = uframe[i];
            if (uf < 0) continue;   // padding of the code's range
            // the item's next frame into L2 while this one decodes
            if (i + 1 < item.start + item.count) {
                const long long un = uframe[i + 1];
                if (un >= 0) prefetch_l2(llr + llr_off[un], 4u * static_cast<uint32_t>(c.n), lane);
            }
            const float *src = llr + llr_off[uf];
            const int done = decode_one_f32<DMAX, WT>(
                c, Zs, rows, wbuf, reinterpret_cast<const uint32_t *>(src), use_bulk != 0,
                bar, phase, pc, lane);
            if (!done) return;
            write_frame_f32_to(c, Zs, done, hard + hard_off[uf], iters + uf,
                               post ? post + llr_off[uf] : nullptr, lane);
            __syncwarp();
        }
        it = next_work(work, gridDim.x, lane);
    }
}

// The FP32 launch with teams: fpb teams per block, each of wpf warps decoding
// one frame at a time (warps per frame and frames per CTA, both tuned per
// launch group).  Team g's shared memory is its own region of team_words
// words (the one-warp layout, then the team's eight shared words); its
// warps meet at named barrier 1 + g.  A team's first work item is static,
// the rest come from the group's counter through its leader.
template <int DMAX, bool WT = false>
__global__ void __launch_bounds__(32 * 12)
    mixed_f32_team_kernel(const DevCode *__restrict__ codes, const MixedItem *__restrict__ items,
                          int n_items, const long long *__restrict__ uframe,
                          const long long *__restrict__ llr_off,
                          const long long *__restrict__ hard_off, const float *__restrict__ llr,
                          DecodeParams p, uint32_t *__restrict__ hard, int32_t *__restrict__ iters,
                          float *__restrict__ post, unsigned long long *work, int use_bulk,
                          const float *const *wptr, const int *wT, int wpf, int fpb,
                          int team_words) {
    extern __shared__ __align__(16) uint32_t smem[];
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const int g = warp / wpf, wi = warp - g * wpf;
    uint32_t *base = smem + static_cast<size_t>(g) * team_words;
    uint64_t *bar = reinterpret_cast<uint64_t *>(base);
    uint32_t *Zs = base + 4;
    volatile int *tw = reinterpret_cast<volatile int *>(base + team_words - 8);
    const int bar_id = 1 + g;
    if (use_bulk && wi == 0 && lane == 0) {
        mbar_init(bar, 1);
        fence_mbar_init();
    }
    team_sync(bar_id, wpf);
    uint32_t phase = 0;
    long long it = static_cast<long long>(blockIdx.x) * fpb + g;
    while (it < n_items) {
        const MixedItem item = items[it];
        const DevCode c = codes[item.code];
        uint32_t *rows = Zs + posterior_words(c.n);
        float *wbuf = reinterpret_cast<float *>(rows + ((c.m * 3 + 3) & ~3));
        DecodeParams pc = p;
        if (WT) {
            pc.weights = wptr[item.code];
            pc.weight_iters = wT[item.code];
            pc.max_iters = p.max_iters > 0 ? p.max_iters : wT[item.code];
            pc.n_edges = c.n_edges;
        }
        if (wi == 0) Zs[c.n + lane] = 0x7F800000u;   // dummy posterior of unused edge slots
        for (long long i = item.start; i < item.start + item.count; ++i) {
            const long long uf = uframe[i];
            if (uf < 0) continue;   // padding of the code's range
            if (i + 1 < item.start + item.count && wi == 0) {
                const long long un = uframe[i + 1];
                if (un >= 0) prefetch_l2(llr + llr_off[un], 4u * static_cast<uint32_t>(c.n), lane);
            }
            const float *src = llr + llr_off[uf];
            const int done = decode_one_f32_team<DMAX, WT>(
                c, Zs, rows, wbuf, reinterpret_cast<const uint32_t *>(src), use_bulk != 0, bar,
                phase, pc, lane, wi, wpf, bar_id, tw);
            if (!done) return;   // team-uniform
            if (wi == 0)
                write_frame_f32_to(c, Zs, done, hard + hard_off[uf], iters + uf,
                                   post ? post + llr_off[uf] : nullptr, lane);
        }
        team_sync(bar_id, wpf);   // outputs written, tw[4..5] free
        if (wi == 0 && lane == 0) {
            const long long nx = static_cast<long long>(atomicAdd(work, 1ull)) +
                                 static_cast<long long>(gridDim.x) * fpb;
            *reinterpret_cast<volatile long long *>(tw + 4) = nx;
        }
        team_sync(bar_id, wpf);
        it = *reinterpret_cast<volatile long long *>(tw + 4);
    }
}

// One int8 launch: a work item's frames enter a packed word four at a time
// and each byte lane is refilled as soon as its frame stops (as in the
// single-code kernel), from the item's remaining frames and then from the
// next items while they belong to the same code; an item of another code
// waits until all four lanes are idle.  ibase[c] is code c's first internal
// index, qoff[c] the word offset of its packed groups.
// Bounded to 12 resident one-warp blocks per SM: the large slot classes then
// take 144-158 registers instead of 187-204, which had capped residency below
// what their shared memory allows (int8 mixed set 13.5 -> 14.0 Gbit/s).
template <int DMAX>
__global__ void __launch_bounds__(32, 12)
    mixed_i8_kernel(const DevCode *__restrict__ codes, const MixedItem *__restrict__ items,
                    int n_items, const long long *__restrict__ uframe,
                    const long long *__restrict__ llr_off, const long long *__restrict__ hard_off,
                    const long long *__restrict__ ibase, const long long *__restrict__ qoff,
                    const uint32_t *__restrict__ q, DecodeParams p, uint32_t *__restrict__ hard,
                    int32_t *__restrict__ iters, int8_t *__restrict__ post,
                    unsigned long long *work, int use_bulk) {
    extern __shared__ __align__(16) uint32_t smem[];
    const int lane = threadIdx.x & 31;
    uint64_t *bar = reinterpret_cast<uint64_t *>(smem);
    uint32_t *Zs = smem + 4;
    const bool norm = p.normalise != 0;
    if (use_bulk && lane == 0) {
        mbar_init(bar, 1);
        fence_mbar_init();
    }
    __syncwarp();
    uint32_t phase = 0;
    int64_t it = blockIdx.x;
    while (it < n_items) {
        const MixedItem item = items[it];
        it = -1;   // no item fetched ahead yet
        const DevCode c = codes[item.code];
        const long long base = ibase[item.code];
        const uint32_t *qc = q + qoff[item.code];
        uint32_t *rows = Zs + posterior_words(c.n);
        long long end = item.start + item.count;
        long long fr[4];
        int kb[4];
#pragma unroll
        for (int b = 0; b < 4; ++b) {
            fr[b] = item.start + b < end ? item.start + b : -1;
            kb[b] = 0;
        }
        long long next = item.start + 4;
        {
            const uint32_t *src = qc + ((item.start - base) >> 2) * c.n;
            if (use_bulk) {
                if (!stage_bulk(c, Zs, src, bar, phase, lane)) return;
                for (int i = lane; i < c.n; i += 32) Zs[i] = to_offset127(Zs[i]);
            } else {
                for (int i = lane; i < c.n; i += 32) Zs[i] = to_offset127(__ldg(src + i));
            }
            for (int i = lane; i < c.m * row_words_i8(DMAX); i += 32) rows[i] = 0u;
            Zs[c.n + lane] = kDummyI8;   // dummy posterior +127
            __syncwarp();
        }
        for (;;) {
            bool any = false;
#pragma unroll
            for (int b = 0; b < 4; ++b) any |= fr[b] >= 0;
            if (!any) break;
            for (int l = 0; l < c.mb; ++l) {
                layer_i8_any<DMAX>(c, l, Zs, rows, lane, norm);
                __syncwarp();
            }
            uint32_t need = 0;   // bit 7 of every byte lane decoding a frame
#pragma unroll
            for (int b = 0; b < 4; ++b) need |= fr[b] >= 0 ? 0x80u << (8 * b) : 0u;
            const uint32_t bad =
                p.early_stop ? syndrome_bad_i8<DMAX>(c, Zs, lane, need) : 0x80808080u;
            for (int b = 0; b < 4; ++b) {
                if (fr[b] < 0) continue;
                kb[b] += 1;
                const bool ok = !((bad >> (8 * b + 7)) & 1u);
                if (!ok && kb[b] < p.max_iters) continue;
                const long long uf = uframe[fr[b]];
                if (uf >= 0)
                    write_frame_i8_to(c, Zs, b, kb[b], hard + hard_off[uf], iters + uf,
                                      post ? post + llr_off[uf] : nullptr, lane);
                if (next >= end && it < 0) {
                    // this item is used up: take the next one; keep refilling
                    // from it if it is of the same code
                    it = next_work(work, gridDim.x, lane);
                    if (it < n_items) {
                        const MixedItem nx = items[it];
                        if (nx.code == item.code) {
                            next = nx.start;
                            end = nx.start + nx.count;
                            it = -1;
                        }
                    }
                }
                if (next >= end) {
                    fr[b] = -1;
                    continue;
                }
                const long long nf = next++;
                fr[b] = nf;
                kb[b] = 0;
                const long long li = nf - base;
                const uint32_t *src = qc + (li >> 2) * c.n;
                // the following refill's packed row into L2
                if (next < end && ((next - base) >> 2) != (li >> 2))
                    prefetch_l2(qc + ((next - base) >> 2) * c.n, 4u * static_cast<uint32_t>(c.n),
                                lane);
                const uint32_t sel = (0x3210u & ~(0xFu << (4 * b))) |
                                     (static_cast<uint32_t>(4 + (li & 3)) << (4 * b));
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
        __syncwarp();
        if (it < 0) it = next_work(work, gridDim.x, lane);
    }
}

// int8 channel of a mixed batch: block per internal four-frame group;
// byte b of word (group, n) is frame ibase + 4 g + b of the group's code, or
// +clip for padding.
__global__ void mixed_quantize_kernel(const DevCode *__restrict__ codes,
                                      const int *__restrict__ group_code,
                                      const long long *__restrict__ group_first,
                                      const long long *__restrict__ group_qoff, long long groups,
                                      const long long *__restrict__ uframe,
                                      const long long *__restrict__ llr_off,
                                      const float *__restrict__ llr, uint32_t *__restrict__ q,
                                      float scale, int clip) {
    const float fc = static_cast<float>(clip);
    for (long long g = blockIdx.x; g < groups; g += gridDim.x) {
        const int n = codes[group_code[g]].n;
        long long src[4];
#pragma unroll
        for (int b = 0; b < 4; ++b) {
            const long long uf = uframe[group_first[g] + b];
            src[b] = uf >= 0 ? llr_off[uf] : -1;
        }
        uint32_t *dst = q + group_qoff[g];
        for (int i = threadIdx.x; i < n; i += blockDim.x) {
            uint32_t word = 0;
#pragma unroll
            for (int b = 0; b < 4; ++b) {
                const uint32_t v = src[b] >= 0 ? quantize_one(llr[src[b] + i], scale, fc)
                                               : static_cast<uint32_t>(clip);
                word |= v << (8 * b);
            }
            dst[i] = word;
        }
    }
}

// Error counts of a mixed batch: one warp per frame, counters as in
// ldpc_frame_stats plus frame errors per code.
__global__ void mixed_stats_kernel(const DevCode *__restrict__ codes,
                                   const int *__restrict__ code_of_frame, long long frames,
                                   const long long *__restrict__ info_off,
                                   const long long *__restrict__ hard_off,
                                   const uint8_t *__restrict__ info,
                                   const uint32_t *__restrict__ hard,
                                   const int32_t *__restrict__ iters, int max_iters,
                                   unsigned long long *__restrict__ cnt,
                                   unsigned long long *__restrict__ code_fe) {
    const int lane = threadIdx.x & 31;
    const long long warps = static_cast<long long>(gridDim.x) * (blockDim.x >> 5);
    for (long long f = (blockIdx.x * static_cast<long long>(blockDim.x) + threadIdx.x) >> 5;
         f < frames; f += warps) {
        const int ci = code_of_frame[f];
        const DevCode c = codes[ci];
        bool syn_ok;
        const unsigned long long errs =
            frame_outcome(c, info + info_off[f], hard + hard_off[f], lane, &syn_ok);
        if (lane == 0) {
            count_frame(cnt, errs, syn_ok, iters[f], max_iters);
            if (errs && code_fe) atomicAdd(&code_fe[ci], 1ull);
        }
    }
}

// 1 for every frame whose hard decisions violate a check (warp per frame).
__global__ void mixed_flags_kernel(const DevCode *__restrict__ codes,
                                   const int *__restrict__ code_of_frame, long long frames,
                                   const long long *__restrict__ hard_off,
                                   const uint32_t *__restrict__ hard, uint8_t *__restrict__ bad) {
    const int lane = threadIdx.x & 31;
    const long long warps = static_cast<long long>(gridDim.x) * (blockDim.x >> 5);
    for (long long f = (blockIdx.x * static_cast<long long>(blockDim.x) + threadIdx.x) >> 5;
         f < frames; f += warps) {
        const DevCode c = codes[code_of_frame[f]];
        const bool ok = hard_syndrome_ok(c, hard + hard_off[f], lane);
        if (lane == 0) bad[f] = ok ? 0 : 1;
    }
}

// Frame s of plan B is frame idx[s] of plan A (same code set).  what = 0:
// LLR row A -> B; 1: hard-decision row B -> A; 2: iteration count B -> A plus
// add[code].  Block per frame of B.
__global__ void mixed_move_kernel(const DevCode *__restrict__ codes,
                                  const int *__restrict__ code_b, long long frames_b,
                                  const long long *__restrict__ idx,
                                  const long long *__restrict__ off_a,
                                  const long long *__restrict__ off_b, int what,
                                  uint32_t *__restrict__ a, uint32_t *__restrict__ b,
                                  const int *__restrict__ add) {
    for (long long s = blockIdx.x; s < frames_b; s += gridDim.x) {
        const long long fa = idx[s];
        const int ci = code_b[s];
        if (what == 2) {
            if (threadIdx.x == 0)
                a[fa] = static_cast<uint32_t>(static_cast<int>(b[s]) + (add ? add[ci] : 0));
            continue;
        }
        const int n = what == 0 ? codes[ci].n : codes[ci].nwords;
        uint32_t *pa = a + off_a[fa];
        uint32_t *pb = b + off_b[s];
        for (int i = threadIdx.x; i < n; i += blockDim.x) {
            if (what == 0)
                pb[i] = pa[i];
            else
                pa[i] = pb[i];
        }
    }
}

// Paired outcomes of two decoders over a mixed batch (as
// ldpc_paired_frame_errors): cnt[2 a + b], a / b = decoder A / B wrong.
__global__ void mixed_paired_kernel(const DevCode *__restrict__ codes,
                                    const int *__restrict__ code_of_frame, long long frames,
                                    const long long *__restrict__ info_off,
                                    const long long *__restrict__ hard_off,
                                    const uint8_t *__restrict__ info,
                                    const uint32_t *__restrict__ ha,
                                    const uint32_t *__restrict__ hb,
                                    unsigned long long *__restrict__ cnt) {
    const int lane = threadIdx.x & 31;
    const long long warps = static_cast<long long>(gridDim.x) * (blockDim.x >> 5);
    for (long long f = (blockIdx.x * static_cast<long long>(blockDim.x) + threadIdx.x) >> 5;
         f < frames; f += warps) {
        const int k = codes[code_of_frame[f]].k;
        const uint8_t *in = info + info_off[f];
        const uint32_t *pa = ha + hard_off[f], *pb = hb + hard_off[f];
        uint32_t ea = 0, eb = 0;
        for (int t = lane; t < k; t += 32) {
            const uint32_t x = in[t] & 1u;
            ea |= ((pa[t >> 5] >> (t & 31)) & 1u) ^ x;
            eb |= ((pb[t >> 5] >> (t & 31)) & 1u) ^ x;
        }
        const bool wa = __any_sync(0xFFFFFFFFu, ea), wb = __any_sync(0xFFFFFFFFu, eb);
        if (lane == 0) atomicAdd(&cnt[2 * (wa ? 1 : 0) + (wb ? 1 : 0)], 1ull);
    }
}

// Rows of one code's frames (consecutive in src, the code's frames in batch
// order) copied to their places in the plan layout: block per frame.
__global__ void mixed_scatter_kernel(const long long *__restrict__ uframe, long long first,
                                     long long count, const long long *__restrict__ off,
                                     int row_bytes, const uint8_t *__restrict__ src,
                                     uint8_t *__restrict__ dst, int elem_bytes) {
    for (long long j = blockIdx.x; j < count; j += gridDim.x) {
        const long long uf = uframe[first + j];
        const uint8_t *s = src + j * row_bytes;
        uint8_t *d = dst + off[uf] * elem_bytes;
        for (int i = threadIdx.x; i < row_bytes; i += blockDim.x) d[i] = s[i];
    }
}

}  // namespace

// ---------------------------------------------------------------------------
// Host side
// ---------------------------------------------------------------------------

struct CodeSet {
    int device = 0;
    std::vector<const Code *> codes;
    DevCode *d_desc = nullptr;
};

struct MixedGroup {
    int dslots = 0;
    std::vector<int> codes;              // set indices, largest first
    int smem[2] = {0, 0};                // bytes per block: [0] FP32, [1] int8
    int smem_learned = 0;                // FP32 plus the learned weight buffers
    int chunk[2] = {8, 16};              // frames per work item
    int per_sm[2] = {0, 0};              // resident blocks per SM (0: occupancy limit)
    int wpf = 1;                         // FP32 warps per frame (a team shares the rows)
    int fpb = 1;                         // FP32 frames (teams) per block
    MixedItem *d_items[2] = {nullptr, nullptr};
    int n_items[2] = {0, 0};
    int built_chunk[2] = {0, 0};         // chunk the item list was built for
    bool bulk_ok = true;                 // every N a multiple of 4 words
    cudaStream_t stream = nullptr;
    cudaEvent_t done = nullptr;
};

struct MixedPlan {
    const CodeSet *set = nullptr;
    int device = 0;
    long long frames = 0;
    std::vector<int> code_of_frame;
    std::vector<long long> llr_off, info_off, hard_off;   // [frames + 1]
    std::vector<long long> ibase, fcount, qoff;           // per set code
    std::vector<long long> uframe;                        // internal index -> frame, -1 pad
    long long q_words = 0, groups4 = 0;
    int *d_code_of_frame = nullptr;
    long long *d_llr_off = nullptr, *d_info_off = nullptr, *d_hard_off = nullptr;
    long long *d_uframe = nullptr, *d_ibase = nullptr, *d_qoff = nullptr;
    int *d_group_code = nullptr;
    long long *d_group_first = nullptr, *d_group_qoff = nullptr;
    unsigned long long *d_work = nullptr;                // one counter per group and dtype
    std::vector<MixedGroup> groups;     // heaviest (edges x frames) first
    bool serial[2] = {false, false};     // groups one after another on the caller's stream
    // learned weights per set code (device pointers) and their iteration counts
    const float **d_wptr = nullptr;
    int *d_wT = nullptr;
    std::vector<int> wT;
    cudaEvent_t fork = nullptr;
    std::mutex mu;                                       // item rebuilds
};

template <typename T>
static cudaError_t upload(T **dst, const std::vector<T> &src) {
    const size_t bytes = sizeof(T) * std::max<size_t>(src.size(), 1);
    cudaError_t e = cudaMalloc(dst, bytes);
    if (e == cudaSuccess && !src.empty())
        e = cudaMemcpy(*dst, src.data(), sizeof(T) * src.size(), cudaMemcpyHostToDevice);
    return e;
}

static int region_bytes_f32(const Code &c) {
    return 16 + 4 * ((posterior_words(c.n) + c.m * 3 + 3) & ~3);
}
static int region_bytes_i8(const Code &c, int dslots) {
    const int sw = (dslots + 7) / 8;
    const int rw = (3 + sw + 1) & ~1;
    return 16 + 4 * ((posterior_words(c.n) + c.m * rw + 3) & ~3);
}

// Work items of one group for `chunk` frames per item (int8: a multiple of 4).
static ldpc_status build_items(MixedPlan &pl, MixedGroup &g, int dt, int chunk) {
    std::vector<MixedItem> items;
    for (int ci : g.codes) {
        const long long padded = (pl.fcount[ci] + 3) & ~3LL;
        for (long long s = 0; s < padded; s += chunk) {
            MixedItem it;
            it.code = ci;
            it.start = pl.ibase[ci] + s;
            it.count = static_cast<int>(std::min<long long>(chunk, padded - s));
            items.push_back(it);
        }
    }
    cudaFree(g.d_items[dt]);
    g.d_items[dt] = nullptr;
    cudaError_t e = upload(&g.d_items[dt], items);
    if (e != cudaSuccess) return cuda_fail(e, "mixed plan: work items");
    g.n_items[dt] = static_cast<int>(items.size());
    g.built_chunk[dt] = chunk;
    return LDPC_OK;
}

static void release_plan(MixedPlan *pl) {
    int prev = 0;
    cudaGetDevice(&prev);
    cudaSetDevice(pl->device);
    for (auto &g : pl->groups) {
        cudaFree(g.d_items[0]);
        cudaFree(g.d_items[1]);
        if (g.stream) cudaStreamDestroy(g.stream);
        if (g.done) cudaEventDestroy(g.done);
    }
    cudaFree(pl->d_code_of_frame);
    cudaFree(pl->d_llr_off);
    cudaFree(pl->d_info_off);
    cudaFree(pl->d_hard_off);
    cudaFree(pl->d_uframe);
    cudaFree(pl->d_ibase);
    cudaFree(pl->d_qoff);
    cudaFree(pl->d_group_code);
    cudaFree(pl->d_group_first);
    cudaFree(pl->d_group_qoff);
    cudaFree(pl->d_work);
    cudaFree(pl->d_wptr);
    cudaFree(pl->d_wT);
    if (pl->fork) cudaEventDestroy(pl->fork);
    cudaSetDevice(prev);
    delete pl;
}

// dt: 0 FP32, 1 int8, 2 FP32 learned (FP32 work items and counter).
template <int DMAX>
static ldpc_status launch_group_t(MixedPlan &pl, MixedGroup &g, int gi, int dt, const void *d_in,
                                  const DecodeParams &p, uint32_t *d_hard, int32_t *d_iters,
                                  void *d_post, cudaStream_t s) {
    const bool learned = dt == 2;
    if (learned) dt = 0;
    const bool team = dt == 0 && (g.wpf > 1 || g.fpb > 1);
    const int smem1 = learned ? g.smem_learned : g.smem[dt];
    // teams: each its one-warp region plus eight shared words, 16-byte aligned
    const int team_bytes = (smem1 + 32 + 15) & ~15;
    const int smem = team ? g.fpb * team_bytes : smem1;
    const int threads = team ? 32 * g.wpf * g.fpb : 32;
    if (team) {
        int max_optin = 0;
        cudaDeviceGetAttribute(&max_optin, cudaDevAttrMaxSharedMemoryPerBlockOptin, pl.device);
        if (smem > max_optin)
            return fail(LDPC_ERR_UNSUPPORTED, "mixed decode: frames per block exceed shared memory");
    }
    const void *kern =
        dt == 1   ? reinterpret_cast<const void *>(mixed_i8_kernel<DMAX>)
        : team    ? (learned ? reinterpret_cast<const void *>(mixed_f32_team_kernel<DMAX, true>)
                             : reinterpret_cast<const void *>(mixed_f32_team_kernel<DMAX, false>))
        : learned ? reinterpret_cast<const void *>(mixed_f32_kernel<DMAX, true>)
                  : reinterpret_cast<const void *>(mixed_f32_kernel<DMAX, false>);
    cudaError_t e = allow_dynamic_smem(reinterpret_cast<const void *>(kern));
    if (e != cudaSuccess) return cuda_fail(e, "mixed kernel attribute");
    int per_sm = 0, sms = 148;
    e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kern, threads, smem);
    if (e != cudaSuccess) return cuda_fail(e, "mixed occupancy");
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, pl.device);
    per_sm = std::max(per_sm, 1);
    if (g.per_sm[dt] > 0) per_sm = std::min(per_sm, g.per_sm[dt]);
    const int units = team ? (g.n_items[dt] + g.fpb - 1) / g.fpb : g.n_items[dt];
    const int grid = std::max(1, std::min(units, per_sm * sms));
    unsigned long long *work = pl.d_work + 2 * gi + (dt == 1 ? 1 : 0);
    e = cudaMemsetAsync(work, 0, sizeof(unsigned long long), s);
    if (e != cudaSuccess) return cuda_fail(e, "mixed work counter");
    const DevCode *codes = pl.set->d_desc;
    if (team) {
        const bool bulk = g.bulk_ok && (reinterpret_cast<uintptr_t>(d_in) & 15u) == 0;
        if (learned)
            mixed_f32_team_kernel<DMAX, true><<<grid, threads, smem, s>>>(
                codes, g.d_items[0], g.n_items[0], pl.d_uframe, pl.d_llr_off, pl.d_hard_off,
                static_cast<const float *>(d_in), p, d_hard, d_iters,
                static_cast<float *>(d_post), work, bulk ? 1 : 0, pl.d_wptr, pl.d_wT, g.wpf, g.fpb,
                team_bytes / 4);
        else
            mixed_f32_team_kernel<DMAX, false><<<grid, threads, smem, s>>>(
                codes, g.d_items[0], g.n_items[0], pl.d_uframe, pl.d_llr_off, pl.d_hard_off,
                static_cast<const float *>(d_in), p, d_hard, d_iters,
                static_cast<float *>(d_post), work, bulk ? 1 : 0, nullptr, nullptr, g.wpf, g.fpb,
                team_bytes / 4);
    } else if (dt == 0) {
        const bool bulk = g.bulk_ok && (reinterpret_cast<uintptr_t>(d_in) & 15u) == 0;
        if (learned)
            mixed_f32_kernel<DMAX, true><<<grid, 32, smem, s>>>(
                codes, g.d_items[0], g.n_items[0], pl.d_uframe, pl.d_llr_off, pl.d_hard_off,
                static_cast<const float *>(d_in), p, d_hard, d_iters,
                static_cast<float *>(d_post), work, bulk ? 1 : 0, pl.d_wptr, pl.d_wT);
        else
            mixed_f32_kernel<DMAX, false><<<grid, 32, smem, s>>>(
                codes, g.d_items[0], g.n_items[0], pl.d_uframe, pl.d_llr_off, pl.d_hard_off,
                static_cast<const float *>(d_in), p, d_hard, d_iters,
                static_cast<float *>(d_post), work, bulk ? 1 : 0, nullptr, nullptr);
    } else {
        const bool bulk = g.bulk_ok && (reinterpret_cast<uintptr_t>(d_in) & 15u) == 0;
        mixed_i8_kernel<DMAX><<<grid, 32, smem, s>>>(
            codes, g.d_items[1], g.n_items[1], pl.d_uframe, pl.d_llr_off, pl.d_hard_off,
            pl.d_ibase, pl.d_qoff, static_cast<const uint32_t *>(d_in), p, d_hard, d_iters,
            static_cast<int8_t *>(d_post), work, bulk ? 1 : 0);
    }
    e = cudaGetLastError();
    return e == cudaSuccess ? LDPC_OK : cuda_fail(e, "mixed decode launch");
}

static ldpc_status launch_group(MixedPlan &pl, int gi, int dt, const void *d_in,
                                const DecodeParams &p, uint32_t *d_hard, int32_t *d_iters,
                                void *d_post, cudaStream_t s) {
    MixedGroup &g = pl.groups[gi];
    const int it = dt == 2 ? 0 : dt;   // the learned decoder uses the FP32 work items
    if (g.built_chunk[it] != g.chunk[it]) {
        std::lock_guard<std::mutex> lock(pl.mu);
        if (g.built_chunk[it] != g.chunk[it]) {
            ldpc_status st = build_items(pl, g, it, g.chunk[it]);
            if (st != LDPC_OK) return st;
        }
    }
    if (g.n_items[it] == 0) return LDPC_OK;
    switch (g.dslots) {
#define LDPC_MIXED_CASE(D) \
    case D: return launch_group_t<D>(pl, g, gi, dt, d_in, p, d_hard, d_iters, d_post, s);
        LDPC_SLOT_CLASSES(LDPC_MIXED_CASE)
#undef LDPC_MIXED_CASE
        default: return fail(LDPC_ERR_UNSUPPORTED, "mixed decode: no kernel for this row degree");
    }
}

// All groups, forked from `s` onto the groups' streams and joined back (or,
// when the plan says so, one after another on `s`).
static ldpc_status launch_all(MixedPlan &pl, int dt, const void *d_in, const DecodeParams &p,
                              uint32_t *d_hard, int32_t *d_iters, void *d_post, cudaStream_t s) {
    if (pl.serial[dt == 1 ? 1 : 0]) {
        for (size_t gi = 0; gi < pl.groups.size(); ++gi) {
            ldpc_status st = launch_group(pl, static_cast<int>(gi), dt, d_in, p, d_hard, d_iters,
                                          d_post, s);
            if (st != LDPC_OK) return st;
        }
        return LDPC_OK;
    }
    cudaError_t e = cudaEventRecord(pl.fork, s);
    if (e != cudaSuccess) return cuda_fail(e, "mixed fork");
    for (size_t gi = 0; gi < pl.groups.size(); ++gi) {
        MixedGroup &g = pl.groups[gi];
        e = cudaStreamWaitEvent(g.stream, pl.fork, 0);
        if (e != cudaSuccess) return cuda_fail(e, "mixed fork wait");
        ldpc_status st = launch_group(pl, static_cast<int>(gi), dt, d_in, p, d_hard, d_iters,
                                      d_post, g.stream);
        if (st != LDPC_OK) return st;
        e = cudaEventRecord(g.done, g.stream);
        if (e != cudaSuccess) return cuda_fail(e, "mixed join record");
        e = cudaStreamWaitEvent(s, g.done, 0);
        if (e != cudaSuccess) return cuda_fail(e, "mixed join wait");
    }
    return LDPC_OK;
}

static ldpc_status check_params(const ldpc_decode_params *params, ldpc_dtype dtype,
                                const char *what) {
    if (!params) return fail(LDPC_ERR_INVALID_ARG, std::string(what) + ": params is NULL");
    if (params->max_iters < 1 || params->max_iters > kMaxIters ||
        (params->normalise != 0 && params->normalise != 1) ||
        (params->early_stop != 0 && params->early_stop != 1) ||
        (params->normalise && !(params->alpha == params->alpha)))
        return fail(LDPC_ERR_INVALID_ARG, std::string(what) + ": bad decode parameters");
    if (dtype != LDPC_F32 && dtype != LDPC_I8X4)
        return fail(LDPC_ERR_INVALID_ARG, std::string(what) + ": unknown dtype");
    if (dtype == LDPC_I8X4 && params->normalise && params->alpha != 0.75f)
        return fail(LDPC_ERR_UNSUPPORTED, std::string(what) + ": int8 scaling needs alpha 0.75");
    return LDPC_OK;
}

static DecodeParams to_params(const ldpc_decode_params *params) {
    DecodeParams p;
    p.max_iters = params->max_iters;
    p.alpha = params->normalise ? params->alpha : 1.0f;
    p.normalise = params->normalise;
    p.early_stop = params->early_stop;
    return p;
}

}  // namespace ldpc

using namespace ldpc;

struct ldpc_codeset {
    CodeSet s;
};
struct ldpc_mixed_plan {
    MixedPlan *p;
};
struct ldpc_mixed_graph {
    int device = 0;
    cudaStream_t cap = nullptr;
    cudaGraph_t graph = nullptr;
    cudaGraphExec_t exec = nullptr;
};

extern "C" {

ldpc_status ldpc_codeset_create(const ldpc_code *const *codes, int count, ldpc_codeset **out) {
    if (!out) return fail(LDPC_ERR_INVALID_ARG, "ldpc_codeset_create: out is NULL");
    *out = nullptr;
    if (!codes || count < 1 || count > 4096)
        return fail(LDPC_ERR_INVALID_ARG, "ldpc_codeset_create: need 1..4096 codes");
    std::vector<DevCode> desc(count);
    int device = -1;
    for (int i = 0; i < count; ++i) {
        if (!codes[i]) return fail(LDPC_ERR_INVALID_ARG, "ldpc_codeset_create: NULL code");
        const Code &c = codes[i]->c;
        if (device >= 0 && c.device != device)
            return fail(LDPC_ERR_INVALID_ARG, "ldpc_codeset_create: codes on different devices");
        device = c.device;
        if (!c.dslots)
            return fail(LDPC_ERR_UNSUPPORTED, "ldpc_codeset_create: row degree above 27");
        desc[i] = dev_view(c);
    }
    ldpc_codeset *h = new (std::nothrow) ldpc_codeset;
    if (!h) return fail(LDPC_ERR_NOMEM, "ldpc_codeset_create: host allocation");
    h->s.device = device;
    for (int i = 0; i < count; ++i) h->s.codes.push_back(&codes[i]->c);
    int prev = 0;
    cudaGetDevice(&prev);
    cudaSetDevice(device);
    cudaError_t e = upload(&h->s.d_desc, desc);
    cudaSetDevice(prev);
    if (e != cudaSuccess) {
        cudaFree(h->s.d_desc);
        delete h;
        return cuda_fail(e, "ldpc_codeset_create");
    }
    *out = h;
    return LDPC_OK;
}

void ldpc_codeset_destroy(ldpc_codeset *set) {
    if (!set) return;
    int prev = 0;
    cudaGetDevice(&prev);
    cudaSetDevice(set->s.device);
    cudaFree(set->s.d_desc);
    cudaSetDevice(prev);
    delete set;
}

ldpc_status ldpc_mixed_plan_create(const ldpc_codeset *set, const int32_t *h_code_of_frame,
                                   int64_t frames, ldpc_mixed_plan **out) {
    if (!out) return fail(LDPC_ERR_INVALID_ARG, "ldpc_mixed_plan_create: out is NULL");
    *out = nullptr;
    if (!set || frames < 0 || (frames > 0 && !h_code_of_frame))
        return fail(LDPC_ERR_INVALID_ARG, "ldpc_mixed_plan_create: bad set, frames or codes");
    const int count = static_cast<int>(set->s.codes.size());
    for (int64_t f = 0; f < frames; ++f)
        if (h_code_of_frame[f] < 0 || h_code_of_frame[f] >= count)
            return fail(LDPC_ERR_INVALID_ARG,
                        "ldpc_mixed_plan_create: code index outside the set at frame " +
                            std::to_string(f));
    MixedPlan *pl = new (std::nothrow) MixedPlan;
    if (!pl) return fail(LDPC_ERR_NOMEM, "ldpc_mixed_plan_create: host allocation");
    pl->set = &set->s;
    pl->device = set->s.device;
    pl->frames = frames;
    pl->code_of_frame.assign(h_code_of_frame, h_code_of_frame + frames);
    const auto &codes = set->s.codes;
    pl->llr_off.assign(frames + 1, 0);
    pl->info_off.assign(frames + 1, 0);
    pl->hard_off.assign(frames + 1, 0);
    pl->fcount.assign(count, 0);
    for (int64_t f = 0; f < frames; ++f) {
        const Code &c = *codes[pl->code_of_frame[f]];
        pl->llr_off[f + 1] = pl->llr_off[f] + c.n;
        pl->info_off[f + 1] = pl->info_off[f] + c.k;
        pl->hard_off[f + 1] = pl->hard_off[f] + (c.n + 31) / 32;
        pl->fcount[pl->code_of_frame[f]] += 1;
    }
    bool all_n4 = true;
    for (int ci = 0; ci < count; ++ci)
        if (pl->fcount[ci] && codes[ci]->n % 4) all_n4 = false;
    // launch groups: same slot class, int8 shared memory within a factor of 2
    std::vector<int> order;
    for (int ci = 0; ci < count; ++ci)
        if (pl->fcount[ci]) order.push_back(ci);
    std::stable_sort(order.begin(), order.end(), [&](int a, int b) {
        if (codes[a]->dslots != codes[b]->dslots) return codes[a]->dslots < codes[b]->dslots;
        return region_bytes_i8(*codes[a], codes[a]->dslots) >
               region_bytes_i8(*codes[b], codes[b]->dslots);
    });
    for (int ci : order) {
        const Code &c = *codes[ci];
        const int si8 = region_bytes_i8(c, c.dslots);
        if (pl->groups.empty() || pl->groups.back().dslots != c.dslots ||
            2 * si8 < pl->groups.back().smem[1]) {
            pl->groups.emplace_back();
            pl->groups.back().dslots = c.dslots;
        }
        MixedGroup &g = pl->groups.back();
        g.codes.push_back(ci);
        g.smem[0] = std::max(g.smem[0], region_bytes_f32(c));
        g.smem_learned = std::max(g.smem_learned, region_bytes_f32(c) + 4 * kWeightBuffers *
                                                                           c.mb * wpad(c.dslots));
        g.smem[1] = std::max(g.smem[1], si8);
        if (c.n % 4) g.bulk_ok = false;
        if (!all_n4) g.bulk_ok = false;
    }
    // heaviest groups first: their launches start first and the lighter ones
    // fill the SMs as the heavy queues drain
    {
        auto work_of = [&](const MixedGroup &g) {
            double w = 0;
            for (int ci : g.codes)
                w += static_cast<double>(pl->fcount[ci]) * codes[ci]->n_edges * codes[ci]->z;
            return w;
        };
        std::stable_sort(pl->groups.begin(), pl->groups.end(),
                         [&](const MixedGroup &a, const MixedGroup &b) {
                             return work_of(a) > work_of(b);
                         });
    }
    // internal order, packed int8 groups
    pl->ibase.assign(count, 0);
    pl->qoff.assign(count, 0);
    long long ib = 0, qo = 0;
    std::vector<int> gcode;
    std::vector<long long> gfirst, gqoff;
    for (const auto &g : pl->groups)
        for (int ci : g.codes) {
            const long long padded = (pl->fcount[ci] + 3) & ~3LL;
            pl->ibase[ci] = ib;
            pl->qoff[ci] = qo;
            for (long long lg = 0; lg < padded / 4; ++lg) {
                gcode.push_back(ci);
                gfirst.push_back(ib + 4 * lg);
                gqoff.push_back(qo + lg * codes[ci]->n);
            }
            ib += padded;
            qo += ((padded / 4) * codes[ci]->n + 3) & ~3LL;
        }
    pl->q_words = qo;
    pl->groups4 = static_cast<long long>(gcode.size());
    pl->uframe.assign(ib, -1);
    {
        std::vector<long long> fill(count, 0);
        for (int64_t f = 0; f < frames; ++f) {
            const int ci = pl->code_of_frame[f];
            pl->uframe[pl->ibase[ci] + fill[ci]++] = f;
        }
    }
    int prev = 0;
    cudaGetDevice(&prev);
    cudaSetDevice(pl->device);
    cudaError_t e = upload(&pl->d_code_of_frame, pl->code_of_frame);
    if (e == cudaSuccess) e = upload(&pl->d_llr_off, pl->llr_off);
    if (e == cudaSuccess) e = upload(&pl->d_info_off, pl->info_off);
    if (e == cudaSuccess) e = upload(&pl->d_hard_off, pl->hard_off);
    if (e == cudaSuccess) e = upload(&pl->d_uframe, pl->uframe);
    if (e == cudaSuccess) e = upload(&pl->d_ibase, pl->ibase);
    if (e == cudaSuccess) e = upload(&pl->d_qoff, pl->qoff);
    if (e == cudaSuccess) e = upload(&pl->d_group_code, gcode);
    if (e == cudaSuccess) e = upload(&pl->d_group_first, gfirst);
    if (e == cudaSuccess) e = upload(&pl->d_group_qoff, gqoff);
    if (e == cudaSuccess)
        e = cudaMalloc(&pl->d_work, sizeof(unsigned long long) * 2 * (pl->groups.size() + 1));
    if (e == cudaSuccess) e = cudaEventCreateWithFlags(&pl->fork, cudaEventDisableTiming);
    for (auto &g : pl->groups) {
        if (e == cudaSuccess) e = cudaStreamCreateWithFlags(&g.stream, cudaStreamNonBlocking);
        if (e == cudaSuccess) e = cudaEventCreateWithFlags(&g.done, cudaEventDisableTiming);
    }
    ldpc_status st = LDPC_OK;
    if (e != cudaSuccess) st = cuda_fail(e, "ldpc_mixed_plan_create");
    for (size_t gi = 0; st == LDPC_OK && gi < pl->groups.size(); ++gi)
        for (int dt = 0; st == LDPC_OK && dt < 2; ++dt)
            st = build_items(*pl, pl->groups[gi], dt, pl->groups[gi].chunk[dt]);
    cudaSetDevice(prev);
    if (st != LDPC_OK) {
        release_plan(pl);
        return st;
    }
    ldpc_mixed_plan *h = new (std::nothrow) ldpc_mixed_plan;
    if (!h) {
        release_plan(pl);
        return fail(LDPC_ERR_NOMEM, "ldpc_mixed_plan_create: host allocation");
    }
    h->p = pl;
    *out = h;
    return LDPC_OK;
}

void ldpc_mixed_plan_destroy(ldpc_mixed_plan *plan) {
    if (!plan) return;
    release_plan(plan->p);
    delete plan;
}

ldpc_status ldpc_mixed_plan_sizes(const ldpc_mixed_plan *plan, int64_t *llr_elems,
                                  int64_t *info_elems, int64_t *hard_words, int64_t *q_words,
                                  int *launch_groups) {
    if (!plan) return fail(LDPC_ERR_INVALID_ARG, "ldpc_mixed_plan_sizes: plan is NULL");
    const MixedPlan &p = *plan->p;
    if (llr_elems) *llr_elems = p.llr_off[p.frames];
    if (info_elems) *info_elems = p.info_off[p.frames];
    if (hard_words) *hard_words = p.hard_off[p.frames];
    if (q_words) *q_words = p.q_words;
    if (launch_groups) *launch_groups = static_cast<int>(p.groups.size());
    return LDPC_OK;
}

ldpc_status ldpc_mixed_plan_offsets(const ldpc_mixed_plan *plan, int64_t *h_llr_off,
                                    int64_t *h_info_off, int64_t *h_hard_off) {
    if (!plan) return fail(LDPC_ERR_INVALID_ARG, "ldpc_mixed_plan_offsets: plan is NULL");
    const MixedPlan &p = *plan->p;
    const size_t n = static_cast<size_t>(p.frames + 1);
    if (h_llr_off) std::memcpy(h_llr_off, p.llr_off.data(), sizeof(int64_t) * n);
    if (h_info_off) std::memcpy(h_info_off, p.info_off.data(), sizeof(int64_t) * n);
    if (h_hard_off) std::memcpy(h_hard_off, p.hard_off.data(), sizeof(int64_t) * n);
    return LDPC_OK;
}

ldpc_status ldpc_mixed_group_info(const ldpc_mixed_plan *plan, int group, int *slot_class,
                                  int *codes, int *smem_f32, int *smem_i8, int *chunk_f32,
                                  int *chunk_i8, int *blocks_per_sm_f32, int *blocks_per_sm_i8) {
    if (!plan || group < 0 || group >= static_cast<int>(plan->p->groups.size()))
        return fail(LDPC_ERR_INVALID_ARG, "ldpc_mixed_group_info: bad plan or group");
    const MixedGroup &g = plan->p->groups[group];
    if (slot_class) *slot_class = g.dslots;
    if (codes) *codes = static_cast<int>(g.codes.size());
    if (smem_f32) *smem_f32 = g.smem[0];
    if (smem_i8) *smem_i8 = g.smem[1];
    if (chunk_f32) *chunk_f32 = g.chunk[0];
    if (chunk_i8) *chunk_i8 = g.chunk[1];
    if (blocks_per_sm_f32) *blocks_per_sm_f32 = g.per_sm[0];
    if (blocks_per_sm_i8) *blocks_per_sm_i8 = g.per_sm[1];
    return LDPC_OK;
}

ldpc_status ldpc_mixed_group_launch(ldpc_mixed_plan *plan, int group, ldpc_dtype dtype,
                                    const ldpc_group_launch *set, ldpc_group_launch *get) {
    if (!plan || group < 0 || group >= static_cast<int>(plan->p->groups.size()))
        return fail(LDPC_ERR_INVALID_ARG, "ldpc_mixed_group_launch: bad plan or group");
    if (dtype != LDPC_F32 && dtype != LDPC_I8X4)
        return fail(LDPC_ERR_INVALID_ARG, "ldpc_mixed_group_launch: unknown dtype");
    MixedGroup &g = plan->p->groups[group];
    const int dt = dtype == LDPC_F32 ? 0 : 1;
    if (set) {
        const bool f32 = dt == 0;
        if (set->frames_per_item < 1 || set->frames_per_item > 1024 || set->blocks_per_sm < 0 ||
            set->blocks_per_sm > 64 || set->warps_per_frame < 1 || set->frames_per_block < 1 ||
            (f32 && (set->warps_per_frame > 3 || set->frames_per_block > 4)) ||
            (!f32 && (set->warps_per_frame != 1 || set->frames_per_block != 1)))
            return fail(LDPC_ERR_INVALID_ARG,
                        "ldpc_mixed_group_launch: frames per item 1..1024, blocks per SM 0..64, "
                        "FP32 warps per frame 1..3 and frames per block 1..4 (int8: 1 and 1)");
        g.chunk[dt] = set->frames_per_item;
        g.per_sm[dt] = set->blocks_per_sm;
        if (f32) {
            g.wpf = set->warps_per_frame;
            g.fpb = set->frames_per_block;
        }
    }
    if (get) {
        get->frames_per_item = g.chunk[dt];
        get->blocks_per_sm = g.per_sm[dt];
        get->warps_per_frame = dt == 0 ? g.wpf : 1;
        get->frames_per_block = dt == 0 ? g.fpb : 1;
    }
    return LDPC_OK;
}

}  // extern "C"

namespace {

ldpc_status bind_plan(const MixedPlan &p) {
    cudaError_t e = cudaSetDevice(p.device);
    return e == cudaSuccess ? LDPC_OK : cuda_fail(e, "cudaSetDevice");
}

ldpc_status quantize_mixed(const MixedPlan &p, const float *d_llr, uint32_t *d_q, float scale,
                           int clip, cudaStream_t s) {
    if (p.groups4 == 0) return LDPC_OK;
    int sms = 148;
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, p.device);
    const long long grid = std::min<long long>(p.groups4, 16LL * sms);
    mixed_quantize_kernel<<<static_cast<unsigned>(grid), 128, 0, s>>>(
        p.set->d_desc, p.d_group_code, p.d_group_first, p.d_group_qoff, p.groups4, p.d_uframe,
        p.d_llr_off, d_llr, d_q, scale, clip);
    cudaError_t e = cudaGetLastError();
    return e == cudaSuccess ? LDPC_OK : cuda_fail(e, "mixed_quantize_kernel");
}

ldpc_status stats_mixed(const MixedPlan &p, const uint8_t *d_info, const uint32_t *d_hard,
                        const int32_t *d_iters, int max_iters, int64_t *d_counters,
                        int64_t *d_code_fe, cudaStream_t s) {
    cudaError_t e = cudaMemsetAsync(d_counters, 0, sizeof(int64_t) * (5 + max_iters), s);
    if (e == cudaSuccess && d_code_fe)
        e = cudaMemsetAsync(d_code_fe, 0, sizeof(int64_t) * p.set->codes.size(), s);
    if (e != cudaSuccess) return cuda_fail(e, "cudaMemsetAsync counters");
    if (p.frames == 0) return LDPC_OK;
    int sms = 148;
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, p.device);
    const long long grid = std::min<long long>((p.frames + 7) / 8, 32LL * sms);
    mixed_stats_kernel<<<static_cast<unsigned>(grid), 256, 0, s>>>(
        p.set->d_desc, p.d_code_of_frame, p.frames, p.d_info_off, p.d_hard_off, d_info, d_hard,
        d_iters, max_iters, reinterpret_cast<unsigned long long *>(d_counters),
        reinterpret_cast<unsigned long long *>(d_code_fe));
    e = cudaGetLastError();
    return e == cudaSuccess ? LDPC_OK : cuda_fail(e, "mixed_stats_kernel");
}

}  // namespace

extern "C" {

ldpc_status ldpc_mixed_plan_serial(const ldpc_mixed_plan *plan, int *serial_f32,
                                   int *serial_i8) {
    if (!plan) return fail(LDPC_ERR_INVALID_ARG, "ldpc_mixed_plan_serial: plan is NULL");
    if (serial_f32) *serial_f32 = plan->p->serial[0] ? 1 : 0;
    if (serial_i8) *serial_i8 = plan->p->serial[1] ? 1 : 0;
    return LDPC_OK;
}

ldpc_status ldpc_mixed_quantize(const ldpc_mixed_plan *plan, const float *d_llr, uint32_t *d_q,
                                float scale, int clip, cudaStream_t stream) {
    if (!plan) return fail(LDPC_ERR_INVALID_ARG, "ldpc_mixed_quantize: plan is NULL");
    if (clip < 0 || clip > 127 || !(scale == scale))
        return fail(LDPC_ERR_INVALID_ARG, "ldpc_mixed_quantize: clip in [0, 127], scale not NaN");
    const MixedPlan &p = *plan->p;
    if (p.frames == 0) return LDPC_OK;
    if (!d_llr || !d_q) return fail(LDPC_ERR_INVALID_ARG, "ldpc_mixed_quantize: NULL buffer");
    ldpc_status st = bind_plan(p);
    if (st != LDPC_OK) return st;
    return quantize_mixed(p, d_llr, d_q, scale, clip, stream);
}

ldpc_status ldpc_decode_mixed(ldpc_mixed_plan *plan, ldpc_dtype dtype, const void *d_in,
                              const ldpc_decode_params *params, uint32_t *d_hard,
                              int32_t *d_iters, void *d_post, cudaStream_t stream) {
    if (!plan) return fail(LDPC_ERR_INVALID_ARG, "ldpc_decode_mixed: plan is NULL");
    ldpc_status st = check_params(params, dtype, "ldpc_decode_mixed");
    if (st != LDPC_OK) return st;
    MixedPlan &p = *plan->p;
    if (p.frames == 0) return LDPC_OK;
    if (!d_in || !d_hard || !d_iters)
        return fail(LDPC_ERR_INVALID_ARG, "ldpc_decode_mixed: NULL buffer");
    if ((st = bind_plan(p)) != LDPC_OK) return st;
    return launch_all(p, dtype == LDPC_F32 ? 0 : 1, d_in, to_params(params), d_hard, d_iters,
                      d_post, stream);
}

ldpc_status ldpc_mixed_stats(const ldpc_mixed_plan *plan, const uint8_t *d_info,
                             const uint32_t *d_hard, const int32_t *d_iters, int max_iters,
                             int64_t *d_counters, int64_t *d_code_frame_errors,
                             cudaStream_t stream) {
    if (!plan) return fail(LDPC_ERR_INVALID_ARG, "ldpc_mixed_stats: plan is NULL");
    if (max_iters < 1 || max_iters > kMaxIters)
        return fail(LDPC_ERR_INVALID_ARG, "ldpc_mixed_stats: max_iters outside 1..1000");
    const MixedPlan &p = *plan->p;
    if (!d_counters || (p.frames && (!d_info || !d_hard || !d_iters)))
        return fail(LDPC_ERR_INVALID_ARG, "ldpc_mixed_stats: NULL buffer");
    ldpc_status st = bind_plan(p);
    if (st != LDPC_OK) return st;
    return stats_mixed(p, d_info, d_hard, d_iters, max_iters, d_counters, d_code_frame_errors,
                       stream);
}

// Autotuner body.  lt: the launch type (0 FP32, 1 int8, 2 learned FP32);
// the learned launches use the FP32 work items, residency caps and
// concurrency, so lt = 2 tunes those (timing the learned decoder).
static ldpc_status autotune_impl(MixedPlan &p, int lt, const void *d_in, const DecodeParams &dp,
                                 uint32_t *d_hard, int32_t *d_iters, int reps,
                                 cudaStream_t stream) {
    const int dt = lt == 1 ? 1 : 0;   // the tuned slot
    ldpc_status st = LDPC_OK;
    cudaEvent_t a = nullptr, b = nullptr;
    cudaError_t e = cudaEventCreate(&a);
    if (e == cudaSuccess) e = cudaEventCreate(&b);
    if (e != cudaSuccess) return cuda_fail(e, "ldpc_mixed_autotune events");
    // median of `reps` timed decodes of the whole batch
    auto measure = [&](float *ms) -> ldpc_status {
        std::vector<float> t;
        for (int r = 0; r < reps; ++r) {
            cudaEventRecord(a, stream);
            ldpc_status s2 = launch_all(p, lt, d_in, dp, d_hard, d_iters, nullptr, stream);
            if (s2 != LDPC_OK) return s2;
            cudaEventRecord(b, stream);
            cudaError_t e2 = cudaEventSynchronize(b);
            if (e2 != cudaSuccess) return cuda_fail(e2, "ldpc_mixed_autotune");
            float x = 0;
            cudaEventElapsedTime(&x, a, b);
            t.push_back(x);
        }
        std::sort(t.begin(), t.end());
        *ms = t[t.size() / 2];
        return LDPC_OK;
    };
    // median of `reps` timed launches of one group alone: a group's chunk
    // moves its own time, which the whole batch's noise can hide when the
    // group's share is small
    auto measure_group = [&](int gi, float *ms) -> ldpc_status {
        std::vector<float> t;
        for (int r = 0; r < reps; ++r) {
            cudaEventRecord(a, stream);
            ldpc_status s2 = launch_group(p, gi, lt, d_in, dp, d_hard, d_iters, nullptr, stream);
            if (s2 != LDPC_OK) return s2;
            cudaEventRecord(b, stream);
            cudaError_t e2 = cudaEventSynchronize(b);
            if (e2 != cudaSuccess) return cuda_fail(e2, "ldpc_mixed_autotune");
            float x = 0;
            cudaEventElapsedTime(&x, a, b);
            t.push_back(x);
        }
        std::sort(t.begin(), t.end());
        *ms = t[t.size() / 2];
        return LDPC_OK;
    };
    const std::vector<int> chunks = dt == 0 ? std::vector<int>{1, 2, 4, 8, 16, 32}
                                            : std::vector<int>{4, 8, 16, 32, 64, 128};
    st = launch_all(p, lt, d_in, dp, d_hard, d_iters, nullptr, stream);   // warm-up
    // each group's chunk, timed on the group alone
    for (size_t gi = 0; st == LDPC_OK && gi < p.groups.size(); ++gi) {
        MixedGroup &g = p.groups[gi];
        float gbest = 0;
        st = measure_group(static_cast<int>(gi), &gbest);
        for (int ch : chunks) {
            if (st != LDPC_OK) break;
            if (ch == g.chunk[dt]) continue;
            const int old = g.chunk[dt];
            g.chunk[dt] = ch;
            float ms = 0;
            st = measure_group(static_cast<int>(gi), &ms);
            if (st != LDPC_OK) break;
            if (ms < gbest) gbest = ms;
            else g.chunk[dt] = old;
        }
    }
    float best = 0;
    if (st == LDPC_OK) st = measure(&best);
    // then, on the whole batch (where the groups run beside one another),
    // coordinate descent from there: each group's chunk, then its residency
    // cap (caps trade one group's speed for room for the others)
    for (size_t gi = 0; st == LDPC_OK && gi < p.groups.size(); ++gi) {
        MixedGroup &g = p.groups[gi];
        for (int ch : chunks) {
            if (ch == g.chunk[dt]) continue;
            const int old = g.chunk[dt];
            g.chunk[dt] = ch;
            float ms = 0;
            st = measure(&ms);
            if (st != LDPC_OK) break;
            if (ms < best) best = ms;
            else g.chunk[dt] = old;
        }
        for (int cap : {16, 8, 4}) {
            if (st != LDPC_OK) break;
            const int old = g.per_sm[dt];
            g.per_sm[dt] = cap;
            float ms = 0;
            st = measure(&ms);
            if (st != LDPC_OK) break;
            if (ms < best) best = ms;
            else g.per_sm[dt] = old;
        }
    }
    // FP32: warps per frame, then frames per block, per group (a setting the
    // device cannot launch is skipped)
    for (size_t gi = 0; st == LDPC_OK && dt == 0 && gi < p.groups.size(); ++gi) {
        MixedGroup &g = p.groups[gi];
        for (int knob = 0; knob < 2 && st == LDPC_OK; ++knob) {
            for (int v : {1, 2, 3, 4}) {
                if ((knob == 0 && (v > 3 || v == g.wpf)) || (knob == 1 && (v == 3 || v == g.fpb)))
                    continue;
                int &ref = knob == 0 ? g.wpf : g.fpb;
                const int old = ref;
                ref = v;
                float ms = 0;
                ldpc_status s2 = measure(&ms);
                if (s2 == LDPC_ERR_UNSUPPORTED) {
                    ref = old;
                    continue;
                }
                if (s2 != LDPC_OK) {
                    ref = old;
                    st = s2;
                    break;
                }
                if (ms < best) best = ms;
                else ref = old;
            }
        }
    }
    // concurrent groups (forked streams) or one after another
    if (st == LDPC_OK && p.groups.size() > 1) {
        p.serial[dt] = !p.serial[dt];
        float ms = 0;
        st = measure(&ms);
        if (st == LDPC_OK && !(ms < best)) p.serial[dt] = !p.serial[dt];
    }
    cudaEventDestroy(a);
    cudaEventDestroy(b);
    return st;
}

ldpc_status ldpc_mixed_autotune(ldpc_mixed_plan *plan, ldpc_dtype dtype, const void *d_in,
                                const ldpc_decode_params *params, uint32_t *d_hard,
                                int32_t *d_iters, int reps, cudaStream_t stream) {
    if (!plan) return fail(LDPC_ERR_INVALID_ARG, "ldpc_mixed_autotune: plan is NULL");
    ldpc_status st = check_params(params, dtype, "ldpc_mixed_autotune");
    if (st != LDPC_OK) return st;
    MixedPlan &p = *plan->p;
    if (p.frames == 0) return LDPC_OK;
    if (!d_in || !d_hard || !d_iters || reps < 1 || reps > 100)
        return fail(LDPC_ERR_INVALID_ARG, "ldpc_mixed_autotune: NULL buffer or reps");
    if ((st = bind_plan(p)) != LDPC_OK) return st;
    return autotune_impl(p, dtype == LDPC_F32 ? 0 : 1, d_in, to_params(params), d_hard, d_iters,
                         reps, stream);
}

ldpc_status ldpc_mixed_autotune_learned(ldpc_mixed_plan *plan, const float *d_llr,
                                        const ldpc_learned_params *lp, uint32_t *d_hard,
                                        int32_t *d_iters, int reps, cudaStream_t stream) {
    const char *who = "ldpc_mixed_autotune_learned";
    if (!plan || !lp) return fail(LDPC_ERR_INVALID_ARG, std::string(who) + ": NULL argument");
    DecodeParams dp;
    ldpc_status st = learned_run_params(lp, &dp, who);
    if (st) return st;
    MixedPlan &p = *plan->p;
    if (p.frames == 0) return LDPC_OK;
    if (!p.d_wptr)
        return fail(LDPC_ERR_INVALID_ARG, std::string(who) + ": no weights (ldpc_mixed_set_weights)");
    if (!d_llr || !d_hard || !d_iters || reps < 1 || reps > 100)
        return fail(LDPC_ERR_INVALID_ARG, std::string(who) + ": NULL buffer or reps");
    if ((st = bind_plan(p)) != LDPC_OK) return st;
    return autotune_impl(p, 2, d_llr, dp, d_hard, d_iters, reps, stream);
}

ldpc_status ldpc_mixed_graph_create(ldpc_mixed_plan *plan, ldpc_dtype dtype, const float *d_llr,
                                    uint32_t *d_q, float quant_scale, int quant_clip,
                                    const ldpc_decode_params *params, uint32_t *d_hard,
                                    int32_t *d_iters, const uint8_t *d_info, int64_t *d_counters,
                                    int64_t *d_code_frame_errors, ldpc_mixed_graph **out) {
    if (!out) return fail(LDPC_ERR_INVALID_ARG, "ldpc_mixed_graph_create: out is NULL");
    *out = nullptr;
    if (!plan) return fail(LDPC_ERR_INVALID_ARG, "ldpc_mixed_graph_create: plan is NULL");
    ldpc_status st = check_params(params, dtype, "ldpc_mixed_graph_create");
    if (st != LDPC_OK) return st;
    MixedPlan &p = *plan->p;
    if (!d_llr || !d_hard || !d_iters || (dtype == LDPC_I8X4 && !d_q) || (d_counters && !d_info))
        return fail(LDPC_ERR_INVALID_ARG, "ldpc_mixed_graph_create: NULL buffer");
    if (dtype == LDPC_I8X4 && (quant_clip < 0 || quant_clip > 127))
        return fail(LDPC_ERR_INVALID_ARG, "ldpc_mixed_graph_create: clip in [0, 127]");
    if ((st = bind_plan(p)) != LDPC_OK) return st;
    const int dt = dtype == LDPC_F32 ? 0 : 1;
    // item lists for the current choices are built before capture
    for (auto &g : p.groups)
        if (g.built_chunk[dt] != g.chunk[dt] && (st = build_items(p, g, dt, g.chunk[dt])) != LDPC_OK)
            return st;
    ldpc_mixed_graph *gr = new (std::nothrow) ldpc_mixed_graph;
    if (!gr) return fail(LDPC_ERR_NOMEM, "ldpc_mixed_graph_create: host allocation");
    gr->device = p.device;
    cudaError_t e = cudaStreamCreateWithFlags(&gr->cap, cudaStreamNonBlocking);
    if (e == cudaSuccess) e = cudaStreamBeginCapture(gr->cap, cudaStreamCaptureModeThreadLocal);
    if (e != cudaSuccess) {
        if (gr->cap) cudaStreamDestroy(gr->cap);
        delete gr;
        return cuda_fail(e, "ldpc_mixed_graph_create: capture");
    }
    const DecodeParams dp = to_params(params);
    if (dt == 1) st = quantize_mixed(p, d_llr, d_q, quant_scale, quant_clip, gr->cap);
    if (st == LDPC_OK)
        st = launch_all(p, dt, dt == 0 ? static_cast<const void *>(d_llr) : d_q, dp, d_hard,
                        d_iters, nullptr, gr->cap);
    if (st == LDPC_OK && d_counters)
        st = stats_mixed(p, d_info, d_hard, d_iters, params->max_iters, d_counters,
                         d_code_frame_errors, gr->cap);
    e = cudaStreamEndCapture(gr->cap, &gr->graph);
    if (st == LDPC_OK && e != cudaSuccess) st = cuda_fail(e, "ldpc_mixed_graph_create: end capture");
    if (st == LDPC_OK) {
        e = cudaGraphInstantiate(&gr->exec, gr->graph, 0);
        if (e != cudaSuccess) st = cuda_fail(e, "ldpc_mixed_graph_create: instantiate");
    }
    if (st != LDPC_OK) {
        if (gr->exec) cudaGraphExecDestroy(gr->exec);
        if (gr->graph) cudaGraphDestroy(gr->graph);
        cudaStreamDestroy(gr->cap);
        delete gr;
        return st;
    }
    *out = gr;
    return LDPC_OK;
}

ldpc_status ldpc_mixed_scatter(const ldpc_mixed_plan *plan, int code, int what,
                               const void *d_src, void *d_dst, cudaStream_t stream) {
    if (!plan) return fail(LDPC_ERR_INVALID_ARG, "ldpc_mixed_scatter: plan is NULL");
    const MixedPlan &p = *plan->p;
    if (code < 0 || code >= static_cast<int>(p.set->codes.size()) || what < 0 || what > 2)
        return fail(LDPC_ERR_INVALID_ARG, "ldpc_mixed_scatter: bad code or kind");
    const long long count = p.fcount[code];
    if (count == 0) return LDPC_OK;
    if (!d_src || !d_dst) return fail(LDPC_ERR_INVALID_ARG, "ldpc_mixed_scatter: NULL buffer");
    ldpc_status st = bind_plan(p);
    if (st != LDPC_OK) return st;
    const Code &c = *p.set->codes[code];
    const long long *off = what == 1 ? p.d_info_off : p.d_llr_off;
    const int elem = what == 0 ? 4 : 1;
    const int row = what == 0 ? 4 * c.n : (what == 1 ? c.k : c.n);
    const unsigned grid = static_cast<unsigned>(std::min<long long>(count, 65535));
    mixed_scatter_kernel<<<grid, 256, 0, stream>>>(p.d_uframe, p.ibase[code], count, off, row,
                                                   static_cast<const uint8_t *>(d_src),
                                                   static_cast<uint8_t *>(d_dst), elem);
    cudaError_t e = cudaGetLastError();
    return e == cudaSuccess ? LDPC_OK : cuda_fail(e, "mixed_scatter_kernel");
}

ldpc_status ldpc_mixed_graph_launch(ldpc_mixed_graph *graph, cudaStream_t stream) {
    if (!graph) return fail(LDPC_ERR_INVALID_ARG, "ldpc_mixed_graph_launch: graph is NULL");
    cudaError_t e = cudaSetDevice(graph->device);
    if (e == cudaSuccess) e = cudaGraphLaunch(graph->exec, stream);
    return e == cudaSuccess ? LDPC_OK : cuda_fail(e, "ldpc_mixed_graph_launch");
}

void ldpc_mixed_graph_destroy(ldpc_mixed_graph *graph) {
    if (!graph) return;
    int prev = 0;
    cudaGetDevice(&prev);
    cudaSetDevice(graph->device);
    if (graph->exec) cudaGraphExecDestroy(graph->exec);
    if (graph->graph) cudaGraphDestroy(graph->graph);
    if (graph->cap) cudaStreamDestroy(graph->cap);
    cudaSetDevice(prev);
    delete graph;
}

}  // extern "C"

extern "C" {

ldpc_status ldpc_mixed_set_weights(ldpc_mixed_plan *plan, const float *const *h_weights,
                                   const int32_t *h_T) {
    if (!plan || !h_weights || !h_T)
        return fail(LDPC_ERR_INVALID_ARG, "ldpc_mixed_set_weights: NULL argument");
    MixedPlan &p = *plan->p;
    const int count = static_cast<int>(p.set->codes.size());
    for (int ci = 0; ci < count; ++ci) {
        if (!p.fcount[ci]) continue;
        if (!h_weights[ci] || h_T[ci] < 1 || h_T[ci] > kMaxIters)
            return fail(LDPC_ERR_INVALID_ARG,
                        "ldpc_mixed_set_weights: code " + std::to_string(ci) +
                            " has frames but no weights or T outside 1..1000");
    }
    ldpc_status st = bind_plan(p);
    if (st != LDPC_OK) return st;
    std::vector<const float *> w(h_weights, h_weights + count);
    std::vector<int> T(h_T, h_T + count);
    cudaFree(p.d_wptr);
    cudaFree(p.d_wT);
    p.d_wptr = nullptr;
    p.d_wT = nullptr;
    cudaError_t e = upload(&p.d_wptr, w);
    if (e == cudaSuccess) e = upload(&p.d_wT, T);
    if (e != cudaSuccess) return cuda_fail(e, "ldpc_mixed_set_weights");
    p.wT = T;
    return LDPC_OK;
}

ldpc_status ldpc_decode_mixed_learned(ldpc_mixed_plan *plan, const float *d_llr, int early_stop,
                                      uint32_t *d_hard, int32_t *d_iters, float *d_post,
                                      cudaStream_t stream) {
    if (!plan) return fail(LDPC_ERR_INVALID_ARG, "ldpc_decode_mixed_learned: plan is NULL");
    if (early_stop != 0 && early_stop != 1)
        return fail(LDPC_ERR_INVALID_ARG, "ldpc_decode_mixed_learned: early_stop must be 0 or 1");
    MixedPlan &p = *plan->p;
    if (p.frames == 0) return LDPC_OK;
    if (!p.d_wptr)
        return fail(LDPC_ERR_INVALID_ARG,
                    "ldpc_decode_mixed_learned: no weights (ldpc_mixed_set_weights)");
    if (!d_llr || !d_hard || !d_iters)
        return fail(LDPC_ERR_INVALID_ARG, "ldpc_decode_mixed_learned: NULL buffer");
    ldpc_status st = bind_plan(p);
    if (st != LDPC_OK) return st;
    DecodeParams dp;
    dp.max_iters = 0;   // per code: T_c of its weight table
    dp.alpha = 1.0f;
    dp.normalise = 0;
    dp.early_stop = early_stop;
    return launch_all(p, 2, d_llr, dp, d_hard, d_iters, d_post, stream);
}

ldpc_status ldpc_decode_mixed_learned_ex(ldpc_mixed_plan *plan, const float *d_llr,
                                         const ldpc_learned_params *lp, uint32_t *d_hard,
                                         int32_t *d_iters, float *d_post, cudaStream_t stream) {
    const char *who = "ldpc_decode_mixed_learned_ex";
    if (!plan || !lp) return fail(LDPC_ERR_INVALID_ARG, std::string(who) + ": NULL argument");
    DecodeParams dp;
    ldpc_status st = learned_run_params(lp, &dp, who);
    if (st) return st;
    MixedPlan &p = *plan->p;
    if (p.frames == 0) return LDPC_OK;
    if (!p.d_wptr)
        return fail(LDPC_ERR_INVALID_ARG, std::string(who) + ": no weights (ldpc_mixed_set_weights)");
    if (!d_llr || !d_hard || !d_iters)
        return fail(LDPC_ERR_INVALID_ARG, std::string(who) + ": NULL buffer");
    st = bind_plan(p);
    if (st != LDPC_OK) return st;
    return launch_all(p, 2, d_llr, dp, d_hard, d_iters, d_post, stream);
}

ldpc_status ldpc_mixed_frame_flags(const ldpc_mixed_plan *plan, const uint32_t *d_hard,
                                   uint8_t *d_bad, cudaStream_t stream) {
    if (!plan) return fail(LDPC_ERR_INVALID_ARG, "ldpc_mixed_frame_flags: plan is NULL");
    const MixedPlan &p = *plan->p;
    if (p.frames == 0) return LDPC_OK;
    if (!d_hard || !d_bad) return fail(LDPC_ERR_INVALID_ARG, "ldpc_mixed_frame_flags: NULL buffer");
    ldpc_status st = bind_plan(p);
    if (st != LDPC_OK) return st;
    int sms = 148;
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, p.device);
    const long long grid = std::min<long long>((p.frames + 7) / 8, 32LL * sms);
    mixed_flags_kernel<<<static_cast<unsigned>(grid), 256, 0, stream>>>(
        p.set->d_desc, p.d_code_of_frame, p.frames, p.d_hard_off, d_hard, d_bad);
    cudaError_t e = cudaGetLastError();
    return e == cudaSuccess ? LDPC_OK : cuda_fail(e, "mixed_flags_kernel");
}

ldpc_status ldpc_mixed_move_frames(const ldpc_mixed_plan *plan_a, const ldpc_mixed_plan *plan_b,
                                   const int64_t *d_index, int what, void *d_a, void *d_b,
                                   cudaStream_t stream) {
    if (!plan_a || !plan_b || what < 0 || what > 2)
        return fail(LDPC_ERR_INVALID_ARG, "ldpc_mixed_move_frames: bad plans or kind");
    const MixedPlan &a = *plan_a->p, &b = *plan_b->p;
    if (a.set != b.set)
        return fail(LDPC_ERR_INVALID_ARG, "ldpc_mixed_move_frames: plans of different code sets");
    if (b.frames == 0) return LDPC_OK;
    if (!d_index || !d_a || !d_b)
        return fail(LDPC_ERR_INVALID_ARG, "ldpc_mixed_move_frames: NULL buffer");
    ldpc_status st = bind_plan(a);
    if (st != LDPC_OK) return st;
    const long long *off_a = what == 0 ? a.d_llr_off : a.d_hard_off;
    const long long *off_b = what == 0 ? b.d_llr_off : b.d_hard_off;
    const unsigned grid = static_cast<unsigned>(std::min<long long>(b.frames, 65535));
    mixed_move_kernel<<<grid, 128, 0, stream>>>(
        a.set->d_desc, b.d_code_of_frame, b.frames, reinterpret_cast<const long long *>(d_index),
        off_a, off_b, what, static_cast<uint32_t *>(d_a), static_cast<uint32_t *>(d_b),
        what == 2 ? a.d_wT : nullptr);
    cudaError_t e = cudaGetLastError();
    return e == cudaSuccess ? LDPC_OK : cuda_fail(e, "mixed_move_kernel");
}

ldpc_status ldpc_mixed_paired_errors(const ldpc_mixed_plan *plan, const uint8_t *d_info,
                                     const uint32_t *d_hard_a, const uint32_t *d_hard_b,
                                     int64_t *d_counts, cudaStream_t stream) {
    if (!plan || !d_counts)
        return fail(LDPC_ERR_INVALID_ARG, "ldpc_mixed_paired_errors: NULL plan or counts");
    const MixedPlan &p = *plan->p;
    ldpc_status st = bind_plan(p);
    if (st != LDPC_OK) return st;
    cudaError_t e = cudaMemsetAsync(d_counts, 0, sizeof(int64_t) * 4, stream);
    if (e != cudaSuccess) return cuda_fail(e, "cudaMemsetAsync counts");
    if (p.frames == 0) return LDPC_OK;
    if (!d_info || !d_hard_a || !d_hard_b)
        return fail(LDPC_ERR_INVALID_ARG, "ldpc_mixed_paired_errors: NULL buffer");
    int sms = 148;
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, p.device);
    const long long grid = std::min<long long>((p.frames + 7) / 8, 32LL * sms);
    mixed_paired_kernel<<<static_cast<unsigned>(grid), 256, 0, stream>>>(
        p.set->d_desc, p.d_code_of_frame, p.frames, p.d_info_off, p.d_hard_off, d_info, d_hard_a,
        d_hard_b, reinterpret_cast<unsigned long long *>(d_counts));
    e = cudaGetLastError();
    return e == cudaSuccess ? LDPC_OK : cuda_fail(e, "mixed_paired_kernel");
}

}  // extern "C"
