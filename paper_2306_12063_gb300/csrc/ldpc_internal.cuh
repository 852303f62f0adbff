// Internal definitions shared by the libldpc translation units.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include <atomic>
#include <string>
#include <vector>

#include "../../include/ldpc.h"

namespace ldpc {

constexpr int kMaxNb = 32;          // block columns (row degree <= nb)
constexpr int kMaxRowDeg = 27;      // sign bits + 5-bit argmin share one word
// Decoder kernels are built for these numbers of edge slots per row; a code
// uses the smallest class that holds its largest row degree.
#define LDPC_SLOT_CLASSES(X) X(8) X(12) X(16) X(20) X(24) X(27)
// (class, slots) pairs of the single-code plain decoders fitted to a code's
// largest row degree d: d itself when it lies in class - 3 .. class, else the
// class (codes of degree <= 4 in class 8, which its 4-slot instance serves).
#define LDPC_FITTED_SLOTS(X)                                                         \
    X(8, 5) X(8, 6) X(8, 7) X(8, 8) X(12, 9) X(12, 10) X(12, 11) X(12, 12) X(16, 13) \
    X(16, 14) X(16, 15) X(16, 16) X(20, 17) X(20, 18) X(20, 19) X(20, 20) X(24, 21)  \
    X(24, 22) X(24, 23) X(24, 24) X(27, 25) X(27, 26) X(27, 27)
inline int slot_class(int max_deg) {
    for (int d : {8, 12, 16, 20, 24, 27})
        if (max_deg <= d) return d;
    return 0;
}
constexpr int kMaxZ = 384;        // 4 N < 65536: byte offsets fit uint16
// Posterior words in shared memory: Z_n for n < N, then one dummy posterior
// word per lane (the unused leading edge slots of lane l read word N + l),
// rounded up to a 16-byte boundary.  4 (N + 31) < 65536 still.
constexpr int kDummyWords = 32;
__host__ __device__ constexpr int posterior_words(int n) { return (n + kDummyWords + 3) & ~3; }
constexpr int kMaxIters = 1000;

// Device status word bits (set by kernels, read and cleared by ldpc_sync).
constexpr int kStatusCopyTimeout = 1;
constexpr int kStatusBadOffset = 2;    // debug builds: an edge offset outside Z_n

// Host-side record of a code; the device tables are built once at creation.
struct Code {
    int device = 0;
    int mb = 0, nb = 0, kb = 0, z = 0, n = 0, k = 0, m = 0, y = 0;
    int max_deg = 0, min_deg = 0, n_edges = 0;
    int rpl = 0;                     // row slots per lane: ceil(z / 32)
    int dslots = 0;                  // edge slots per row in the offset table
    std::vector<int16_t> hbm;        // [mb][nb]
    std::vector<int> layer_off;      // [mb + 1] into the edge list
    std::vector<int> edge_col;       // block column j of each edge (sorted per layer)
    std::vector<int> edge_shift;     // its cyclic shift s
    // device copies
    int16_t *d_hbm = nullptr;        // [mb][nb] (encoder)
    uint16_t *d_voff = nullptr;      // per-lane variable offsets (see ldpc_code_create)
    uint32_t *d_rowinfo = nullptr;   // [mb] layer degree and first edge
    uint32_t *d_edges = nullptr;     // [n_edges] (block column << 16) | shift
    int16_t *d_wgather = nullptr;    // [mb][(dslots + 3) & ~3] block edge of each slot, -1 unused
    uint32_t *d_colent = nullptr;    // [n_edges] per block column, block rows increasing:
                                     //   (block row << 20) | (block edge << 9) | shift
    int *d_coloff = nullptr;         // [nb + 1] start of each block column in d_colent
    int *d_status = nullptr;         // device status word; 8 bytes on, the int8 decoder's
                                     // saturation count (debug builds)
    cudaStream_t aux[2] = {nullptr, nullptr};   // host-decode pipeline
    cudaEvent_t ev[3] = {nullptr, nullptr, nullptr};
    size_t voff_words = 0;           // uint16 entries in d_voff
    // Work counters of the decode kernels' dynamic frame scheduling: one
    // 64-bit slot per launch, taken round-robin and zeroed on the launch's
    // stream, so up to kWorkSlots launches may be in flight at once.
    unsigned long long *d_work = nullptr;
    mutable std::atomic<unsigned> work_seq{0};
};
constexpr int kWorkSlots = 64;

// Kernel-side view of a code, passed by value.
struct DevCode {
    int n, k, m, z, mb, nb, kb, y;
    int nwords;        // ceil(n / 32)
    int rpl;           // row slots per lane
    int dslots;        // edge slots per row in the offset table
    int n_edges;       // block edges (nonzeros of H_bm)
    const int16_t *hbm;
    const uint16_t *voff;     // [mb][rpl][dslots][32] byte offset of each edge's variable
    const uint32_t *rowinfo;  // [mb] (first_edge << 8) | degree
    const uint32_t *edges;    // [n_edges] (block column << 16) | shift
    const int16_t *wgather;   // [mb][(dslots + 3) & ~3] block edge of each slot, -1 unused
    const uint32_t *colent;   // [n_edges] column entries (block row, block edge, shift)
    const int *coloff;        // [nb + 1]
    int *status;
    unsigned long long *sat;  // debug builds: int8 clamps taken (NULL: not counted)
};

inline DevCode dev_view(const Code &c) {
    DevCode d;
    d.n = c.n; d.k = c.k; d.m = c.m; d.z = c.z; d.mb = c.mb; d.nb = c.nb;
    d.kb = c.kb; d.y = c.y; d.nwords = (c.n + 31) / 32; d.rpl = c.rpl; d.dslots = c.dslots;
    d.n_edges = c.n_edges; d.hbm = c.d_hbm; d.voff = c.d_voff;
    d.rowinfo = c.d_rowinfo; d.edges = c.d_edges; d.wgather = c.d_wgather;
    d.colent = c.d_colent; d.coloff = c.d_coloff; d.status = c.d_status;
    d.sat = c.d_status ? reinterpret_cast<unsigned long long *>(c.d_status + 2) : nullptr;
    return d;
}

// Lets `kern` take up to the current device's opt-in maximum of dynamic
// shared memory; every launcher calls it before launching with its own size.
// The attribute belongs to the kernel, not to a launch, so setting it to one
// launch's size would race with another host thread launching the same
// kernel for a larger code.
inline cudaError_t allow_dynamic_smem(const void *kern) {
    int dev = 0, mx = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e == cudaSuccess)
        e = cudaDeviceGetAttribute(&mx, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev);
    if (e == cudaSuccess) e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, mx);
    return e;
}

// Thread-local last-error message, set by fail().
void set_error(const std::string &msg);
ldpc_status fail(ldpc_status st, const std::string &msg);
ldpc_status cuda_fail(cudaError_t e, const char *what);

struct DecodeParams {
    int max_iters;
    float alpha;
    int normalise;
    int early_stop;
    // learned normalised min-sum (FP32 only): weights[T][n_edges], NULL for
    // the plain / alpha-scaled decoder; T = weight_iters (0: max_iters), and
    // iterations past T use row T - 1
    const float *weights = nullptr;
    int n_edges = 0;
    int weight_iters = 0;
    // give-up checkpoints (0: none; need early_stop): at iteration
    // stop_iter[j] a frame with more than floor(stop_frac[j] * M) unsatisfied
    // checks stops
    int stop_iter[2] = {0, 0};
    float stop_frac[2] = {0.0f, 0.0f};
};

// Launchers (defined in the .cu files).
ldpc_status launch_gen_info(uint64_t seed, int64_t frame0, int64_t frames, int k,
                            uint8_t *d_info, cudaStream_t s);
ldpc_status launch_encode(const Code &c, const uint8_t *d_info, uint8_t *d_code,
                          int64_t frames, cudaStream_t s);
ldpc_status launch_awgn(const uint8_t *d_code, int64_t frame0, int64_t frames, int n,
                        uint64_t seed, float sigma, float scale, float *d_llr,
                        cudaStream_t s);
ldpc_status launch_awgn_frames(const uint8_t *d_code, int64_t frame0, int64_t frames, int n,
                               uint64_t seed, const float *d_sigma, float *d_llr,
                               cudaStream_t s);
ldpc_status launch_snr_sigma(uint64_t seed, int64_t frame0, int64_t frames, double lo,
                             double hi, double rate, float *d_sigma, cudaStream_t s);
ldpc_status launch_quantize(const float *d_llr, uint32_t *d_q, int64_t frames, int n,
                            float scale, int clip, cudaStream_t s);
ldpc_status launch_stats(const Code &c, const uint8_t *d_info, const uint32_t *d_hard,
                         const int32_t *d_iters, int64_t frames, int max_iters,
                         int64_t *d_counters, cudaStream_t s);
ldpc_status launch_paired(const Code &c, const uint8_t *d_info, const uint32_t *d_hard_a,
                          const uint32_t *d_hard_b, int64_t frames, int64_t *d_counts,
                          cudaStream_t s);
ldpc_status launch_wait_check(const Code &c, uint32_t polls, cudaStream_t s);
// A persistent grid size lowered to the cap set by ldpc_test_set_grid_cap.
int64_t grid_cap(int64_t cap);
// Zeroes the next work-counter slot on stream s and returns it (NULL and an
// error message on failure).
unsigned long long *work_slot(const Code &c, cudaStream_t s);
ldpc_status launch_decode(const Code &c, ldpc_dtype dtype, const void *d_llr,
                          int64_t frames, const DecodeParams &p, uint32_t *d_hard,
                          int32_t *d_iters, void *d_post, cudaStream_t s);

// Section 5 int16 decoder with wrap-around arithmetic (ldpc_variants.cu).
ldpc_status launch_decode_i16w(const Code &c, const int16_t *d_llr, int64_t frames,
                               const DecodeParams &p, uint32_t *d_hard, int32_t *d_iters,
                               int16_t *d_post, cudaStream_t s);

// Learned normalised min-sum (FP32): per-iteration, per-block-edge weights.
ldpc_status launch_decode_learned(const Code &c, const float *d_llr, int64_t frames,
                                  const DecodeParams &p, uint32_t *d_hard, int32_t *d_iters,
                                  float *d_post, cudaStream_t s);

// Learned decoding followed by the int8 plain min-sum fallback for the
// frames that still violate a parity check (ldpc_learned.cu).
size_t learned_fallback_workspace(const Code &c, int64_t frames);
ldpc_status learned_fallback(const Code &c, const float *d_llr, int64_t frames,
                             const DecodeParams &learned, const DecodeParams &fb, float scale,
                             int clip, uint32_t *d_hard, int32_t *d_iters, int64_t *h_count,
                             void *d_ws, cudaStream_t s);

// Validates the learned decoder's run limits and copies them into dp
// (max_iters 0 means "the weight table's T").
ldpc_status learned_run_params(const ldpc_learned_params *lp, DecodeParams *dp, const char *who);

// Decode launch on a caller-assembled code view (tables, status word and work
// counter supplied by the caller); no allocation.
ldpc_status launch_decode_view(const DevCode &dc, ldpc_dtype dtype, const void *d_llr,
                               int64_t frames, const DecodeParams &p, uint32_t *d_hard,
                               int32_t *d_iters, void *d_post, unsigned long long *work,
                               cudaStream_t s);

}  // namespace ldpc

// The opaque handle of the C-ABI.
struct ldpc_code {
    ldpc::Code c;
};

// ---------------------------------------------------------------------------
// Device helpers
// ---------------------------------------------------------------------------
#ifdef __CUDACC__
namespace ldpc {

__device__ __forceinline__ uint32_t smem_addr(const void *p) {
    return static_cast<uint32_t>(__cvta_generic_to_shared(p));
}

__device__ __forceinline__ void mbar_init(uint64_t *bar, uint32_t count) {
    asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_addr(bar)), "r"(count)
                 : "memory");
}

// Make the barrier initialisation visible to the asynchronous (bulk copy) proxy.
__device__ __forceinline__ void fence_mbar_init() {
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
}

// Order this thread's earlier generic-proxy shared-memory accesses before
// later async-proxy (bulk copy) writes to the same addresses.
__device__ __forceinline__ void fence_proxy_async_smem() {
    asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
}

__device__ __forceinline__ void mbar_arrive_expect_tx(uint64_t *bar, uint32_t bytes) {
    asm volatile(
        "{ .reg .b64 st; mbarrier.arrive.expect_tx.shared::cta.b64 st, [%0], %1; }" ::"r"(
            smem_addr(bar)),
        "r"(bytes)
        : "memory");
}

// 1-D bulk copy global -> shared (TMA engine), completion counted on `bar`.
// dst, src 16-byte aligned; bytes a multiple of 16.
__device__ __forceinline__ void bulk_copy_g2s(void *dst, const void *src, uint32_t bytes,
                                              uint64_t *bar) {
    asm volatile(
        "cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, "
        "[%3];" ::"r"(smem_addr(dst)),
        "l"(src), "r"(bytes), "r"(smem_addr(bar))
        : "memory");
}

__device__ __forceinline__ bool mbar_try_wait(uint64_t *bar, uint32_t parity) {
    uint32_t ok;
    asm volatile(
        "{ .reg .pred p; mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2; selp.u32 %0, 1, "
        "0, p; }"
        : "=r"(ok)
        : "r"(smem_addr(bar)), "r"(parity)
        : "memory");
    return ok != 0;
}

// Bounded wait: gives up after `limit` polls and reports false.
__device__ __forceinline__ bool mbar_wait_bounded(uint64_t *bar, uint32_t parity,
                                                  uint32_t limit) {
    for (uint32_t i = 0; i < limit; ++i)
        if (mbar_try_wait(bar, parity)) return true;
    return false;
}

// Asynchronous 4-byte copy global -> shared (no register staging); copies
// issued since the last commit form one group, and wait_group<n> returns
// once at most n of this thread's groups are still in flight.
__device__ __forceinline__ void cp_async4(void *dst, const void *src) {
    asm volatile("cp.async.ca.shared.global [%0], [%1], 4;" ::"r"(smem_addr(dst)), "l"(src)
                 : "memory");
}
__device__ __forceinline__ void cp_async_commit() {
    asm volatile("cp.async.commit_group;" ::: "memory");
}
template <int N>
__device__ __forceinline__ void cp_async_wait() {
    asm volatile("cp.async.wait_group %0;" ::"n"(N) : "memory");
}

// Byte-wise mask from the top bit of each byte: 0xFF where bit 7 is set.
__device__ __forceinline__ uint32_t msb_bytes_to_mask(uint32_t x) {
    uint32_t r;   // prmt selector nibble with bit 3 set replicates the byte's sign
    asm("prmt.b32 %0, %1, 0, 0xBA98;" : "=r"(r) : "r"(x));
    return r;
}

// Bitwise select: bits of b where m is 1, bits of a where m is 0.
__device__ __forceinline__ uint32_t bsel(uint32_t a, uint32_t b, uint32_t m) {
    return (a & ~m) | (b & m);
}

}  // namespace ldpc
#endif
