// C-ABI of libldpc: code handles, argument checks and launches.
// The operations are those of arXiv 2306.12063 (Palenik & Szitkey): the
// base-matrix code model of Section 1, the direct encoder of Section 2 and
// the layered min-sum decoder of Section 4; see include/ldpc.h.
#include <algorithm>
#include <chrono>
#include <cstring>
#include <new>
#include <string>
#include <thread>

#include "ldpc_internal.cuh"

namespace ldpc {

static thread_local std::string g_last_error;

void set_error(const std::string &msg) { g_last_error = msg; }

ldpc_status fail(ldpc_status st, const std::string &msg) {
    g_last_error = msg;
    return st;
}

ldpc_status cuda_fail(cudaError_t e, const char *what) {
    g_last_error = std::string(what) + ": " + cudaGetErrorString(e);
    return LDPC_ERR_CUDA;
}

#define LDPC_CUDA_TRY(expr, what)                   \
    do {                                            \
        cudaError_t _e = (expr);                    \
        if (_e != cudaSuccess) return cuda_fail(_e, what); \
    } while (0)

// Structure required by the direct encoder (eq. 3-7): h_b = column Kb has
// equal non-negative entries in rows 0 and Mb-1 and exactly one more
// non-negative entry at a row y in 1..Mb-2; H_b2' is the dual diagonal.
static bool encodable_structure(const int16_t *h, int mb, int nb, int *y_out,
                                std::string *why) {
    const int kb = nb - mb;
    if (h[kb] < 0 || h[kb] != h[(mb - 1) * nb + kb]) {
        *why = "h_b entries of rows 0 and mb-1 must be equal and non-negative";
        return false;
    }
    int y = -1;
    for (int i = 1; i < mb - 1; ++i) {
        if (h[i * nb + kb] >= 0) {
            if (y >= 0) {
                *why = "h_b has more than one entry between its first and last rows";
                return false;
            }
            y = i;
        }
    }
    if (y < 0) {
        *why = "h_b has no entry between its first and last rows";
        return false;
    }
    for (int i = 0; i < mb; ++i)
        for (int t = 0; t < mb - 1; ++t) {
            const int v = h[i * nb + kb + 1 + t];
            const bool diag = (i == t || i == t + 1);
            if ((diag && v != 0) || (!diag && v != -1)) {
                *why = "columns Kb+1.. must be the dual diagonal of zeros (H_b2')";
                return false;
            }
        }
    *y_out = y;
    return true;
}

static void release(Code &c) {
    int prev = 0;
    cudaGetDevice(&prev);
    cudaSetDevice(c.device);
    cudaFree(c.d_hbm);
    cudaFree(c.d_voff);
    cudaFree(c.d_rowinfo);
    cudaFree(c.d_edges);
    cudaFree(c.d_wgather);
    cudaFree(c.d_colent);
    cudaFree(c.d_coloff);
    cudaFree(c.d_status);
    cudaFree(c.d_work);
    for (auto &s : c.aux)
        if (s) cudaStreamDestroy(s);
    for (auto &e : c.ev)
        if (e) cudaEventDestroy(e);
    cudaSetDevice(prev);
}

unsigned long long *work_slot(const Code &c, cudaStream_t s) {
    const unsigned k = c.work_seq.fetch_add(1u) % kWorkSlots;
    unsigned long long *p = c.d_work + k;
    cudaError_t e = cudaMemsetAsync(p, 0, sizeof(unsigned long long), s);
    if (e != cudaSuccess) {
        cuda_fail(e, "cudaMemsetAsync work counter");
        return nullptr;
    }
    return p;
}

static ldpc_status bind(const Code *c) {
    LDPC_CUDA_TRY(cudaSetDevice(c->device), "cudaSetDevice");
    return LDPC_OK;
}

}  // namespace ldpc

using namespace ldpc;


extern "C" {

const char *ldpc_last_error(void) { return g_last_error.c_str(); }

ldpc_status ldpc_set_device(int device) {
    int count = 0;
    cudaError_t e = cudaGetDeviceCount(&count);
    if (e != cudaSuccess) return cuda_fail(e, "cudaGetDeviceCount");
    if (device < 0 || device >= count)
        return fail(LDPC_ERR_INVALID_ARG, "ldpc_set_device: no such device");
    e = cudaSetDevice(device);
    if (e != cudaSuccess) return cuda_fail(e, "cudaSetDevice");
    return LDPC_OK;
}

ldpc_status ldpc_code_create(const int16_t *hbm, int mb, int nb, int z, ldpc_code **out) {
    if (!out) return fail(LDPC_ERR_INVALID_ARG, "ldpc_code_create: out is NULL");
    *out = nullptr;
    if (!hbm) return fail(LDPC_ERR_INVALID_ARG, "ldpc_code_create: hbm is NULL");
    if (mb < 3 || nb <= mb || nb > kMaxNb)
        return fail(LDPC_ERR_INVALID_ARG, "ldpc_code_create: need 3 <= mb < nb <= 32");
    if (z < 1 || z > kMaxZ)
        return fail(LDPC_ERR_INVALID_ARG, "ldpc_code_create: need 1 <= z <= 384");
    for (int i = 0; i < mb * nb; ++i)
        if (hbm[i] < -1 || hbm[i] >= z)
            return fail(LDPC_ERR_BAD_STRUCTURE,
                        "ldpc_code_create: entry outside [-1, z) at index " + std::to_string(i));
    int y = -1;
    std::string why;
    if (!encodable_structure(hbm, mb, nb, &y, &why))
        return fail(LDPC_ERR_BAD_STRUCTURE, "ldpc_code_create: " + why);

    ldpc_code *h = new (std::nothrow) ldpc_code;
    if (!h) return fail(LDPC_ERR_NOMEM, "ldpc_code_create: host allocation");
    Code &c = h->c;
    cudaGetDevice(&c.device);
    c.mb = mb; c.nb = nb; c.kb = nb - mb; c.z = z;
    c.n = nb * z; c.k = (nb - mb) * z; c.m = mb * z; c.y = y;
    c.rpl = (z + 31) / 32;
    c.hbm.assign(hbm, hbm + mb * nb);
    // Per-layer edge list (block column j, shift s), increasing j (Section 1:
    // the row neighbourhood N(m) of every row in block row i).
    c.layer_off.assign(mb + 1, 0);
    c.max_deg = 0;
    c.min_deg = nb;
    for (int i = 0; i < mb; ++i) {
        c.layer_off[i] = static_cast<int>(c.edge_col.size());
        for (int j = 0; j < nb; ++j) {
            const int s = hbm[i * nb + j];
            if (s < 0) continue;
            c.edge_col.push_back(j);
            c.edge_shift.push_back(s);
        }
        const int d = static_cast<int>(c.edge_col.size()) - c.layer_off[i];
        c.max_deg = std::max(c.max_deg, d);
        c.min_deg = std::min(c.min_deg, d);
    }
    c.layer_off[mb] = static_cast<int>(c.edge_col.size());
    c.n_edges = c.layer_off[mb];

    c.dslots = slot_class(c.max_deg);
    const int D = c.dslots ? c.dslots : kMaxRowDeg;
    // Per-lane variable offsets: lane l of row slot t handles row r = l + 32 t
    // of a layer; its variable on edge (j, s) is n = j Z + (r + s) mod Z.
    // Layout [layer][t][edge slot][lane] with D edge slots per row (the
    // kernel's slot class); a layer of degree d fills slots D-d .. D-1 in edge
    // order, so a slot sits at a fixed stride of 32 entries from the row's
    // first one.  Entries are byte offsets into a 4-byte posterior array.  The
    // unused leading slots of lane l point at word N + l, that lane's own
    // dummy posterior holding a value that cannot affect a row (the decoders
    // run every slot unconditionally); lanes r >= Z never read the table.
    std::vector<uint16_t> voff(static_cast<size_t>(mb) * c.rpl * D * 32);
    for (size_t q = 0; q < voff.size(); ++q)
        voff[q] = static_cast<uint16_t>(4 * (c.n + static_cast<int>(q % 32)));
    for (int i = 0; i < mb; ++i) {
        const int d = c.layer_off[i + 1] - c.layer_off[i];
        if (d > D) continue;   // rows above 27 edges are rejected by the decoders
        for (int e = 0; e < d; ++e) {
            const int q = c.layer_off[i] + e;
            const int slot = D - d + e;
            for (int t = 0; t < c.rpl; ++t)
                for (int l = 0; l < 32; ++l) {
                    const int r = l + 32 * t;
                    if (r >= z) continue;
                    const int v = c.edge_col[q] * z + (r + c.edge_shift[q]) % z;
                    voff[((static_cast<size_t>(i) * c.rpl + t) * D + slot) * 32 + l] =
                        static_cast<uint16_t>(4 * v);
                }
        }
    }
    std::vector<uint32_t> rowinfo(mb);
    for (int i = 0; i < mb; ++i)
        rowinfo[i] = (static_cast<uint32_t>(c.layer_off[i]) << 8) |
                     static_cast<uint32_t>(c.layer_off[i + 1] - c.layer_off[i]);
    c.voff_words = voff.size();
    // Learned-weight gather table: slot i of layer l (slot order of the
    // offset table, padded to a multiple of 4) holds block edge
    // layer_off[l] + i - (D - d), or -1 for a leading unused slot or padding.
    const int wp = (D + 3) & ~3;
    std::vector<int16_t> wgather(static_cast<size_t>(mb) * wp, static_cast<int16_t>(-1));
    for (int i = 0; i < mb; ++i) {
        const int d = c.layer_off[i + 1] - c.layer_off[i];
        if (d > D) continue;
        for (int e = 0; e < d; ++e)
            wgather[static_cast<size_t>(i) * wp + (D - d + e)] =
                static_cast<int16_t>(c.layer_off[i] + e);
    }
    // Column table: for each block column j, its nonzero blocks in increasing
    // block row (the neighbourhood M(n) of every variable of the column).
    std::vector<int> coloff(nb + 1, 0);
    std::vector<uint32_t> colent;
    for (int j = 0; j < nb; ++j) {
        coloff[j] = static_cast<int>(colent.size());
        for (int i = 0; i < mb; ++i) {
            const int s = hbm[i * nb + j];
            if (s < 0) continue;
            int q = c.layer_off[i];
            while (c.edge_col[q] != j) ++q;
            colent.push_back((static_cast<uint32_t>(i) << 20) | (static_cast<uint32_t>(q) << 9) |
                             static_cast<uint32_t>(s));
        }
    }
    coloff[nb] = static_cast<int>(colent.size());
    std::vector<uint32_t> edges(c.n_edges);
    for (int q = 0; q < c.n_edges; ++q)
        edges[q] = (static_cast<uint32_t>(c.edge_col[q]) << 16) |
                   static_cast<uint32_t>(c.edge_shift[q]);

    cudaError_t e = cudaSuccess;
    if (e == cudaSuccess) e = cudaMalloc(&c.d_hbm, sizeof(int16_t) * mb * nb);
    if (e == cudaSuccess) e = cudaMalloc(&c.d_voff, sizeof(uint16_t) * voff.size());
    if (e == cudaSuccess) e = cudaMalloc(&c.d_rowinfo, sizeof(uint32_t) * mb);
    if (e == cudaSuccess) e = cudaMalloc(&c.d_edges, sizeof(uint32_t) * c.n_edges);
    if (e == cudaSuccess) e = cudaMalloc(&c.d_wgather, sizeof(int16_t) * wgather.size());
    if (e == cudaSuccess) e = cudaMalloc(&c.d_colent, sizeof(uint32_t) * colent.size());
    if (e == cudaSuccess) e = cudaMalloc(&c.d_coloff, sizeof(int) * coloff.size());
    if (e == cudaSuccess) e = cudaMalloc(&c.d_status, 16);   // status word, saturation count
    if (e == cudaSuccess) e = cudaMalloc(&c.d_work, sizeof(unsigned long long) * kWorkSlots);
    if (e == cudaSuccess)
        e = cudaMemcpy(c.d_hbm, hbm, sizeof(int16_t) * mb * nb, cudaMemcpyHostToDevice);
    if (e == cudaSuccess)
        e = cudaMemcpy(c.d_voff, voff.data(), sizeof(uint16_t) * voff.size(),
                       cudaMemcpyHostToDevice);
    if (e == cudaSuccess)
        e = cudaMemcpy(c.d_rowinfo, rowinfo.data(), sizeof(uint32_t) * mb,
                       cudaMemcpyHostToDevice);
    if (e == cudaSuccess)
        e = cudaMemcpy(c.d_edges, edges.data(), sizeof(uint32_t) * c.n_edges,
                       cudaMemcpyHostToDevice);
    if (e == cudaSuccess)
        e = cudaMemcpy(c.d_wgather, wgather.data(), sizeof(int16_t) * wgather.size(),
                       cudaMemcpyHostToDevice);
    if (e == cudaSuccess)
        e = cudaMemcpy(c.d_colent, colent.data(), sizeof(uint32_t) * colent.size(),
                       cudaMemcpyHostToDevice);
    if (e == cudaSuccess)
        e = cudaMemcpy(c.d_coloff, coloff.data(), sizeof(int) * coloff.size(),
                       cudaMemcpyHostToDevice);
    if (e == cudaSuccess) e = cudaMemset(c.d_status, 0, 16);
    if (e != cudaSuccess) {
        ldpc_status st = (e == cudaErrorMemoryAllocation)
                             ? fail(LDPC_ERR_NOMEM, "ldpc_code_create: device allocation")
                             : cuda_fail(e, "ldpc_code_create");
        release(c);
        delete h;
        return st;
    }
    *out = h;
    return LDPC_OK;
}

void ldpc_code_destroy(ldpc_code *code) {
    if (!code) return;
    release(code->c);
    delete code;
}

ldpc_status ldpc_code_info(const ldpc_code *code, int *n, int *k, int *m, int *z,
                           int *max_row_deg) {
    if (!code) return fail(LDPC_ERR_INVALID_ARG, "ldpc_code_info: code is NULL");
    const Code &c = code->c;
    if (n) *n = c.n;
    if (k) *k = c.k;
    if (m) *m = c.m;
    if (z) *z = c.z;
    if (max_row_deg) *max_row_deg = c.max_deg;
    return LDPC_OK;
}

ldpc_status ldpc_gen_info(uint64_t seed, int64_t frame0, int64_t frames, int k,
                          uint8_t *d_info, cudaStream_t stream) {
    if (frames < 0 || frame0 < 0 || k < 0)
        return fail(LDPC_ERR_INVALID_ARG, "ldpc_gen_info: negative size");
    if (frames == 0 || k == 0) return LDPC_OK;
    if (!d_info) return fail(LDPC_ERR_INVALID_ARG, "ldpc_gen_info: d_info is NULL");
    return launch_gen_info(seed, frame0, frames, k, d_info, stream);
}

ldpc_status ldpc_encode(const ldpc_code *code, const uint8_t *d_info, uint8_t *d_code,
                        int64_t frames, cudaStream_t stream) {
    if (!code) return fail(LDPC_ERR_INVALID_ARG, "ldpc_encode: code is NULL");
    if (frames < 0) return fail(LDPC_ERR_INVALID_ARG, "ldpc_encode: frames < 0");
    if (frames == 0) return LDPC_OK;
    if (!d_info || !d_code) return fail(LDPC_ERR_INVALID_ARG, "ldpc_encode: NULL buffer");
    ldpc_status st = bind(&code->c);
    if (st) return st;
    return launch_encode(code->c, d_info, d_code, frames, stream);
}

ldpc_status ldpc_awgn_llr(const uint8_t *d_code, int64_t frame0, int64_t frames, int n,
                          uint64_t seed, float sigma, float llr_scale, float *d_llr,
                          cudaStream_t stream) {
    if (frames < 0 || frame0 < 0 || n < 0)
        return fail(LDPC_ERR_INVALID_ARG, "ldpc_awgn_llr: negative size");
    if (frames == 0 || n == 0) return LDPC_OK;
    if (!d_code || !d_llr) return fail(LDPC_ERR_INVALID_ARG, "ldpc_awgn_llr: NULL buffer");
    if (!(sigma >= 0.0f) || !(llr_scale == llr_scale))
        return fail(LDPC_ERR_INVALID_ARG, "ldpc_awgn_llr: sigma must be >= 0");
    return launch_awgn(d_code, frame0, frames, n, seed, sigma, llr_scale, d_llr, stream);
}

ldpc_status ldpc_awgn_llr_frames(const uint8_t *d_code, int64_t frame0, int64_t frames, int n,
                                 uint64_t seed, const float *d_sigma, float *d_llr,
                                 cudaStream_t stream) {
    if (frames < 0 || frame0 < 0 || n < 0)
        return fail(LDPC_ERR_INVALID_ARG, "ldpc_awgn_llr_frames: negative size");
    if (frames == 0 || n == 0) return LDPC_OK;
    if (!d_code || !d_llr || !d_sigma)
        return fail(LDPC_ERR_INVALID_ARG, "ldpc_awgn_llr_frames: NULL buffer");
    return launch_awgn_frames(d_code, frame0, frames, n, seed, d_sigma, d_llr, stream);
}

ldpc_status ldpc_snr_sigma(uint64_t seed, int64_t frame0, int64_t frames, float ebn0_lo_db,
                           float ebn0_hi_db, float rate, float *d_sigma, cudaStream_t stream) {
    if (frames < 0 || frame0 < 0)
        return fail(LDPC_ERR_INVALID_ARG, "ldpc_snr_sigma: negative size");
    if (!(rate > 0.0f && rate <= 1.0f) || !(ebn0_lo_db <= ebn0_hi_db) ||
        !(ebn0_lo_db > -100.0f && ebn0_hi_db < 100.0f))
        return fail(LDPC_ERR_INVALID_ARG, "ldpc_snr_sigma: bad rate or Eb/N0 range");
    if (frames == 0) return LDPC_OK;
    if (!d_sigma) return fail(LDPC_ERR_INVALID_ARG, "ldpc_snr_sigma: NULL buffer");
    return launch_snr_sigma(seed, frame0, frames, ebn0_lo_db, ebn0_hi_db, rate, d_sigma, stream);
}

ldpc_status ldpc_quantize_pack_i8(const float *d_llr, uint32_t *d_q, int64_t frames, int n,
                                  float scale, int clip, cudaStream_t stream) {
    if (frames < 0 || n < 0)
        return fail(LDPC_ERR_INVALID_ARG, "ldpc_quantize_pack_i8: negative size");
    if (clip < 0 || clip > 127)
        return fail(LDPC_ERR_INVALID_ARG, "ldpc_quantize_pack_i8: clip must be in [0, 127]");
    if (!(scale == scale))
        return fail(LDPC_ERR_INVALID_ARG, "ldpc_quantize_pack_i8: scale is NaN");
    if (frames == 0 || n == 0) return LDPC_OK;
    if (!d_llr || !d_q) return fail(LDPC_ERR_INVALID_ARG, "ldpc_quantize_pack_i8: NULL buffer");
    return launch_quantize(d_llr, d_q, frames, n, scale, clip, stream);
}

static ldpc_status check_decode_args(const ldpc_code *code, ldpc_dtype dtype, int64_t frames,
                                     const ldpc_decode_params *params, DecodeParams *p,
                                     const char *who) {
    std::string w(who);
    if (!code) return fail(LDPC_ERR_INVALID_ARG, w + ": code is NULL");
    if (!params) return fail(LDPC_ERR_INVALID_ARG, w + ": params is NULL");
    if (dtype != LDPC_F32 && dtype != LDPC_I8X4 && dtype != LDPC_I16W)
        return fail(LDPC_ERR_INVALID_ARG, w + ": unknown dtype");
    if (frames < 0) return fail(LDPC_ERR_INVALID_ARG, w + ": frames < 0");
    if (params->max_iters < 1 || params->max_iters > kMaxIters)
        return fail(LDPC_ERR_INVALID_ARG, w + ": max_iters must be in [1, 1000]");
    if (params->normalise != 0 && params->normalise != 1)
        return fail(LDPC_ERR_INVALID_ARG, w + ": normalise must be 0 or 1");
    if (params->early_stop != 0 && params->early_stop != 1)
        return fail(LDPC_ERR_INVALID_ARG, w + ": early_stop must be 0 or 1");
    if (params->normalise && !(params->alpha == params->alpha))
        return fail(LDPC_ERR_INVALID_ARG, w + ": alpha is NaN");
    if (dtype != LDPC_F32 && params->normalise && params->alpha != 0.75f)
        return fail(LDPC_ERR_UNSUPPORTED,
                    w + ": the integer decoders scale by (3m)>>2, which needs alpha == 0.75");
    if (code->c.max_deg > kMaxRowDeg)
        return fail(LDPC_ERR_UNSUPPORTED, w + ": row degree above 27");
    p->max_iters = params->max_iters;
    p->alpha = params->normalise ? params->alpha : 1.0f;
    p->normalise = params->normalise;
    p->early_stop = params->early_stop;
    return LDPC_OK;
}

ldpc_status ldpc_decode_layered_minsum(const ldpc_code *code, ldpc_dtype dtype,
                                       const void *d_llr, int64_t frames,
                                       const ldpc_decode_params *params, uint32_t *d_hard,
                                       int32_t *d_iters, void *d_post, cudaStream_t stream) {
    DecodeParams p;
    ldpc_status st = check_decode_args(code, dtype, frames, params, &p,
                                       "ldpc_decode_layered_minsum");
    if (st) return st;
    if (frames == 0) return LDPC_OK;
    if (!d_llr || !d_hard || !d_iters)
        return fail(LDPC_ERR_INVALID_ARG, "ldpc_decode_layered_minsum: NULL buffer");
    st = bind(&code->c);
    if (st) return st;
    if (dtype == LDPC_I16W)
        return launch_decode_i16w(code->c, static_cast<const int16_t *>(d_llr), frames, p,
                                  d_hard, d_iters, static_cast<int16_t *>(d_post), stream);
    return launch_decode(code->c, dtype, d_llr, frames, p, d_hard, d_iters, d_post, stream);
}

ldpc_status ldpc_frame_stats(const ldpc_code *code, const uint8_t *d_info,
                             const uint32_t *d_hard, const int32_t *d_iters, int64_t frames,
                             int max_iters, int64_t *d_counters, cudaStream_t stream) {
    if (!code) return fail(LDPC_ERR_INVALID_ARG, "ldpc_frame_stats: code is NULL");
    if (frames < 0 || max_iters < 1 || max_iters > kMaxIters)
        return fail(LDPC_ERR_INVALID_ARG, "ldpc_frame_stats: bad frames or max_iters");
    if (!d_counters || (frames && (!d_info || !d_hard || !d_iters)))
        return fail(LDPC_ERR_INVALID_ARG, "ldpc_frame_stats: NULL buffer");
    ldpc_status st = bind(&code->c);
    if (st) return st;
    return launch_stats(code->c, d_info, d_hard, d_iters, frames, max_iters, d_counters,
                        stream);
}

ldpc_status ldpc_paired_frame_errors(const ldpc_code *code, const uint8_t *d_info,
                                     const uint32_t *d_hard_a, const uint32_t *d_hard_b,
                                     int64_t frames, int64_t *d_counts, cudaStream_t stream) {
    if (!code) return fail(LDPC_ERR_INVALID_ARG, "ldpc_paired_frame_errors: code is NULL");
    if (frames < 0) return fail(LDPC_ERR_INVALID_ARG, "ldpc_paired_frame_errors: frames < 0");
    if (!d_counts || (frames && (!d_info || !d_hard_a || !d_hard_b)))
        return fail(LDPC_ERR_INVALID_ARG, "ldpc_paired_frame_errors: NULL buffer");
    ldpc_status st = bind(&code->c);
    if (st) return st;
    return launch_paired(code->c, d_info, d_hard_a, d_hard_b, frames, d_counts, stream);
}

static size_t align256(size_t x) { return (x + 255) & ~static_cast<size_t>(255); }

static void host_chunk_bytes(const Code &c, ldpc_dtype dtype, int64_t chunk, size_t *llr,
                             size_t *hard, size_t *iters) {
    const int64_t groups = (chunk + 3) / 4;
    *llr = align256(dtype == LDPC_F32 ? static_cast<size_t>(chunk) * c.n * 4
                                      : static_cast<size_t>(groups) * c.n * 4);
    *hard = align256(static_cast<size_t>(chunk) * ((c.n + 31) / 32) * 4);
    *iters = align256(static_cast<size_t>(chunk) * 4);
}

size_t ldpc_decode_host_workspace_bytes(const ldpc_code *code, ldpc_dtype dtype,
                                        int64_t chunk_frames) {
    if (!code || chunk_frames <= 0) return 0;
    size_t a, b, c;
    host_chunk_bytes(code->c, dtype, chunk_frames, &a, &b, &c);
    return 2 * (a + b + c);
}

ldpc_status ldpc_decode_host(const ldpc_code *code, ldpc_dtype dtype, const void *h_llr,
                             int64_t frames, const ldpc_decode_params *params,
                             uint32_t *h_hard, int32_t *h_iters, void *d_workspace,
                             size_t workspace_bytes, int64_t chunk_frames,
                             cudaStream_t stream) {
    DecodeParams p;
    ldpc_status st = check_decode_args(code, dtype, frames, params, &p, "ldpc_decode_host");
    if (st) return st;
    if (dtype == LDPC_I16W)
        return fail(LDPC_ERR_UNSUPPORTED, "ldpc_decode_host: LDPC_F32 or LDPC_I8X4 only");
    if (frames == 0) return LDPC_OK;
    if (!h_llr || !h_hard || !h_iters || !d_workspace)
        return fail(LDPC_ERR_INVALID_ARG, "ldpc_decode_host: NULL buffer");
    if (chunk_frames <= 0 || chunk_frames % 4)
        return fail(LDPC_ERR_INVALID_ARG, "ldpc_decode_host: chunk_frames must be a positive "
                                          "multiple of 4");
    if (workspace_bytes < ldpc_decode_host_workspace_bytes(code, dtype, chunk_frames))
        return fail(LDPC_ERR_INVALID_ARG, "ldpc_decode_host: workspace too small");
    Code &c = const_cast<Code &>(code->c);
    st = bind(&c);
    if (st) return st;
    for (auto &s : c.aux)
        if (!s) LDPC_CUDA_TRY(cudaStreamCreateWithFlags(&s, cudaStreamNonBlocking),
                              "cudaStreamCreateWithFlags");
    for (auto &e : c.ev)
        if (!e) LDPC_CUDA_TRY(cudaEventCreateWithFlags(&e, cudaEventDisableTiming),
                              "cudaEventCreateWithFlags");
    size_t bl, bh, bi;
    host_chunk_bytes(c, dtype, chunk_frames, &bl, &bh, &bi);
    char *ws = static_cast<char *>(d_workspace);
    const int nw = (c.n + 31) / 32;
    LDPC_CUDA_TRY(cudaEventRecord(c.ev[0], stream), "cudaEventRecord");
    for (int b = 0; b < 2; ++b)
        LDPC_CUDA_TRY(cudaStreamWaitEvent(c.aux[b], c.ev[0], 0), "cudaStreamWaitEvent");
    int64_t idx = 0;
    // a short first chunk: the pipeline waits only for its copy
    const int64_t first = std::min(chunk_frames, ((chunk_frames / 4 + 3) / 4) * 4);
    for (int64_t f0 = 0, fc = 0; f0 < frames; f0 += fc, ++idx) {
        fc = std::min(idx == 0 ? first : chunk_frames, frames - f0);
        const int b = static_cast<int>(idx & 1);
        cudaStream_t s = c.aux[b];
        char *base = ws + b * (bl + bh + bi);
        void *d_llr = base;
        uint32_t *d_hard = reinterpret_cast<uint32_t *>(base + bl);
        int32_t *d_iters = reinterpret_cast<int32_t *>(base + bl + bh);
        const size_t in_bytes = dtype == LDPC_F32
                                    ? static_cast<size_t>(fc) * c.n * 4
                                    : static_cast<size_t>((fc + 3) / 4) * c.n * 4;
        const char *src = static_cast<const char *>(h_llr) +
                          (dtype == LDPC_F32 ? static_cast<size_t>(f0) * c.n * 4
                                             : static_cast<size_t>(f0 / 4) * c.n * 4);
        LDPC_CUDA_TRY(cudaMemcpyAsync(d_llr, src, in_bytes, cudaMemcpyHostToDevice, s),
                      "cudaMemcpyAsync H2D");
        st = launch_decode(c, dtype, d_llr, fc, p, d_hard, d_iters, nullptr, s);
        if (st) return st;
        LDPC_CUDA_TRY(cudaMemcpyAsync(h_hard + f0 * nw, d_hard, static_cast<size_t>(fc) * nw * 4,
                                      cudaMemcpyDeviceToHost, s),
                      "cudaMemcpyAsync D2H");
        LDPC_CUDA_TRY(cudaMemcpyAsync(h_iters + f0, d_iters, static_cast<size_t>(fc) * 4,
                                      cudaMemcpyDeviceToHost, s),
                      "cudaMemcpyAsync D2H");
    }
    LDPC_CUDA_TRY(cudaEventRecord(c.ev[1], c.aux[0]), "cudaEventRecord");
    LDPC_CUDA_TRY(cudaEventRecord(c.ev[2], c.aux[1]), "cudaEventRecord");
    LDPC_CUDA_TRY(cudaStreamWaitEvent(stream, c.ev[1], 0), "cudaStreamWaitEvent");
    LDPC_CUDA_TRY(cudaStreamWaitEvent(stream, c.ev[2], 0), "cudaStreamWaitEvent");
    return LDPC_OK;
}

ldpc_status ldpc_check_bounded_wait(const ldpc_code *code, uint32_t polls,
                                    cudaStream_t stream) {
    if (!code) return fail(LDPC_ERR_INVALID_ARG, "ldpc_check_bounded_wait: code is NULL");
    if (polls < 1 || polls > (1u << 22))
        return fail(LDPC_ERR_INVALID_ARG, "ldpc_check_bounded_wait: polls outside 1..2^22");
    ldpc_status st = bind(&code->c);
    if (st) return st;
    return launch_wait_check(code->c, polls, stream);
}

ldpc_status ldpc_debug_saturation_count(const ldpc_code *code, cudaStream_t stream,
                                        int64_t *count) {
    if (!code || !count)
        return fail(LDPC_ERR_INVALID_ARG, "ldpc_debug_saturation_count: NULL argument");
#ifdef LDPC_DEBUG
    ldpc_status st = bind(&code->c);
    if (st) return st;
    LDPC_CUDA_TRY(cudaStreamSynchronize(stream), "cudaStreamSynchronize");
    unsigned long long v = 0;
    LDPC_CUDA_TRY(cudaMemcpy(&v, code->c.d_status + 2, sizeof(v), cudaMemcpyDeviceToHost),
                  "cudaMemcpy saturation count");
    LDPC_CUDA_TRY(cudaMemset(code->c.d_status + 2, 0, sizeof(v)), "cudaMemset saturation count");
    *count = static_cast<int64_t>(v);
    return LDPC_OK;
#else
    (void)stream;
    *count = 0;
    return fail(LDPC_ERR_UNSUPPORTED,
                "ldpc_debug_saturation_count: the library was built without -DLDPC_DEBUG");
#endif
}

ldpc_status ldpc_sync(const ldpc_code *code, cudaStream_t stream, double timeout_s) {
    if (!code) return fail(LDPC_ERR_INVALID_ARG, "ldpc_sync: code is NULL");
    if (!(timeout_s >= 0.0)) return fail(LDPC_ERR_INVALID_ARG, "ldpc_sync: bad timeout");
    ldpc_status st = bind(&code->c);
    if (st) return st;
    const auto t0 = std::chrono::steady_clock::now();
    for (;;) {
        cudaError_t e = cudaStreamQuery(stream);
        if (e == cudaSuccess) break;
        if (e != cudaErrorNotReady) return cuda_fail(e, "cudaStreamQuery");
        const double el =
            std::chrono::duration<double>(std::chrono::steady_clock::now() - t0).count();
        if (el > timeout_s)
            return fail(LDPC_ERR_TIMEOUT, "ldpc_sync: stream still busy after the time limit");
        std::this_thread::sleep_for(std::chrono::microseconds(50));
    }
    int status = 0;
    LDPC_CUDA_TRY(cudaMemcpy(&status, code->c.d_status, sizeof(int), cudaMemcpyDeviceToHost),
                  "cudaMemcpy status");
    if (status) {
        LDPC_CUDA_TRY(cudaMemset(code->c.d_status, 0, sizeof(int)), "cudaMemset status");
        if (status & kStatusCopyTimeout)
            return fail(LDPC_ERR_TIMEOUT, "ldpc_sync: a kernel's wait for its bulk copy ran out");
        if (status & kStatusBadOffset)
            return fail(LDPC_ERR_CUDA, "ldpc_sync: a kernel read an edge offset outside the "
                                       "posterior region (debug build check)");
        return fail(LDPC_ERR_CUDA, "ldpc_sync: device status " + std::to_string(status));
    }
    return LDPC_OK;
}

}  // extern "C"
