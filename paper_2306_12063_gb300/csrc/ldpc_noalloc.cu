// ldpc_decode_layered_minsum_noalloc: the layered min-sum decoder for callers
// that cannot allocate device memory.
//
// Every other decode call uses a code handle, whose creation allocates the
// per-code tables and work counters with cudaMalloc.  Some callers cannot do
// that: a real-time thread with a fixed memory budget, a process whose
// framework owns every device allocation (a caching allocator or a pool that
// must account for each byte), or a steady-state path where cudaMalloc and
// cudaFree, which can synchronise the device, are not allowed.  This entry
// point needs nothing but the caller's own input and output buffers: its
// scratch memory -- the work counter and status word of the decode kernel
// and the per-lane offset table that a handle would hold -- lives in one
// file-scope static device array that every GPU loading the library keeps
// until the process exits.
#include <string>

#include "ldpc_internal.cuh"

namespace ldpc {

// Static scratch, shared by every call on a device.  Layout (bytes):
//   [0, 8)      work counter of the decode kernel's frame hand-out
//   [8, 12)     device status word (bulk-copy timeouts)
//   [64, 256)   per-layer row info, one word per block row
//   [256, ...)  per-lane offset table, [mb][rpl][dslots][32] uint16
constexpr size_t kStaticScratchBytes = 64 * 1024;
constexpr size_t kScratchRowInfo = 64;
constexpr size_t kScratchOffsets = 256;
static __device__ __align__(256) unsigned char g_static_scratch[kStaticScratchBytes];

struct HbmArg {
    int16_t v[kMaxNb * kMaxNb];   // row-major mb x nb base matrix
};

// Clears the counter and status word and writes the row info and offset
// table for the given base matrix into the scratch array.
__global__ void noalloc_setup_kernel(HbmArg h, int mb, int nb, int z, int rpl, int dslots,
                                     unsigned char *scratch) {
    unsigned long long *work = reinterpret_cast<unsigned long long *>(scratch);
    int *status = reinterpret_cast<int *>(scratch + 8);
    uint32_t *rowinfo = reinterpret_cast<uint32_t *>(scratch + kScratchRowInfo);
    uint16_t *voff = reinterpret_cast<uint16_t *>(scratch + kScratchOffsets);
    if (threadIdx.x == 0) {
        *work = 0ull;
        *status = 0;
    }
    for (int i = threadIdx.x; i < mb; i += blockDim.x) {
        int d = 0;
        for (int j = 0; j < nb; ++j) d += h.v[i * nb + j] >= 0;
        rowinfo[i] = static_cast<uint32_t>(d);
    }
    const int total = mb * rpl * dslots * 32;
    for (int q = threadIdx.x; q < total; q += blockDim.x) {
        const int lane = q % 32;
        const int slot = (q / 32) % dslots;
        const int t = (q / (32 * dslots)) % rpl;
        const int i = q / (32 * dslots * rpl);
        int d = 0;
        for (int j = 0; j < nb; ++j) d += h.v[i * nb + j] >= 0;
        const int e = slot - (dslots - d);   // edge index within the row, if any
        const int r = lane + 32 * t;
        // leading unused slots point at the lane's dummy posterior word N + lane
        uint16_t val = static_cast<uint16_t>(4 * (nb * z + lane));
        if (e >= 0 && r < z) {
            int seen = 0;
            for (int j = 0; j < nb; ++j) {
                const int s = h.v[i * nb + j];
                if (s < 0) continue;
                if (seen++ == e) {
                    val = static_cast<uint16_t>(4 * (j * z + (r + s) % z));
                    break;
                }
            }
        }
        voff[q] = val;
    }
}

// Device address of the static array on the current device.  Looked up on
// every call (the lookup allocates nothing): after a device reset the module
// is loaded again and the array may sit at another address.
static ldpc_status scratch_address(unsigned char **out) {
    void *p = nullptr;
    const cudaError_t e = cudaGetSymbolAddress(&p, g_static_scratch);
    if (e != cudaSuccess) return cuda_fail(e, "cudaGetSymbolAddress of the static scratch");
    *out = static_cast<unsigned char *>(p);
    return LDPC_OK;
}

// The parity structure the direct encoder needs (eq. 3-7), checked the same
// way as at code creation; returns a reason or NULL.
static const char *structure_problem(const int16_t *h, int mb, int nb, int z) {
    for (int q = 0; q < mb * nb; ++q)
        if (h[q] < -1 || h[q] >= z) return "base matrix entry outside [-1, z)";
    const int kb = nb - mb;
    if (h[kb] < 0 || h[kb] != h[(mb - 1) * nb + kb])
        return "h_b entries of rows 0 and mb-1 must be equal and non-negative";
    int y = -1;
    for (int i = 1; i < mb - 1; ++i)
        if (h[i * nb + kb] >= 0) {
            if (y >= 0) return "h_b has more than one entry between its first and last rows";
            y = i;
        }
    if (y < 0) return "h_b has no entry between its first and last rows";
    for (int i = 0; i < mb; ++i)
        for (int t = 0; t < mb - 1; ++t) {
            const int v = h[i * nb + kb + 1 + t];
            const bool diag = (i == t || i == t + 1);
            if ((diag && v != 0) || (!diag && v != -1))
                return "columns Kb+1.. must be the dual diagonal of zeros (H_b2')";
        }
    return nullptr;
}

}  // namespace ldpc

using namespace ldpc;

extern "C" ldpc_status ldpc_decode_layered_minsum_noalloc(
    const int16_t *hbm, int mb, int nb, int z, ldpc_dtype dtype, const void *d_llr,
    int64_t frames, const ldpc_decode_params *params, uint32_t *d_hard, int32_t *d_iters,
    void *d_post, cudaStream_t stream) {
    if (!hbm || !params)
        return fail(LDPC_ERR_INVALID_ARG, "ldpc_decode_layered_minsum_noalloc: NULL argument");
    if (mb < 3 || nb <= mb || nb > kMaxNb || z < 1 || z > kMaxZ)
        return fail(LDPC_ERR_INVALID_ARG,
                    "ldpc_decode_layered_minsum_noalloc: need 3 <= mb < nb <= 32, 1 <= z <= 384");
    if (dtype != LDPC_F32 && dtype != LDPC_I8X4)
        return fail(LDPC_ERR_INVALID_ARG, "ldpc_decode_layered_minsum_noalloc: unknown dtype");
    if (frames < 0 || params->max_iters < 1 || params->max_iters > kMaxIters ||
        (params->normalise != 0 && params->normalise != 1) ||
        (params->early_stop != 0 && params->early_stop != 1) ||
        (params->normalise && !(params->alpha == params->alpha)))
        return fail(LDPC_ERR_INVALID_ARG,
                    "ldpc_decode_layered_minsum_noalloc: bad frames or decode parameters");
    if (dtype == LDPC_I8X4 && params->normalise && params->alpha != 0.75f)
        return fail(LDPC_ERR_UNSUPPORTED,
                    "ldpc_decode_layered_minsum_noalloc: int8 scaling needs alpha == 0.75");
    if (const char *why = structure_problem(hbm, mb, nb, z))
        return fail(LDPC_ERR_BAD_STRUCTURE, why);
    int max_deg = 0;
    for (int i = 0; i < mb; ++i) {
        int d = 0;
        for (int j = 0; j < nb; ++j) d += hbm[i * nb + j] >= 0;
        max_deg = d > max_deg ? d : max_deg;
    }
    const int dslots = slot_class(max_deg);
    if (!dslots)
        return fail(LDPC_ERR_UNSUPPORTED,
                    "ldpc_decode_layered_minsum_noalloc: row degree above 27");
    const int rpl = (z + 31) / 32;
    const size_t table_bytes = static_cast<size_t>(mb) * rpl * dslots * 32 * sizeof(uint16_t);
    if (kScratchOffsets + table_bytes > kStaticScratchBytes)
        return fail(LDPC_ERR_UNSUPPORTED,
                    "ldpc_decode_layered_minsum_noalloc: offset table of mb * ceil(z/32) * "
                    "slots * 64 bytes exceeds the 65280 bytes of static scratch");
    if (frames == 0) return LDPC_OK;
    if (!d_llr || !d_hard || !d_iters)
        return fail(LDPC_ERR_INVALID_ARG, "ldpc_decode_layered_minsum_noalloc: NULL buffer");

    unsigned char *scratch = nullptr;
    ldpc_status st = scratch_address(&scratch);
    if (st) return st;

    HbmArg h;
    for (int q = 0; q < kMaxNb * kMaxNb; ++q) h.v[q] = q < mb * nb ? hbm[q] : -1;
    noalloc_setup_kernel<<<1, 256, 0, stream>>>(h, mb, nb, z, rpl, dslots, scratch);
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return cuda_fail(e, "noalloc_setup_kernel");

    DevCode dc;
    dc.n = nb * z; dc.k = (nb - mb) * z; dc.m = mb * z; dc.z = z;
    dc.mb = mb; dc.nb = nb; dc.kb = nb - mb; dc.y = -1;
    dc.nwords = (dc.n + 31) / 32; dc.rpl = rpl; dc.dslots = dslots; dc.n_edges = 0;
    dc.hbm = nullptr;
    dc.voff = reinterpret_cast<const uint16_t *>(scratch + kScratchOffsets);
    dc.rowinfo = reinterpret_cast<const uint32_t *>(scratch + kScratchRowInfo);
    dc.edges = nullptr;   // the plain decoders read only the offset table
    dc.wgather = nullptr;
    dc.colent = nullptr;
    dc.coloff = nullptr;
    dc.status = reinterpret_cast<int *>(scratch + 8);
    dc.sat = nullptr;   // the debug saturation count needs a code handle
    DecodeParams p;
    p.max_iters = params->max_iters;
    p.alpha = params->normalise ? params->alpha : 1.0f;
    p.normalise = params->normalise;
    p.early_stop = params->early_stop;
    st = launch_decode_view(dc, dtype, d_llr, frames, p, d_hard, d_iters, d_post,
                            reinterpret_cast<unsigned long long *>(scratch), stream);
    if (st) return st;
    // With no handle there is no ldpc_sync to read the status word later, so
    // read it here (into a host int: no allocation) once the decode is done.
    int status = 0;
    e = cudaMemcpyFromSymbolAsync(&status, g_static_scratch, sizeof(int), 8,
                                  cudaMemcpyDeviceToHost, stream);
    if (e != cudaSuccess) return cuda_fail(e, "reading the static status word");
    e = cudaStreamSynchronize(stream);
    if (e != cudaSuccess) return cuda_fail(e, "cudaStreamSynchronize");
    if (status & kStatusCopyTimeout)
        return fail(LDPC_ERR_TIMEOUT,
                    "ldpc_decode_layered_minsum_noalloc: a kernel's wait for its bulk copy ran out");
    if (status & kStatusBadOffset)
        return fail(LDPC_ERR_CUDA, "ldpc_decode_layered_minsum_noalloc: a kernel read an edge "
                                   "offset outside the posterior region (debug build check)");
    if (status)
        return fail(LDPC_ERR_CUDA, "ldpc_decode_layered_minsum_noalloc: device status " +
                                       std::to_string(status));
    return LDPC_OK;
}
