// Training of the learned normalised min-sum decoder: the unrolled layered
// decoder (Section 4, eq. 22, 23, 20, with a learned factor per iteration and
// per nonzero block of H_bm in place of a fixed normalisation), its
// cross-entropy loss on the posteriors of every iteration, and its
// hand-written reverse-mode derivative.
//
// Forward.  One warp per frame; lane l handles rows l, l + 32, ... of each
// layer with the posteriors in shared memory.  After every iteration t the
// warp writes the posteriors Z^(t) and the compressed state of every check
// row (unscaled smallest and second smallest |Z_mn|, the argmin edge and the
// message signs) to global memory: these checkpoints are all the backward
// pass needs.
//
// Backward.  One warp per frame, iterations t = T .. 1.  The warp reloads
// Z^(t-1) and the row state of iteration t-1, runs iteration t forward again
// keeping every Z_mn in shared memory, then walks the layers in reverse:
//   Z_n' = Q_e + L_e,  L_e = w[t][b_e] sigma_e M_e,  Q_e = Z_n - L_e^old,
// with M_e the smallest |Q| of the row's other edges, so the adjoint of M_e
// reaches |Q| of the row's argmin (or, for the argmin itself, of the second
// argmin) and, through sign(Q), Q itself.  The adjoint of L_e^old is carried
// per edge into the previous iteration, where that message was produced.
// Shared memory per frame: Z, its adjoint, Q and the message adjoint
// (4 (2 N + 2 E) bytes, E = edges of H).
#include <algorithm>
#include <cmath>
#include <string>

#include "ldpc_internal.cuh"

namespace ldpc {
namespace {

constexpr uint32_t kFullMask = 0xFFFFFFFFu;
constexpr int kTrainWarps = 4;   // frames per block (upper bound)

__device__ __forceinline__ int edge_var(uint32_t ed, int r, int z) {
    int rr = r + static_cast<int>(ed & 0xFFFFu);
    rr = rr >= z ? rr - z : rr;
    return static_cast<int>(ed >> 16) * z + rr;
}

__device__ __forceinline__ float sign_xor(float x, uint32_t s) {
    return __uint_as_float(__float_as_uint(x) ^ s);
}

template <typename T>
__device__ __forceinline__ T warp_sum(T v) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(kFullMask, v, o);
    return v;
}

// One check row of one layer, iteration t: eq. 22 for every edge, the two
// smallest |Z_mn| and the sign product, then eq. 23 (weighted) and eq. 20.
// The rounding is that of the oracle's weighted decoder: w m is rounded,
// then added or subtracted (the learned inference decoder fuses the two, so
// its posteriors differ from these by rounding only).  Q and v receive Z_mn
// and the variable of each edge; returns the row's new state.
template <int DMAX>
__device__ __forceinline__ uint4 row_forward(const DevCode &c, int e0, int d, int r, float *Zs,
                                             uint4 st, const float *wprev, const float *wcur,
                                             float (&Q)[DMAX], int (&v)[DMAX]) {
    const float m1o = __uint_as_float(st.x), m2o = __uint_as_float(st.y);
    const int idxo = static_cast<int>(st.z);
    float mn1 = __int_as_float(0x7F800000), mn2 = mn1;
    int idx = 0;
    uint32_t S = 0;
#pragma unroll
    for (int i = 0; i < DMAX; ++i) {
        if (i < d) {
            v[i] = edge_var(__ldg(c.edges + e0 + i), r, c.z);
            const float mag = (i == idxo) ? m2o : m1o;
            const float L = sign_xor(__fmul_rn(__ldg(wprev + e0 + i), mag), ((st.w >> i) & 1u) << 31);
            const float q = __fsub_rn(Zs[v[i]], L);
            Q[i] = q;
            const float a = fabsf(q);
            if (a < mn1) {
                mn2 = mn1;
                mn1 = a;
                idx = i;
            } else if (a < mn2) {
                mn2 = a;
            }
            S ^= __float_as_uint(q);
        }
    }
    S &= 0x80000000u;
    uint32_t sg = 0;
#pragma unroll
    for (int i = 0; i < DMAX; ++i) {
        if (i < d) {
            const float M = (i == idx) ? mn2 : mn1;
            const uint32_t sb = S ^ (__float_as_uint(Q[i]) & 0x80000000u);
            const float L = sign_xor(__fmul_rn(__ldg(wcur + e0 + i), M), sb);
            Zs[v[i]] = __fadd_rn(Q[i], L);
            sg |= (sb >> 31) << i;
        }
    }
    return make_uint4(__float_as_uint(mn1), __float_as_uint(mn2), static_cast<uint32_t>(idx), sg);
}

// BCE(sigmoid(-Z), c) = softplus(-Z) + c Z, overflow-free.
__device__ __forceinline__ float bce_post(float zz, float cb) {
    return fmaxf(-zz, 0.0f) + log1pf(expf(-fabsf(zz))) + cb * zz;
}

template <int DMAX>
__global__ void __launch_bounds__(32 * kTrainWarps)
    train_forward_kernel(DevCode c, const float *__restrict__ llr, const uint8_t *__restrict__ bits,
                         int64_t frames, const float *__restrict__ w, int T,
                         float *__restrict__ post, uint4 *__restrict__ rows,
                         float *__restrict__ loss, int zstride) {
    extern __shared__ float smem[];
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int64_t f = static_cast<int64_t>(blockIdx.x) * (blockDim.x >> 5) + warp;
    if (f >= frames) return;   // the whole warp leaves together
    const int n = c.n, z = c.z, m = c.m, E = c.n_edges;
    float *Zs = smem + warp * zstride;
#pragma unroll 8
    for (int i = lane; i < n; i += 32) Zs[i] = llr[f * n + i];
    __syncwarp();
    double acc = 0.0;
    for (int t = 1; t <= T; ++t) {
        const float *wcur = w + static_cast<size_t>(t - 1) * E;
        const float *wprev = w + static_cast<size_t>(t >= 2 ? t - 2 : 0) * E;
        const uint4 *rin = t >= 2 ? rows + (static_cast<size_t>(t - 2) * frames + f) * m : nullptr;
        uint4 *rout = t < T ? rows + (static_cast<size_t>(t - 1) * frames + f) * m : nullptr;
        for (int l = 0; l < c.mb; ++l) {
            const uint32_t ri = __ldg(c.rowinfo + l);
            const int d = ri & 255, e0 = static_cast<int>(ri >> 8);
            for (int r = lane; r < z; r += 32) {
                const uint4 st = rin ? rin[l * z + r] : make_uint4(0u, 0u, 0u, 0u);
                float Q[DMAX];
                int v[DMAX];
                const uint4 ns = row_forward<DMAX>(c, e0, d, r, Zs, st, wprev, wcur, Q, v);
                if (rout) rout[l * z + r] = ns;
            }
            __syncwarp();
        }
        float *pout = post + (static_cast<size_t>(t - 1) * frames + f) * n;
        const uint8_t *cb = bits + f * n;
        for (int i = lane; i < n; i += 32) {
            const float zz = Zs[i];
            pout[i] = zz;
            acc += static_cast<double>(bce_post(zz, static_cast<float>(cb[i] & 1u)));
        }
        __syncwarp();
    }
    acc = warp_sum(acc);
    if (lane == 0) loss[f] = static_cast<float>(acc);
}

// Shared memory of one backward warp: Z [zstride], adjoint of Z [zstride],
// Q [E z] (reused for the per-row weight-gradient terms), adjoint of the
// messages [E z].
template <int DMAX>
__global__ void __launch_bounds__(32 * kTrainWarps)
    train_backward_kernel(DevCode c, const float *__restrict__ llr,
                          const uint8_t *__restrict__ bits, int64_t frames,
                          const float *__restrict__ w, int T, const float *__restrict__ post,
                          const uint4 *__restrict__ rows, float loss_scale,
                          float *__restrict__ gw_frame, float *__restrict__ gllr, int zstride,
                          int warp_floats) {
    extern __shared__ float smem[];
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int64_t f = static_cast<int64_t>(blockIdx.x) * (blockDim.x >> 5) + warp;
    if (f >= frames) return;
    const int n = c.n, z = c.z, m = c.m, E = c.n_edges;
    float *Zs = smem + static_cast<size_t>(warp) * warp_floats;
    float *gZ = Zs + zstride;
    float *Qs = gZ + zstride;
    float *gL = Qs + E * z;
    for (int i = lane; i < n; i += 32) gZ[i] = 0.0f;
    for (int i = lane; i < E * z; i += 32) gL[i] = 0.0f;
    const uint8_t *cb = bits + f * n;
    for (int t = T; t >= 1; --t) {
        // adjoint of the loss term of iteration t: d BCE / d Z = c - sigmoid(-Z)
        const float *pt = post + (static_cast<size_t>(t - 1) * frames + f) * n;
        const float *zin = t >= 2 ? post + (static_cast<size_t>(t - 2) * frames + f) * n
                                  : llr + f * n;
        // the loads of eight positions in flight per lane
#pragma unroll 8
        for (int i = lane; i < n; i += 32) {
            const float p1 = 1.0f / (1.0f + expf(pt[i]));
            gZ[i] += loss_scale * (static_cast<float>(cb[i] & 1u) - p1);
            Zs[i] = zin[i];
        }
        __syncwarp();
        // iteration t again, keeping Z_mn of every edge
        const float *wcur = w + static_cast<size_t>(t - 1) * E;
        const float *wprev = w + static_cast<size_t>(t >= 2 ? t - 2 : 0) * E;
        const uint4 *rin = t >= 2 ? rows + (static_cast<size_t>(t - 2) * frames + f) * m : nullptr;
        for (int l = 0; l < c.mb; ++l) {
            const uint32_t ri = __ldg(c.rowinfo + l);
            const int d = ri & 255, e0 = static_cast<int>(ri >> 8);
            for (int r = lane; r < z; r += 32) {
                const uint4 st = rin ? rin[l * z + r] : make_uint4(0u, 0u, 0u, 0u);
                float Q[DMAX];
                int v[DMAX];
                row_forward<DMAX>(c, e0, d, r, Zs, st, wprev, wcur, Q, v);
#pragma unroll
                for (int i = 0; i < DMAX; ++i)
                    if (i < d) Qs[(e0 + i) * z + r] = Q[i];
            }
            __syncwarp();
        }
        // layers in reverse
        for (int l = c.mb - 1; l >= 0; --l) {
            const uint32_t ri = __ldg(c.rowinfo + l);
            const int d = ri & 255, e0 = static_cast<int>(ri >> 8);
            for (int r = lane; r < z; r += 32) {
                float Q[DMAX], gq[DMAX];
                int v[DMAX];
                float mn1 = __int_as_float(0x7F800000), mn2 = mn1;
                int idx = 0, idx2 = 0;
                uint32_t S = 0;
#pragma unroll
                for (int i = 0; i < DMAX; ++i) {
                    if (i < d) {
                        v[i] = edge_var(__ldg(c.edges + e0 + i), r, z);
                        const float q = Qs[(e0 + i) * z + r];
                        Q[i] = q;
                        const float a = fabsf(q);
                        if (a < mn1) {
                            mn2 = mn1;
                            idx2 = idx;
                            mn1 = a;
                            idx = i;
                        } else if (a < mn2) {
                            mn2 = a;
                            idx2 = i;
                        }
                        S ^= __float_as_uint(q);
                    }
                }
                S &= 0x80000000u;
                float g_others = 0.0f, g_argmin = 0.0f;
#pragma unroll
                for (int i = 0; i < DMAX; ++i) {
                    if (i < d) {
                        const float gz = gZ[v[i]];
                        gq[i] = gz;   // Z_n' = Q + L: the direct path
                        const float gl = gz + gL[(e0 + i) * z + r];   // adjoint of L_e
                        const float M = (i == idx) ? mn2 : mn1;
                        const uint32_t sb = S ^ (__float_as_uint(Q[i]) & 0x80000000u);
                        Qs[(e0 + i) * z + r] = sign_xor(gl * M, sb);            // d/dw
                        const float gm = sign_xor(gl * __ldg(wcur + e0 + i), sb);   // d/dM
                        if (i == idx)
                            g_argmin = gm;
                        else
                            g_others += gm;
                    }
                }
                // M = |Q_idx| for every other edge, |Q_idx2| for the argmin edge
#pragma unroll
                for (int i = 0; i < DMAX; ++i) {
                    if (i < d) {
                        const uint32_t qs = __float_as_uint(Q[i]) & 0x80000000u;
                        float g = gq[i];
                        if (i == idx) g += sign_xor(g_others, qs);
                        if (i == idx2) g += sign_xor(g_argmin, qs);
                        gZ[v[i]] = g;                        // adjoint of Z_n before the layer
                        gL[(e0 + i) * z + r] = -g;           // adjoint of the previous message
                    }
                }
            }
            __syncwarp();
            // weight gradient of this layer: sum of the row terms per block
            // edge, the d warp reductions interleaved (independent shuffles)
            float *gw = gw_frame + (static_cast<size_t>(f) * T + (t - 1)) * E;
            float s[DMAX];
#pragma unroll
            for (int i = 0; i < DMAX; ++i) {
                s[i] = 0.0f;
                if (i < d)
                    for (int r = lane; r < z; r += 32) s[i] += Qs[(e0 + i) * z + r];
            }
#pragma unroll
            for (int o = 16; o >= 1; o >>= 1) {
#pragma unroll
                for (int i = 0; i < DMAX; ++i) s[i] += __shfl_xor_sync(0xFFFFFFFFu, s[i], o);
            }
            if (lane == 0) {
#pragma unroll
                for (int i = 0; i < DMAX; ++i)
                    if (i < d) gw[e0 + i] = s[i];
            }
        }
        __syncwarp();
    }
    if (gllr)
        for (int i = lane; i < n; i += 32) gllr[f * n + i] = gZ[i];
}

// out[j] = scale * sum over rows i of x[i][j], summed in a fixed order (the
// result does not depend on the launch).  Block: 32 columns x 32 row slices.
__global__ void __launch_bounds__(1024)
    sum_rows_kernel(const float *__restrict__ x, int64_t rows, int cols, float scale,
                    float *__restrict__ out) {
    __shared__ double part[32][33];
    const int col = blockIdx.x * 32 + threadIdx.x;
    double s0 = 0.0, s1 = 0.0;
    if (col < cols) {
        int64_t i = threadIdx.y;
        for (; i + 32 < rows; i += 64) {
            s0 += x[i * cols + col];
            s1 += x[(i + 32) * cols + col];
        }
        if (i < rows) s0 += x[i * cols + col];
    }
    part[threadIdx.y][threadIdx.x] = s0 + s1;
    __syncthreads();
    if (threadIdx.y == 0 && col < cols) {
        double s = 0.0;
        for (int k = 0; k < 32; ++k) s += part[k][threadIdx.x];
        out[col] = static_cast<float>(s * static_cast<double>(scale));
    }
}

// Adam (Kingma and Ba, 2015) on a flat parameter vector; c1 = 1 / (1 - b1^t)
// and c2 = 1 / (1 - b2^t) are the bias corrections of step t.
__global__ void adam_kernel(float *__restrict__ p, const float *__restrict__ g,
                            float *__restrict__ m, float *__restrict__ v, int64_t count, float lr,
                            float b1, float b2, float eps, float c1, float c2) {
    for (int64_t i = blockIdx.x * static_cast<int64_t>(blockDim.x) + threadIdx.x; i < count;
         i += static_cast<int64_t>(gridDim.x) * blockDim.x) {
        const float gi = g[i];
        const float mi = b1 * m[i] + (1.0f - b1) * gi;
        const float vi = b2 * v[i] + (1.0f - b2) * gi * gi;
        m[i] = mi;
        v[i] = vi;
        p[i] -= lr * (mi * c1) / (sqrtf(vi * c2) + eps);
    }
}

}  // namespace

// ---------------------------------------------------------------------------
// Host side
// ---------------------------------------------------------------------------
namespace {

ldpc_status bind_device(const Code &c) {
    cudaError_t e = cudaSetDevice(c.device);
    return e == cudaSuccess ? LDPC_OK : cuda_fail(e, "cudaSetDevice");
}

int zstride_of(const Code &c) { return (c.n + 3) & ~3; }
size_t backward_warp_floats(const Code &c) {
    return 2 * static_cast<size_t>(zstride_of(c)) + 2 * static_cast<size_t>(c.n_edges) * c.z;
}

int max_smem_optin(int device) {
    int v = 0;
    if (cudaDeviceGetAttribute(&v, cudaDevAttrMaxSharedMemoryPerBlockOptin, device) != cudaSuccess)
        v = 48 * 1024;
    return v;
}

// Frames per block (1..kTrainWarps): the count that keeps the most frames
// resident per SM, given the SM's shared memory and the 1 KB each block
// reserves; ties go to the larger block.  0 if one frame does not fit.
int warps_for(size_t warp_bytes, int device) {
    const size_t limit = static_cast<size_t>(max_smem_optin(device));
    if (warp_bytes > limit) return 0;
    int per_sm = 0;
    if (cudaDeviceGetAttribute(&per_sm, cudaDevAttrMaxSharedMemoryPerMultiprocessor, device) !=
        cudaSuccess)
        per_sm = static_cast<int>(limit);
    int best = 1, best_frames = 0;
    for (int w = 1; w <= kTrainWarps; ++w) {
        const size_t block = w * warp_bytes + 1024;
        if (w * warp_bytes > limit) break;
        const int frames = static_cast<int>(static_cast<size_t>(per_sm) / block) * w;
        if (frames >= best_frames) {
            best = w;
            best_frames = frames;
        }
    }
    return best;
}

ldpc_status check_common(const char *what, const ldpc_code *code, const float *d_llr,
                         const uint8_t *d_bits, int64_t frames, const float *d_w, int T) {
    if (!code) return fail(LDPC_ERR_INVALID_ARG, std::string(what) + ": code is NULL");
    if (frames < 0) return fail(LDPC_ERR_INVALID_ARG, std::string(what) + ": frames < 0");
    if (T < 1 || T > kMaxIters)
        return fail(LDPC_ERR_INVALID_ARG, std::string(what) + ": T outside 1..1000");
    if (frames > 0 && (!d_llr || !d_bits || !d_w))
        return fail(LDPC_ERR_INVALID_ARG, std::string(what) + ": NULL buffer");
    const Code &c = code->c;
    if (c.dslots == 0)
        return fail(LDPC_ERR_UNSUPPORTED,
                    std::string(what) + ": rows of more than 27 edges are not supported");
    return LDPC_OK;
}

bool aligned(const void *p, size_t a) { return (reinterpret_cast<uintptr_t>(p) % a) == 0; }

template <int DMAX>
ldpc_status launch_forward_t(const Code &c, const float *llr, const uint8_t *bits,
                             int64_t frames, const float *w, int T, float *post, uint32_t *rows,
                             float *loss, cudaStream_t s) {
    const int zs = zstride_of(c);
    const size_t warp_bytes = sizeof(float) * zs;
    const int wpb = warps_for(warp_bytes, c.device);
    if (wpb == 0) return fail(LDPC_ERR_UNSUPPORTED, "ldpc_learned_train_forward: code too large");
    const size_t smem = warp_bytes * wpb;
    cudaError_t e = allow_dynamic_smem(reinterpret_cast<const void *>(train_forward_kernel<DMAX>));
    if (e != cudaSuccess) return cuda_fail(e, "cudaFuncSetAttribute");
    const int64_t blocks = (frames + wpb - 1) / wpb;
    train_forward_kernel<DMAX><<<static_cast<unsigned>(blocks), 32 * wpb, smem, s>>>(
        dev_view(c), llr, bits, frames, w, T, post, reinterpret_cast<uint4 *>(rows), loss, zs);
    e = cudaGetLastError();
    return e == cudaSuccess ? LDPC_OK : cuda_fail(e, "train_forward_kernel");
}

template <int DMAX>
ldpc_status launch_backward_t(const Code &c, const float *llr, const uint8_t *bits,
                              int64_t frames, const float *w, int T, const float *post,
                              const uint32_t *rows, float loss_scale, float *gw_frame,
                              float *gllr, cudaStream_t s) {
    const int zs = zstride_of(c);
    const size_t wf = backward_warp_floats(c);
    const int wpb = warps_for(sizeof(float) * wf, c.device);
    if (wpb == 0) return fail(LDPC_ERR_UNSUPPORTED, "ldpc_learned_train_backward: code too large");
    const size_t smem = sizeof(float) * wf * wpb;
    cudaError_t e = allow_dynamic_smem(reinterpret_cast<const void *>(train_backward_kernel<DMAX>));
    if (e != cudaSuccess) return cuda_fail(e, "cudaFuncSetAttribute");
    const int64_t blocks = (frames + wpb - 1) / wpb;
    train_backward_kernel<DMAX><<<static_cast<unsigned>(blocks), 32 * wpb, smem, s>>>(
        dev_view(c), llr, bits, frames, w, T, post, reinterpret_cast<const uint4 *>(rows),
        loss_scale, gw_frame, gllr, zs, static_cast<int>(wf));
    e = cudaGetLastError();
    return e == cudaSuccess ? LDPC_OK : cuda_fail(e, "train_backward_kernel");
}

ldpc_status launch_sum_rows(const float *x, int64_t rows, int cols, float scale, float *out,
                            cudaStream_t s) {
    if (cols <= 0) return LDPC_OK;
    sum_rows_kernel<<<(cols + 31) / 32, dim3(32, 32), 0, s>>>(x, rows, cols, scale, out);
    cudaError_t e = cudaGetLastError();
    return e == cudaSuccess ? LDPC_OK : cuda_fail(e, "sum_rows_kernel");
}

}  // namespace
}  // namespace ldpc

using namespace ldpc;

extern "C" {

ldpc_status ldpc_learned_train_forward(const ldpc_code *code, const float *d_llr,
                                       const uint8_t *d_bits, int64_t frames,
                                       const float *d_weights, int T, float *d_post,
                                       uint32_t *d_rows, float *d_loss, float loss_scale,
                                       float *d_loss_sum, cudaStream_t stream) {
    static const char *kWhat = "ldpc_learned_train_forward";
    ldpc_status st = check_common(kWhat, code, d_llr, d_bits, frames, d_weights, T);
    if (st != LDPC_OK) return st;
    if (frames > 0 && (!d_post || !d_loss || (T > 1 && !d_rows)))
        return fail(LDPC_ERR_INVALID_ARG, std::string(kWhat) + ": NULL output buffer");
    if (d_rows && !aligned(d_rows, 16))
        return fail(LDPC_ERR_INVALID_ARG, std::string(kWhat) + ": d_rows not 16-byte aligned");
    const Code &c = code->c;
    if ((st = bind_device(c)) != LDPC_OK) return st;
    if (frames > 0) {
        switch (c.dslots) {
#define LDPC_TRAIN_FWD_CASE(D)                                                                 \
    case D:                                                                                    \
        st = launch_forward_t<D>(c, d_llr, d_bits, frames, d_weights, T, d_post, d_rows,       \
                                 d_loss, stream);                                              \
        break;
            LDPC_SLOT_CLASSES(LDPC_TRAIN_FWD_CASE)
#undef LDPC_TRAIN_FWD_CASE
            default:
                return fail(LDPC_ERR_UNSUPPORTED, std::string(kWhat) + ": row degree");
        }
        if (st != LDPC_OK) return st;
    }
    if (d_loss_sum) {
        if (frames == 0) {
            cudaError_t e = cudaMemsetAsync(d_loss_sum, 0, sizeof(float), stream);
            if (e != cudaSuccess) return cuda_fail(e, "cudaMemsetAsync");
            return LDPC_OK;
        }
        return launch_sum_rows(d_loss, frames, 1, loss_scale, d_loss_sum, stream);
    }
    return LDPC_OK;
}

size_t ldpc_learned_train_workspace_bytes(const ldpc_code *code, int64_t frames, int T) {
    if (!code || frames <= 0 || T < 1) return 0;
    return sizeof(float) * static_cast<size_t>(frames) * T * code->c.n_edges;
}

ldpc_status ldpc_learned_train_backward(const ldpc_code *code, const float *d_llr,
                                        const uint8_t *d_bits, int64_t frames,
                                        const float *d_weights, int T, const float *d_post,
                                        const uint32_t *d_rows, float loss_scale,
                                        float *d_grad_weights, float *d_grad_llr,
                                        void *d_workspace, size_t workspace_bytes,
                                        cudaStream_t stream) {
    static const char *kWhat = "ldpc_learned_train_backward";
    ldpc_status st = check_common(kWhat, code, d_llr, d_bits, frames, d_weights, T);
    if (st != LDPC_OK) return st;
    if (!d_grad_weights) return fail(LDPC_ERR_INVALID_ARG, std::string(kWhat) + ": NULL gradient");
    if (frames > 0 && (!d_post || (T > 1 && !d_rows) || !d_workspace))
        return fail(LDPC_ERR_INVALID_ARG, std::string(kWhat) + ": NULL buffer");
    if (d_rows && !aligned(d_rows, 16))
        return fail(LDPC_ERR_INVALID_ARG, std::string(kWhat) + ": d_rows not 16-byte aligned");
    if (workspace_bytes < ldpc_learned_train_workspace_bytes(code, frames, T))
        return fail(LDPC_ERR_INVALID_ARG, std::string(kWhat) + ": workspace too small");
    const Code &c = code->c;
    if ((st = bind_device(c)) != LDPC_OK) return st;
    const int cols = T * c.n_edges;
    if (frames == 0) {
        cudaError_t e = cudaMemsetAsync(d_grad_weights, 0, sizeof(float) * cols, stream);
        return e == cudaSuccess ? LDPC_OK : cuda_fail(e, "cudaMemsetAsync");
    }
    float *gw_frame = static_cast<float *>(d_workspace);
    switch (c.dslots) {
#define LDPC_TRAIN_BWD_CASE(D)                                                                 \
    case D:                                                                                    \
        st = launch_backward_t<D>(c, d_llr, d_bits, frames, d_weights, T, d_post, d_rows,      \
                                  loss_scale, gw_frame, d_grad_llr, stream);                   \
        break;
        LDPC_SLOT_CLASSES(LDPC_TRAIN_BWD_CASE)
#undef LDPC_TRAIN_BWD_CASE
        default:
            return fail(LDPC_ERR_UNSUPPORTED, std::string(kWhat) + ": row degree");
    }
    if (st != LDPC_OK) return st;
    return launch_sum_rows(gw_frame, frames, cols, 1.0f, d_grad_weights, stream);
}

ldpc_status ldpc_adam_step(float *d_param, const float *d_grad, float *d_m, float *d_v,
                           int64_t count, int step, float lr, float beta1, float beta2, float eps,
                           cudaStream_t stream) {
    if (count < 0 || step < 1 || !(beta1 >= 0.0f && beta1 < 1.0f) ||
        !(beta2 >= 0.0f && beta2 < 1.0f) || !(eps >= 0.0f))
        return fail(LDPC_ERR_INVALID_ARG, "ldpc_adam_step: bad count, step or coefficients");
    if (count == 0) return LDPC_OK;
    if (!d_param || !d_grad || !d_m || !d_v)
        return fail(LDPC_ERR_INVALID_ARG, "ldpc_adam_step: NULL buffer");
    const double c1 = 1.0 / (1.0 - std::pow(static_cast<double>(beta1), step));
    const double c2 = 1.0 / (1.0 - std::pow(static_cast<double>(beta2), step));
    const int threads = 256;
    const int64_t blocks = std::min<int64_t>((count + threads - 1) / threads, 4096);
    adam_kernel<<<static_cast<unsigned>(blocks), threads, 0, stream>>>(
        d_param, d_grad, d_m, d_v, count, lr, beta1, beta2, eps, static_cast<float>(c1),
        static_cast<float>(c2));
    cudaError_t e = cudaGetLastError();
    return e == cudaSuccess ? LDPC_OK : cuda_fail(e, "adam_kernel");
}

}  // extern "C"
