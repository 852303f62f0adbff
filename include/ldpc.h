/*
 * libldpc -- layered single-scan min-sum decoding and direct encoding of
 * QC-LDPC codes shaped like the IEEE 802.11 (Wi-Fi 6) and IEEE 802.16
 * (WiMAX) codes, on NVIDIA GB300 (sm_103a).
 *
 * The operations follow Palenik & Szitkey, "High Throughput Open-Source
 * Implementation of Wi-Fi 6 and WiMAX LDPC Encoder and Decoder"
 * (arXiv 2306.12063), cited below by section and equation.
 *
 * Conventions for every entry point:
 *  - Pointers named d_* are CUDA device pointers, h_* are host pointers.
 *    The caller owns every buffer; the library owns only the code handle and
 *    the small device tables inside it.
 *  - Work is enqueued on the given stream and returns before it runs.
 *    Argument errors are detected on the host and returned at once; nothing
 *    is enqueued then.  No call aborts, exits or traps.
 *  - A status other than LDPC_OK leaves a message for ldpc_last_error() on
 *    the calling thread.
 *  - Circulant convention: base-matrix entry s >= 0 at block (i, j) places
 *    the one of check row i*Z + r at variable j*Z + (r + s) mod Z.
 *  - Bits are one per byte (0/1) unless stated; packed hard decisions use
 *    bit (n % 32) of 32-bit word n / 32, ceil(N / 32) words per frame.
 *  - Hard decision, eq. (21): bit = 0 if the posterior is > 0, else 1.
 */
#ifndef LDPC_H
#define LDPC_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

/* The CUDA runtime's stream handle type (declared here so that this header
 * needs no CUDA include).  NULL is the legacy default stream. */
typedef struct CUstream_st *cudaStream_t;

typedef enum {
    LDPC_OK = 0,
    LDPC_ERR_INVALID_ARG = 1,    /* a pointer, size or flag is out of range */
    LDPC_ERR_BAD_STRUCTURE = 2,  /* base matrix lacks the eq. (3)-(7) shape */
    LDPC_ERR_NOMEM = 3,          /* a host or device allocation failed */
    LDPC_ERR_CUDA = 4,           /* a CUDA runtime call failed */
    LDPC_ERR_TIMEOUT = 5,        /* a bounded wait ran out */
    LDPC_ERR_UNSUPPORTED = 6     /* valid input outside what the kernels handle */
} ldpc_status;

typedef enum {
    LDPC_F32 = 0,   /* channel LLRs float[F][N]; posteriors float[F][N] */
    LDPC_I8X4 = 1,  /* channel LLRs int8 packed four frames per 32-bit word,
                       uint32[ceil(F/4)][N], byte b of word (g, n) = frame
                       4g + b; posteriors int8[F][N] */
    LDPC_I16W = 2   /* Section 5's fixed-point decoder: channel int16[F][N]
                       (ldpc_quantize_i16), int16 arithmetic with native
                       wrap-around (every Z_mn, |Z_mn|, message and Z_n is
                       reduced modulo 2^16 into [-32768, 32767], so
                       |-32768| = -32768); posteriors int16[F][N].  Only
                       ldpc_decode_layered_minsum takes it. */
} ldpc_dtype;

typedef struct ldpc_code ldpc_code;   /* opaque; created and freed here */

/* Selects the GPU that later calls (and code handles created afterwards)
 * use.  Call it once per host thread before the first ldpc_code_create when
 * the process uses a GPU other than 0. */
ldpc_status ldpc_set_device(int device);

/* Builds a code from its base (model) matrix H_bm (Section 1, eq. 2):
 * hbm is a host array, row-major mb x nb int16, entries -1 (zero block) or a
 * cyclic shift in [0, z).  The array is copied.
 * Requires 3 <= mb < nb <= 32, 1 <= z <= 384 and the parity structure the
 * direct encoder needs (eq. 3-7): column Kb = nb - mb (h_b) has equal
 * non-negative entries in rows 0 and mb-1 and exactly one more non-negative
 * entry, at a row y in 1..mb-2; columns Kb+1+t, t = 0..mb-2 (H_b2') hold 0
 * at rows t and t+1 and -1 elsewhere.  Otherwise LDPC_ERR_BAD_STRUCTURE.
 * On success *out receives a handle bound to the current device; it holds a
 * few kilobytes of device memory for the per-layer edge table. */
ldpc_status ldpc_code_create(const int16_t *hbm, int mb, int nb, int z,
                             ldpc_code **out);

/* Frees the handle (no-op on NULL).  Pending work that uses it must have
 * finished. */
void ldpc_code_destroy(ldpc_code *code);

/* N = nb z, K = (nb - mb) z, M = mb z, z, and the largest check-row degree
 * max g(m) (Section 1).  Any output pointer may be NULL. */
ldpc_status ldpc_code_info(const ldpc_code *code, int *n, int *k, int *m,
                           int *z, int *max_row_deg);

/* Synthetic info bits: bit k of frame f = frame0 + i is bit (k % 32) of
 * word (k / 32) % 4 of Philox4x32-10 (Salmon et al., SC'11) at counter
 * {k / 128, f mod 2^32, f / 2^32, 0} under key {seed mod 2^32,
 * (seed / 2^32) ^ 0x494E464F}.  d_info: uint8[frames][k]. */
ldpc_status ldpc_gen_info(uint64_t seed, int64_t frame0, int64_t frames, int k,
                          uint8_t *d_info, cudaStream_t stream);

/* Direct encoder of Section 2, eq. (8)-(15): d_info uint8[frames][K] (0/1)
 * -> d_code uint8[frames][N] = [info | v_0 | v_1 | ... | v_{Mb-1}] with
 * S_i = sum_j P_{H(i,j)} u_j (eq. 15), v_0 = P^{-1}_{H(y,Kb)} sum_i S_i
 * (eq. 12), v_1 = P_{H(0,Kb)} v_0 + S_0 (eq. 13) and
 * v_{i+1} = v_i + P_{H(i,Kb)} v_0 + S_i (eq. 14), all over GF(2). */
ldpc_status ldpc_encode(const ldpc_code *code, const uint8_t *d_info,
                        uint8_t *d_code, int64_t frames, cudaStream_t stream);

/* BPSK over AWGN and the channel LLR, eq. (16)-(17): for frame
 * f = frame0 + i and position n, g is Gaussian number n % 4 of the
 * Box-Muller pair-of-pairs drawn from Philox4x32-10 at counter
 * {n / 4, f mod 2^32, f / 2^32, 0} under key {seed mod 2^32,
 * (seed / 2^32) ^ 0x4E4F4953}; y = (1 - 2 c) + sigma g and
 * llr = y * llr_scale (llr_scale = 2 / sigma^2 for eq. 17).  The logarithm,
 * sine and cosine are evaluated with fixed series in correctly rounded
 * float arithmetic, so the output does not depend on the math library.
 * d_code uint8[frames][n] -> d_llr float[frames][n]. */
ldpc_status ldpc_awgn_llr(const uint8_t *d_code, int64_t frame0, int64_t frames,
                          int n, uint64_t seed, float sigma, float llr_scale,
                          float *d_llr, cudaStream_t stream);

/* Section 5's fixed-point channel: q = rint(clamp(scale * llr, -(2^qb - 1),
 * 2^qb - 1)) with round-half-to-even, stored as int16 (Q_B = qb; the paper's
 * default qb = 10 gives -1023..1023).  d_llr float[count] -> d_q int16[count];
 * 1 <= qb <= 14. */
ldpc_status ldpc_quantize_i16(const float *d_llr, int16_t *d_q, int64_t count, float scale,
                              int qb, cudaStream_t stream);

/* Bitmap encoder (Section 3, Alg. A1), for Z a multiple of 32: the direct
 * encoder of eq. (12)-(15) on packed words.  Bit r of block j sits at bit
 * (j Z + r) % 32 of word (j Z + r) / 32; each cyclic shift P_s (out bit r =
 * in bit (r + s) mod Z) is split as in Alg. A1 into s / 32 whole words and
 * s % 32 bits, combined in one pass over the block.  d_info
 * uint32[frames][K/32] -> d_code uint32[frames][N/32].  Z % 32 != 0 gives
 * LDPC_ERR_UNSUPPORTED. */
ldpc_status ldpc_encode_bitmap(const ldpc_code *code, const uint32_t *d_info, uint32_t *d_code,
                               int64_t frames, cudaStream_t stream);

/* Fixed-point channel input (Section 5, narrowed to 8 bits):
 * q = rint(clamp(scale * llr, -clip, clip)) with round-half-to-even, packed
 * four frames per word: d_llr float[frames][n] -> d_q uint32[ceil(frames/4)][n],
 * byte b of word (g, n) = frame 4g + b.  Bytes of frames >= frames (the pad
 * of the last group) are set to +clip.  0 <= clip <= 127. */
ldpc_status ldpc_quantize_pack_i8(const float *d_llr, uint32_t *d_q,
                                  int64_t frames, int n, float scale, int clip,
                                  cudaStream_t stream);

typedef struct {
    int max_iters;   /* 1..1000 full iterations */
    float alpha;     /* message scale when normalise = 1 (FP32 path) */
    int normalise;   /* 0: plain min-sum, eq. (23); 1: scaled messages.
                        LDPC_I8X4 scales by (3 |m|) >> 2 and requires
                        alpha == 0.75 */
    int early_stop;  /* 1: stop a frame after the first full iteration whose
                        hard decisions satisfy H x^T = 0 (Section 4, step 4) */
} ldpc_decode_params;

/* Layered single-scan min-sum decoding (Section 4, eq. 20, 22, 23): for
 * every iteration, block rows (layers) 0..Mb-1 in order; within a layer each
 * check row m computes Z_mn = Z_n - L_mn for its variables, the new
 * messages L_mn = s * min_{n' != n} |Z_mn'| * prod_{n' != n} sgn Z_mn' (s =
 * alpha or 1), and writes Z_n = Z_mn + L_mn.  Only the compressed messages
 * (two magnitudes, the argmin and the sign bits per row) are kept.
 *   d_llr   LDPC_F32: float[frames][N];  LDPC_I8X4: uint32[ceil(frames/4)][N]
 *           (as written by ldpc_quantize_pack_i8; int8 values must lie in
 *           [-127, 127]).  16-byte alignment enables the bulk-copy path.
 *   d_hard  uint32[frames][ceil(N/32)] hard decisions of eq. (21).
 *   d_iters int32[frames]: the iteration at which the syndrome became zero,
 *           or max_iters.
 *   d_post  NULL, or posteriors Z_n: float[frames][N] / int8[frames][N].
 * A frame that stops early has its outputs written at that iteration and
 * never changed afterwards.  LDPC_I8X4 saturates every Z_mn and Z_n to
 * [-127, 127].  Rows of degree above 27 are LDPC_ERR_UNSUPPORTED. */
ldpc_status ldpc_decode_layered_minsum(const ldpc_code *code, ldpc_dtype dtype,
                                       const void *d_llr, int64_t frames,
                                       const ldpc_decode_params *params,
                                       uint32_t *d_hard, int32_t *d_iters,
                                       void *d_post, cudaStream_t stream);

/* Learned (neural) normalised min-sum: the FP32 decoder above with the
 * message of eq. (23) scaled, in iteration k = 1..T, by a trained weight per
 * nonzero block of H_bm: L_mn = w[k-1][q] * min_{n' != n} |Z_mn'| *
 * prod sgn Z_mn', where q numbers the nonzero blocks of H_bm row by row in
 * increasing block column (q = 0 .. nnz(H_bm)-1).  The paper's decoder is
 * the special case of all weights 1 (eq. 23).  The weighted message is
 * applied with one rounding per update: Z_mn = Z_n - w' m_old and
 * Z_n = Z_mn + w m are fused multiply-adds (w' the weight m_old was made
 * with).  d_weights: device float[T][nnz(H_bm)]; at most T iterations, with
 * the syndrome stop when early_stop = 1.  Other arguments and layouts as in
 * ldpc_decode_layered_minsum with dtype LDPC_F32. */
ldpc_status ldpc_decode_learned_minsum(const ldpc_code *code, const float *d_llr,
                                       int64_t frames, const float *d_weights, int T,
                                       int early_stop, uint32_t *d_hard, int32_t *d_iters,
                                       float *d_post, cudaStream_t stream);

/* Run limits of the learned decoder beyond the weight table and a give-up
 * rule (extensions; the paper has neither).  Iteration k uses weight row
 * min(k, T) - 1, so iterations past the table's T rows repeat its last row.
 * With early_stop the unsatisfied checks u of the hard decisions are counted
 * after every iteration; a frame stops when u = 0 (eq. 21) or when k equals
 * stop_iter[j] (j = 0, 1; 0 = no checkpoint) and u > floor(stop_frac[j] * M),
 * the product rounded in FP32: a frame still far from a codeword there is
 * given up (its outputs are those of iteration k, its count k).
 * Checkpoints need early_stop = 1; stop_frac must be >= 0. */
typedef struct {
    int max_iters;       /* 1..1000 iterations at most; 0 = T (the table's rows) */
    int early_stop;      /* 0 or 1 */
    int stop_iter[2];    /* give-up checkpoints, 0..1000 (0 = none) */
    float stop_frac[2];  /* their limits as fractions of M */
} ldpc_learned_params;

/* ldpc_decode_learned_minsum with the run limits above (lp->max_iters may
 * exceed T).  With max_iters = T and no checkpoints it is
 * ldpc_decode_learned_minsum. */
ldpc_status ldpc_decode_learned_minsum_ex(const ldpc_code *code, const float *d_llr,
                                          int64_t frames, const float *d_weights, int T,
                                          const ldpc_learned_params *lp, uint32_t *d_hard,
                                          int32_t *d_iters, float *d_post, cudaStream_t stream);

/* Flooding min-sum (Section 4, eq. 18-21) in FP32, the schedule the layered
 * decoder improves on: each iteration first computes every check message
 * from the previous iteration's messages, Z_mn = Z_n^(0) + sum over the
 * variable's other checks of L (eq. 19, summed in increasing check index),
 * L_mn = s * min over the row's other edges of |Z_mn'| * their sign product
 * (eq. 18; s = alpha if normalise, else 1), then every posterior
 * Z_n = Z_n^(0) + sum of its L (eq. 20, increasing check index), and the
 * syndrome stop (eq. 21).  Arguments as for ldpc_decode_layered_minsum with
 * LDPC_F32.  Shared memory per frame is 4 (2 N + 2 nnz(H)) bytes; larger
 * codes return LDPC_ERR_UNSUPPORTED. */
ldpc_status ldpc_decode_flooding_minsum(const ldpc_code *code, const float *d_llr,
                                        int64_t frames, const ldpc_decode_params *params,
                                        uint32_t *d_hard, int32_t *d_iters, float *d_post,
                                        cudaStream_t stream);

/* Device workspace bytes of ldpc_decode_learned_fallback for `frames`. */
size_t ldpc_learned_fallback_workspace_bytes(const ldpc_code *code, int64_t frames);

/* Learned decoding with a plain min-sum fallback: ldpc_decode_learned_minsum
 * (T iterations, syndrome stop), then every frame whose hard decisions still
 * violate a parity check (Section 4, step 4) is decoded again from its
 * channel LLRs by the int8 decoder with `fallback` parameters (channel
 * quantised as in ldpc_quantize_pack_i8 with quant_scale, quant_clip), and
 * its outputs replace the learned ones; its d_iters entry becomes T plus the
 * fallback's count.  *h_fallback_frames receives the number of such frames:
 * the call reads it back and so waits for the learned pass to finish.
 * d_workspace: ldpc_learned_fallback_workspace_bytes bytes of device memory. */
ldpc_status ldpc_decode_learned_fallback(const ldpc_code *code, const float *d_llr,
                                         int64_t frames, const float *d_weights, int T,
                                         const ldpc_decode_params *fallback,
                                         float quant_scale, int quant_clip,
                                         uint32_t *d_hard, int32_t *d_iters,
                                         int64_t *h_fallback_frames, void *d_workspace,
                                         size_t workspace_bytes, cudaStream_t stream);

/* ---- Training of the learned weights (the paper has no counterpart: it
 * decodes with fixed messages; this is the unrolled layered decoder of
 * Section 4 differentiated in reverse mode). ---- */

/* Training forward: exactly T iterations of the learned decoder (no
 * syndrome stop) on every frame, with the weighted message w m rounded
 * before it is added or subtracted (the form the gradients below are exact
 * for; inference fuses the two), and its loss
 *   loss[f] = sum over t = 1..T and n of BCE(sigmoid(-Z_n^(t)), c_n)
 *           = softplus(-Z) + c Z,
 * the cross-entropy of each iteration's posterior bit probability against
 * the sent bit.  Inputs: d_llr float[frames][n]; d_bits uint8[frames][n]
 * (0/1 code bits); d_weights float[T][nnz(H_bm)] (as in
 * ldpc_decode_learned_minsum).  Outputs, kept for the backward pass:
 * d_post float[T][frames][n] = Z^(1..T); d_rows uint32[T-1][frames][m][4],
 * 16-byte aligned, the compressed row state after iterations 1..T-1
 * (unscaled smallest and second smallest |Z_mn| as float bits, argmin
 * edge, message sign bits; may be NULL when T = 1); d_loss float[frames];
 * d_loss_sum (float[1] or NULL) = loss_scale * sum_f d_loss[f], summed in a
 * fixed order. */
ldpc_status ldpc_learned_train_forward(const ldpc_code *code, const float *d_llr,
                                       const uint8_t *d_bits, int64_t frames,
                                       const float *d_weights, int T, float *d_post,
                                       uint32_t *d_rows, float *d_loss, float loss_scale,
                                       float *d_loss_sum, cudaStream_t stream);

/* Device workspace bytes of ldpc_learned_train_backward (one gradient row
 * per frame: frames * T * nnz(H_bm) floats). */
size_t ldpc_learned_train_workspace_bytes(const ldpc_code *code, int64_t frames, int T);

/* Training backward: gradients of loss_scale * sum_f loss[f] with respect
 * to the weights (d_grad_weights float[T][nnz(H_bm)], overwritten; the sum
 * over frames is taken in a fixed order, so the result is reproducible) and,
 * if d_grad_llr is not NULL, to the channel LLRs (float[frames][n]).  Takes
 * the forward's inputs and its d_post / d_rows unchanged.  The derivative of
 * |x| is sign(x); the smallest |Z_mn| of a row passes its gradient to the
 * first edge attaining it, the second smallest to the first attaining edge
 * among the others (one subgradient at exact ties); signs have derivative 0.
 * Shared memory per frame is 4 (2 n + 2 nnz(H)) bytes, so codes above the
 * device limit return LDPC_ERR_UNSUPPORTED. */
ldpc_status ldpc_learned_train_backward(const ldpc_code *code, const float *d_llr,
                                        const uint8_t *d_bits, int64_t frames,
                                        const float *d_weights, int T, const float *d_post,
                                        const uint32_t *d_rows, float loss_scale,
                                        float *d_grad_weights, float *d_grad_llr,
                                        void *d_workspace, size_t workspace_bytes,
                                        cudaStream_t stream);

/* One Adam step (Kingma and Ba, 2015) on count floats, step = 1, 2, ...:
 * m = b1 m + (1 - b1) g, v = b2 v + (1 - b2) g^2,
 * p -= lr (m / (1 - b1^step)) / (sqrt(v / (1 - b2^step)) + eps).
 * All four arrays are device memory, updated in place. */
ldpc_status ldpc_adam_step(float *d_param, const float *d_grad, float *d_m, float *d_v,
                           int64_t count, int step, float lr, float beta1, float beta2,
                           float eps, cudaStream_t stream);

/* Per-frame noise level for training batches: for frame f = frame0 + i,
 * Eb/N0 (dB) = lo + (hi - lo) u with u = ((x >> 8) + 1/2) / 2^24, x word 0 of
 * Philox4x32-10 at counter {0, f mod 2^32, f / 2^32, 0} under key
 * {seed mod 2^32, (seed / 2^32) ^ 0x534E5253}; then
 * d_sigma[i] = sqrt(1 / (2 rate 10^(Eb/N0 / 10))), computed in double
 * precision from the float arguments, each operation rounded once, and
 * rounded to float. */
ldpc_status ldpc_snr_sigma(uint64_t seed, int64_t frame0, int64_t frames, float ebn0_lo_db,
                           float ebn0_hi_db, float rate, float *d_sigma, cudaStream_t stream);

/* ldpc_awgn_llr with a noise level per frame: frame i uses
 * sigma = d_sigma[i] and llr_scale = 2 / sigma^2 (eq. 17; each float
 * operation rounded once).  d_sigma float[frames], device memory. */
ldpc_status ldpc_awgn_llr_frames(const uint8_t *d_code, int64_t frame0, int64_t frames,
                                 int n, uint64_t seed, const float *d_sigma, float *d_llr,
                                 cudaStream_t stream);

/* ---- Mixed-code batches (no counterpart in the paper, which decodes one
 * code per call): frames of several codes decoded together. ---- */

typedef struct ldpc_codeset ldpc_codeset;         /* opaque */
typedef struct ldpc_mixed_plan ldpc_mixed_plan;   /* opaque */
typedef struct ldpc_mixed_graph ldpc_mixed_graph; /* opaque */

/* A set of 1..4096 codes (host array of handles, all on one device; the
 * handles must outlive the set).  The kernel-side descriptor of each code
 * (sizes and device table pointers) is copied to device memory. */
ldpc_status ldpc_codeset_create(const ldpc_code *const *codes, int count, ldpc_codeset **out);
void ldpc_codeset_destroy(ldpc_codeset *set);

/* A batch layout: frame f = 0..frames-1 uses code h_code_of_frame[f] (an
 * index into the set; host array, copied).  Buffers of a mixed batch hold
 * the frames back to back in frame order: LLRs (float, or int8 posteriors)
 * from element llr_off[f] = sum over earlier frames of N, info bits (uint8)
 * from info_off[f] = sum of K, hard decisions (uint32) from hard_off[f] =
 * sum of ceil(N/32) words, iteration counts int32[frames].  Internally the
 * frames are grouped by code (each code's run padded to a multiple of four
 * frames) and the codes are split into launch groups: one per slot class of
 * the largest row degree (8, 12, 16, 20, 24, 27), split further so that
 * shared memory within a group differs by at most a factor of two, ordered
 * by work (frames x edges), heaviest first.  The set must outlive the
 * plan. */
ldpc_status ldpc_mixed_plan_create(const ldpc_codeset *set, const int32_t *h_code_of_frame,
                                   int64_t frames, ldpc_mixed_plan **out);
void ldpc_mixed_plan_destroy(ldpc_mixed_plan *plan);

/* Buffer sizes of the plan: LLR elements, info bytes, hard-decision words,
 * packed int8 words (ldpc_mixed_quantize) and the number of launch groups.
 * Any output pointer may be NULL. */
ldpc_status ldpc_mixed_plan_sizes(const ldpc_mixed_plan *plan, int64_t *llr_elems,
                                  int64_t *info_elems, int64_t *hard_words, int64_t *q_words,
                                  int *launch_groups);

/* The per-frame offsets (host arrays of frames + 1 int64 each, the last
 * entry the total; any may be NULL). */
ldpc_status ldpc_mixed_plan_offsets(const ldpc_mixed_plan *plan, int64_t *h_llr_off,
                                    int64_t *h_info_off, int64_t *h_hard_off);

/* Launch group `group`: slot class, number of codes, shared-memory bytes per
 * block (FP32 / int8), frames per work item and resident-block cap per SM
 * (0 = occupancy limit) as currently chosen.  Outputs may be NULL. */
ldpc_status ldpc_mixed_group_info(const ldpc_mixed_plan *plan, int group, int *slot_class,
                                  int *codes, int *smem_f32, int *smem_i8, int *chunk_f32,
                                  int *chunk_i8, int *blocks_per_sm_f32, int *blocks_per_sm_i8);

/* Whether the plan launches its groups one after another on the caller's
 * stream (1) or concurrently on forked streams (0), per dtype; the autotuner
 * picks it.  Outputs may be NULL. */
ldpc_status ldpc_mixed_plan_serial(const ldpc_mixed_plan *plan, int *serial_f32, int *serial_i8);

/* int8 input of a mixed batch: each LLR quantised as in ldpc_quantize_pack_i8
 * (scale, clip) and packed four frames of the same code per word in the
 * plan's internal order; padding bytes are +clip.  d_llr float (plan
 * layout) -> d_q uint32[q_words]. */
ldpc_status ldpc_mixed_quantize(const ldpc_mixed_plan *plan, const float *d_llr, uint32_t *d_q,
                                float scale, int clip, cudaStream_t stream);

/* Layered min-sum decoding (as ldpc_decode_layered_minsum, same parameters
 * for every frame) of a mixed batch: LDPC_F32 reads d_in = LLRs (float, plan
 * layout; 16-byte aligned with every N a multiple of 4 enables the
 * bulk-copy path), LDPC_I8X4 reads the words of ldpc_mixed_quantize.  Each
 * launch group is one persistent kernel launch whose warps take work items
 * (runs of consecutive frames of one code, largest codes first) from an
 * atomic counter; the groups' launches are forked from `stream` onto the
 * plan's own streams and joined back, so later work on `stream` sees the
 * results.  d_hard, d_iters, d_post (NULL, or float / int8 at llr_off) in
 * the plan layout.  Calls on one plan must not overlap in time. */
ldpc_status ldpc_decode_mixed(ldpc_mixed_plan *plan, ldpc_dtype dtype, const void *d_in,
                              const ldpc_decode_params *params, uint32_t *d_hard,
                              int32_t *d_iters, void *d_post, cudaStream_t stream);

/* Error counts of a decoded mixed batch: d_counters int64[5 + max_iters] as
 * in ldpc_frame_stats over all frames; d_code_frame_errors (NULL or
 * int64[set size]) receives the frame errors per code of the set. */
ldpc_status ldpc_mixed_stats(const ldpc_mixed_plan *plan, const uint8_t *d_info,
                             const uint32_t *d_hard, const int32_t *d_iters, int max_iters,
                             int64_t *d_counters, int64_t *d_code_frame_errors,
                             cudaStream_t stream);

/* Autotuner: for each launch group in turn, picks the frames per work item
 * (FP32 1..32, int8 4..128) and then a resident-block cap per SM (none, 16,
 * 8, 4) that minimise the median time of `reps` decodes of this batch, the
 * other groups' choices held fixed; for FP32 then the warps per frame (1..3)
 * and frames per block (1, 2, 4) of each group, and finally concurrent or
 * serial groups.  Runs and synchronises `stream`; the choices stay in the
 * plan (ldpc_mixed_group_launch and ldpc_mixed_group_info report them). */
ldpc_status ldpc_mixed_autotune(ldpc_mixed_plan *plan, ldpc_dtype dtype, const void *d_in,
                                const ldpc_decode_params *params, uint32_t *d_hard,
                                int32_t *d_iters, int reps, cudaStream_t stream);

/* Assembly of a mixed batch from per-code buffers: the rows of code
 * `code`'s frames, stored consecutively in d_src in batch order, are copied
 * to their places in the plan layout of d_dst.  what = 0: float LLR rows
 * (N floats, at llr_off); 1: info bits (K bytes, at info_off); 2: code bits
 * (N bytes, at llr_off counted in bytes). */
ldpc_status ldpc_mixed_scatter(const ldpc_mixed_plan *plan, int code, int what,
                               const void *d_src, void *d_dst, cudaStream_t stream);

/* Learned weights of a mixed batch: h_weights[c] (device pointer to
 * float[T_c][nnz(H_bm of code c)], as for ldpc_decode_learned_minsum) and
 * h_T[c] = T_c for every code c of the set (host arrays of the set's size;
 * entries of codes without frames may be NULL / 0).  The pointers are copied;
 * the weight arrays must stay valid while the plan decodes with them. */
ldpc_status ldpc_mixed_set_weights(ldpc_mixed_plan *plan, const float *const *h_weights,
                                   const int32_t *h_T);

/* Learned normalised min-sum over a mixed batch: every frame decoded by the
 * learned FP32 decoder of its code (at most T_c iterations, syndrome stop if
 * early_stop) in the plan's launches.  d_llr float (plan layout); d_hard,
 * d_iters, d_post (NULL or float at llr_off) in the plan layout. */
ldpc_status ldpc_decode_mixed_learned(ldpc_mixed_plan *plan, const float *d_llr, int early_stop,
                                      uint32_t *d_hard, int32_t *d_iters, float *d_post,
                                      cudaStream_t stream);

/* ldpc_decode_mixed_learned with the run limits of ldpc_learned_params
 * (lp->max_iters = 0: T_c per code; otherwise every code runs up to
 * lp->max_iters iterations, rows past T_c repeating its last row; the
 * give-up limits are fractions of each code's M). */
ldpc_status ldpc_decode_mixed_learned_ex(ldpc_mixed_plan *plan, const float *d_llr,
                                         const ldpc_learned_params *lp, uint32_t *d_hard,
                                         int32_t *d_iters, float *d_post, cudaStream_t stream);

/* ldpc_mixed_autotune for the learned decoder: the learned launches share
 * the FP32 launches' work items, residency caps and concurrency; this tunes
 * them by timing ldpc_decode_mixed_learned_ex with `lp` (so the FP32 plain
 * decoder runs with them afterwards too).  Needs ldpc_mixed_set_weights. */
ldpc_status ldpc_mixed_autotune_learned(ldpc_mixed_plan *plan, const float *d_llr,
                                        const ldpc_learned_params *lp, uint32_t *d_hard,
                                        int32_t *d_iters, int reps, cudaStream_t stream);

/* Launch settings of one launch group (not in the paper: tuning of the
 * batched decoders).  frames_per_item: frames per work item taken from the
 * group's counter; blocks_per_sm: resident blocks per SM, 0 = as many as fit;
 * warps_per_frame (FP32, 1..3): warps that decode one frame together, each
 * taking every warps_per_frame-th round of a layer's rows, with a barrier
 * between layers; frames_per_block (FP32, 1..4): such teams per block.  The
 * int8 launches use 1 and 1.  The FP32 settings also serve the learned
 * launches. */
typedef struct {
    int frames_per_item;
    int blocks_per_sm;
    int warps_per_frame;
    int frames_per_block;
} ldpc_group_launch;

/* Reads (get) and/or replaces (set) the settings of `group` for `dtype`;
 * either pointer may be NULL.  ldpc_mixed_autotune searches the same
 * settings.  Results do not depend on them. */
ldpc_status ldpc_mixed_group_launch(ldpc_mixed_plan *plan, int group, ldpc_dtype dtype,
                                    const ldpc_group_launch *set, ldpc_group_launch *get);

/* d_bad uint8[frames]: 1 where a frame's hard decisions (plan layout)
 * violate a parity check (eq. 21 termination test), else 0. */
ldpc_status ldpc_mixed_frame_flags(const ldpc_mixed_plan *plan, const uint32_t *d_hard,
                                   uint8_t *d_bad, cudaStream_t stream);

/* Moves frames between two plans of the same code set, where frame s of
 * plan B is frame d_index[s] (int64, device) of plan A: what = 0 copies LLR
 * rows A -> B (float, plan layouts), 1 copies hard-decision rows B -> A,
 * 2 writes iteration counts B -> A adding T_c of plan A's weights (the
 * fallback's count after T_c learned iterations). */
ldpc_status ldpc_mixed_move_frames(const ldpc_mixed_plan *plan_a, const ldpc_mixed_plan *plan_b,
                                   const int64_t *d_index, int what, void *d_a, void *d_b,
                                   cudaStream_t stream);

/* Paired outcomes of two decoders over a mixed batch (as
 * ldpc_paired_frame_errors): d_counts int64[4] = both right, only B wrong,
 * only A wrong, both wrong. */
ldpc_status ldpc_mixed_paired_errors(const ldpc_mixed_plan *plan, const uint8_t *d_info,
                                     const uint32_t *d_hard_a, const uint32_t *d_hard_b,
                                     int64_t *d_counts, cudaStream_t stream);

/* A CUDA graph of one whole step on fixed buffers: [LDPC_I8X4: quantise
 * d_llr into d_q] -> the decode launches of every group (parallel branches)
 * -> [if d_counters: ldpc_mixed_stats against d_info with max_iters =
 * params->max_iters].  Captured from the plan's current choices; replay with
 * ldpc_mixed_graph_launch.  The plan and the buffers must outlive it. */
ldpc_status ldpc_mixed_graph_create(ldpc_mixed_plan *plan, ldpc_dtype dtype, const float *d_llr,
                                    uint32_t *d_q, float quant_scale, int quant_clip,
                                    const ldpc_decode_params *params, uint32_t *d_hard,
                                    int32_t *d_iters, const uint8_t *d_info, int64_t *d_counters,
                                    int64_t *d_code_frame_errors, ldpc_mixed_graph **out);
ldpc_status ldpc_mixed_graph_launch(ldpc_mixed_graph *graph, cudaStream_t stream);
void ldpc_mixed_graph_destroy(ldpc_mixed_graph *graph);

/* Error counts of decoded frames against the sent info bits (the
 * evaluation of Section 6.1).  d_counters int64[4 + max_iters + 1] is
 * overwritten with: [0] info-bit errors, [1] frame errors (any info bit
 * wrong), [2] undetected frame errors (hard decisions satisfy every check
 * but the info bits are wrong), [3] sum of d_iters, [4 + t] number of frames
 * with d_iters == t. */
ldpc_status ldpc_frame_stats(const ldpc_code *code, const uint8_t *d_info,
                             const uint32_t *d_hard, const int32_t *d_iters,
                             int64_t frames, int max_iters, int64_t *d_counters,
                             cudaStream_t stream);

/* Paired outcomes of two decoders on the same frames (for the McNemar
 * comparison of their frame-error rates): d_counts int64[4] is overwritten
 * with [0] both right, [1] only B wrong, [2] only A wrong, [3] both wrong,
 * where a frame is wrong when any of its K info bits (the first K hard
 * decisions) differs from d_info uint8[frames][K].  d_hard_a, d_hard_b as
 * written by the decoders. */
ldpc_status ldpc_paired_frame_errors(const ldpc_code *code, const uint8_t *d_info,
                                     const uint32_t *d_hard_a, const uint32_t *d_hard_b,
                                     int64_t frames, int64_t *d_counts, cudaStream_t stream);

/* Device bytes that ldpc_decode_host needs as workspace for a given chunk
 * of frames (a multiple of 4). */
size_t ldpc_decode_host_workspace_bytes(const ldpc_code *code, ldpc_dtype dtype,
                                        int64_t chunk_frames);

/* End-to-end decode of host-resident data: copies h_llr to the device in
 * chunks of chunk_frames frames, decodes each chunk, and copies hard
 * decisions and iteration counts back, overlapping the copies of one chunk
 * with the decoding of the next on two internal streams ordered after and
 * before `stream`.  The first chunk is a quarter of chunk_frames (rounded
 * up to a multiple of 4), so that decoding starts after a short copy.  Host buffers should be page-locked for the copies to run
 * asynchronously.  d_workspace must hold ldpc_decode_host_workspace_bytes.
 * Layouts as in ldpc_decode_layered_minsum (no posteriors). */
ldpc_status ldpc_decode_host(const ldpc_code *code, ldpc_dtype dtype,
                             const void *h_llr, int64_t frames,
                             const ldpc_decode_params *params,
                             uint32_t *h_hard, int32_t *h_iters,
                             void *d_workspace, size_t workspace_bytes,
                             int64_t chunk_frames, cudaStream_t stream);

/* Waits for `stream` to drain, polling for at most timeout_s seconds
 * (LDPC_ERR_TIMEOUT if it has not), then reads the handle's device status
 * word: a kernel whose bounded wait on a bulk copy ran out reports it there
 * and the call returns LDPC_ERR_TIMEOUT.  The status word is cleared. */
ldpc_status ldpc_sync(const ldpc_code *code, cudaStream_t stream,
                      double timeout_s);

/* The decoder of ldpc_decode_layered_minsum for callers that cannot allocate
 * device memory (no counterpart in the paper: it exists for integration).
 * Creating a code handle allocates its tables with cudaMalloc; some callers
 * cannot do that -- a real-time thread with a fixed memory budget, a process
 * whose framework owns every device allocation (a caching allocator or a
 * pool that accounts for each byte), or a steady-state path where cudaMalloc
 * and cudaFree, which can synchronise the device, are not allowed.  This
 * call takes the base matrix itself (host array, same rules as
 * ldpc_code_create) plus the caller's own buffers, laid out as for
 * ldpc_decode_layered_minsum, and allocates nothing: no cudaMalloc, cudaFree
 * or allocating library routine.  Its scratch (the per-lane offset table,
 * the work counter and the status word) lives in a 64 KiB static device
 * array that each GPU loading the library holds until the process exits;
 * codes whose offset table, mb * ceil(z/32) * slots * 64 bytes (slots = 8,
 * 12, 16, 20, 24 or 27, the smallest that holds the largest row degree),
 * exceeds 65280 bytes are rejected with LDPC_ERR_UNSUPPORTED.  Each call
 * clears the counter and status word and rewrites the table on `stream`
 * before decoding.  All calls on a device share the one array and it keeps
 * the last call's contents, so calls whose GPU work overlaps (on different
 * streams or from different host threads) race; serialise them.
 * Unlike the other decode calls this one is synchronous: with no handle
 * there is no ldpc_sync, so it waits for `stream` to drain and reads the
 * status word itself, returning LDPC_ERR_TIMEOUT when a kernel's bounded
 * wait for its bulk copy ran out (those frames are not decoded) and
 * LDPC_ERR_CUDA for a debug-build offset check.  Each call looks up the
 * array's device address (cudaGetSymbolAddress); the first lookup on a
 * device loads the library's device code, so make the first call before
 * any stream capture. */
ldpc_status ldpc_decode_layered_minsum_noalloc(const int16_t *hbm, int mb, int nb, int z,
                                               ldpc_dtype dtype, const void *d_llr,
                                               int64_t frames,
                                               const ldpc_decode_params *params,
                                               uint32_t *d_hard, int32_t *d_iters,
                                               void *d_post, cudaStream_t stream);

/* Failure-path check (no counterpart in the paper): one warp waits, with
 * the decoders' bounded wait of `polls` polls (1..2^22), on a bulk-copy
 * barrier that expects bytes no copy will deliver; the wait gives up, the
 * kernel sets the code's device status word and returns.  A following
 * ldpc_sync reports LDPC_ERR_TIMEOUT (and clears the word); the context
 * stays usable.  Nothing faults, traps or hangs. */
ldpc_status ldpc_check_bounded_wait(const ldpc_code *code, uint32_t polls,
                                    cudaStream_t stream);

/* Debug builds (-DLDPC_DEBUG) only: the number of clamps to [-127, 127]
 * that the single-code int8 decoder took on real edges of decoded frames
 * (eq. 22 and eq. 20 results, as the oracle counts them) since the last
 * call; waits for `stream`, then reads and clears the count.  Release
 * builds, which keep the decoder's instruction budget, return
 * LDPC_ERR_UNSUPPORTED.  Saturation is the int8 decoder's specified
 * arithmetic; the count tells how often it acted. */
ldpc_status ldpc_debug_saturation_count(const ldpc_code *code, cudaStream_t stream,
                                        int64_t *count);

/* Testing aid (no counterpart in the paper): caps the number of blocks in
 * the persistent grids of the single-code FP32, int8, int16 and learned
 * decode kernels for every later launch in the process; 0 (the default)
 * removes the cap.  Under a small cap each block decodes many frames, which
 * drives the dynamic frame hand-out (per byte or 16-bit lane for the packed
 * decoders) on small batches.
 * A negative cap returns LDPC_ERR_INVALID_ARG. */
ldpc_status ldpc_test_set_grid_cap(int blocks);

/* Message for the last failed call on this thread ("" if none). */
const char *ldpc_last_error(void);

#ifdef __cplusplus
}
#endif

#endif /* LDPC_H */
