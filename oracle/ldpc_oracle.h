/*
 * CPU oracle for layered min-sum QC-LDPC decoding and direct encoding.
 *
 * TEST INFRASTRUCTURE ONLY.  This is a plain, slow, single-threaded C
 * restatement of Palenik & Szitkey, "High Throughput Open-Source
 * Implementation of Wi-Fi 6 and WiMAX LDPC Encoder and Decoder"
 * (arXiv 2306.12063).  It exists to check the CUDA library against; it shares
 * no code, header or table with it, and the library never calls it.
 *
 * Conventions (the paper leaves the circulant direction open):
 *   H_bm(i,j) = s >= 0 expands to the Z x Z block P_s with
 *   P_s[r][(r + s) mod Z] = 1, i.e. (P_s u)[r] = u[(r + s) mod Z].
 *   Variable n = j*Z + c is column c of block column j; check m = i*Z + r.
 *   Hard decisions (eq. 21): bit = 0 if Z_n > 0, else 1.
 *   Packed hard bits: bit (n % 32) of word n / 32, words [F][ceil(N/32)].
 *
 * Every function returns 0 on success or a positive status code.
 *
 * Pins (CPU tests that fix each part against the paper or the mathematics,
 * not against itself):
 *   code set-up, encoder: H c^T = 0 over the explicit H, systematic form,
 *     linearity, equality with a textbook GF(2) elimination, the hand-worked
 *     Z = 2 example (tests/test_oracle_encoder.py, tests/golden/);
 *   Philox, Box-Muller, channel, quantisers: published known-answer vectors,
 *     distribution and rounding properties (tests/test_oracle_channel.py);
 *   layered FP32 / int8 decoders: the hand-worked Z = 2 traces, one-iteration
 *     recovery of noiseless input, single-parity-check ML, brute-force ML
 *     bounds, FP32 = int8 where nothing saturates, the counted saturations
 *     (tests/test_oracle_decoder.py);
 *   weighted (learned) decoder: the worked example with weights, constant
 *     weights = the alpha decoder (tests/test_oracle_decoder.py); the
 *     inference form (fused updates, run past its table, give-up
 *     checkpoints): an exact-rational trace on tiny codes, power-of-two
 *     weights = the alpha decoder, equal to an explicitly extended table, to
 *     a shorter decode where a checkpoint always fires, to the plain run
 *     where it never does, and checkpoint decisions against syndrome
 *     weights from a dense H (tests/test_oracle_learned_gated.py);
 *   flooding: equal to layered on one layer (tests/test_oracle_decoder.py);
 *   int16 wrap decoder, bitmap encoder: hand-worked overflow traces, FP32 /
 *     int8 equivalence without overflow, brute-force rotation, the byte
 *     encoder (tests/test_oracle_variants.py, tests/golden/).
 * FER values of the seeded stand-in codes are parity unpinned: the standard
 * matrices and the paper's reference decoder are not available.
 */
#ifndef LDPC_ORACLE_H
#define LDPC_ORACLE_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

enum {
    LDPC_REF_OK = 0,
    LDPC_REF_ERR_INVALID_ARG = 1,
    LDPC_REF_ERR_BAD_STRUCTURE = 2,
    LDPC_REF_ERR_NOMEM = 3,
    LDPC_REF_ERR_UNSUPPORTED = 6
};

typedef struct ldpc_ref_code ldpc_ref_code;

/* Build a code from its base matrix (eq. 2), host row-major mb*nb int16.
 * Entries must lie in [-1, z).  If require_encodable, the parity part must
 * have the structure of eq. (3)-(7) (h_b paired first/last entries, one more
 * non-negative entry at a row y in 1..mb-2, dual diagonal of zeros), else
 * LDPC_REF_ERR_BAD_STRUCTURE.  Without it any base matrix is accepted and
 * only the decoders may be used. */
int ldpc_ref_code_create(const int16_t *hbm, int mb, int nb, int z,
                         int require_encodable, ldpc_ref_code **out);
void ldpc_ref_code_destroy(ldpc_ref_code *code);
/* n, k, m, z, max row degree, y (-1 if not encodable), encodable flag. */
int ldpc_ref_code_info(const ldpc_ref_code *code, int *n, int *k, int *m,
                       int *z, int *max_row_deg, int *y, int *encodable);
/* Variables N(m) of check row m (Section 1), in increasing block column;
 * writes at most cap entries and returns the degree g(m) (or -1). */
int ldpc_ref_row_vars(const ldpc_ref_code *code, int row, int *vars, int cap);

/* Direct encoder, eq. (8)-(15): info u8[frames][K] (0/1) ->
 * codeword u8[frames][N] = [info | v_0 | v_1 | ... | v_{Mb-1}]. */
int ldpc_ref_encode(const ldpc_ref_code *code, const uint8_t *info,
                    uint8_t *cw, int64_t frames);
/* Number of unsatisfied checks of one word bits u8[N] (0 means H x^T = 0). */
int ldpc_ref_syndrome_weight(const ldpc_ref_code *code, const uint8_t *bits);

/* Philox4x32-10 (Salmon, Moraes, Dror & Shaw, SC'11). */
void ldpc_ref_philox4x32_10(const uint32_t ctr[4], const uint32_t key[2],
                            uint32_t out[4]);
/* Uniform info bits: bit k of frame f is bit (k % 32) of word (k / 32) % 4 of
 * Philox(ctr = {k / 128, f_lo, f_hi, 0}, key = {seed_lo, seed_hi ^ 0x494E464F}). */
int ldpc_ref_gen_info(uint64_t seed, int64_t frame0, int64_t frames, int k,
                      uint8_t *info);
/* Standard normal pair by Box-Muller from two Philox words; the logarithm
 * and the sine/cosine are evaluated with the series given in ldpc_oracle.c
 * using only correctly rounded float + - * / sqrt. */
void ldpc_ref_box_muller(uint32_t w0, uint32_t w1, float *g0, float *g1);
float ldpc_ref_lnf(float u);
void ldpc_ref_sincos_turn(uint32_t k24, float *s, float *c);
/* BPSK + AWGN + channel LLR, eq. (16)-(17): for frame f = frame0 + i and
 * position n, g = Gaussian number n % 4 of noise call n / 4 (Philox ctr =
 * {n / 4, f_lo, f_hi, 0}, key = {seed_lo, seed_hi ^ 0x4E4F4953}),
 * y = (1 - 2 c) + sigma * g, llr = y * llr_scale (llr_scale = 2 / sigma^2).
 * cw u8[frames][n], llr f32[frames][n]. */
int ldpc_ref_awgn_llr(const uint8_t *cw, int64_t frame0, int64_t frames, int n,
                      uint64_t seed, float sigma, float llr_scale, float *llr);

/* Fixed-point channel input: q = rint(clamp(scale * llr, -clip, clip)),
 * round half to even. */
int ldpc_ref_quantize_i8(const float *llr, int8_t *q, int64_t count,
                         float scale, int clip);

typedef struct {
    int max_iters;   /* >= 1 */
    float alpha;     /* normalisation factor, FP32 decoder */
    int normalise;   /* 0: plain min-sum (eq. 23); 1: scaled messages */
    int early_stop;  /* 1: stop at the first iteration with H x^T = 0 */
} ldpc_ref_params;

/* Layered single-scan min-sum (Section 4, eq. 20, 22, 23), FP32.
 * llr f32[frames][N]; hard u32[frames][ceil(N/32)]; iters i32[frames];
 * post f32[frames][N] or NULL. */
int ldpc_ref_decode_layered_f32(const ldpc_ref_code *code, const float *llr,
                                int64_t frames, const ldpc_ref_params *p,
                                uint32_t *hard, int32_t *iters, float *post);
/* The same schedule in saturating int8 (values in [-127, 127]); normalise
 * means m -> (3 m) >> 2 and requires alpha == 0.75.  sat_events (or NULL)
 * receives the number of clamps taken. */
int ldpc_ref_decode_layered_i8(const ldpc_ref_code *code, const int8_t *llr,
                               int64_t frames, const ldpc_ref_params *p,
                               uint32_t *hard, int32_t *iters, int8_t *post,
                               int64_t *sat_events);
/* Learned (neural) normalised min-sum: the layered decoder above with the
 * message of eq. (23) scaled by one weight per iteration and nonzero block of
 * H_bm, L_mn = w[k-1][q] * min_{n' != n} |Z_mn'| * prod sgn, where q numbers
 * the nonzero blocks of H_bm row by row in increasing block column and
 * k = 1..T.  weights f32[T][nnz(H_bm)]; at most T iterations, syndrome stop
 * if early_stop.  Outputs as for ldpc_ref_decode_layered_f32. */
int ldpc_ref_decode_layered_weighted_f32(const ldpc_ref_code *code, const float *llr,
                                         int64_t frames, const float *weights, int T,
                                         int early_stop, uint32_t *hard, int32_t *iters,
                                         float *post);
/* The learned decoder as the library runs it for inference (extensions, not
 * in the paper): the message of edge e in iteration k is w[row][q] * m with
 * m the eq. (23) min-sum message and row = min(k, T) - 1, so iterations
 * past T repeat the last row; the posterior updates Z_mn = Z_n - w' m_old
 * (w' the weight m_old was made with) and Z_n = Z_mn + w m are each rounded
 * once (fused multiply-add, C99 fmaf).  The weighted decoder above rounds
 * w * m first (the training arithmetic).  With early_stop the unsatisfied
 * checks u of the hard decisions are counted after every iteration; the
 * frame stops at iteration k when u = 0, or when k equals stop_iter[j]
 * (j = 0, 1; 0 means no checkpoint) and u > floor(stop_frac[j] * M) with
 * the product rounded in FP32.  stop_iter / stop_frac may be NULL (no
 * checkpoints); checkpoints need early_stop. */
int ldpc_ref_decode_learned_f32(const ldpc_ref_code *code, const float *llr, int64_t frames,
                                const float *weights, int T, int max_iters, int early_stop,
                                const int *stop_iter, const float *stop_frac, uint32_t *hard,
                                int32_t *iters, float *post);
/* Flooding min-sum, eq. (18)-(21), FP32: all checks from the previous
 * iteration's variable messages, then all posteriors. */
int ldpc_ref_decode_flooding_f32(const ldpc_ref_code *code, const float *llr,
                                 int64_t frames, const ldpc_ref_params *p,
                                 uint32_t *hard, int32_t *iters, float *post);

/* Section 5's fixed-point channel: q = rint(clamp(scale * llr, -(2^qb - 1),
 * 2^qb - 1)), round half to even, stored in int16 (qb = 10: -1023..1023). */
int ldpc_ref_quantize_i16(const float *llr, int16_t *q, int64_t count,
                          float scale, int qb);
/* The layered decoder in Section 5's int16 arithmetic with native wrap-around
 * (no saturation): every Z_mn and Z_n write, every |Z_mn| and every message
 * is reduced modulo 2^16 into [-32768, 32767] (so |-32768| = -32768, the
 * smallest value under the signed comparisons of the minimum).  normalise
 * means m -> (3 m) >> 2 (arithmetic shift) and requires alpha == 0.75.
 * wrap_events (or NULL) receives the number of reductions that changed a
 * value. */
int ldpc_ref_decode_layered_i16w(const ldpc_ref_code *code, const int16_t *llr,
                                 int64_t frames, const ldpc_ref_params *p,
                                 uint32_t *hard, int32_t *iters, int16_t *post,
                                 int64_t *wrap_events);

/* Bitmap encoder (Section 3, Alg. A1) for Z a multiple of 32: the direct
 * encoder of eq. (12)-(15) on packed words, bit r of block j at bit
 * (j Z + r) % 32 of word (j Z + r) / 32 (LSB first).  Each cyclic shift
 * P_s is split as in Alg. A1 into a rotation by sw = s / 32 whole words and
 * sb = s % 32 bits, the two combined in one pass over the block's words.
 * info u32[frames][K/32] -> cw u32[frames][N/32]; Z % 32 != 0 gives
 * LDPC_REF_ERR_UNSUPPORTED. */
int ldpc_ref_encode_bitmap(const ldpc_ref_code *code, const uint32_t *info,
                           uint32_t *cw, int64_t frames);
/* out = P_s in on one packed block of zw = Z/32 words (the rotation used by
 * ldpc_ref_encode_bitmap): out bit r = in bit (r + s) mod Z. */
void ldpc_ref_rotate_block(const uint32_t *in, int zw, int s, uint32_t *out);

#ifdef __cplusplus
}
#endif

#endif /* LDPC_ORACLE_H */
