/*
 * CPU oracle: plain restatement of arXiv 2306.12063 (Palenik & Szitkey).
 *
 * TEST INFRASTRUCTURE ONLY -- it is the yardstick the CUDA library is checked
 * against, never a code path of the library.  Clarity over speed: the
 * explicit sparse H is built from the base matrix, every check message L_mn
 * is stored uncompressed, and eq. (23)'s "minimum over the other edges" is
 * evaluated literally with a double loop.  Build with -ffp-contract=off so
 * that every float operation is rounded on its own.
 *
 * Parity status: every function here is pinned by the tests under tests/
 * (worked example, closed forms, brute force, published test vectors); see
 * the test files for which pin covers which function.
 */
#include "ldpc_oracle.h"

#include <math.h>
#include <stdlib.h>
#include <string.h>

struct ldpc_ref_code {
    int mb, nb, kb, z;
    int n, k, m;
    int16_t *hbm;     /* [mb][nb] */
    int encodable;
    int y;            /* row of the middle h_b entry, eq. (12) */
    int max_deg;
    /* explicit H (Section 1: neighbourhoods N(m), M(n)) */
    int *row_start;   /* [m + 1] */
    int *row_var;     /* [nnz]   variables of each row, increasing column block */
    int *col_start;   /* [n + 1] */
    int *col_row;     /* [nnz]   rows of each column */
    int nnz;
};

static int mod_z(int a, int z) {
    int r = a % z;
    return r < 0 ? r + z : r;
}

/* Structure required by the direct encoder, eq. (3)-(7) and the text around
 * them: h_b = column Kb has equal entries in rows 0 and Mb-1 and exactly one
 * other non-negative entry, at a row y in 1..Mb-2; H_b2' has zeros exactly on
 * the two diagonals (t, Kb+1+t) and (t+1, Kb+1+t). */
static int check_encodable(const int16_t *h, int mb, int nb, int *y_out) {
    int kb = nb - mb;
    if (mb < 3 || kb < 1) return 0;
    if (h[0 * nb + kb] < 0 || h[0 * nb + kb] != h[(mb - 1) * nb + kb]) return 0;
    int y = -1;
    for (int i = 1; i < mb - 1; i++) {
        if (h[i * nb + kb] >= 0) {
            if (y >= 0) return 0;
            y = i;
        }
    }
    if (y < 0) return 0;
    for (int i = 0; i < mb; i++) {
        for (int t = 0; t < mb - 1; t++) {
            int v = h[i * nb + kb + 1 + t];
            int on_diag = (i == t || i == t + 1);
            if (on_diag && v != 0) return 0;
            if (!on_diag && v != -1) return 0;
        }
    }
    *y_out = y;
    return 1;
}

int ldpc_ref_code_create(const int16_t *hbm, int mb, int nb, int z,
                         int require_encodable, ldpc_ref_code **out) {
    if (!hbm || !out || mb < 1 || nb <= mb || z < 1) return LDPC_REF_ERR_INVALID_ARG;
    *out = NULL;
    for (int i = 0; i < mb * nb; i++)
        if (hbm[i] < -1 || hbm[i] >= z) return LDPC_REF_ERR_BAD_STRUCTURE;
    int y = -1;
    int enc = check_encodable(hbm, mb, nb, &y);
    if (require_encodable && !enc) return LDPC_REF_ERR_BAD_STRUCTURE;

    ldpc_ref_code *c = (ldpc_ref_code *)calloc(1, sizeof(*c));
    if (!c) return LDPC_REF_ERR_NOMEM;
    c->mb = mb; c->nb = nb; c->kb = nb - mb; c->z = z;
    c->n = nb * z; c->k = (nb - mb) * z; c->m = mb * z;
    c->encodable = enc; c->y = enc ? y : -1;
    c->hbm = (int16_t *)malloc(sizeof(int16_t) * mb * nb);
    memcpy(c->hbm, hbm, sizeof(int16_t) * mb * nb);

    int nnz_b = 0;
    for (int i = 0; i < mb * nb; i++) nnz_b += hbm[i] >= 0;
    c->nnz = nnz_b * z;
    c->row_start = (int *)calloc(c->m + 1, sizeof(int));
    c->row_var = (int *)malloc(sizeof(int) * (c->nnz ? c->nnz : 1));
    c->col_start = (int *)calloc(c->n + 1, sizeof(int));
    c->col_row = (int *)malloc(sizeof(int) * (c->nnz ? c->nnz : 1));
    if (!c->hbm || !c->row_start || !c->row_var || !c->col_start || !c->col_row) {
        ldpc_ref_code_destroy(c);
        return LDPC_REF_ERR_NOMEM;
    }
    /* Expand each block (eq. 2): row r of block (i, j) with shift s has its
     * one in column (r + s) mod Z. */
    int e = 0;
    c->max_deg = 0;
    for (int i = 0; i < mb; i++) {
        for (int r = 0; r < z; r++) {
            int row = i * z + r;
            c->row_start[row] = e;
            for (int j = 0; j < nb; j++) {
                int s = hbm[i * nb + j];
                if (s < 0) continue;
                c->row_var[e++] = j * z + mod_z(r + s, z);
            }
            int d = e - c->row_start[row];
            if (d > c->max_deg) c->max_deg = d;
        }
    }
    c->row_start[c->m] = e;
    /* Column lists M(n) by counting sort over the row lists. */
    for (int t = 0; t < c->nnz; t++) c->col_start[c->row_var[t] + 1]++;
    for (int n = 0; n < c->n; n++) c->col_start[n + 1] += c->col_start[n];
    int *fill = (int *)calloc(c->n, sizeof(int));
    if (!fill) { ldpc_ref_code_destroy(c); return LDPC_REF_ERR_NOMEM; }
    for (int row = 0; row < c->m; row++)
        for (int t = c->row_start[row]; t < c->row_start[row + 1]; t++) {
            int n = c->row_var[t];
            c->col_row[c->col_start[n] + fill[n]++] = row;
        }
    free(fill);
    *out = c;
    return LDPC_REF_OK;
}

void ldpc_ref_code_destroy(ldpc_ref_code *c) {
    if (!c) return;
    free(c->hbm); free(c->row_start); free(c->row_var);
    free(c->col_start); free(c->col_row);
    free(c);
}

int ldpc_ref_code_info(const ldpc_ref_code *c, int *n, int *k, int *m, int *z,
                       int *max_row_deg, int *y, int *encodable) {
    if (!c) return LDPC_REF_ERR_INVALID_ARG;
    if (n) *n = c->n;
    if (k) *k = c->k;
    if (m) *m = c->m;
    if (z) *z = c->z;
    if (max_row_deg) *max_row_deg = c->max_deg;
    if (y) *y = c->y;
    if (encodable) *encodable = c->encodable;
    return LDPC_REF_OK;
}

int ldpc_ref_row_vars(const ldpc_ref_code *c, int row, int *vars, int cap) {
    if (!c || row < 0 || row >= c->m) return -1;
    int d = c->row_start[row + 1] - c->row_start[row];
    for (int t = 0; t < d && t < cap; t++) vars[t] = c->row_var[c->row_start[row] + t];
    return d;
}

int ldpc_ref_syndrome_weight(const ldpc_ref_code *c, const uint8_t *bits) {
    int w = 0;
    for (int row = 0; row < c->m; row++) {
        int par = 0;
        for (int t = c->row_start[row]; t < c->row_start[row + 1]; t++)
            par ^= bits[c->row_var[t]] & 1;
        w += par;
    }
    return w;
}

/* ---------------------------------------------------------------------------
 * Direct encoder (Section 2), on one bit per byte as in the paper's universal
 * array encoder (Section 3).
 * ------------------------------------------------------------------------- */

/* out = P_s in, i.e. out[r] = in[(r + s) mod Z]. */
static void circ_apply(const uint8_t *in, int s, int z, uint8_t *out) {
    for (int r = 0; r < z; r++) out[r] = in[mod_z(r + s, z)];
}

/* out = P_s^{-1} in, i.e. out[r] = in[(r - s) mod Z] (shift the other way). */
static void circ_apply_inv(const uint8_t *in, int s, int z, uint8_t *out) {
    for (int r = 0; r < z; r++) out[r] = in[mod_z(r - s, z)];
}

static void xor_into(uint8_t *acc, const uint8_t *x, int z) {
    for (int r = 0; r < z; r++) acc[r] ^= x[r];
}

int ldpc_ref_encode(const ldpc_ref_code *c, const uint8_t *info, uint8_t *cw,
                    int64_t frames) {
    if (!c || (!info && frames) || (!cw && frames) || frames < 0)
        return LDPC_REF_ERR_INVALID_ARG;
    if (!c->encodable) return LDPC_REF_ERR_BAD_STRUCTURE;
    const int z = c->z, mb = c->mb, nb = c->nb, kb = c->kb;
    uint8_t *S = (uint8_t *)malloc((size_t)mb * z);   /* S_i, eq. (15) */
    uint8_t *tmp = (uint8_t *)malloc(z);
    uint8_t *sum = (uint8_t *)malloc(z);
    if (!S || !tmp || !sum) { free(S); free(tmp); free(sum); return LDPC_REF_ERR_NOMEM; }

    for (int64_t f = 0; f < frames; f++) {
        const uint8_t *u = info + f * (int64_t)c->k;       /* u_j, eq. (8)-(9) */
        uint8_t *out = cw + f * (int64_t)c->n;
        for (int t = 0; t < c->k; t++) out[t] = u[t] & 1;  /* s = i, eq. (1) */
        uint8_t *v = out + c->k;                             /* v_i, eq. (10)-(11) */

        /* eq. (15): S_i = sum_j P_{H(i,j)} u_j over the info block columns */
        for (int i = 0; i < mb; i++) {
            uint8_t *Si = S + (size_t)i * z;
            memset(Si, 0, z);
            for (int j = 0; j < kb; j++) {
                int s = c->hbm[i * nb + j];
                if (s < 0) continue;            /* zero block: term skipped */
                circ_apply(out + j * z, s, z, tmp);
                xor_into(Si, tmp, z);
            }
        }
        /* eq. (12): v_0 = P^{-1}_{H(y,Kb)} sum_i S_i */
        memset(sum, 0, z);
        for (int i = 0; i < mb; i++) xor_into(sum, S + (size_t)i * z, z);
        circ_apply_inv(sum, c->hbm[c->y * nb + kb], z, v);
        /* eq. (13): v_1 = P_{H(0,Kb)} v_0 + S_0 */
        circ_apply(v, c->hbm[0 * nb + kb], z, v + z);
        xor_into(v + z, S, z);
        /* eq. (14): v_{i+1} = v_i + P_{H(i,Kb)} v_0 + S_i, i = 1..Mb-2 */
        for (int i = 1; i < mb - 1; i++) {
            uint8_t *vn = v + (size_t)(i + 1) * z;
            memcpy(vn, v + (size_t)i * z, z);
            int s = c->hbm[i * nb + kb];
            if (s >= 0) {
                circ_apply(v, s, z, tmp);
                xor_into(vn, tmp, z);
            }
            xor_into(vn, S + (size_t)i * z, z);
        }
    }
    free(S); free(tmp); free(sum);
    return LDPC_REF_OK;
}

/* ---------------------------------------------------------------------------
 * Counter-based random numbers for the synthetic channel (inputs only).
 * Philox4x32-10 as published by Salmon, Moraes, Dror & Shaw (SC'11): ten
 * rounds of two 32x32->64 multiplies, key bumped by the Weyl constants
 * between rounds.
 * ------------------------------------------------------------------------- */
void ldpc_ref_philox4x32_10(const uint32_t ctr[4], const uint32_t key[2],
                            uint32_t out[4]) {
    uint32_t c0 = ctr[0], c1 = ctr[1], c2 = ctr[2], c3 = ctr[3];
    uint32_t k0 = key[0], k1 = key[1];
    for (int round = 0; round < 10; round++) {
        if (round > 0) { k0 += 0x9E3779B9u; k1 += 0xBB67AE85u; }
        uint64_t p0 = (uint64_t)0xD2511F53u * c0;
        uint64_t p1 = (uint64_t)0xCD9E8D57u * c2;
        uint32_t hi0 = (uint32_t)(p0 >> 32), lo0 = (uint32_t)p0;
        uint32_t hi1 = (uint32_t)(p1 >> 32), lo1 = (uint32_t)p1;
        uint32_t n0 = hi1 ^ c1 ^ k0;
        uint32_t n2 = hi0 ^ c3 ^ k1;
        c0 = n0; c1 = lo1; c2 = n2; c3 = lo0;
    }
    out[0] = c0; out[1] = c1; out[2] = c2; out[3] = c3;
}

int ldpc_ref_gen_info(uint64_t seed, int64_t frame0, int64_t frames, int k,
                      uint8_t *info) {
    if ((!info && frames) || frames < 0 || k < 0 || frame0 < 0) return LDPC_REF_ERR_INVALID_ARG;
    uint32_t key[2] = {(uint32_t)seed, (uint32_t)(seed >> 32) ^ 0x494E464Fu};
    for (int64_t i = 0; i < frames; i++) {
        uint64_t f = (uint64_t)(frame0 + i);
        for (int b = 0; b < k; b++) {
            uint32_t ctr[4] = {(uint32_t)(b / 128), (uint32_t)f, (uint32_t)(f >> 32), 0u};
            uint32_t w[4];
            ldpc_ref_philox4x32_10(ctr, key, w);
            info[i * (int64_t)k + b] = (uint8_t)((w[(b / 32) % 4] >> (b % 32)) & 1u);
        }
    }
    return LDPC_REF_OK;
}

/* Natural logarithm of a positive normal float from its definition: write
 * u = m 2^e with m in [sqrt(1/2), sqrt(2)), then ln m = 2 atanh(t) with
 * t = (m - 1)/(m + 1), |t| < 0.172, summed as the odd power series
 * 2 t (1 + t^2/3 + t^4/5 + ... + t^10/11) by Horner's rule in t^2; the
 * truncation error is below 1e-10 relative.  Every step is one correctly
 * rounded float operation. */
float ldpc_ref_lnf(float u) {
    uint32_t b;
    memcpy(&b, &u, sizeof b);
    int e = (int)((b >> 23) & 0xFFu) - 127;
    uint32_t mbits = (b & 0x007FFFFFu) | 0x3F800000u;
    if (mbits > 0x3FB504F3u) { mbits -= 0x00800000u; e += 1; }
    float m;
    memcpy(&m, &mbits, sizeof m);
    float t = (m - 1.0f) / (m + 1.0f);
    float t2 = t * t;
    float s = 0x1.745d18p-4f;            /* 1/11 */
    s = s * t2 + 0x1.c71c72p-4f;        /* 1/9  */
    s = s * t2 + 0x1.24924ap-3f;        /* 1/7  */
    s = s * t2 + 0x1.99999ap-3f;        /* 1/5  */
    s = s * t2 + 0x1.555556p-2f;        /* 1/3  */
    s = s * t2 + 1.0f;
    float lnm = (2.0f * t) * s;
    return (float)e * 0x1.62e430p-1f + lnm;   /* e ln 2 + ln m */
}

/* sin and cos of the angle 2 pi k / 2^24 for an integer k < 2^24.  The turn
 * is split exactly into a quadrant q = k >> 22 and a remainder; the
 * remainder is reflected into [0, pi/4] so that the Taylor series of sin and
 * cos (coefficients 1/n!, through x^11 and x^12) converge to below 1e-10. */
void ldpc_ref_sincos_turn(uint32_t k24, float *s_out, float *c_out) {
    uint32_t q = (k24 >> 22) & 3u;
    uint32_t rem = k24 & 0x3FFFFFu;
    int swap = rem > 0x200000u;
    uint32_t red = swap ? 0x400000u - rem : rem;      /* <= 2^21 */
    float phi = (float)red * 0x1.921fb6p-22f;          /* red * pi / 2^23 */
    float x = phi * phi;
    float ps = -0x1.ae6456p-26f;                       /* -1/11! */
    ps = ps * x + 0x1.71de3ap-19f;                     /*  1/9!  */
    ps = ps * x - 0x1.a01a02p-13f;                     /* -1/7!  */
    ps = ps * x + 0x1.111112p-7f;                      /*  1/5!  */
    ps = ps * x - 0x1.555556p-3f;                      /* -1/3!  */
    ps = ps * x + 1.0f;
    float sinp = phi * ps;
    float pc = 0x1.1eed8ep-29f;                        /*  1/12! */
    pc = pc * x - 0x1.27e4fcp-22f;                     /* -1/10! */
    pc = pc * x + 0x1.a01a02p-16f;                     /*  1/8!  */
    pc = pc * x - 0x1.6c16c2p-10f;                     /* -1/6!  */
    pc = pc * x + 0x1.555556p-5f;                      /*  1/4!  */
    pc = pc * x - 0.5f;                                /* -1/2!  */
    pc = pc * x + 1.0f;
    float cosp = pc;
    float ct = swap ? sinp : cosp;   /* cos and sin of the in-quadrant angle */
    float st = swap ? cosp : sinp;
    float c, s;
    switch (q) {
        case 0: c = ct;  s = st;  break;
        case 1: c = -st; s = ct;  break;
        case 2: c = -ct; s = -st; break;
        default: c = st; s = -ct; break;
    }
    *s_out = s;
    *c_out = c;
}

/* Box-Muller (1958): u1 in (0, 1] and u2 in [0, 1) from the top 24 bits of
 * two words, R = sqrt(-2 ln u1), (g0, g1) = R (cos 2 pi u2, sin 2 pi u2). */
void ldpc_ref_box_muller(uint32_t w0, uint32_t w1, float *g0, float *g1) {
    float u1 = (float)((w0 >> 8) + 1u) * 0x1p-24f;
    float r = sqrtf(-2.0f * ldpc_ref_lnf(u1));
    float s, c;
    ldpc_ref_sincos_turn(w1 >> 8, &s, &c);
    *g0 = r * c;
    *g1 = r * s;
}

int ldpc_ref_awgn_llr(const uint8_t *cw, int64_t frame0, int64_t frames, int n,
                      uint64_t seed, float sigma, float llr_scale, float *llr) {
    if ((!cw && frames) || (!llr && frames) || frames < 0 || n < 0 || frame0 < 0)
        return LDPC_REF_ERR_INVALID_ARG;
    uint32_t key[2] = {(uint32_t)seed, (uint32_t)(seed >> 32) ^ 0x4E4F4953u};
    for (int64_t i = 0; i < frames; i++) {
        uint64_t f = (uint64_t)(frame0 + i);
        for (int p = 0; p < n; p++) {
            uint32_t ctr[4] = {(uint32_t)(p / 4), (uint32_t)f, (uint32_t)(f >> 32), 0u};
            uint32_t w[4];
            ldpc_ref_philox4x32_10(ctr, key, w);
            float g[4];
            ldpc_ref_box_muller(w[0], w[1], &g[0], &g[1]);
            ldpc_ref_box_muller(w[2], w[3], &g[2], &g[3]);
            /* eq. (16): BPSK x -> 1 - 2x plus noise; eq. (17): 2 y / sigma^2 */
            float x = (cw[i * (int64_t)n + p] & 1) ? -1.0f : 1.0f;
            float y = x + sigma * g[p % 4];
            llr[i * (int64_t)n + p] = y * llr_scale;
        }
    }
    return LDPC_REF_OK;
}

int ldpc_ref_quantize_i8(const float *llr, int8_t *q, int64_t count, float scale,
                         int clip) {
    if ((!llr && count) || (!q && count) || count < 0 || clip < 0 || clip > 127)
        return LDPC_REF_ERR_INVALID_ARG;
    for (int64_t i = 0; i < count; i++) {
        float v = scale * llr[i];
        if (v > (float)clip) v = (float)clip;
        if (v < -(float)clip) v = -(float)clip;
        q[i] = (int8_t)nearbyintf(v);   /* default rounding: half to even */
    }
    return LDPC_REF_OK;
}

/* ---------------------------------------------------------------------------
 * Decoders (Section 4).  Notation follows the paper: Z_n posterior LLR of
 * variable n, L_mn check message from row m to variable n, Z_mn = Z_n - L_mn
 * the variable message (eq. 22).
 * ------------------------------------------------------------------------- */

static int min_row_degree(const ldpc_ref_code *c) {
    int dmin = c->nb + 1;
    for (int row = 0; row < c->m; row++) {
        int d = c->row_start[row + 1] - c->row_start[row];
        if (d < dmin) dmin = d;
    }
    return dmin;
}

static int check_params(const ldpc_ref_code *c, const ldpc_ref_params *p,
                        int64_t frames, const void *llr, const void *hard,
                        const void *iters) {
    if (!c || !p || frames < 0) return LDPC_REF_ERR_INVALID_ARG;
    if (frames && (!llr || !hard || !iters)) return LDPC_REF_ERR_INVALID_ARG;
    if (p->max_iters < 1) return LDPC_REF_ERR_INVALID_ARG;
    if (min_row_degree(c) < 2) return LDPC_REF_ERR_UNSUPPORTED;
    return LDPC_REF_OK;
}

/* eq. (21): bit n = 0 if Z_n > 0, else 1; packed LSB-first in 32-bit words. */
static void hard_from_f32(const float *Zn, int n, uint32_t *words, uint8_t *bits) {
    int nw = (n + 31) / 32;
    for (int w = 0; w < nw; w++) words[w] = 0;
    for (int v = 0; v < n; v++) {
        int b = !(Zn[v] > 0.0f);
        bits[v] = (uint8_t)b;
        words[v / 32] |= (uint32_t)b << (v % 32);
    }
}

static void hard_from_int(const int *Zn, int n, uint32_t *words, uint8_t *bits) {
    int nw = (n + 31) / 32;
    for (int w = 0; w < nw; w++) words[w] = 0;
    for (int v = 0; v < n; v++) {
        int b = !(Zn[v] > 0);
        bits[v] = (uint8_t)b;
        words[v / 32] |= (uint32_t)b << (v % 32);
    }
}

/* eq. (18) / (23) for one edge t of a row with variable messages Q[0..d-1]:
 * the smallest |Q| and the product of signs over the OTHER edges. */
static float minsum_excl_f32(const float *Q, int d, int t) {
    float mn = INFINITY;
    int neg = 0;
    for (int u = 0; u < d; u++) {
        if (u == t) continue;
        float a = fabsf(Q[u]);
        if (a < mn) mn = a;
        if (Q[u] < 0.0f) neg ^= 1;
    }
    return neg ? -mn : mn;
}

static int minsum_excl_int(const int *Q, int d, int t) {
    int mn = 1 << 30;
    int neg = 0;
    for (int u = 0; u < d; u++) {
        if (u == t) continue;
        int a = Q[u] < 0 ? -Q[u] : Q[u];
        if (a < mn) mn = a;
        if (Q[u] < 0) neg ^= 1;
    }
    return neg ? -mn : mn;
}

int ldpc_ref_decode_layered_f32(const ldpc_ref_code *c, const float *llr,
                                int64_t frames, const ldpc_ref_params *p,
                                uint32_t *hard, int32_t *iters, float *post) {
    int st = check_params(c, p, frames, llr, hard, iters);
    if (st) return st;
    const int n = c->n, nw = (n + 31) / 32;
    float *Zn = (float *)malloc(sizeof(float) * n);
    float *L = (float *)malloc(sizeof(float) * (c->nnz ? c->nnz : 1));
    float *Q = (float *)malloc(sizeof(float) * (c->max_deg ? c->max_deg : 1));
    float *Ln = (float *)malloc(sizeof(float) * (c->max_deg ? c->max_deg : 1));
    uint8_t *bits = (uint8_t *)malloc(n);
    if (!Zn || !L || !Q || !Ln || !bits) {
        free(Zn); free(L); free(Q); free(Ln); free(bits);
        return LDPC_REF_ERR_NOMEM;
    }
    const float alpha = p->normalise ? p->alpha : 1.0f;

    for (int64_t f = 0; f < frames; f++) {
        /* Z_n^(0) = channel LLR; Z_mn^(0) := Z_n^(0), i.e. every L_mn = 0 */
        for (int v = 0; v < n; v++) Zn[v] = llr[f * (int64_t)n + v];
        for (int e = 0; e < c->nnz; e++) L[e] = 0.0f;
        int done = p->max_iters;
        for (int k = 1; k <= p->max_iters; k++) {
            /* layered schedule: tiers of Z rows, block rows in natural order */
            for (int i = 0; i < c->mb; i++) {
                for (int r = 0; r < c->z; r++) {
                    int row = i * c->z + r;
                    int b = c->row_start[row];
                    int d = c->row_start[row + 1] - b;
                    for (int t = 0; t < d; t++)                       /* eq. (22) */
                        Q[t] = Zn[c->row_var[b + t]] - L[b + t];
                    for (int t = 0; t < d; t++) {                     /* eq. (23) */
                        float m = minsum_excl_f32(Q, d, t);
                        Ln[t] = p->normalise ? alpha * m : m;
                    }
                    for (int t = 0; t < d; t++) {                     /* eq. (20) */
                        L[b + t] = Ln[t];
                        Zn[c->row_var[b + t]] = Q[t] + Ln[t];
                    }
                }
            }
            if (p->early_stop) {                                       /* eq. (21) */
                hard_from_f32(Zn, n, hard + f * (int64_t)nw, bits);
                if (ldpc_ref_syndrome_weight(c, bits) == 0) { done = k; break; }
            }
        }
        hard_from_f32(Zn, n, hard + f * (int64_t)nw, bits);
        iters[f] = done;
        if (post) for (int v = 0; v < n; v++) post[f * (int64_t)n + v] = Zn[v];
    }
    free(Zn); free(L); free(Q); free(Ln); free(bits);
    return LDPC_REF_OK;
}

static int sat127(int x, int64_t *events) {
    if (x > 127) { (*events)++; return 127; }
    if (x < -127) { (*events)++; return -127; }
    return x;
}

int ldpc_ref_decode_layered_i8(const ldpc_ref_code *c, const int8_t *llr,
                               int64_t frames, const ldpc_ref_params *p,
                               uint32_t *hard, int32_t *iters, int8_t *post,
                               int64_t *sat_events) {
    int st = check_params(c, p, frames, llr, hard, iters);
    if (st) return st;
    if (p->normalise && p->alpha != 0.75f) return LDPC_REF_ERR_UNSUPPORTED;
    const int n = c->n, nw = (n + 31) / 32;
    int *Zn = (int *)malloc(sizeof(int) * n);
    int *L = (int *)malloc(sizeof(int) * (c->nnz ? c->nnz : 1));
    int *Q = (int *)malloc(sizeof(int) * (c->max_deg ? c->max_deg : 1));
    int *Ln = (int *)malloc(sizeof(int) * (c->max_deg ? c->max_deg : 1));
    uint8_t *bits = (uint8_t *)malloc(n);
    if (!Zn || !L || !Q || !Ln || !bits) {
        free(Zn); free(L); free(Q); free(Ln); free(bits);
        return LDPC_REF_ERR_NOMEM;
    }
    int64_t events = 0;
    for (int64_t f = 0; f < frames; f++) {
        for (int v = 0; v < n; v++) Zn[v] = llr[f * (int64_t)n + v];
        for (int e = 0; e < c->nnz; e++) L[e] = 0;
        int done = p->max_iters;
        for (int k = 1; k <= p->max_iters; k++) {
            for (int i = 0; i < c->mb; i++) {
                for (int r = 0; r < c->z; r++) {
                    int row = i * c->z + r;
                    int b = c->row_start[row];
                    int d = c->row_start[row + 1] - b;
                    for (int t = 0; t < d; t++)
                        Q[t] = sat127(Zn[c->row_var[b + t]] - L[b + t], &events);
                    for (int t = 0; t < d; t++) {
                        int m = minsum_excl_int(Q, d, t);
                        if (p->normalise) {
                            int a = m < 0 ? -m : m;
                            a = (3 * a) >> 2;        /* 3/4 scaling by shift */
                            m = m < 0 ? -a : a;
                        }
                        Ln[t] = m;
                    }
                    for (int t = 0; t < d; t++) {
                        L[b + t] = Ln[t];
                        Zn[c->row_var[b + t]] = sat127(Q[t] + Ln[t], &events);
                    }
                }
            }
            if (p->early_stop) {
                hard_from_int(Zn, n, hard + f * (int64_t)nw, bits);
                if (ldpc_ref_syndrome_weight(c, bits) == 0) { done = k; break; }
            }
        }
        hard_from_int(Zn, n, hard + f * (int64_t)nw, bits);
        iters[f] = done;
        if (post) for (int v = 0; v < n; v++) post[f * (int64_t)n + v] = (int8_t)Zn[v];
    }
    if (sat_events) *sat_events = events;
    free(Zn); free(L); free(Q); free(Ln); free(bits);
    return LDPC_REF_OK;
}

int ldpc_ref_decode_flooding_f32(const ldpc_ref_code *c, const float *llr,
                                 int64_t frames, const ldpc_ref_params *p,
                                 uint32_t *hard, int32_t *iters, float *post) {
    int st = check_params(c, p, frames, llr, hard, iters);
    if (st) return st;
    const int n = c->n, nw = (n + 31) / 32;
    float *Z0 = (float *)malloc(sizeof(float) * n);
    float *Zn = (float *)malloc(sizeof(float) * n);
    float *L = (float *)malloc(sizeof(float) * (c->nnz ? c->nnz : 1));
    float *Lnew = (float *)malloc(sizeof(float) * (c->nnz ? c->nnz : 1));
    float *Q = (float *)malloc(sizeof(float) * (c->max_deg ? c->max_deg : 1));
    uint8_t *bits = (uint8_t *)malloc(n);
    if (!Z0 || !Zn || !L || !Lnew || !Q || !bits) {
        free(Z0); free(Zn); free(L); free(Lnew); free(Q); free(bits);
        return LDPC_REF_ERR_NOMEM;
    }
    const float alpha = p->normalise ? p->alpha : 1.0f;
    for (int64_t f = 0; f < frames; f++) {
        for (int v = 0; v < n; v++) Z0[v] = Zn[v] = llr[f * (int64_t)n + v];
        for (int e = 0; e < c->nnz; e++) L[e] = 0.0f;
        int done = p->max_iters;
        for (int k = 1; k <= p->max_iters; k++) {
            /* horizontal scan, eq. (18), on variable messages of eq. (19) */
            for (int row = 0; row < c->m; row++) {
                int b = c->row_start[row];
                int d = c->row_start[row + 1] - b;
                for (int t = 0; t < d; t++) {
                    int v = c->row_var[b + t];
                    float s = Z0[v];                      /* eq. (19) */
                    for (int q = c->col_start[v]; q < c->col_start[v + 1]; q++) {
                        int m2 = c->col_row[q];
                        if (m2 == row) continue;
                        int b2 = c->row_start[m2];
                        for (int u = b2; u < c->row_start[m2 + 1]; u++)
                            if (c->row_var[u] == v) { s = s + L[u]; break; }
                    }
                    Q[t] = s;
                }
                for (int t = 0; t < d; t++) {
                    float m = minsum_excl_f32(Q, d, t);
                    Lnew[b + t] = p->normalise ? alpha * m : m;
                }
            }
            memcpy(L, Lnew, sizeof(float) * c->nnz);
            /* posterior, eq. (20) */
            for (int v = 0; v < n; v++) {
                float s = Z0[v];
                for (int q = c->col_start[v]; q < c->col_start[v + 1]; q++) {
                    int m2 = c->col_row[q];
                    for (int u = c->row_start[m2]; u < c->row_start[m2 + 1]; u++)
                        if (c->row_var[u] == v) { s = s + L[u]; break; }
                }
                Zn[v] = s;
            }
            if (p->early_stop) {
                hard_from_f32(Zn, n, hard + f * (int64_t)nw, bits);
                if (ldpc_ref_syndrome_weight(c, bits) == 0) { done = k; break; }
            }
        }
        hard_from_f32(Zn, n, hard + f * (int64_t)nw, bits);
        iters[f] = done;
        if (post) for (int v = 0; v < n; v++) post[f * (int64_t)n + v] = Zn[v];
    }
    free(Z0); free(Zn); free(L); free(Lnew); free(Q); free(bits);
    return LDPC_REF_OK;
}

/* ---------------------------------------------------------------------------
 * Section 5: int16 fixed point with wrap-around arithmetic.
 * ------------------------------------------------------------------------- */
int ldpc_ref_quantize_i16(const float *llr, int16_t *q, int64_t count, float scale,
                          int qb) {
    if ((!llr && count) || (!q && count) || count < 0 || qb < 1 || qb > 14)
        return LDPC_REF_ERR_INVALID_ARG;
    const float lim = (float)((1 << qb) - 1);
    for (int64_t i = 0; i < count; i++) {
        float v = scale * llr[i];
        if (v > lim) v = lim;
        if (v < -lim) v = -lim;
        q[i] = (int16_t)nearbyintf(v);   /* default rounding: half to even */
    }
    return LDPC_REF_OK;
}

/* x reduced modulo 2^16 into [-32768, 32767], counting changes. */
static int wrap16(int x, int64_t *events) {
    int y = x & 0xFFFF;
    if (y >= 32768) y -= 65536;
    if (y != x) (*events)++;
    return y;
}

int ldpc_ref_decode_layered_i16w(const ldpc_ref_code *c, const int16_t *llr,
                                 int64_t frames, const ldpc_ref_params *p,
                                 uint32_t *hard, int32_t *iters, int16_t *post,
                                 int64_t *wrap_events) {
    int st = check_params(c, p, frames, llr, hard, iters);
    if (st) return st;
    if (p->normalise && p->alpha != 0.75f) return LDPC_REF_ERR_UNSUPPORTED;
    const int n = c->n, nw = (n + 31) / 32;
    int *Zn = (int *)malloc(sizeof(int) * n);
    int *L = (int *)malloc(sizeof(int) * (c->nnz ? c->nnz : 1));
    int *Q = (int *)malloc(sizeof(int) * (c->max_deg ? c->max_deg : 1));
    int *A = (int *)malloc(sizeof(int) * (c->max_deg ? c->max_deg : 1));
    int *Ln = (int *)malloc(sizeof(int) * (c->max_deg ? c->max_deg : 1));
    uint8_t *bits = (uint8_t *)malloc(n);
    if (!Zn || !L || !Q || !A || !Ln || !bits) {
        free(Zn); free(L); free(Q); free(A); free(Ln); free(bits);
        return LDPC_REF_ERR_NOMEM;
    }
    int64_t events = 0;
    for (int64_t f = 0; f < frames; f++) {
        for (int v = 0; v < n; v++) Zn[v] = llr[f * (int64_t)n + v];
        for (int e = 0; e < c->nnz; e++) L[e] = 0;
        int done = p->max_iters;
        for (int k = 1; k <= p->max_iters; k++) {
            for (int i = 0; i < c->mb; i++) {
                for (int r = 0; r < c->z; r++) {
                    int row = i * c->z + r;
                    int b = c->row_start[row];
                    int d = c->row_start[row + 1] - b;
                    for (int t = 0; t < d; t++) {                      /* eq. (22) */
                        Q[t] = wrap16(Zn[c->row_var[b + t]] - L[b + t], &events);
                        A[t] = wrap16(Q[t] < 0 ? -Q[t] : Q[t], &events);   /* |Z_mn| */
                    }
                    for (int t = 0; t < d; t++) {                      /* eq. (23) */
                        int mn = 1 << 30, neg = 0;
                        for (int u = 0; u < d; u++) {
                            if (u == t) continue;
                            if (A[u] < mn) mn = A[u];
                            if (Q[u] < 0) neg ^= 1;
                        }
                        if (p->normalise) mn = wrap16((3 * mn) >> 2, &events);
                        Ln[t] = neg ? wrap16(-mn, &events) : mn;
                    }
                    for (int t = 0; t < d; t++) {                      /* eq. (20) */
                        L[b + t] = Ln[t];
                        Zn[c->row_var[b + t]] = wrap16(Q[t] + Ln[t], &events);
                    }
                }
            }
            if (p->early_stop) {
                hard_from_int(Zn, n, hard + f * (int64_t)nw, bits);
                if (ldpc_ref_syndrome_weight(c, bits) == 0) { done = k; break; }
            }
        }
        hard_from_int(Zn, n, hard + f * (int64_t)nw, bits);
        iters[f] = done;
        if (post) for (int v = 0; v < n; v++) post[f * (int64_t)n + v] = (int16_t)Zn[v];
    }
    if (wrap_events) *wrap_events = events;
    free(Zn); free(L); free(Q); free(A); free(Ln); free(bits);
    return LDPC_REF_OK;
}

/* ---------------------------------------------------------------------------
 * Section 3: bitmap encoder.  A packed block of Z = 32 zw bits, bit r at bit
 * r % 32 of word r / 32.  P_s (out bit r = in bit (r + s) mod Z) splits, as
 * in Alg. A1, into sw = s / 32 whole words and sb = s % 32 bits: output word
 * w takes the top 32 - sb bits of input word (w + sw) mod zw (shifted down)
 * and the low sb bits of the next input word (shifted up).
 * ------------------------------------------------------------------------- */
void ldpc_ref_rotate_block(const uint32_t *in, int zw, int s, uint32_t *out) {
    const int sw = s / 32, sb = s % 32;
    for (int w = 0; w < zw; w++) {
        uint32_t lo = in[(w + sw) % zw];
        uint32_t hi = in[(w + sw + 1) % zw];
        out[w] = sb ? (lo >> sb) | (hi << (32 - sb)) : lo;
    }
}

int ldpc_ref_encode_bitmap(const ldpc_ref_code *c, const uint32_t *info, uint32_t *cw,
                           int64_t frames) {
    if (!c || (!info && frames) || (!cw && frames) || frames < 0)
        return LDPC_REF_ERR_INVALID_ARG;
    if (!c->encodable) return LDPC_REF_ERR_BAD_STRUCTURE;
    if (c->z % 32) return LDPC_REF_ERR_UNSUPPORTED;
    const int zw = c->z / 32, mb = c->mb, nb = c->nb, kb = c->kb;
    uint32_t *S = (uint32_t *)malloc(sizeof(uint32_t) * mb * zw);
    uint32_t *tmp = (uint32_t *)malloc(sizeof(uint32_t) * zw);
    uint32_t *sum = (uint32_t *)malloc(sizeof(uint32_t) * zw);
    if (!S || !tmp || !sum) { free(S); free(tmp); free(sum); return LDPC_REF_ERR_NOMEM; }
    for (int64_t f = 0; f < frames; f++) {
        const uint32_t *u = info + f * (int64_t)(kb * zw);
        uint32_t *out = cw + f * (int64_t)(nb * zw);
        for (int w = 0; w < kb * zw; w++) out[w] = u[w];
        uint32_t *v = out + kb * zw;
        for (int i = 0; i < mb; i++) {                   /* eq. (15) */
            uint32_t *Si = S + i * zw;
            for (int w = 0; w < zw; w++) Si[w] = 0;
            for (int j = 0; j < kb; j++) {
                int s = c->hbm[i * nb + j];
                if (s < 0) continue;
                ldpc_ref_rotate_block(u + j * zw, zw, s, tmp);
                for (int w = 0; w < zw; w++) Si[w] ^= tmp[w];
            }
        }
        for (int w = 0; w < zw; w++) sum[w] = 0;        /* eq. (12) */
        for (int i = 0; i < mb; i++)
            for (int w = 0; w < zw; w++) sum[w] ^= S[i * zw + w];
        {
            int b = c->hbm[c->y * nb + kb];             /* P_b^{-1} = P_{Z-b} */
            ldpc_ref_rotate_block(sum, zw, (c->z - b) % c->z, v);
        }
        ldpc_ref_rotate_block(v, zw, c->hbm[kb], v + zw);   /* eq. (13) */
        for (int w = 0; w < zw; w++) v[zw + w] ^= S[w];
        for (int i = 1; i < mb - 1; i++) {                   /* eq. (14) */
            uint32_t *vn = v + (i + 1) * zw;
            for (int w = 0; w < zw; w++) vn[w] = v[i * zw + w] ^ S[i * zw + w];
            int s = c->hbm[i * nb + kb];
            if (s >= 0) {
                ldpc_ref_rotate_block(v, zw, s, tmp);
                for (int w = 0; w < zw; w++) vn[w] ^= tmp[w];
            }
        }
    }
    free(S); free(tmp); free(sum);
    return LDPC_REF_OK;
}

/* Index of the first nonzero block of H_bm block row i in row-major order. */
static int block_edge_base(const ldpc_ref_code *c, int i) {
    int q = 0;
    for (int a = 0; a < i; a++)
        for (int j = 0; j < c->nb; j++) q += c->hbm[a * c->nb + j] >= 0;
    return q;
}

/* Give-up checkpoint j (0 when there is none). */
static int stop_iter_of(const int *stop_iter, int j) { return stop_iter ? stop_iter[j] : 0; }

/* Learned normalised min-sum (see the header).  The weights of iteration k
 * are row min(k, T) - 1 of the table, so iterations past T repeat the last
 * row.  fused = 0 is the training arithmetic: the weighted message
 * w * m is rounded, then added to or subtracted from the posterior; fused = 1
 * is the inference arithmetic: Z - w m and Z + w m each with one rounding
 * (fmaf), the unweighted messages m being kept per edge.  After each
 * iteration with early_stop the unsatisfied checks u are counted: u = 0
 * stops the frame (eq. 21, Section 4 step 4); so does u > floor(stop_frac[j]
 * * M) at iteration stop_iter[j] (the give-up rule for frames the decoder is
 * not converging on). */
static int decode_learned(const ldpc_ref_code *c, const float *llr, int64_t frames,
                          const float *weights, int T, int max_iters, int early_stop,
                          const int *stop_iter, const float *stop_frac, int fused,
                          uint32_t *hard, int32_t *iters, float *post) {
    ldpc_ref_params p = {max_iters, 1.0f, 0, early_stop};
    int st = check_params(c, &p, frames, llr, hard, iters);
    if (st) return st;
    if ((!weights && frames) || T < 1) return LDPC_REF_ERR_INVALID_ARG;
    int limit[2] = {-1, -1};
    for (int j = 0; j < 2; j++) {
        if (!stop_iter || stop_iter[j] == 0) continue;
        if (stop_iter[j] < 1 || !early_stop || !(stop_frac[j] >= 0.0f))
            return LDPC_REF_ERR_INVALID_ARG;
        limit[j] = (int)floorf(stop_frac[j] * (float)c->m);
    }
    const int n = c->n, nw = (n + 31) / 32;
    int nnzb = 0;
    for (int q = 0; q < c->mb * c->nb; q++) nnzb += c->hbm[q] >= 0;
    float *Zn = (float *)malloc(sizeof(float) * n);
    float *L = (float *)malloc(sizeof(float) * (c->nnz ? c->nnz : 1));
    float *Q = (float *)malloc(sizeof(float) * (c->max_deg ? c->max_deg : 1));
    float *Ln = (float *)malloc(sizeof(float) * (c->max_deg ? c->max_deg : 1));
    uint8_t *bits = (uint8_t *)malloc(n);
    if (!Zn || !L || !Q || !Ln || !bits) {
        free(Zn); free(L); free(Q); free(Ln); free(bits);
        return LDPC_REF_ERR_NOMEM;
    }
    for (int64_t f = 0; f < frames; f++) {
        for (int v = 0; v < n; v++) Zn[v] = llr[f * (int64_t)n + v];
        /* L: the messages, weighted (fused = 0) or unweighted (fused = 1) */
        for (int e = 0; e < c->nnz; e++) L[e] = 0.0f;
        int done = max_iters;
        for (int k = 1; k <= max_iters; k++) {
            const float *wk = weights + (size_t)((k < T ? k : T) - 1) * nnzb;
            /* the weights the old messages were made with (iteration k - 1;
               iteration 1 has no old messages) */
            const int kp = k > 1 ? k - 1 : 1;
            const float *wp = weights + (size_t)((kp < T ? kp : T) - 1) * nnzb;
            for (int i = 0; i < c->mb; i++) {
                const int q0 = block_edge_base(c, i);
                for (int r = 0; r < c->z; r++) {
                    int row = i * c->z + r;
                    int b = c->row_start[row];
                    int d = c->row_start[row + 1] - b;
                    for (int t = 0; t < d; t++)                       /* eq. (22) */
                        Q[t] = fused ? fmaf(-wp[q0 + t], L[b + t], Zn[c->row_var[b + t]])
                                     : Zn[c->row_var[b + t]] - L[b + t];
                    for (int t = 0; t < d; t++) {                     /* eq. (23) */
                        const float m = minsum_excl_f32(Q, d, t);
                        Ln[t] = fused ? m : wk[q0 + t] * m;
                    }
                    for (int t = 0; t < d; t++) {                     /* eq. (20) */
                        L[b + t] = Ln[t];
                        Zn[c->row_var[b + t]] = fused ? fmaf(wk[q0 + t], Ln[t], Q[t])
                                                      : Q[t] + Ln[t];
                    }
                }
            }
            if (early_stop) {
                hard_from_f32(Zn, n, hard + f * (int64_t)nw, bits);
                const int u = ldpc_ref_syndrome_weight(c, bits);
                if (u == 0 || (k == stop_iter_of(stop_iter, 0) && u > limit[0]) ||
                    (k == stop_iter_of(stop_iter, 1) && u > limit[1])) {
                    done = k;
                    break;
                }
            }
        }
        hard_from_f32(Zn, n, hard + f * (int64_t)nw, bits);
        iters[f] = done;
        if (post) for (int v = 0; v < n; v++) post[f * (int64_t)n + v] = Zn[v];
    }
    free(Zn); free(L); free(Q); free(Ln); free(bits);
    return LDPC_REF_OK;
}

int ldpc_ref_decode_learned_f32(const ldpc_ref_code *c, const float *llr, int64_t frames,
                                const float *weights, int T, int max_iters, int early_stop,
                                const int *stop_iter, const float *stop_frac, uint32_t *hard,
                                int32_t *iters, float *post) {
    return decode_learned(c, llr, frames, weights, T, max_iters, early_stop, stop_iter,
                          stop_frac, 1, hard, iters, post);
}

int ldpc_ref_decode_layered_weighted_f32(const ldpc_ref_code *c, const float *llr,
                                         int64_t frames, const float *weights, int T,
                                         int early_stop, uint32_t *hard, int32_t *iters,
                                         float *post) {
    return decode_learned(c, llr, frames, weights, T, T, early_stop, NULL, NULL, 0, hard,
                          iters, post);
}
