/*
 * mlmc_oracle.c -- plain FP64 CPU oracle of the MLMC estimator for E[AB]
 * (Wu & Polydorides, arXiv:1904.00429).  TEST INFRASTRUCTURE ONLY: used by
 * tests, the smoke check and the CPU-baseline leg of the benchmark, never by
 * the product path.  See mlmc_oracle.h for the contract of every function.
 *
 * The code is deliberately slow and literal: it materialises one realisation
 * of the sampled columns of A and rows of B, forms the fine and the coarse
 * sketches separately as the paper writes them (Sec. 3.1, Alg. 1) and only then
 * takes their difference, and accumulates statistics with Welford updates in
 * sample order.  No blocking, fusion or reordering.
 */
#include "mlmc_oracle.h"

#include <math.h>
#include <stdlib.h>
#include <string.h>

/* ------------------------------------------------------------------------- */
/* Philox (Salmon et al., SC'11): a 10-round keyed bijection on a 4-word
 * counter.  Each round multiplies words 0 and 2 by fixed odd constants, keeps
 * the high and low halves of the double-width products, and mixes the high
 * halves with the other two words and the round key; the key is advanced by
 * the Weyl constants (golden ratio, sqrt(3) - 1) between rounds. */

#define PHILOX32_M0 0xD2511F53u
#define PHILOX32_M1 0xCD9E8D57u
#define PHILOX32_W0 0x9E3779B9u
#define PHILOX32_W1 0xBB67AE85u

void orc_philox4x32_10(const uint32_t ctr[4], const uint32_t key[2], uint32_t out[4])
{
    uint32_t c0 = ctr[0], c1 = ctr[1], c2 = ctr[2], c3 = ctr[3];
    uint32_t k0 = key[0], k1 = key[1];
    for (int round = 0; round < 10; ++round) {
        if (round > 0) {
            k0 += PHILOX32_W0;
            k1 += PHILOX32_W1;
        }
        uint64_t prod0 = (uint64_t)PHILOX32_M0 * (uint64_t)c0;
        uint64_t prod1 = (uint64_t)PHILOX32_M1 * (uint64_t)c2;
        uint32_t hi0 = (uint32_t)(prod0 >> 32), lo0 = (uint32_t)prod0;
        uint32_t hi1 = (uint32_t)(prod1 >> 32), lo1 = (uint32_t)prod1;
        uint32_t n0 = hi1 ^ c1 ^ k0;
        uint32_t n1 = lo1;
        uint32_t n2 = hi0 ^ c3 ^ k1;
        uint32_t n3 = lo0;
        c0 = n0; c1 = n1; c2 = n2; c3 = n3;
    }
    out[0] = c0; out[1] = c1; out[2] = c2; out[3] = c3;
}

#define PHILOX64_M0 0xD2E7470EE14C6C93ull
#define PHILOX64_M1 0xCA5A826395121157ull
#define PHILOX64_W0 0x9E3779B97F4A7C15ull
#define PHILOX64_W1 0xBB67AE8584CAA73Bull

void orc_philox4x64_10(const uint64_t ctr[4], const uint64_t key[2], uint64_t out[4])
{
    uint64_t c0 = ctr[0], c1 = ctr[1], c2 = ctr[2], c3 = ctr[3];
    uint64_t k0 = key[0], k1 = key[1];
    for (int round = 0; round < 10; ++round) {
        if (round > 0) {
            k0 += PHILOX64_W0;
            k1 += PHILOX64_W1;
        }
        unsigned __int128 prod0 = (unsigned __int128)PHILOX64_M0 * c0;
        unsigned __int128 prod1 = (unsigned __int128)PHILOX64_M1 * c2;
        uint64_t hi0 = (uint64_t)(prod0 >> 64), lo0 = (uint64_t)prod0;
        uint64_t hi1 = (uint64_t)(prod1 >> 64), lo1 = (uint64_t)prod1;
        uint64_t n0 = hi1 ^ c1 ^ k0;
        uint64_t n1 = lo1;
        uint64_t n2 = hi0 ^ c3 ^ k1;
        uint64_t n3 = lo0;
        c0 = n0; c1 = n1; c2 = n2; c3 = n3;
    }
    out[0] = c0; out[1] = c1; out[2] = c2; out[3] = c3;
}

/* ------------------------------------------------------------------------- */
/* Maps from Philox words to the draws the method needs. */

double orc_uniform(uint32_t w)
{
    return ((double)w + 0.5) * 0x1p-32;
}

/* Fourth counter word: level in the low 8 bits, sample bits 32..55 above. */
static uint32_t level_sample_word(int l, uint64_t s)
{
    return (uint32_t)(((s >> 32) << 8) | (uint64_t)(l & 0xFF));
}

double orc_normal(uint32_t seed, uint32_t problem_id, int l, uint64_t s, int64_t row, int64_t k)
{
    const double two_pi = 6.283185307179586476925286766559;
    uint32_t ctr[4] = { (uint32_t)(row >> 2), (uint32_t)k, (uint32_t)s, level_sample_word(l, s) };
    uint32_t key[2] = { seed, problem_id };
    uint32_t w[4];
    orc_philox4x32_10(ctr, key, w);
    int q = (int)(row & 3);
    int pair = q >> 1;
    double u_radius = orc_uniform(w[2 * pair]);
    double u_angle = orc_uniform(w[2 * pair + 1]);
    /* Box-Muller: two independent N(0,1) from two independent U(0,1). */
    double radius = sqrt(-2.0 * log(u_radius));
    double angle = two_pi * u_angle;
    return (q & 1) ? radius * sin(angle) : radius * cos(angle);
}

int64_t orc_index(uint32_t seed_idx, uint32_t problem_id, int l, uint64_t s, int64_t t, int64_t n)
{
    uint32_t ctr[4] = { (uint32_t)(t >> 1), 0xFFFFFFFFu, (uint32_t)s, level_sample_word(l, s) };
    uint32_t key[2] = { seed_idx, problem_id };
    uint32_t w[4];
    orc_philox4x32_10(ctr, key, w);
    uint64_t word = (t & 1) ? (((uint64_t)w[3] << 32) | w[2]) : (((uint64_t)w[1] << 32) | w[0]);
    /* floor(word * n / 2^64): every index in 0..n-1 gets either floor or ceil
     * of 2^64 / n words, so the law is uniform up to n / 2^64 (Eq. unique). */
    unsigned __int128 prod = (unsigned __int128)word * (unsigned __int128)(uint64_t)n;
    return (int64_t)(uint64_t)(prod >> 64);
}

void orc_xi_optimal(const orc_problem* pr, double* q, double* Q)
{
    int64_t m = pr->m, n = pr->n, p = pr->p;
    double run = 0.0;
    for (int64_t j = 0; j < n; ++j) {
        double ea = 0.0, eb = 0.0;   /* E||A_{:,j}||^2 and E||B_{j,:}||^2: E[(M + S Z)^2] = M^2 + S^2 */
        for (int64_t i = 0; i < m; ++i) {
            double mm = pr->M[i * n + j] * pr->M[i * n + j];
            double ss = pr->S[i * n + j] * pr->S[i * n + j];
            ea += mm + ss;
        }
        for (int64_t k = 0; k < p; ++k) {
            double mm = pr->Mp[j * p + k] * pr->Mp[j * p + k];
            double ss = pr->Sp[j * p + k] * pr->Sp[j * p + k];
            eb += mm + ss;
        }
        q[j] = sqrt(ea * eb);
        run += q[j];
        Q[j] = run;
    }
}

int64_t orc_index_xi(uint32_t seed_idx, uint32_t problem_id, int l, uint64_t s, int64_t t, int64_t n,
                     const double* q, const double* Q)
{
    uint32_t ctr[4] = { (uint32_t)(t >> 1), 0xFFFFFFFFu, (uint32_t)s, level_sample_word(l, s) };
    uint32_t key[2] = { seed_idx, problem_id };
    uint32_t w[4];
    orc_philox4x32_10(ctr, key, w);
    uint64_t word = (t & 1) ? (((uint64_t)w[3] << 32) | w[2]) : (((uint64_t)w[1] << 32) | w[0]);
    double u = (double)(word >> 11) * 0x1p-53;
    double x = u * Q[n - 1];
    if (!(x < Q[n - 1])) {
        int64_t j = n - 1;
        while (j > 0 && !(q[j] > 0.0)) --j;
        return j;
    }
    /* smallest j with x < Q[j] */
    int64_t lo = 0, hi = n - 1;
    while (lo < hi) {
        int64_t mid = lo + (hi - lo) / 2;
        if (x < Q[mid])
            hi = mid;
        else
            lo = mid + 1;
    }
    return lo;
}

int64_t orc_cl(const orc_levels* lv, int l)
{
    int64_t c = lv->c0;
    for (int i = 0; i < l; ++i) c *= lv->R;
    return c;
}

double orc_cost(const orc_levels* lv, int l)
{
    if (l == 0) return (double)orc_cl(lv, 0);
    return (double)orc_cl(lv, l) + (double)orc_cl(lv, l - 1);
}

/* ------------------------------------------------------------------------- */
/* Reduced-precision roundings, written from the format definitions:
 *   bfloat16: 1 sign, 8 exponent (bias 127), 7 fraction bits; same exponent
 *             range as binary32, so the spacing below 2^-126 is 2^-133.
 *   OCP FP8 E4M3: 1 sign, 4 exponent (bias 7), 3 fraction bits; normal
 *             numbers from 2^-6 up to 448 = 1.75 * 2^8, subnormal spacing 2^-9,
 *             no infinities.  Saturating conversion clamps to +-448. */

static double round_to_spacing(double x, double spacing)
{
    /* x / spacing and the product below are exact (spacing is a power of two
     * inside the double range); rint rounds half to even in the default mode. */
    return rint(x / spacing) * spacing;
}

double orc_round_bf16(double x)
{
    if (x == 0.0 || isnan(x) || isinf(x)) return x;
    int e = ilogb(x); /* |x| in [2^e, 2^(e+1)) */
    if (e < -126) e = -126;
    return round_to_spacing(x, ldexp(1.0, e - 7));
}

double orc_round_e4m3(double x)
{
    if (x == 0.0 || isnan(x)) return x;
    double ax = fabs(x);
    if (ax >= 448.0) return copysign(448.0, x);
    int e = ilogb(ax);
    if (e < -6) e = -6;
    double r = round_to_spacing(ax, ldexp(1.0, e - 3));
    if (r > 448.0) r = 448.0;
    return copysign(r, x);
}

/* Stochastic rounding to the E4M3 grid: |y| lies in [lo, lo + h) with lo on the grid and h the
 * grid spacing there; the result is lo + h when (d + 1/2) 2^-16 < (|y| - lo) / h for the 16-bit
 * dither d, else lo, with the sign of y.  A uniform d makes the rounding unbiased up to the
 * dither's resolution: averaged over the 2^16 dithers the result is y within 2^-17 h. */
double orc_round_e4m3_sr(double y, uint32_t d)
{
    if (y == 0.0 || isnan(y)) return y;
    double ay = fabs(y);
    if (ay >= 448.0) return copysign(448.0, y);
    int e = ilogb(ay);
    if (e < -6) e = -6;
    double h = ldexp(1.0, e - 3);
    double lo = floor(ay / h) * h;
    double f = (ay - lo) / h;                       /* exact: h is a power of two */
    double r = (f * 65536.0 > (double)(d & 0xFFFFu) + 0.5) ? lo + h : lo;
    return copysign(r, y);
}

/* Dither of the E4M3 rounding of the sampled entry in row `row` (a row of A, or a column of B)
 * and slot t of sample s of level l: Philox4x32-10 with the entry's key (seed_A or seed_B,
 * problem) and counter (row / 4, 2^31 + t / 2, s_lo, level word) -- a stream of its own: the
 * normals use counter word 1 = k < 2^31 and the indices 2^32 - 1 -- word row mod 4, its low 16
 * bits for even t and its high 16 bits for odd t. */
uint32_t orc_e4m3_dither(uint32_t seed, uint32_t problem_id, int l, uint64_t s, int64_t row, int64_t t)
{
    uint32_t ctr[4] = { (uint32_t)(row >> 2), 0x80000000u | (uint32_t)(t >> 1), (uint32_t)s, level_sample_word(l, s) };
    uint32_t key[2] = { seed, problem_id };
    uint32_t w[4];
    orc_philox4x32_10(ctr, key, w);
    uint32_t word = w[row & 3];
    return (t & 1) ? (word >> 16) : (word & 0xFFFFu);
}

double orc_e4m3_block_scale(double absmax)
{
    if (!(absmax > 0.0)) return 1.0;
    /* smallest integer e with absmax <= 448 * 2^e */
    int e = ilogb(absmax) - 9;
    while (absmax > ldexp(448.0, e)) ++e;
    return ldexp(1.0, e);
}

/* ------------------------------------------------------------------------- */
/* The sketch (Eq. matrixsketch, uniform xi): (1/cnt) sum A[:,r] B[r,:] / (1/n). */

void orc_sketch(int64_t m, int64_t n, int64_t p, const double* A, const double* B,
                const int64_t* idx, int64_t off, int64_t stride, int64_t cnt, double* out)
{
    memset(out, 0, sizeof(double) * (size_t)(m * p));
    for (int64_t j = 0; j < cnt; ++j) {
        int64_t r = idx[off + j * stride];
        for (int64_t i = 0; i < m; ++i) {
            double a = A[i * n + r];
            for (int64_t c = 0; c < p; ++c) out[i * p + c] += a * B[r * p + c];
        }
    }
    double scale = (double)n / (double)cnt;
    for (int64_t e = 0; e < m * p; ++e) out[e] *= scale;
}

/* ------------------------------------------------------------------------- */
/* One coupled sample (Alg. 1): one realisation of A and B, c_l draws, the fine
 * estimate from all draws and the coarse one from draws r_{jR}. */

typedef struct {
    int64_t c;       /* c_l */
    int64_t* r;      /* c_l drawn indices */
    double* Asel;    /* m x c_l: column t is A[:, r_t] of this realisation */
    double* Bsel;    /* c_l x p: row t is B[r_t, :] of this realisation */
    double* Aabs;    /* m x c_l: |M| + |S| |Z| of the same entries */
    double* Babs;    /* c_l x p: |M'| + |S'| |Z'| of the same entries */
    double* g;       /* c_l: 1 under xi^u (the n is in the estimate's scale); Q[n-1] / q[r_t] = 1 / xi**_{r_t} */
} realisation;

/* Block-scaled E4M3 of the sampled A (along_rows: blocks of 32 consecutive slots within each row)
 * or of the sampled B (blocks of 32 consecutive slots within each column): the block's scale
 * 2^e from its absmax, then every entry x -> 2^e q(x / 2^e), q the E4M3 rounding -- stochastic
 * (orc_round_e4m3_sr with the entry's dither, seed = the seed of A or of B) when sr is set, else
 * round to nearest even. */
static void quantise_e4m3_blocks(double* X, int64_t rows, int64_t cols, int along_rows, int sr,
                                 uint32_t seed, uint32_t problem_id, int l, uint64_t s)
{
    int64_t outer = along_rows ? rows : cols;
    int64_t inner = along_rows ? cols : rows;
    for (int64_t o = 0; o < outer; ++o) {
        for (int64_t b0 = 0; b0 < inner; b0 += 32) {
            int64_t b1 = b0 + 32 < inner ? b0 + 32 : inner;
            double absmax = 0.0;
            for (int64_t t = b0; t < b1; ++t) {
                double v = along_rows ? X[o * cols + t] : X[t * cols + o];
                if (fabs(v) > absmax) absmax = fabs(v);
            }
            double scale = orc_e4m3_block_scale(absmax);
            for (int64_t t = b0; t < b1; ++t) {
                double* v = along_rows ? &X[o * cols + t] : &X[t * cols + o];
                double q = sr ? orc_round_e4m3_sr(*v / scale, orc_e4m3_dither(seed, problem_id, l, s, o, t))
                              : orc_round_e4m3(*v / scale);
                *v = q * scale;
            }
        }
    }
}

static int draw_realisation(const orc_problem* pr, const orc_levels* lv, int l, uint64_t s,
                            int quant, realisation* rz)
{
    int64_t m = pr->m, n = pr->n, p = pr->p;
    int64_t c = orc_cl(lv, l);
    rz->c = c;
    rz->r = NULL; rz->Asel = rz->Bsel = rz->Aabs = rz->Babs = rz->g = NULL;
    rz->r = (int64_t*)malloc(sizeof(int64_t) * (size_t)c);
    rz->g = (double*)malloc(sizeof(double) * (size_t)c);
    rz->Asel = (double*)malloc(sizeof(double) * (size_t)(m * c));
    rz->Bsel = (double*)malloc(sizeof(double) * (size_t)(c * p));
    rz->Aabs = (double*)malloc(sizeof(double) * (size_t)(m * c));
    rz->Babs = (double*)malloc(sizeof(double) * (size_t)(c * p));
    if (!rz->r || !rz->g || !rz->Asel || !rz->Bsel || !rz->Aabs || !rz->Babs) return -1;
    for (int64_t t = 0; t < c; ++t) {
        if (pr->Q) {
            rz->r[t] = orc_index_xi(pr->seed_idx, pr->problem_id, l, s, t, n, pr->q, pr->Q);
            rz->g[t] = pr->Q[n - 1] / pr->q[rz->r[t]];
        } else {
            rz->r[t] = orc_index(pr->seed_idx, pr->problem_id, l, s, t, n);
            rz->g[t] = 1.0;
        }
    }
    for (int64_t t = 0; t < c; ++t) {
        int64_t k = rz->r[t];
        for (int64_t i = 0; i < m; ++i) {
            double z = orc_normal(pr->seed_A, pr->problem_id, l, s, i, k);
            rz->Asel[i * c + t] = pr->M[i * n + k] + pr->S[i * n + k] * z;
            rz->Aabs[i * c + t] = fabs(pr->M[i * n + k]) + fabs(pr->S[i * n + k] * z);
        }
        for (int64_t j = 0; j < p; ++j) {
            double z = orc_normal(pr->seed_B, pr->problem_id, l, s, j, k);
            rz->Bsel[t * p + j] = pr->Mp[k * p + j] + pr->Sp[k * p + j] * z;
            rz->Babs[t * p + j] = fabs(pr->Mp[k * p + j]) + fabs(pr->Sp[k * p + j] * z);
        }
    }
    if (quant == ORC_QUANT_BF16) {
        for (int64_t e = 0; e < m * c; ++e) rz->Asel[e] = orc_round_bf16(rz->Asel[e]);
        for (int64_t e = 0; e < c * p; ++e) rz->Bsel[e] = orc_round_bf16(rz->Bsel[e]);
    } else if (quant == ORC_QUANT_E4M3 || quant == ORC_QUANT_E4M3_RNE) {
        int sr = quant == ORC_QUANT_E4M3;
        quantise_e4m3_blocks(rz->Asel, m, c, 1, sr, pr->seed_A, pr->problem_id, l, s);
        quantise_e4m3_blocks(rz->Bsel, c, p, 0, sr, pr->seed_B, pr->problem_id, l, s);
    }
    return 0;
}

static void free_realisation(realisation* rz)
{
    free(rz->r);
    free(rz->g);
    free(rz->Asel);
    free(rz->Bsel);
    free(rz->Aabs);
    free(rz->Babs);
}

/* out = scale * sum_{slots t = first, first+stride, ...} Asel[:,t] Bsel[t,:];
 * if mag != NULL, mag += |scale| * sum Aabs[i,t] Babs[t,j] over the same t. */
static void sampled_sum(int64_t m, int64_t p, const realisation* rz, int64_t first, int64_t stride,
                        double scale, double* out, double* mag)
{
    int64_t c = rz->c;
    memset(out, 0, sizeof(double) * (size_t)(m * p));
    for (int64_t t = first; t < c; t += stride) {
        double g = rz->g[t];
        for (int64_t i = 0; i < m; ++i) {
            double a = rz->Asel[i * c + t];
            for (int64_t j = 0; j < p; ++j) {
                double b = rz->Bsel[t * p + j];
                out[i * p + j] += a * (g * b);
                if (mag) mag[i * p + j] += fabs(scale) * g * rz->Aabs[i * c + t] * rz->Babs[t * p + j];
            }
        }
    }
    for (int64_t e = 0; e < m * p; ++e) out[e] *= scale;
}

double orc_f(int fkind, double x)
{
    switch (fkind) {
    case ORC_F_IDENTITY: return x;
    case ORC_F_ABS_STEP: return (2.0 - x >= 0.0) ? fabs(x) : 0.0;   /* |x| H(2 - x), H(0) = 1 */
    default: return NAN;
    }
}

void orc_sample_f(const orc_problem* pr, const orc_levels* lv, int l, uint64_t s, int quant, int fkind,
                  double* D, double* Pf, double* Pc, double* mag)
{
    int64_t m = pr->m, n = pr->n, p = pr->p;
    size_t sz = sizeof(double) * (size_t)(m * p);
    realisation rz;
    double* fine = (double*)malloc(sz);
    double* coarse = (double*)calloc((size_t)(m * p), sizeof(double));
    if (mag) memset(mag, 0, sz);
    int drawn = draw_realisation(pr, lv, l, s, quant, &rz);
    if (!fine || !coarse || drawn != 0) {
        for (int64_t e = 0; e < m * p; ++e) D[e] = NAN;
        free_realisation(&rz);
        free(fine);
        free(coarse);
        return;
    }
    int64_t c = rz.c;
    /* fine: all c_l draws, scale n / c_l */
    /* under xi** the 1 / xi_{r_t} are per slot (in g) and the scale is 1 / c */
    double nn = pr->Q ? 1.0 : (double)n;
    sampled_sum(m, p, &rz, 0, 1, nn / (double)c, fine, mag);
    if (l > 0) {
        /* coarse: draws r_{jR}, j = 1..c_{l-1} (0-based slots jR - 1), scale n / c_{l-1} */
        int64_t cc = c / lv->R;
        sampled_sum(m, p, &rz, lv->R - 1, lv->R, nn / (double)cc, coarse, mag);
    }
    /* P_l - P_{l-1} with the targeted function applied to each estimate (Alg. 1); at l = 0
     * there is no coarse estimate */
    for (int64_t e = 0; e < m * p; ++e)
        D[e] = l > 0 ? orc_f(fkind, fine[e]) - orc_f(fkind, coarse[e]) : orc_f(fkind, fine[e]);
    if (Pf) memcpy(Pf, fine, sz);
    if (Pc) memcpy(Pc, coarse, sz);
    free_realisation(&rz);
    free(fine);
    free(coarse);
}

void orc_sample(const orc_problem* pr, const orc_levels* lv, int l, uint64_t s, int quant,
                double* D, double* Pf, double* Pc, double* mag)
{
    orc_sample_f(pr, lv, l, s, quant, ORC_F_IDENTITY, D, Pf, Pc, mag);
}

/* ------------------------------------------------------------------------- */
/* Per-level statistics (Eq. hatYl and the single-sample variance V_l of
 * Remark 3.6): Welford's running mean and second moment per entry. */

typedef struct {
    uint64_t count;
    double* mean;  /* m x p */
    double* m2;    /* m x p */
    double* mag;   /* m x p running mean of mag, may be NULL */
} welford;

static void welford_add_samples(const orc_problem* pr, const orc_levels* lv, int l, uint64_t s0,
                                uint64_t N, int quant, int fkind, welford* w)
{
    int64_t mp = pr->m * pr->p;
    double* D = (double*)malloc(sizeof(double) * (size_t)mp);
    double* mg = w->mag ? (double*)malloc(sizeof(double) * (size_t)mp) : NULL;
    for (uint64_t k = 0; k < N; ++k) {
        orc_sample_f(pr, lv, l, s0 + k, quant, fkind, D, NULL, NULL, mg);
        w->count += 1;
        double inv = 1.0 / (double)w->count;
        for (int64_t e = 0; e < mp; ++e) {
            double delta = D[e] - w->mean[e];
            w->mean[e] += delta * inv;
            w->m2[e] += delta * (D[e] - w->mean[e]);
            if (mg) w->mag[e] += (mg[e] - w->mag[e]) * inv;
        }
    }
    free(D);
    free(mg);
}

static double welford_total_m2(const welford* w, int64_t mp)
{
    double t = 0.0;
    for (int64_t e = 0; e < mp; ++e) t += w->m2[e];
    return t;
}

void orc_level_stats_f(const orc_problem* pr, const orc_levels* lv, int l, uint64_t s0, uint64_t N,
                       int quant, int fkind, double* mean, double* M2, double* mag_mean)
{
    int64_t mp = pr->m * pr->p;
    welford w;
    w.count = 0;
    w.mean = mean;
    w.m2 = (double*)calloc((size_t)mp, sizeof(double));
    w.mag = mag_mean;
    memset(mean, 0, sizeof(double) * (size_t)mp);
    if (mag_mean) memset(mag_mean, 0, sizeof(double) * (size_t)mp);
    welford_add_samples(pr, lv, l, s0, N, quant, fkind, &w);
    *M2 = welford_total_m2(&w, mp);
    free(w.m2);
}

void orc_level_stats(const orc_problem* pr, const orc_levels* lv, int l, uint64_t s0, uint64_t N,
                     int quant, double* mean, double* M2, double* mag_mean)
{
    orc_level_stats_f(pr, lv, l, s0, N, quant, ORC_F_IDENTITY, mean, M2, mag_mean);
}

/* ------------------------------------------------------------------------- */
/* Allocation (Remark 3.6) and the driver (Alg. 2 with a fixed finest level). */

int orc_allocate(int L, const double* V, const double* C, double eps, double nl_scale,
                 int64_t pilot, int64_t* Nl)
{
    if (L < 0 || !(eps > 0.0) || !(nl_scale > 0.0)) return -1;
    double sum = 0.0;
    for (int j = 0; j <= L; ++j) {
        if (!(V[j] >= 0.0) || !(C[j] > 0.0)) return -1;
        sum += sqrt(V[j] * C[j]);
    }
    for (int l = 0; l <= L; ++l) {
        double target = nl_scale * 2.0 / (eps * eps) * sqrt(V[l] / C[l]) * sum;
        int64_t n_l = (int64_t)ceil(target);
        Nl[l] = n_l > pilot ? n_l : pilot;
    }
    return 0;
}

static double mean_norm(const welford* w, int64_t mp)
{
    double t = 0.0;
    for (int64_t e = 0; e < mp; ++e) t += w->mean[e] * w->mean[e];
    return sqrt(t);
}

int orc_estimate_f(const orc_problem* pr, const orc_levels* lv, double eps, int64_t pilot, double nl_scale,
                   int quant, int fkind, int adaptive, double* Yhat, int* L_used, int64_t* Nl, double* V,
                   double* means)
{
    int Lmax = lv->L;
    int64_t mp = pr->m * pr->p;
    if (Lmax < 0 || pilot < 2 || !(eps > 0.0)) return -1;
    welford* acc = (welford*)calloc((size_t)(Lmax + 1), sizeof(welford));
    double* C = (double*)malloc(sizeof(double) * (size_t)(Lmax + 1));
    for (int l = 0; l <= Lmax; ++l) {
        acc[l].mean = (double*)calloc((size_t)mp, sizeof(double));
        acc[l].m2 = (double*)calloc((size_t)mp, sizeof(double));
        acc[l].mag = NULL;
        C[l] = orc_cost(lv, l);
    }
    /* Alg. 2: fixed L runs one round on levels 0..L.  Adaptive: rounds on levels 0..L for
     * L = 0, 1, ...; each round pilots the new finest level, re-allocates every level from the
     * variances of all samples held and tops them up (never discarding samples); the loop stops
     * once at least three levels are in and the finest level's mean satisfies
     * ||Y_L||_F < (sqrt(R) + 1) eps / sqrt(2) (Remark 3.5, Eq. L_num_bound_matrix), or at the
     * largest L. */
    int L = adaptive ? 0 : Lmax;
    int rc = 0;
    for (;;) {
        for (int l = 0; l <= L; ++l) {
            uint64_t have = acc[l].count;
            if (have < (uint64_t)pilot) welford_add_samples(pr, lv, l, have, (uint64_t)pilot - have, quant, fkind, &acc[l]);
            V[l] = welford_total_m2(&acc[l], mp) / (double)(acc[l].count - 1);
        }
        rc = orc_allocate(L, V, C, eps, nl_scale, pilot, Nl);
        if (rc != 0) break;
        for (int l = 0; l <= L; ++l) {
            uint64_t have = acc[l].count;
            if ((uint64_t)Nl[l] > have)
                welford_add_samples(pr, lv, l, have, (uint64_t)Nl[l] - have, quant, fkind, &acc[l]);
            Nl[l] = (int64_t)acc[l].count;
            V[l] = welford_total_m2(&acc[l], mp) / (double)(acc[l].count - 1);
        }
        if (!adaptive || L == Lmax) break;
        if (L >= 2 && mean_norm(&acc[L], mp) < (sqrt((double)lv->R) + 1.0) * eps / sqrt(2.0)) break;
        L += 1;
    }
    if (rc == 0) {
        /* telescoping sum (Eq. hatY) */
        for (int64_t e = 0; e < mp; ++e) {
            double y = 0.0;
            for (int l = 0; l <= L; ++l) y += acc[l].mean[e];
            Yhat[e] = y;
        }
        if (means)
            for (int l = 0; l <= L; ++l)
                memcpy(means + (size_t)l * (size_t)mp, acc[l].mean, sizeof(double) * (size_t)mp);
        if (L_used) *L_used = L;
    }
    for (int l = 0; l <= Lmax; ++l) {
        free(acc[l].mean);
        free(acc[l].m2);
    }
    free(acc);
    free(C);
    return rc;
}

int orc_estimate(const orc_problem* pr, const orc_levels* lv, double eps, int64_t pilot,
                 double nl_scale, int quant, double* Yhat, int64_t* Nl, double* V, double* means)
{
    return orc_estimate_f(pr, lv, eps, pilot, nl_scale, quant, ORC_F_IDENTITY, 0, Yhat, NULL, Nl, V, means);
}

/* ------------------------------------------------------------------------- */
/* Reparameterised adjoint.  Yhat is linear in each sampled product a b^T with
 * a = A[:, r_t], b = B[r_t, :]; d<G, w a b^T>/da = w G b and /db = w G^T a.
 * With A = M + S o Z: dM += dA, dS += Z o dA (likewise for B). */

static void adjoint_terms(const orc_problem* pr, const realisation* rz, int l, uint64_t s,
                          int64_t first, int64_t stride, double weight, const double* G,
                          double* dM, double* dS, double* dMp, double* dSp)
{
    int64_t m = pr->m, n = pr->n, p = pr->p, c = rz->c;
    for (int64_t t = first; t < c; t += stride) {
        int64_t k = rz->r[t];
        for (int64_t i = 0; i < m; ++i) {
            double g = 0.0; /* (G b)_i */
            for (int64_t j = 0; j < p; ++j) g += G[i * p + j] * rz->Bsel[t * p + j];
            g *= weight * rz->g[t];
            double z = orc_normal(pr->seed_A, pr->problem_id, l, s, i, k);
            dM[i * n + k] += g;
            dS[i * n + k] += g * z;
        }
        for (int64_t j = 0; j < p; ++j) {
            double h = 0.0; /* (G^T a)_j */
            for (int64_t i = 0; i < m; ++i) h += G[i * p + j] * rz->Asel[i * c + t];
            h *= weight * rz->g[t];
            double z = orc_normal(pr->seed_B, pr->problem_id, l, s, j, k);
            dMp[k * p + j] += h;
            dSp[k * p + j] += h * z;
        }
    }
}

void orc_adjoint(const orc_problem* pr, const orc_levels* lv, const int64_t* Nl, const double* G,
                 int quant, double* dM, double* dS, double* dMp, double* dSp)
{
    int64_t m = pr->m, n = pr->n, p = pr->p;
    memset(dM, 0, sizeof(double) * (size_t)(m * n));
    memset(dS, 0, sizeof(double) * (size_t)(m * n));
    memset(dMp, 0, sizeof(double) * (size_t)(n * p));
    memset(dSp, 0, sizeof(double) * (size_t)(n * p));
    for (int l = 0; l <= lv->L; ++l) {
        if (Nl[l] <= 0) continue;
        double inv_n = 1.0 / (double)Nl[l];
        for (int64_t s = 0; s < Nl[l]; ++s) {
            realisation rz;
            if (draw_realisation(pr, lv, l, (uint64_t)s, quant, &rz) != 0) {
                free_realisation(&rz);
                return;
            }
            int64_t c = rz.c;
            /* + fine estimate */
            double nn = pr->Q ? 1.0 : (double)n;   /* xi**: the 1 / xi are per slot */
            adjoint_terms(pr, &rz, l, (uint64_t)s, 0, 1, inv_n * nn / (double)c, G,
                          dM, dS, dMp, dSp);
            if (l > 0) {
                /* - coarse estimate */
                int64_t cc = c / lv->R;
                adjoint_terms(pr, &rz, l, (uint64_t)s, lv->R - 1, lv->R,
                              -inv_n * nn / (double)cc, G, dM, dS, dMp, dSp);
            }
            free_realisation(&rz);
        }
    }
}
