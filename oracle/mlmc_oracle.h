/*
 * mlmc_oracle.h -- plain FP64 CPU oracle for the multilevel Monte Carlo (MLMC)
 * estimator of E[AB] (Wu & Polydorides, "A Multilevel Monte Carlo Estimator for
 * Matrix Multiplication", arXiv:1904.00429).
 *
 * TEST INFRASTRUCTURE ONLY.  This library exists so that the tests, the smoke
 * check and the CPU-baseline leg of the benchmark can compare the CUDA path
 * against an obviously correct restatement of the paper.  The product path
 * (the CUDA library and its Python binding) never links, loads or calls it,
 * and it shares no code, header, table or constant with the CUDA sources.
 *
 * Everything is single-threaded, unblocked and in the order the paper states:
 *   - the sketch Z_L = (1/c) sum_t A[:,r_t] B[r_t,:] / xi_{r_t}   (Sec. 3, Eq. matrixsketch)
 *     with uniform xi_j = 1/n                                    (Eq. unique)
 *   - coupled fine/coarse estimates of one realisation, the coarse one using
 *     every R-th draw r_{jR}                                     (Sec. 3.1, Alg. 1)
 *   - per-level sample mean Y_l and single-sample variance V_l   (Eq. hatYl, Remark 3.6)
 *   - the N_l allocation and the telescoping sum                 (Remark 3.6, Eq. hatY, Alg. 2)
 *   - the reparameterised adjoint of <G, Yhat> with respect to M, S, M', S'.
 *
 * Random numbers.  The paper leaves the generator unspecified.  Both sides of
 * the comparison implement, independently, Philox4x32-10 (Salmon, Moraes, Dror,
 * Shaw, "Parallel random numbers: as easy as 1, 2, 3", SC'11) with the counter
 * layout below, so that every draw is a pure function of its coordinates:
 *   normal of A entry (i, k), level l, sample s:
 *       key = (seed_A, problem_id), ctr = (i/4, k, s mod 2^32, (s >> 32) << 8 | l)
 *   normal of B entry (k, j): the same with seed_B and j in place of i
 *   index of slot t:
 *       key = (seed_idx, problem_id), ctr = (t/2, 0xFFFFFFFF, s mod 2^32, (s >> 32) << 8 | l)
 * A call returns four 32-bit words w0..w3.  Normals: entry q = i mod 4 uses the
 * Box-Muller pair (w0, w1) for q < 2 and (w2, w3) for q >= 2; the radius comes
 * from the first word of the pair, the angle from the second; even q takes the
 * cosine branch, odd q the sine branch.  Uniforms are u = (w + 1/2) 2^-32.
 * Indices: slot t uses the 64-bit word (w1 << 32 | w0) for even t and
 * (w3 << 32 | w2) for odd t, and r = floor(word * n / 2^64).
 * Limits: l < 256, s < 2^56, k < 2^32.
 */
#ifndef MLMC_ORACLE_H
#define MLMC_ORACLE_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

/* One problem: A = M + S o Z (m x n), B = M' + S' o Z' (n x p).  All four
 * parameter matrices are dense row-major FP64 owned by the caller. */
typedef struct {
    int64_t m, n, p;
    const double *M, *S;    /* m x n, row-major */
    const double *Mp, *Sp;  /* n x p, row-major */
    uint32_t seed_A, seed_B, seed_idx, problem_id;
    /* Sampling law of the indices: NULL for the uniform xi^u (Eq. unique); else the
     * variance-optimal xi** of Thm 3.1 (Eq. optproM) given by q[j] = sqrt(E||A_{:,j}||^2
     * E||B_{j,:}||^2) and its running sums Q[j] = q[0] + ... + q[j] (orc_xi_optimal), so that
     * xi**_j = q[j] / Q[n-1]. */
    const double* q;
    const double* Q;
} orc_problem;

/* Level schedule: c_l = c0 * R^l sampled indices at level l = 0..L. */
typedef struct {
    int64_t c0;
    int64_t R;
    int L;
} orc_levels;

/* Operand rounding applied to every sampled entry before the products
 * (emulation of the reduced-precision forms; none for the plain method). */
/* ORC_QUANT_E4M3: block-scaled E4M3 with stochastic rounding (the library's FP8 form);
 * ORC_QUANT_E4M3_RNE: the same with round to nearest even (kept to measure its bias). */
enum { ORC_QUANT_NONE = 0, ORC_QUANT_BF16 = 1, ORC_QUANT_E4M3 = 2, ORC_QUANT_E4M3_RNE = 3 };

/* The targeted function f of f^(AB), applied entrywise (Sec. 3): the identity (the
 * estimator of E[AB]), or f(x) = |x| H(2 - x) with H the Heaviside step, H(0) = 1 (the function
 * of the paper's matrix example, Sec. 5.2). */
enum { ORC_F_IDENTITY = 0, ORC_F_ABS_STEP = 1 };
double orc_f(int fkind, double x);

/* Philox4x32-10 and Philox4x64-10 block functions (Salmon et al., SC'11). */
void orc_philox4x32_10(const uint32_t ctr[4], const uint32_t key[2], uint32_t out[4]);
void orc_philox4x64_10(const uint64_t ctr[4], const uint64_t key[2], uint64_t out[4]);

/* u = (w + 1/2) 2^-32, exact in FP64, strictly inside (0, 1). */
double orc_uniform(uint32_t w);

/* Standard normal Z for entry (row, k) of level l, sample s; row is i for A and
 * j for B, k the inner (column of A / row of B) index. */
double orc_normal(uint32_t seed, uint32_t problem_id, int l, uint64_t s, int64_t row, int64_t k);

/* Sampled index r_t in {0..n-1} of slot t (uniform xi, Eq. unique). */
int64_t orc_index(uint32_t seed_idx, uint32_t problem_id, int l, uint64_t s, int64_t t, int64_t n);

/* The weights of xi** (Thm 3.1, Eq. optproM) from the entry laws: E||A_{:,j}||^2 =
 * sum_i (M_ij^2 + S_ij^2) and E||B_{j,:}||^2 = sum_k (M'_jk^2 + S'_jk^2), summed in index order;
 * q[j] = sqrt of their product; Q[j] = q[0] + ... + q[j] in index order.  n entries each. */
void orc_xi_optimal(const orc_problem* pr, double* q, double* Q);

/* Sampled index of slot t under xi**: the slot's 64-bit word (as in orc_index) gives
 * u = (word >> 11) 2^-53 in [0, 1); x = u Q[n-1] (one rounding); r_t is the smallest j with
 * x < Q[j] (inverse of the cumulative law), or the last j with q[j] > 0 if there is none. */
int64_t orc_index_xi(uint32_t seed_idx, uint32_t problem_id, int l, uint64_t s, int64_t t, int64_t n,
                     const double* q, const double* Q);

/* c_l = c0 R^l. */
int64_t orc_cl(const orc_levels* lv, int l);

/* Cost model of one sample at level l (Cor. 3.4): C_0 = c_0, C_l = c_l + c_{l-1}. */
double orc_cost(const orc_levels* lv, int l);

/* Rounding of one value to bfloat16 (round to nearest even) and to OCP FP8
 * E4M3 (round to nearest even, saturating to +-448), returned as FP64. */
double orc_round_bf16(double x);
double orc_round_e4m3(double x);

/* Stochastic rounding of y (|y| <= 448) to the E4M3 grid with the 16-bit dither d: the upper of
 * the two neighbouring grid values when (d + 1/2) 2^-16 < the fractional position of |y| between
 * them, else the lower one; unbiased over a uniform d up to 2^-17 of the spacing. */
double orc_round_e4m3_sr(double y, uint32_t d);

/* The 16-bit dither of sampled entry (row, slot t) of sample s of level l: Philox4x32-10 with key
 * (seed, problem_id) and counter (row / 4, 2^31 + t / 2, s mod 2^32, level word), word row mod 4,
 * low half for even t, high half for odd t. */
uint32_t orc_e4m3_dither(uint32_t seed, uint32_t problem_id, int l, uint64_t s, int64_t row, int64_t t);

/* The sketch of Eq. matrixsketch for given operands and index positions:
 *   out = (n / cnt) * sum_{j=0}^{cnt-1} A[:, idx[off + j*stride]] B[idx[off + j*stride], :]
 * A is m x n and B is n x p, both row-major; out is m x p. */
void orc_sketch(int64_t m, int64_t n, int64_t p, const double* A, const double* B,
                const int64_t* idx, int64_t off, int64_t stride, int64_t cnt, double* out);

/* One coupled sample of level l (Alg. 1, one loop iteration).  Outputs (each
 * m x p, row-major, any may be NULL except D):
 *   Pf  = fine estimate from all c_l draws, (1/c_l) sum_t A[:,r_t] B[r_t,:] / xi_{r_t}
 *         (Eq. matrixsketch: n/c_l times the plain sum under xi^u),
 *   Pc  = coarse estimate from the draws r_{jR}, j = 1..c_{l-1} (zero at l = 0),
 *   D   = Pf - Pc,
 *   mag = sum over the products that enter D of |weight| (|M_ik| + |S_ik Z_ik|)
 *         (|M'_kj| + |S'_kj Z'_kj|) with k = r_t: the magnitude against which
 *         rounding error, including that of the generated entries, is measured.
 * quant rounds every sampled A and B entry first (ORC_QUANT_*); for E4M3 the
 * scales are the power-of-two absmax block scales described in
 * orc_e4m3_block_scale, and the rounding is stochastic with the entries'
 * dithers (orc_e4m3_dither) unless ORC_QUANT_E4M3_RNE asks for nearest even. */
void orc_sample(const orc_problem* pr, const orc_levels* lv, int l, uint64_t s, int quant,
                double* D, double* Pf, double* Pc, double* mag);

/* The same with the targeted function: D = f(Pf) - f(Pc) entrywise for l > 0 and D = f(Pf) at
 * l = 0 (Alg. 1 with f^); Pf, Pc and mag are as above (before f). */
void orc_sample_f(const orc_problem* pr, const orc_levels* lv, int l, uint64_t s, int quant, int fkind,
                  double* D, double* Pf, double* Pc, double* mag);

/* Power-of-two scale of one block of 32 consecutive slots of one row of the
 * sampled A (or one column of the sampled B): 2^ceil(log2(absmax / 448)),
 * 1 when the block is all zero. */
double orc_e4m3_block_scale(double absmax);

/* Statistics of level l over samples s0 .. s0+N-1 (Eq. hatYl): per-entry mean
 * (m x p), the summed second central moment M2 = sum_ij sum_s (D_s,ij - mean_ij)^2,
 * and the per-entry mean of mag (may be NULL).  Welford updates in sample order. */
void orc_level_stats(const orc_problem* pr, const orc_levels* lv, int l, uint64_t s0, uint64_t N,
                     int quant, double* mean, double* M2, double* mag_mean);

/* The same with the targeted function (D as in orc_sample_f). */
void orc_level_stats_f(const orc_problem* pr, const orc_levels* lv, int l, uint64_t s0, uint64_t N,
                       int quant, int fkind, double* mean, double* M2, double* mag_mean);

/* N_l from the variance-optimal allocation (Remark 3.6, Giles' Eq. 12 with the
 * sum running over V_j C_j):  N_l = ceil(nl_scale * 2 eps^-2 sqrt(V_l / C_l)
 * sum_j sqrt(V_j C_j)), then at least `pilot`.  Returns 0, or -1 on bad input. */
int orc_allocate(int L, const double* V, const double* C, double eps, double nl_scale,
                 int64_t pilot, int64_t* Nl);

/* Alg. 2 with L fixed: `pilot` samples per level, V_l, N_l, top-ups that keep
 * the pilot samples, then Yhat = sum_l Y_l (Eq. hatY).  Outputs Yhat (m x p),
 * Nl[L+1], V[L+1] (from all samples) and, if non-NULL, the level means
 * ((L+1) x m x p).  Returns 0, or -1 on bad input. */
int orc_estimate(const orc_problem* pr, const orc_levels* lv, double eps, int64_t pilot,
                 double nl_scale, int quant, double* Yhat, int64_t* Nl, double* V, double* means);

/* Alg. 2 with the targeted function and, if adaptive, the choice of L: rounds on levels 0..L
 * for L = 0, 1, ... (each round: pilot samples on the new finest level, V_l from all samples
 * held, N_l by orc_allocate over levels 0..L, top-ups from the next unused sample id); the loop
 * ends after the first round with at least three levels whose finest mean satisfies
 * ||Y_L||_F < (sqrt(R) + 1) eps / sqrt(2) (Remark 3.5, Eq. L_num_bound_matrix), or after the
 * round with L = lv->L.  adaptive = 0: one round with L = lv->L (orc_estimate).  Outputs as in
 * orc_estimate over levels 0..*L_used; Nl and V hold the final sample counts and variances. */
int orc_estimate_f(const orc_problem* pr, const orc_levels* lv, double eps, int64_t pilot, double nl_scale,
                   int quant, int fkind, int adaptive, double* Yhat, int* L_used, int64_t* Nl, double* V,
                   double* means);

/* Gradient of <G, Yhat> for Yhat = sum_l (1/N_l) sum_{s<N_l} D_{l,s}, with the
 * draws (indices and Z) held fixed: dM, dS (m x n), dMp, dSp (n x p).  The
 * outputs are overwritten.  quant as in orc_sample (rounding treated as the
 * identity in the derivative, operands taken as rounded in the forward). */
void orc_adjoint(const orc_problem* pr, const orc_levels* lv, const int64_t* Nl, const double* G,
                 int quant, double* dM, double* dS, double* dMp, double* dSp);

#ifdef __cplusplus
}
#endif

#endif /* MLMC_ORACLE_H */
