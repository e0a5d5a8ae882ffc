/*
 * mlmc.h -- C ABI of the GB300 (sm_103a) multilevel Monte Carlo estimator of
 * E[AB] for random matrices (Wu & Polydorides, "A Multilevel Monte Carlo
 * Estimator for Matrix Multiplication", arXiv:1904.00429).
 *
 * The problem (Sec. 3): A is a random m x n matrix and B a random n x p
 * matrix with independent entries; the target is E[AB].  Entries follow the
 * Gaussian reparameterisation
 *     A_ik = M_ik + S_ik Z_ik,   B_kj = M'_kj + S'_kj Z'_kj,   Z, Z' ~ N(0,1),
 * so the caller supplies the four parameter matrices M, S (m x n) and
 * M', S' (n x p).  Level l draws c_l = c0 R^l indices r_t uniformly from
 * {0..n-1} (Eq. unique) and forms, from one realisation of A and B, the fine
 * sketch P_l = (n/c_l) sum_t A[:,r_t] B[r_t,:] (Eq. matrixsketch) and the
 * coarse sketch P_{l-1} = (n/c_{l-1}) sum_j A[:,r_{jR}] B[r_{jR},:] from every
 * R-th draw (Sec. 3.1, Alg. 1).  Sample s of level l is D = P_l - P_{l-1}
 * (D = P_0 at l = 0).  The estimator is Yhat = sum_l Y_l with Y_l the mean of
 * N_l samples of level l (Eq. hatYl, Eq. hatY); the N_l follow the
 * variance-optimal allocation of Remark 3.6 from pilot variances (Alg. 2).
 *
 * Random numbers are counter-based (Philox4x32-10, Salmon et al., SC'11), so
 * every draw is a pure function of (seed, problem, level, sample, entry):
 *   Z of A entry (i, k): key (seed_A, problem_id), counter (i/4, k, s_lo, s_hi<<8 | l)
 *   Z' of B entry (k, j): key (seed_B, problem_id), counter (j/4, k, s_lo, s_hi<<8 | l)
 *   index of slot t:      key (seed_idx, problem_id), counter (t/2, 0xFFFFFFFF, s_lo, s_hi<<8 | l)
 * with Box-Muller on word pairs (w0,w1), (w2,w3) (cosine branch for even
 * i mod 4, sine for odd), uniforms (w + 1/2) 2^-32, and indices
 * floor(word64 * n / 2^64) from (w1:w0) for even t and (w3:w2) for odd t.
 * Results therefore do not depend on grid shapes, on how sample ranges are
 * split across calls, or on the device.
 *
 * Conventions for every entry point:
 *   - Pointers named *_dev are device pointers (cudaMalloc'd or torch CUDA
 *     storage) on the device that was current when the plan was made; every
 *     other pointer is host memory.  The caller owns all memory it passes;
 *     the plan owns only its internal scratch.
 *   - Matrices are dense row-major with the stated leading dimension.
 *   - No entry point aborts, throws or prints.  Each returns an mlmc_status;
 *     the first error seen by a plan sticks and is returned by every later
 *     call on that plan.  mlmc_last_error() gives a thread-local message.
 *   - Work is enqueued on the plan's stream and is asynchronous unless the
 *     function says otherwise.  (mlmc_level_stats runs its chunk merges on a
 *     stream the plan owns, forked from the plan's stream after each level
 *     kernel and joined back into it before the call returns, so every later
 *     work on the plan's stream sees the merged statistics.)
 */
#ifndef MLMC_H
#define MLMC_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

#define MLMC_MAX_LEVELS 32

#if defined(__GNUC__)
#define MLMC_API __attribute__((visibility("default")))
#else
#define MLMC_API
#endif

typedef enum {
    MLMC_OK = 0,
    MLMC_ERR_INVALID_ARG = 1,  /* a size, pointer, level or option is out of range */
    MLMC_ERR_CUDA = 2,         /* a CUDA runtime call or kernel launch failed */
    MLMC_ERR_OOM = 3,          /* device allocation of the plan's scratch failed */
    MLMC_ERR_TIMEOUT = 4,      /* a bounded device wait gave up */
    MLMC_ERR_NUMERIC = 5,      /* a statistic became NaN or infinite */
    MLMC_ERR_UNSUPPORTED = 6,  /* valid request the library does not implement */
    MLMC_ERR_STATE = 7         /* call out of order (e.g. backward before estimate) */
} mlmc_status;

/* Arithmetic of the sampled entries and of the rank-c_l contraction.  The
 * per-level statistics, the allocation and the telescoping sum are FP64 in
 * every precision. */
typedef enum {
    MLMC_FP64 = 0,     /* FP64 entries, FP64 CUDA-core contraction */
    MLMC_FP32 = 1,     /* FP32 entries, FP32 CUDA-core contraction */
    MLMC_BF16 = 2,     /* FP32 entries rounded to bfloat16, tensor-core contraction, FP32 accumulation */
    MLMC_FP8_E4M3 = 3  /* FP32 entries scaled per 32-slot block (power of two from the block's absmax)
                          and rounded to E4M3 stochastically (a 16-bit dither per entry from a Philox
                          stream of its own), FP32 accumulation: unbiased, where rounding to nearest
                          on the E4M3 grid shrinks the entries by about 1e-3 of their mean */
} mlmc_precision;

/* Element type of the caller's parameter matrices. */
typedef enum { MLMC_DTYPE_F64 = 0, MLMC_DTYPE_F32 = 1 } mlmc_dtype;

/* One problem.  M, S: m x n with leading dimension ldA >= n; Mp, Sp: n x p
 * with leading dimension ldB >= p; all four of element type `dtype`, device
 * memory.  The plan copies them once (mlmc_plan) into its own sample-major
 * layout, so they may be freed or changed afterwards without affecting it.
 * Limits: 1 <= m, p <= 65536, 1 <= n < 2^31. */
typedef struct {
    int64_t m, n, p;
    const void* M_dev;
    const void* S_dev;
    int64_t ldA;
    const void* Mp_dev;
    const void* Sp_dev;
    int64_t ldB;
    int32_t dtype;       /* mlmc_dtype */
    int32_t L;           /* finest level of this problem; < 0 means options.L */
    uint32_t seed_A, seed_B, seed_idx, problem_id;
} mlmc_problem;

/* Level schedule and method options shared by the problems of a plan. */
typedef struct {
    int32_t c0;          /* c_0 >= 1 indices at level 0 */
    int32_t ratio;       /* R >= 2: c_l = c0 R^l (the paper's base number M) */
    int32_t L;           /* default finest level, 0 <= L < MLMC_MAX_LEVELS */
    int32_t precision;   /* mlmc_precision */
    int64_t pilot_n;     /* pilot samples per level used by mlmc_estimate (>= 2) */
    double nl_scale;     /* factor on the allocated N_l (Remark 2.6 oversampling control), > 0 */
    int64_t timeout_ns;  /* bound on any device-side wait; 0 = 2 s */
    int32_t tile_override; /* tensor-core tile: 0 = automatic; else 1000 * (rows / 128) + columns,
                              one of 1032 1064 1128 1256 2032 2064 2128 2256 (e.g. 2128 = 256 x 128;
                              E4M3: 1032 1064 1128 2032 2064), or 3256: a cluster of two CTAs of
                              128 x 256 sharing one 256 x 256 tile (BF16 and E4M3, single-problem
                              and batched launches; the BF16 default for outputs above 128 x 128,
                              whose levels with c_l >= 4096 then run on 2256, measured faster there),
                              or 4256: the same pair with 16 generator warps on 4-slot items (the
                              E4M3 default for outputs above 128 x 128; single-problem launches).  CUDA-core plans: 1000 * rows + columns
                              of the output tile, 64064; FP32 with f = identity also 128064 (its
                              default above 64 rows) and 128128 */
    int32_t adjoint_batch_log2; /* mlmc_backward replays at most 2^this sampled products per batch
                                   (0 = 26; at least c_L + 1 are always taken); scratch is 8 B each */
    int32_t f;           /* mlmc_function applied entrywise to each sketch (Sec. 3): the estimator then
                            targets E[f(AB)] with D = f(P_l) - f(P_{l-1}) (Alg. 1).  Anything but the
                            identity needs MLMC_FP64, MLMC_FP32 or MLMC_BF16 (not E4M3) and has no
                            mlmc_backward.  BF16 keeps the fine and coarse sums of a sample in two
                            tensor-memory accumulators (FP32) and applies f to each in FP32; its
                            tiles are 128 rows by 32, 64 or 128 columns (tile_override 1032, 1064,
                            1128), and mlmc_level_stats_batch evaluates its ranges in turn */
    int32_t adaptive_L;  /* 0: mlmc_estimate uses the problem's L.  1: Alg. 2 chooses L: rounds on
                            levels 0..L for L = 0, 1, ... (the new finest level gets pilot_n samples,
                            every level is re-allocated from the variances of all samples held and
                            topped up), stopping after the first round with at least three levels
                            whose finest mean satisfies ||Y_L||_F < (sqrt(R) + 1) eps / sqrt(2)
                            (Remark 3.5, Eq. L_num_bound_matrix), or at the problem's L */
    int32_t sampling;    /* mlmc_sampling: the law of the sampled indices.  MLMC_XI_OPTIMAL needs
                            MLMC_FP64, MLMC_FP32 or MLMC_BF16 (not E4M3) and has no mlmc_backward;
                            BF16 multiplies each entry of B by its slot's weight Q_{n-1} / q_k (FP32)
                            before rounding, applies 1 / c_l to the accumulator, and evaluates
                            mlmc_level_stats_batch ranges in turn */
} mlmc_options;

/* Index laws (mlmc_options.sampling). */
typedef enum {
    MLMC_XI_UNIFORM = 0, /* xi_j = 1/n (Eq. unique); index floor(word64 n / 2^64) */
    MLMC_XI_OPTIMAL = 1  /* xi**_j proportional to q_j = sqrt(E||A_{:,j}||^2 E||B_{j,:}||^2), E[(M + S Z)^2]
                            = M^2 + S^2 (Thm 3.1, Eq. optproM).  mlmc_plan computes q_j (sums over i and
                            k in index order, FP64) and Q_j = q_0 + ... + q_j (one sequential pass, so
                            plan time grows with n).  Slot t draws u = (word64 >> 11) 2^-53, x = u Q_{n-1}
                            and takes the smallest j with x < Q_j; its weight is Q_{n-1} / (c q_j) in the
                            fine estimate (and Q_{n-1} / (c_{l-1} q_j) in the coarse one) */
} mlmc_sampling;

/* Targeted functions f (mlmc_options.f). */
typedef enum {
    MLMC_F_IDENTITY = 0, /* f(x) = x: the estimator of E[AB] */
    MLMC_F_ABS_STEP = 1  /* f(x) = |x| H(2 - x), H the Heaviside step with H(0) = 1 (the paper's
                            matrix example, Sec. 5.2) */
} mlmc_function;

/* Report of one problem after mlmc_estimate. */
typedef struct {
    int32_t L;                      /* finest level used (chosen by Alg. 2 when adaptive_L) */
    int32_t bias_unmet;             /* adaptive_L: 1 if the problem's L was reached without the
                                       finest mean meeting the bound, else 0 */
    int64_t N[MLMC_MAX_LEVELS];     /* samples per level */
    double V[MLMC_MAX_LEVELS];      /* single-sample variance V_l (Remark 3.6) */
    double cost[MLMC_MAX_LEVELS];   /* C_l of the allocation: c_0, then c_l + c_{l-1} */
    double mean_norm[MLMC_MAX_LEVELS]; /* ||Y_l||_F */
    double rmse_pred;               /* sqrt(sum_l V_l / N_l) */
    double eps_abs;                 /* the requested tolerance */
    double outer_products;          /* sum_l N_l c_l sampled outer products evaluated */
} mlmc_report;

typedef struct mlmc_plan_s mlmc_plan_t;

/* ---- plan ---------------------------------------------------------------- */

/* mlmc_plan: validate `nprob` problems and the options, allocate the plan's
 * device scratch, and copy each problem's parameters into the plan's
 * sample-major layout (one gathered column of [M|S] and one gathered row of
 * [M'|S'] become contiguous).  `stream` is a cudaStream_t (NULL = legacy
 * default stream) on which every later call enqueues its work.  Statistics
 * of every (problem, level) start empty.  Synchronous with respect to the
 * host only in that the layout copy has been enqueued on return.
 * Problem statement: inputs L_A, L_B, the base number and the tolerance
 * (Alg. 1, Alg. 2). */
MLMC_API mlmc_status mlmc_plan(const mlmc_problem* problems, int32_t nprob, const mlmc_options* options,
                      void* stream, mlmc_plan_t** plan_out);

/* mlmc_plan_host: as mlmc_plan, for parameters in HOST memory (pinned or pageable): the
 * problems' M_dev, S_dev, Mp_dev, Sp_dev fields point to host arrays with the same layout and
 * leading dimensions.  The plan allocates device copies (owned by it until mlmc_plan_destroy),
 * copies the parameters on `stream` and builds its layout from them; the host arrays may be
 * reused once the stream has reached the layout copy (mlmc_synchronize).  Such a plan also owns
 * a device buffer for mlmc_telescoping_sum_host.  Problem statement as for mlmc_plan. */
MLMC_API mlmc_status mlmc_plan_host(const mlmc_problem* problems, int32_t nprob, const mlmc_options* options,
                                    void* stream, mlmc_plan_t** plan_out);

/* Release everything the plan owns (after draining its stream).  NULL is a no-op. */
MLMC_API mlmc_status mlmc_plan_destroy(mlmc_plan_t* plan);

/* ---- level statistics (Alg. 1, incremental) ---------------------------------------- */

/* mlmc_level_stats: evaluate samples s = sample_begin .. sample_begin+count-1
 * of level `level` of problem `prob` (Alg. 1, one loop iteration each) and
 * fold them into that level's running statistics: the count N, the FP64
 * per-entry sum of D and the FP64 M2 = sum_s ||D_s - mean||_F^2.  Within a
 * chunk of consecutive sample ids the kernels grow M2 by Welford's update;
 * chunks are folded into the level in chunk order by Chan's pairwise update
 * (the variance of Remark 3.6 without the cancellation of a one-pass formula).
 * Samples are pure functions of their ids, so disjoint ranges may be
 * evaluated in any order and split across calls: for any split at multiples
 * of 64 sample ids N and the per-entry sums are bit-identical (one chain of
 * FP64 additions per entry in chunk order) and M2 equal up to the rounding of
 * its between-chunk terms, which are summed per launch of chunks (bit-identical
 * too where the launches coincide, e.g. a first call of one chunk); any split
 * gives the same statistics up to rounding.  count = 0 is a no-op. */
MLMC_API mlmc_status mlmc_level_stats(mlmc_plan_t* plan, int32_t prob, int32_t level, uint64_t sample_begin,
                             uint64_t count);

/* Read the statistics of one level (synchronises the plan's stream):
 * N = samples folded so far; mean_dev (m x p FP64, device, may be NULL) =
 * Y_l = mean of D (Eq. hatYl); M2 (host, may be NULL) = sum_s ||D_s - Y_l||_F^2,
 * so V_l = M2 / (N - 1) (Remark 3.6). */
MLMC_API mlmc_status mlmc_get_level_stats(mlmc_plan_t* plan, int32_t prob, int32_t level, uint64_t* N,
                                 double* mean_dev, double* M2);

/* Accumulator state of one level for checkpointing and for merging the
 * statistics of several processes: N, the per-entry sum of D (m x p FP64,
 * device) and M2 = sum_s ||D_s - mean||_F^2 (host FP64).  Get synchronises the
 * plan's stream; set replaces the state (resume continues at sample id N; the
 * caller vouches that the state holds the sample ids 0 .. N-1, which
 * mlmc_backward relies on).  M2 must be finite and >= 0, else
 * MLMC_ERR_INVALID_ARG. */
MLMC_API mlmc_status mlmc_get_level_state(mlmc_plan_t* plan, int32_t prob, int32_t level, uint64_t* N,
                                 double* sum_dev, double* M2);
MLMC_API mlmc_status mlmc_set_level_state(mlmc_plan_t* plan, int32_t prob, int32_t level, uint64_t N,
                                 const double* sum_dev, double M2);

/* mlmc_merge_level_state: fold another state of the same level (N samples
 * disjoint from the held ones; sum_dev m x p FP64 on the plan's device; M2
 * host FP64, finite and >= 0) into the held one with Chan's pairwise update
 * (Eq. hatYl and Remark 3.6 over the union of the samples):
 *     M2 <- M2 + M2' + N N' / (N + N') ||sum/N - sum'/N'||_F^2,
 *     sum <- sum + sum',  N <- N + N'.
 * Several processes that evaluate disjoint sample ranges obtain the same
 * statistics by merging every process's state in one fixed order.  N = 0 is a
 * no-op.  The flag of mlmc_backward (ids 0 .. N-1 held) is left as it was.
 * Synchronises the plan's stream. */
MLMC_API mlmc_status mlmc_merge_level_state(mlmc_plan_t* plan, int32_t prob, int32_t level, uint64_t N,
                                            const double* sum_dev, double M2);

/* Empty the statistics of one level (level < 0: every level of the problem). */
MLMC_API mlmc_status mlmc_reset_level_stats(mlmc_plan_t* plan, int32_t prob, int32_t level);

/* ---- batched form: many problems and levels in one persistent launch ------------------ */

typedef struct {
    int32_t prob;
    int32_t level;
    uint64_t sample_begin;
    uint64_t count;
} mlmc_range;

/* mlmc_level_stats_batch: evaluate every range (samples sample_begin ..
 * sample_begin+count-1 of level `level` of problem `prob`) and fold it into
 * that level's statistics, as mlmc_level_stats on the ranges one by one in the
 * given order would.  BF16: the ranges are cut into (problem, level, chunk of
 * samples, output tile) work items, packed into waves (at most 1 GiB of chunk
 * partials, 4096 (problem, level) runs and 2^20 items each), balanced over
 * persistent CTAs longest item first, and each wave runs as one persistent
 * kernel launch plus two merge launches; up to four waves are captured in one
 * CUDA graph, which is replayed while the tile, the CTA count and the number of
 * waves stay the same.  The tile is options->tile_override if set, else the
 * autotuner's: the first call times every candidate tile on the first chunk
 * of each range and keeps the fastest for the plan (mlmc_get_batch_tile).
 * Tiles of at most 256 accumulator columns per CTA (all but 2256, including
 * the pair 3256) keep each chunk's running sum of D in tensor memory, so with
 * any of them the per-level sums of D are the same bit for bit; the 2256 tile
 * adds scaled samples in global memory and agrees with them up to FP32
 * rounding.  The CTA pair 3256 runs batched launches as clusters of two CTAs,
 * each cluster walking its own list of (job, chunks, 256 x 256 tile) items;
 * the 16-warp pair 4256 serves single-problem launches only.  The M2
 * are grouped by output tile, so they agree across tiles up to rounding; with
 * the same tile a batched call and the same ranges run one by one give the
 * same bits.  Other
 * precisions: one launch sequence per range, as mlmc_level_stats.  Problems
 * whose m x p FP32 partial exceeds 1 GiB: MLMC_ERR_UNSUPPORTED.
 * Scratch: the first BF16 call allocates 1 GiB of partials and about 40 MiB
 * of device tables (plus the same in pinned host memory) for the plan. */
MLMC_API mlmc_status mlmc_level_stats_batch(mlmc_plan_t* plan, const mlmc_range* ranges, int32_t count);

/* Tile of the batched BF16 launches as a tile id (see mlmc_options), 0 before
 * the first batched call.  timings_ms (host array of 9, may be NULL) receives
 * the autotuner's time in ms of each candidate in the order 1032 1064 1128
 * 1256 2032 2064 2128 2256 3256 (negative: not tried). */
MLMC_API mlmc_status mlmc_get_batch_tile(const mlmc_plan_t* plan, int32_t* tile_id, double* timings_ms);

/* ---- estimator (Alg. 2) ------------------------------------------------------------- */

/* mlmc_estimate: for every problem, run pilot_n samples on every level not
 * yet holding that many, take V_l, allocate N_l = ceil(nl_scale 2 eps^-2
 * sqrt(V_l/C_l) sum_j sqrt(V_j C_j)) with C_0 = c_0, C_l = c_l + c_{l-1}
 * (Remark 3.6; at least pilot_n), evaluate the missing samples pilot_n ..
 * N_l - 1 (earlier samples are kept, as Alg. 2 reuses them), and write
 * Yhat = sum_l Y_l (Eq. hatY).  With options.adaptive_L the levels are taken
 * one round at a time as described there, and Yhat sums the levels up to the
 * finest one used (mlmc_report.L).  eps_abs: host array of nprob absolute
 * Frobenius tolerances (> 0).  yhat_dev: device FP64 buffer holding every
 * problem's m x p estimate back to back in problem order.  reports: host
 * array of nprob reports, or NULL.  Synchronises the plan's stream (the
 * allocation needs the pilot variances on the host); the N_l are recorded in
 * the plan for mlmc_backward. */
MLMC_API mlmc_status mlmc_estimate(mlmc_plan_t* plan, const double* eps_abs, double* yhat_dev,
                          mlmc_report* reports);

/* The allocation step of Alg. 2 alone: from the statistics currently held
 * (every level needs N >= 2 samples), N_l = max(ceil(nl_scale 2 eps^-2
 * sqrt(V_l/C_l) sum_j sqrt(V_j C_j)), pilot_n) (Remark 3.6) for every problem,
 * without evaluating any sample.  eps_abs: host array of nprob tolerances;
 * Nl: host array of nprob x MLMC_MAX_LEVELS (row q holds problem q's levels
 * 0..L, the rest zero).  Synchronises the plan's stream. */
MLMC_API mlmc_status mlmc_allocate(mlmc_plan_t* plan, const double* eps_abs, int64_t* Nl);

/* The allocation of Remark 3.6 over levels 0..L of problem `prob` only (L at
 * most the problem's finest level; every level 0..L needs N >= 2): Nl (host
 * array of L + 1) as in mlmc_allocate for the absolute tolerance eps_abs
 * (> 0).  This is the allocation step of one round of Alg. 2's while loop,
 * for drivers that run the rounds themselves (several processes).
 * Synchronises the plan's stream. */
MLMC_API mlmc_status mlmc_allocate_levels(mlmc_plan_t* plan, int32_t prob, int32_t L, double eps_abs, int64_t* Nl);

/* The stopping test of Alg. 2's while loop on level L of problem `prob`
 * (Remark 3.5, matrix form): *met = 1 if L >= 2 and
 * ||Y_L||_F < (sqrt(R) + 1) eps_abs / sqrt(2), else 0; *mean_norm (may be
 * NULL) = ||Y_L||_F.  Synchronises the plan's stream. */
MLMC_API mlmc_status mlmc_bias_test(mlmc_plan_t* plan, int32_t prob, int32_t L, double eps_abs, int32_t* met,
                                    double* mean_norm);

/* Yhat of the current statistics without new samples: yhat_dev as above. */
MLMC_API mlmc_status mlmc_telescoping_sum(mlmc_plan_t* plan, double* yhat_dev);

/* The same written to HOST memory (every problem's m x p FP64 estimate back to back), for plans
 * made by mlmc_plan_host (else MLMC_ERR_STATE); synchronises the plan's stream (Eq. hatY). */
MLMC_API mlmc_status mlmc_telescoping_sum_host(mlmc_plan_t* plan, double* yhat_host);

/* ---- level statistics without allocation ------------------------------------------------
 * The paper has no counterpart to this entry point; it exists for callers
 * that cannot allocate device memory: code running while a stream is being
 * captured into a CUDA graph, inference-runtime plugins whose enqueue step
 * must not allocate, and applications that give all device memory to their
 * own pool at start-up.  mlmc_plan allocates (its layout copy and scratch),
 * so such callers use this instead.
 *
 * mlmc_level_stats_noalloc: evaluate samples s = sample_begin ..
 * sample_begin+count-1 of level `level` of one problem, with the same draws
 * and arithmetic as mlmc_level_stats, reading the caller's row-major
 * parameters in place (problem->M_dev etc.; dtype F64 with precision FP64,
 * or F32 with FP32; other precisions: MLMC_ERR_UNSUPPORTED).  Writes (does
 * not accumulate) sum_dev (m x p FP64, device) = sum_s D_s and *M2_dev
 * (one FP64, device) = sum_s ||D_s - mean||_F^2 (Welford within chunks of 8
 * sample ids, Chan's update across them); count = 0 writes zeros.  Of the
 * options, c0, ratio and precision are read, and f and sampling must be
 * MLMC_F_IDENTITY and MLMC_XI_UNIFORM (else MLMC_ERR_UNSUPPORTED).  Enqueued
 * on `stream` (cudaStream_t, NULL = legacy default stream).
 * Memory: calls no cudaMalloc, cudaFree or allocating library routine.  Its
 * scratch is a fixed 4 MiB array in the library's device image, present on
 * every GPU that loads the library until the process exits.  A problem is
 * accepted only if one chunk of partials fits: m*p*(8 for FP64, 4 for FP32)
 * + 8*ceil(m/64)*ceil(p/64) + 8*ceil(m*p/64), each part rounded up to 256
 * bytes, <= 4 MiB (for FP64, about m*p <= 515000); larger sizes return
 * MLMC_ERR_INVALID_ARG with a message.
 * Set-up: the first call on each device looks up the array's device address
 * (cudaGetSymbolAddress, with that device current); make that first call
 * before any stream capture starts.  The address is kept for the life of the
 * process; after cudaDeviceReset (or another teardown of the device's primary
 * context) do not call this entry point again in that process.
 * Concurrency: all calls share the one array and each call overwrites it, so
 * calls whose GPU work overlaps (different streams or threads without
 * ordering) race and give wrong results; order them on one stream or with
 * events. */
MLMC_API mlmc_status mlmc_level_stats_noalloc(const mlmc_problem* problem, const mlmc_options* options,
                                              int32_t level, uint64_t sample_begin, uint64_t count,
                                              double* sum_dev, double* M2_dev, void* stream);

/* ---- reparameterised adjoint ---------------------------------------------------------- */

/* mlmc_backward: gradient of <G, Yhat> with respect to the caller's M, S, M',
 * S' of every problem, with the draws (indices and Z) held fixed as in the
 * reparameterisation A = M + S o Z (the estimator is bilinear in (A, B), so
 * for omega_t = w_t / N_l and k = r_t the sampled product a_t b_t^T gives
 * dM[:, k] += omega G b_t, dS[:, k] += omega z_t o G b_t and the mirrored
 * terms for M', S'; Eq. matrixsketch, Eq. hatYl, Eq. hatY).  Yhat here is the
 * estimate of the statistics the plan holds, sum_l (sum of D) / N_l over the
 * levels with N_l > 0; the samples are replayed (indices and Z recomputed from
 * Philox, nothing stored by the forward), so every level must hold exactly
 * the sample ids 0 .. N_l - 1 (true after mlmc_estimate, and after
 * mlmc_level_stats calls that each start at the level's current N), else
 * MLMC_ERR_STATE; a problem with no samples at all is MLMC_ERR_STATE too.
 * G_dev: device FP64, every problem's m x p upstream gradient (row-major)
 * back to back in problem order.  dM_dev, dS_dev, dMp_dev, dSp_dev: host
 * arrays of nprob device pointers, one per problem, to m x n (leading
 * dimension ldA) and n x p (ldB) buffers of the problem's parameter dtype.
 * Gradients are written, not accumulated.  In BF16 precision the rounding of
 * the entries to bfloat16 is treated as the identity and the rounded
 * operands are used (straight-through).  Limits: n <= 2^30; the CUDA-core
 * contraction keeps a block of G with all p columns (A side) or all m rows
 * (B side) in shared memory, so m, p <= 696 (FP64) or 1584 (FP32, BF16),
 * else MLMC_ERR_UNSUPPORTED.  Scratch: the plan grows a device buffer to
 * 20n + 8 (2nm + 2np) bytes + 8 B per record of a batch (options
 * adjoint_batch_log2, default 2^26 records = 512 MiB) and keeps it until
 * mlmc_plan_destroy.  Enqueued on the plan's stream; within a problem the
 * records of one sampled column are summed in an order the sort leaves
 * unspecified, so repeated calls agree to FP64 rounding, not bitwise. */
MLMC_API mlmc_status mlmc_backward(mlmc_plan_t* plan, const double* G_dev, void* const* dM_dev,
                          void* const* dS_dev, void* const* dMp_dev, void* const* dSp_dev);

/* ---- status ------------------------------------------------------------------------ */

/* Wait for the plan's stream and return its sticky status. */
MLMC_API mlmc_status mlmc_synchronize(mlmc_plan_t* plan);

/* Number of kernels the plan has launched so far (all entry points). */
MLMC_API mlmc_status mlmc_launch_count(const mlmc_plan_t* plan, uint64_t* count);

/* Thread-local description of the last error returned on this thread ("" if none). */
MLMC_API const char* mlmc_last_error(void);

/* ---- verification hooks ----------------------------------------------------------------
 * The same device functions the kernels use, exposed so tests can compare
 * them with an independent implementation.  All write device buffers. */

/* Philox4x32-10 blocks: ctr_dev holds count counters of 4 words, key_dev
 * count keys of 2 words; out_dev receives count blocks of 4 words. */
MLMC_API mlmc_status mlmc_debug_philox(const uint32_t* ctr_dev, const uint32_t* key_dev, int64_t count,
                              uint32_t* out_dev, void* stream);

/* Indices r_t, t = t0 .. t0+count-1, of sample s at level l of problem prob. */
MLMC_API mlmc_status mlmc_debug_indices(mlmc_plan_t* plan, int32_t prob, int32_t level, uint64_t sample,
                               int64_t t0, int64_t count, int64_t* idx_dev);

/* Normals Z (which = 0, for A: rows i = row0 .. row0+count-1 of column k) or
 * Z' (which = 1, for B: columns j = row0 .. of row k), in the precision of
 * the plan's arithmetic, widened to FP64. */
MLMC_API mlmc_status mlmc_debug_normals(mlmc_plan_t* plan, int32_t prob, int32_t which, int32_t level,
                               uint64_t sample, int64_t k, int64_t row0, int64_t count, double* z_dev);

/* One sample D (m x p FP64) of level `level` computed by the same kernel
 * mlmc_level_stats launches, without touching the level's statistics. */
MLMC_API mlmc_status mlmc_debug_sample(mlmc_plan_t* plan, int32_t prob, int32_t level, uint64_t sample,
                              double* D_dev);

/* Failure detection (no counterpart in the paper): launch on the plan's stream
 * a kernel whose bounded wait can never be satisfied (an mbarrier that nothing
 * arrives on).  After timeout_ns (0 < timeout_ns <= 10 s) it gives up and
 * records MLMC_ERR_TIMEOUT in the plan's device error word, exactly as a level
 * kernel whose wait gave up does, so the next synchronising call returns
 * MLMC_ERR_TIMEOUT and the error sticks to the plan.  Nothing faults; the
 * CUDA context stays usable for other plans. */
MLMC_API mlmc_status mlmc_debug_bounded_wait(mlmc_plan_t* plan, int64_t timeout_ns);

/* Measurement (no counterpart in the paper): the rate, in entries per second, at which this GPU
 * generates the sampled entries of the reduced-precision paths on their own -- one Philox4x32-10
 * block per four normals, special-function-unit Box-Muller per pair (rng counter layout and
 * transforms as in the level kernels), A = M + S z in FP32 and the bfloat16 rounding -- with no
 * gathers, contraction or statistics, at full occupancy.  Each sampled outer product of an
 * m x p problem needs m + p entries, so (m + p) / rate is the generation bound per outer product
 * beside the HBM and tensor bounds.  Runs a warm-up and three timed launches (about 1.5 ms each
 * on a GB300) on `cuda_stream` (a cudaStream_t, NULL for the legacy default stream) and
 * synchronises it; allocates 1 KiB of device memory for the duration of the call.  Returns
 * MLMC_ERR_INVALID_ARG for a null output pointer, MLMC_ERR_CUDA on a CUDA error. */
MLMC_API mlmc_status mlmc_measure_generation_rate(void* cuda_stream, double* entries_per_s);

/* Measurement (no counterpart in the paper): arithmetic throughput of this GPU, the denominators
 * of the ALU rooflines.  ops_per_s (host array of 4) receives operations per second of
 * [0] FP32 fused multiply-add, [1] FP64 fused multiply-add, [2] INT32 multiply-add and
 * [3] special-function sine (sin.approx), each from 8 independent dependency chains per thread
 * at full occupancy (best of three launches after a warm-up; FLOP/s = 2 x FMA/s).  Runs on
 * `cuda_stream` and synchronises it; allocates 1 KiB of device memory for the call.  Returns
 * MLMC_ERR_INVALID_ARG for a null output pointer, MLMC_ERR_CUDA on a CUDA error. */
MLMC_API mlmc_status mlmc_measure_peaks(void* cuda_stream, double* ops_per_s);

#ifdef __cplusplus
}
#endif

#endif /* MLMC_H */
