// internal.h -- declarations shared by the CUDA sources of libmlmc (not part of the ABI).
#pragma once

#include <cstdint>
#include <cuda.h>
#include <cuda_runtime.h>

#include "mlmc.h"
#include "rng.cuh"

namespace mlmc {

// Samples are grouped into fixed chunks of consecutive sample ids (chunk c of a
// level holds ids c*chunk .. c*chunk+chunk-1).  Partial statistics are produced
// per chunk and folded into a level in chunk order, so the result does not
// depend on grid shapes, and a split of sample ranges at chunk boundaries
// changes only the rounding of M2's between-chunk terms (summed per launch).
// The plan's kernels use chunk_samples(c_l) (8 to 64, a power of two: cheap
// samples get longer chunks: the longest with at most 8192 sampled products, or 8
// samples; this bounds the FP32 accumulation of a chunk sum); the no-allocation
// entry point uses kChunk.
constexpr int kChunk = 8;
constexpr int kMaxChunkSamples = 64;
inline int chunk_samples(int64_t c_l)
{
    int ch = 8;
    while (ch < kMaxChunkSamples && int64_t(ch) * 2 * c_l <= 8192) ch *= 2;
    return ch;
}

// Tensor maps of the interleaved parameter table for the tensor-core kernel's row gathers: the
// table seen as n rows of (m_pad + p_pad) 8-byte (M, S) pairs, with a box of one row and
// `wa` (A part) or `wb` (B part) pairs.  valid = 0: gather with plain bulk copies instead.
struct TcMaps {   // CUtensorMap brings its own 64-byte alignment
    CUtensorMap a;
    CUtensorMap b;
    int wa, wb, valid, pad;
};

// Arguments of one level-kernel launch over samples [s_begin, s_end).
struct LevelParams {
    const void* PA;       // row k: (M_ik, S_ik) pairs, i < m_pad (gathered column k of [M|S])
    const void* PB;       // row k: (M'_kj, S'_kj) pairs, j < p_pad (gathered row k of [M'|S'])
    int64_t ldPA, ldPB;   // elements between consecutive rows k of PA / PB
    int64_t n;
    int m, p, m_pad, p_pad;
    int l;                // level
    int c;                // c_l sampled indices
    int R;                // ratio; slot t is also coarse iff t % R == R - 1 (and l > 0)
    double w_fine;        // n / c_l
    double w_coarse;      // n / c_l - n / c_{l-1}
    uint2 keyA, keyB, keyI;
    PhiloxRoundKeys rkA, rkB;  // round keys of keyA and keyB
    uint64_t s_begin, s_end;
    uint64_t chunk0;      // absolute chunk id handled by blockIdx.y == 0
    int chunk;            // samples per chunk
    int nchunks;
    int tiles_m, tiles_p;
    void* partial_sum;    // [nchunks][m][p] of T
    double* partial_q;    // [nchunks][tiles_m * tiles_p]: each chunk's M2 over the tile's entries
    const double* xi_q;   // xi** (CUDA-core kernel): weights q (n), or null for the uniform law
    const double* xi_Q;   // their running sums (n)
    double xi_Qtot;       // Q[n-1]
    const int* xi_G;      // guide table of the running sums (n buckets)
    int cc_tile;          // CUDA-core kernel: output tile id 1000 rows + columns (0 or 64064: 64 x 64)
    int pack;             // tensor-core kernel, 128-row tiles: two samples per accumulator (m <= 64, c % 16 == 0)
    int welford;          // tensor-core kernel: grow each chunk's M2 sample by sample (Welford); 0: levels whose
                          // mean is zero by construction keep the raw sum of ||D||^2 and subtract ||S||^2 / n
                          // at the chunk's end (no cancellation when the mean is zero)
    TcMaps maps;          // tensor-core kernel only
};

// Tile geometry of the CUDA-core level kernel.
struct CudaCoreTile {
    int tm, tp;
};

// Launchers (return the launch error, if any).
// f: the targeted function (mlmc_function), applied to the fine and coarse estimates apart.
cudaError_t launch_level_cuda_core_f64(const LevelParams& prm, int f, cudaStream_t st);
cudaError_t launch_level_cuda_core_f32(const LevelParams& prm, int f, cudaStream_t st);
bool cuda_core_tile_valid(int precision, int f, int id);   // id = 1000 rows + columns: 64064, 128064, 128128
int cuda_core_default_tile(int precision, int f, int64_t m);
CudaCoreTile cuda_core_tile(int id);
// The inner-product case m = p = 1 (uniform law): one warp per sample, FP64 or FP32.
cudaError_t launch_level_inner(const LevelParams& prm, bool f64, int f, cudaStream_t st);

// Tensor-core (BF16) level kernel: tile of (128 * mh) rows x bn columns per CTA.
// Tensor-core tile: mh x 128 rows x bn columns per CTA; pair = 1: a cluster of two CTAs of 128
// rows each shares one 256 x bn tile (bn = 256), each generating half of B for both.
struct TcTile {
    int mh, bn, rows, pair;   // pair: 0 single CTA, 1 cluster pair, 2 cluster pair with 16 generator warps
};
struct TcLaunch {
    int* err_flag;        // device word set to an mlmc_status when a bounded wait gives up
    uint64_t timeout_ns;  // bound on every device-side wait
    float scale;          // n / c_l, applied to the FP32 accumulator
    int num_sms;
};
// Batched launch: CTA b processes items[cta_begin[b] .. cta_begin[b+1]); an item packs
// job (bits 0-15, index into jobs), the first chunk cy of a run (bits 16-39), the run length
// (bits 40-47, 1..255 chunks) and the output tile (bits 48-63).
struct TcBatch {
    const LevelParams* jobs;
    const uint64_t* items;
    const int* cta_begin;
};

// Tensor-core level kernel.  q selects the operand format: 0 = bfloat16, 1 = FP8 E4M3 with
// per-(row, 32-slot block) power-of-two scales (dequantised into the same bf16 MMA).
// Encode the row-gather maps of a table (base, n rows, ld floats per row) for a tile whose A part
// spans wa pairs and B part wb pairs (<= 256 each); returns false if the driver lacks the call.
bool tc_encode_maps(TcMaps* maps, const void* base, int64_t n, int64_t ld, int wa, int wb);
// One warp waits (bounded by timeout_ns) on an mbarrier that nothing arrives on and records
// MLMC_ERR_TIMEOUT in err_flag when it gives up.
cudaError_t launch_bounded_wait_probe(int* err_flag, uint64_t timeout_ns, cudaStream_t st);
// Pairs of the A and B parts a tile's CTA stages per slot.
int tc_stage_width_a(const TcTile& t);
int tc_stage_width_b(const TcTile& t);
// Default tile: bf16 outputs with more than 128 rows and columns use the cluster pair (single-
// problem launches, allow_pair); otherwise mh = 1 or 2 and the narrowest bn covering p.
TcTile tc_tile_for(int64_t m, int64_t p, int q, bool allow_pair);
bool tc_tile_valid(const TcTile& t, int q);
cudaError_t launch_level_tc(const LevelParams& prm, const TcTile& tile, int q, const TcLaunch& tl, cudaStream_t st);
// BF16 with a targeted function (f = 1): fine and coarse sums in two accumulators, tiles of 128
// rows and 32, 64 or 128 columns
TcTile tc_tile_for_f(int64_t p);
bool tc_tile_valid_f(const TcTile& t);
// BF16 under xi**: the CTA pair above 128 x 128, else tiles of 128 rows and at most 128 columns
TcTile tc_tile_for_xi(int64_t m, int64_t p);
bool tc_tile_valid_xi(const TcTile& t);
cudaError_t launch_level_tc_f(const LevelParams& prm, const TcTile& tile, int f, const TcLaunch& tl, cudaStream_t st);
// Whether a launch of `tile` over a level with c slots packs two samples per accumulator.
bool tc_pack(const TcTile& tile, int q, int64_t m, int64_t c);
// CTAs of a batched launch for this tile (resident CTAs per SM x SMs); 0 on error.  Also sets
// the kernel's shared-memory attribute, which launch_level_tc_batch relies on.
int tc_batch_grid(const TcTile& tile, int q, int num_sms);
cudaError_t launch_level_tc_batch(const TcBatch& bt, const TcTile& tile, int q, int grid, const TcLaunch& tl,
                                  cudaStream_t st);

// The chunks of one launch: chunk c (0-based) is absolute chunk chunk0 + c of the level and holds
// the sample ids [max(s_begin, (chunk0 + c) chunk), min(s_end, (chunk0 + c + 1) chunk)); the
// level held n_before samples before the first of them.
struct ChunkRun {
    uint64_t s_begin, s_end, chunk0, chunk;
    uint64_t n_before;
    int nchunks;
};
__host__ __device__ inline uint64_t chunk_count(const ChunkRun& r, int c)
{
    const uint64_t lo = (r.chunk0 + uint64_t(c)) * r.chunk, hi = lo + r.chunk;
    const uint64_t a = r.s_begin > lo ? r.s_begin : lo;
    const uint64_t b = r.s_end < hi ? r.s_end : hi;
    return b - a;
}

// Entry groups of the merge (one per kMergeGroup entries): the length of its scratch of
// between-chunk terms.
constexpr int kMergeGroup = 64;
int merge_groups(int64_t mp);

// One job of a batched merge: the FP32 chunk partials of an m x p level (mp entries) and their
// per-tile M2, folded into the level's FP64 sum and M2; `chan` holds merge_groups(mp) doubles.
struct MergeJob {
    const float* partial;
    const double* partial_q;
    double* sum;
    double* M2;
    double* chan;
    int64_t mp;
    ChunkRun run;   // run.nchunks <= 4096
    int tiles;
};
cudaError_t launch_merge_batch(const MergeJob* jobs, const int* njobs_dev, cudaStream_t st);

// Fold the partials of one launch into a level's FP64 state (sum, M2), in chunk order, with
// Chan's pairwise update; chan_scratch holds merge_groups(mp) doubles.
cudaError_t launch_merge_partials(const void* partial_sum, bool partial_f64, const double* partial_q, int tiles,
                                  int64_t mp, const ChunkRun& run, double* level_sum, double* level_M2,
                                  double* chan_scratch, cudaStream_t st);

// Sample counts of the levels of one problem, passed by value to kernels.
struct LevelCounts {
    uint64_t v[MLMC_MAX_LEVELS];
};

// mean = sum / N for `count` levels laid out back to back (sum, mean: count x mp),
// N[l] = counts.v[first + l].
cudaError_t launch_finalize(const double* sum, LevelCounts counts, int first, int count, int64_t mp, double* mean,
                            cudaStream_t st);

// yhat[e] = sum_l sum_l[e] / N_l over levels with N_l > 0.
cudaError_t launch_telescoping(const double* sum, LevelCounts counts, int levels, int64_t mp, double* yhat,
                               cudaStream_t st);

// Copy row-major parameters into the sample-major pair layout: element (k, i) of [M|S] goes to
// PA[k * ld_dst + 2 i + {0, 1}], element (k, j) of [M'|S'] to PB[k * ld_dst + 2 j + {0, 1}].
cudaError_t launch_layout_A(const void* M, const void* S, int src_dtype, int64_t ldA, int64_t m,
                            int64_t n, int64_t m_pad, void* PA, int64_t ld_dst, bool dst_f64, cudaStream_t st);
cudaError_t launch_layout_B(const void* Mp, const void* Sp, int src_dtype, int64_t ldB, int64_t n,
                            int64_t p, int64_t p_pad, void* PB, int64_t ld_dst, bool dst_f64, cudaStream_t st);

// ---- adjoint ----------------------------------------------------------------------------
// One batch of the adjoint's replay: entry e covers samples s0[e] .. s0[e] + (pairs of the entry)
// / ceil(c[e] / 2) - 1 of level lev[e]; pair_begin[e] is the entry's first Philox block (two
// slots) in the batch's flattened enumeration.
struct AdjLevels {
    int count;
    int lev[MLMC_MAX_LEVELS];
    int64_t c[MLMC_MAX_LEVELS];
    uint64_t s0[MLMC_MAX_LEVELS];
    int64_t pair_begin[MLMC_MAX_LEVELS];
    int64_t total_pairs;
};

struct AdjSegmentParams {
    const void* PAB;        // plan layout: row k = [(M, S) pairs of A | (M', S') pairs of B]
    int64_t ld;             // elements per row
    int m, p, m_pad;
    int64_t n;
    PhiloxRoundKeys rkA, rkB;
    const double* G;        // m x p upstream gradient
    const int64_t* offsets; // segment starts (n)
    int64_t total;          // number of records
    const uint64_t* records;
    double w_fine[MLMC_MAX_LEVELS];        // n / c_l
    double w_coarse_extra[MLMC_MAX_LEVELS];  // -n / c_{l-1} (l > 0), added on coarse slots
    double inv_N[MLMC_MAX_LEVELS];
    int bf16;               // round the regenerated operands to bfloat16 (straight-through)
    int ob;                 // register-tile width: the CTA owns 32 * ob outputs (adjoint_output_block)
    double* gM_t;           // n x m staging of dM (the kernels add to the staging)
    double* gS_t;           // n x m staging of dS
    double* gMp;            // n x p
    double* gSp;            // n x p
};

cudaError_t adjoint_count(const AdjLevels& lv, uint2 keyI, int64_t n, int R, int* counts, cudaStream_t st);
cudaError_t adjoint_scatter(const AdjLevels& lv, uint2 keyI, int64_t n, int R, int64_t* cursor, uint64_t* records,
                            cudaStream_t st);
int64_t adjoint_scan_scratch(int64_t n);
cudaError_t adjoint_scan(const int* counts, int64_t n, int64_t* offsets, int64_t* scratch, cudaStream_t st);
size_t adjoint_segment_smem(int kin, int opt, bool f64);
// Register-tile width (1, 2 or 4) for kin contracted entries; 0 if none fits in shared memory.
int adjoint_output_block(int kin, bool f64);
cudaError_t adjoint_segments(const AdjSegmentParams& prm, bool f64, int side, int num_sms, cudaStream_t st);
// Tensor-core segment reduction for BF16 plans (vectors exact in bfloat16, G split into bfloat16
// hi and lo parts): contracted dimension up to 256.
bool adjoint_tc_supported(int kin);
cudaError_t adjoint_segments_tc(const AdjSegmentParams& prm, int side, const TcLaunch& tl, cudaStream_t st);
cudaError_t adjoint_write_A(const double* src, int64_t n, int64_t m, void* dst, int64_t ld, int dtype, cudaStream_t st);
cudaError_t adjoint_write_B(const double* src, int64_t n, int64_t p, void* dst, int64_t ld, int dtype, cudaStream_t st);

// Entries per second of the generation alone (Philox4x32-10, special-function Box-Muller,
// M + S z, bfloat16) at full occupancy: the ceiling of the reduced-precision level kernels'
// entry generation.  Synchronises `st`.
cudaError_t measure_generation_rate(cudaStream_t st, int num_sms, double* entries_per_s);
// Measured operations per second of FP32 FMA, FP64 FMA, INT32 multiply-add and special-function
// sine (out[0..3]), from independent dependency chains at full occupancy.  Synchronises `st`.
cudaError_t measure_peaks(cudaStream_t st, int num_sms, double out[4]);

// xi** of Thm 3.1 from the plan's parameter layout (rows k of PA / PB hold the (M, S) pairs of
// column k of A / row k of B): q[k] = sqrt(sum_i (M^2 + S^2) * sum_j (M'^2 + S'^2)) in index order
// without contraction, Q[k] = q[0] + ... + q[k] in one sequential pass, and the guide table G
// (G[b] = the smallest j with Q[j] > b Q[n-1] / n) that lets a draw start its search near the answer.
cudaError_t launch_xi_optimal(const void* PAB, bool f64, int64_t ld, int64_t m, int64_t m_pad, int64_t n,
                              int64_t p, double* q, double* Q, int* G, cudaStream_t st);
cudaError_t launch_debug_indices_xi(uint2 keyI, int l, uint64_t s, int64_t n, int64_t t0, int64_t count,
                                    const double* Q, const double* q, const int* G, int64_t* out, cudaStream_t st);

// Set the thread-local message returned by mlmc_last_error().
mlmc_status report_error(mlmc_status st, const char* msg);

// Verification hooks.
cudaError_t launch_debug_philox(const uint32_t* ctr, const uint32_t* key, int64_t count, uint32_t* out,
                                cudaStream_t st);
cudaError_t launch_debug_indices(uint2 keyI, int l, uint64_t s, int64_t n, int64_t t0, int64_t count,
                                 int64_t* out, cudaStream_t st);
cudaError_t launch_debug_normals(uint2 key, bool f64, int l, uint64_t s, int64_t k, int64_t row0,
                                 int64_t count, double* out, cudaStream_t st);

}  // namespace mlmc
