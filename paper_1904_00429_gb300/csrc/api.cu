// api.cu -- host side of the C ABI declared in include/mlmc.h.
//
// The plan holds, per problem, the parameters in sample-major layout and the
// FP64 state of every level; level_stats enqueues the fused level kernel over
// bounded batches of sample chunks followed by the in-order merge; estimate
// runs Alg. 2 with the finest level fixed: pilot samples, V_l, the allocation
// of Remark 3.6 in FP64 on the host, top-ups from the next unused sample id,
// and the telescoping sum of Eq. hatY.
#include <algorithm>
#include <cmath>
#include <cstdarg>
#include <cstdio>
#include <cstdlib>
#include <cstring>
#include <new>
#include <numeric>
#include <string>
#include <vector>

#include <cuda_runtime.h>
#include <nvtx3/nvToolsExt.h>

#include "internal.h"
#include "mlmc.h"

using namespace mlmc;

namespace {

thread_local std::string g_last_error;

mlmc_status fail(mlmc_status st, const char* fmt, ...)
{
    char buf[512];
    va_list ap;
    va_start(ap, fmt);
    vsnprintf(buf, sizeof(buf), fmt, ap);
    va_end(ap);
    g_last_error = buf;
    return st;
}

constexpr size_t kPartialBudget = size_t(64) << 20;     // bytes of chunk partials per launch (CUDA cores)
constexpr size_t kPartialBudgetTc = size_t(256) << 20;  // tensor-core path: more chunks per persistent launch
constexpr int kMaxChunksPerLaunch = 4096;
constexpr int64_t kMaxCl = int64_t(1) << 30;

}  // namespace

namespace mlmc {
// Record a message for mlmc_last_error() from another translation unit.
mlmc_status report_error(mlmc_status st, const char* msg)
{
    g_last_error = msg;
    return st;
}
}  // namespace mlmc

struct ProblemState {
    mlmc_problem desc;
    int L = 0;
    int64_t m = 0, n = 0, p = 0, m_pad = 0, p_pad = 0;
    void* PAB = nullptr;   // row k: [(M_ik, S_ik) for i < m_pad | (M'_kj, S'_kj) for j < p_pad]
    int64_t ld = 0;        // elements per row of PAB
    double* sum = nullptr;    // (L+1) x m x p
    double* M2 = nullptr;     // (L+1): sum over the level's samples of ||D - mean||_F^2
    LevelCounts N{};
    int64_t Nl_est[MLMC_MAX_LEVELS] = {};
    bool prefix[MLMC_MAX_LEVELS];   // level l holds exactly the samples 0 .. N_l - 1
    bool has_estimate = false;
    ProblemState() { std::fill(prefix, prefix + MLMC_MAX_LEVELS, true); }
    int tiles_m = 1, tiles_p = 1;
    TcTile tile{0, 0, 0};   // tensor-core tile of the single-problem launches
    TcMaps maps{};          // row-gather maps of PAB for `tile`
    // BF16 problems on the CTA pair: levels with c_l >= c_wide run on the single-CTA 256 x 256
    // tile instead, which measured faster there (the pair's per-sub-block exchange outweighs its
    // cheaper per-sample drain once a sample has hundreds of sub-blocks)
    TcTile tile_wide{0, 0, 0};
    TcMaps maps_wide{};
    int tiles_m_wide = 1, tiles_p_wide = 1;
    int64_t c_wide = INT64_MAX;
    TcMaps batch_maps{};    // ... and for the plan's batched tile
    int32_t batch_maps_tile = 0;
    int max_chunks = 1;
    int cc_tile = 64064;      // CUDA-core output tile id (1000 rows + columns)
    double* xi_q = nullptr;   // xi** (MLMC_XI_OPTIMAL): weights q_k and their running sums Q_k (n each)
    double* xi_Q = nullptr;
    int* xi_G = nullptr;      // guide table of Q (n buckets)
    double xi_Qtot = 0.0;
};

struct mlmc_plan_s {
    int device = 0;
    cudaStream_t stream = nullptr;
    mlmc_options opt{};
    bool f64 = false;
    size_t elem = 4;
    std::vector<ProblemState> probs;
    // Chunk partials of a level call, two sets: the level kernel of one batch of chunks writes one
    // set while the merges of the batch before read the other, on merge_stream (forked from the
    // plan's stream by `produced`, joined back by `merged` before the call returns).
    void* partial_sum[2] = {nullptr, nullptr};
    double* partial_q[2] = {nullptr, nullptr};
    cudaStream_t merge_stream = nullptr;
    cudaEvent_t produced[2] = {nullptr, nullptr};   // a batch's partials are written (plan's stream)
    cudaEvent_t merged[2] = {nullptr, nullptr};     // a batch's partials are folded (merge_stream)
    double* dbg_sum = nullptr;    // one level's state for debug_sample
    double* dbg_M2 = nullptr;
    double* chan = nullptr;       // between-chunk terms of a merge (merge_groups(m p) of the largest problem)
    double* ext_q = nullptr;      // one M2 handed to mlmc_merge_level_state
    int* err_flag = nullptr;      // set by kernels whose bounded waits give up
    int num_sms = 1;
    uint64_t timeout_ns = 2000000000ull;
    mlmc_status sticky = MLMC_OK;
    std::string sticky_msg;
    uint64_t launches = 0;
    // adjoint scratch, grown on demand
    void* adj_buf = nullptr;
    size_t adj_bytes = 0;
    // batched launches (created on the first mlmc_level_stats_batch)
    TcTile batch_tile{0, 0, 0};
    double tune_ms[9] = {-1, -1, -1, -1, -1, -1, -1, -1, -1};
    int batch_grid = 0;
    float* batch_partial = nullptr;
    double* batch_q = nullptr;
    double* batch_chan = nullptr;   // between-chunk terms of one wave's merges
    unsigned char* batch_dev = nullptr;    // tables of kBatchMaxWaves waves
    unsigned char* batch_host = nullptr;   // pinned staging of the same
    cudaEvent_t batch_copied = nullptr;    // recorded after the last table upload
    cudaStream_t capture_stream = nullptr;
    cudaGraphExec_t batch_exec = nullptr;
    std::vector<int64_t> batch_key;
    // plans made from host buffers (mlmc_plan_host): the device copies of the parameters, and the
    // device buffer of mlmc_telescoping_sum_host
    std::vector<void*> owned;
    double* yhat_dev = nullptr;
};

namespace {

// Makes the plan's device current for the duration of a call.
struct DeviceGuard {
    int prev = -1;
    bool ok = false;
    explicit DeviceGuard(int dev)
    {
        if (cudaGetDevice(&prev) != cudaSuccess) prev = -1;
        ok = cudaSetDevice(dev) == cudaSuccess;
    }
    ~DeviceGuard()
    {
        if (prev >= 0) cudaSetDevice(prev);
    }
};

// Host-side fault injection for testing the error paths (nothing reaches the GPU):
// MLMC_FAULT=alloc  -> mlmc_plan fails as if a device allocation failed (MLMC_ERR_OOM), before
//                      any CUDA call;
// MLMC_FAULT=launch -> every level launch fails as if the launch had been refused (MLMC_ERR_CUDA);
// MLMC_FAULT=cancel -> the first call after mlmc_plan cancels the plan (MLMC_ERR_CUDA, sticky).
bool fault_is(const char* what)
{
    const char* f = std::getenv("MLMC_FAULT");
    return f && std::strcmp(f, what) == 0;
}

mlmc_status set_sticky(mlmc_plan_t* plan, mlmc_status st)
{
    if (plan && plan->sticky == MLMC_OK && st != MLMC_OK) {
        plan->sticky = st;
        plan->sticky_msg = g_last_error;
    }
    return st;
}

mlmc_status check_cuda(mlmc_plan_t* plan, cudaError_t err, const char* what)
{
    if (err == cudaSuccess) return MLMC_OK;
    fail(err == cudaErrorMemoryAllocation ? MLMC_ERR_OOM : MLMC_ERR_CUDA, "%s: %s", what, cudaGetErrorString(err));
    return set_sticky(plan, err == cudaErrorMemoryAllocation ? MLMC_ERR_OOM : MLMC_ERR_CUDA);
}

mlmc_status enter(mlmc_plan_t* plan)
{
    if (!plan) return fail(MLMC_ERR_INVALID_ARG, "null plan");
    if (plan->sticky == MLMC_OK && fault_is("cancel"))
        return set_sticky(plan, fail(MLMC_ERR_CUDA, "injected fault: plan cancelled"));
    if (plan->sticky != MLMC_OK) {
        g_last_error = plan->sticky_msg;
        return plan->sticky;
    }
    return MLMC_OK;
}

int64_t level_c(const mlmc_options& o, int l)
{
    int64_t c = o.c0;
    for (int i = 0; i < l; ++i) c *= o.ratio;
    return c;
}

double level_cost(const mlmc_options& o, int l)
{
    return l == 0 ? double(level_c(o, 0)) : double(level_c(o, l)) + double(level_c(o, l - 1));
}

uint2 key(uint32_t seed, uint32_t pid) { return make_uint2(seed, pid); }

// Tile ids: 1000 * (rows / 128) + columns, e.g. 2128 = 256 rows x 128 columns.
// 3256 = a cluster pair of 128 x 256 CTAs sharing one 256 x 256 tile.
TcTile decode_tile(int32_t id)
{
    if (id / 1000 == 3) return TcTile{1, id % 1000, 128, 1};
    if (id / 1000 == 4) return TcTile{1, id % 1000, 128, 2};   // pair with 16 generator warps
    TcTile t{id / 1000, id % 1000, 128 * (id / 1000), 0};
    return t;
}

int32_t encode_tile(const TcTile& t)
{
    if (t.mh <= 0) return 0;
    return t.pair ? (t.pair == 2 ? 4000 : 3000) + t.bn : 1000 * t.mh + t.bn;
}

const int32_t kTileIds[9] = {1032, 1064, 1128, 1256, 2032, 2064, 2128, 2256, 3256};
// BF16 single-problem launches on the CTA pair switch to the 256 x 256 single-CTA tile from this
// many slots per sample on (measured on 256 x 65536 x 256: at c_l = 4096, 8192, 16384 the single
// CTA took 4 %, 8 %, 10 % less time than the pair; at 2048 and below it took more)
constexpr int64_t kWideTileFromC = 4096;

mlmc_status validate(const mlmc_problem* problems, int32_t nprob, const mlmc_options* o)
{
    if (!problems || nprob < 1) return fail(MLMC_ERR_INVALID_ARG, "need at least one problem");
    if (!o) return fail(MLMC_ERR_INVALID_ARG, "null options");
    if (o->c0 < 1) return fail(MLMC_ERR_INVALID_ARG, "c0 must be >= 1 (got %d)", o->c0);
    if (o->ratio < 2) return fail(MLMC_ERR_INVALID_ARG, "ratio must be >= 2 (got %d)", o->ratio);
    if (o->precision < MLMC_FP64 || o->precision > MLMC_FP8_E4M3)
        return fail(MLMC_ERR_INVALID_ARG, "unknown precision %d", o->precision);
    if (o->pilot_n < 2) return fail(MLMC_ERR_INVALID_ARG, "pilot_n must be >= 2");
    if ((o->precision == MLMC_BF16 || o->precision == MLMC_FP8_E4M3) && o->ratio != 2)
        return fail(MLMC_ERR_UNSUPPORTED, "the tensor-core precisions fold the coupling sign into B and need ratio 2");
    if (!(o->nl_scale > 0.0) || !std::isfinite(o->nl_scale)) return fail(MLMC_ERR_INVALID_ARG, "nl_scale must be > 0");
    if (o->timeout_ns < 0) return fail(MLMC_ERR_INVALID_ARG, "timeout_ns must be >= 0");
    const bool tc_prec = o->precision == MLMC_BF16 || o->precision == MLMC_FP8_E4M3;
    if (!tc_prec && o->tile_override != 0 && !cuda_core_tile_valid(o->precision, o->f, o->tile_override))
        return fail(MLMC_ERR_INVALID_ARG, "tile_override %d is not a CUDA-core tile of this plan (64064; FP32 with "
                    "f = identity: 128064, 128128)", o->tile_override);
    if (tc_prec && o->f == MLMC_F_IDENTITY && o->tile_override != 0 &&
        !tc_tile_valid(decode_tile(o->tile_override), o->precision == MLMC_FP8_E4M3 ? 1 : 0))
        return fail(MLMC_ERR_INVALID_ARG, "tile_override %d is not a tile id of this precision (1032 .. 2256; "
                    "E4M3: 1032 1064 1128 2032 2064; pairs 3256, 4256)", o->tile_override);
    if (tc_prec && o->f == MLMC_F_IDENTITY && o->sampling == MLMC_XI_OPTIMAL && o->tile_override != 0 &&
        !tc_tile_valid_xi(decode_tile(o->tile_override)))
        return fail(MLMC_ERR_INVALID_ARG, "tile_override %d: xi** takes tiles 1032, 1064, 1128 or 3256",
                    o->tile_override);
    if (tc_prec && o->f != MLMC_F_IDENTITY && o->tile_override != 0 && !tc_tile_valid_f(decode_tile(o->tile_override)))
        return fail(MLMC_ERR_INVALID_ARG, "tile_override %d: a targeted function takes tiles 1032, 1064 or 1128",
                    o->tile_override);
    if (o->adjoint_batch_log2 < 0 || o->adjoint_batch_log2 > 40)
        return fail(MLMC_ERR_INVALID_ARG, "adjoint_batch_log2 must be in [0, 40]");
    if (o->f != MLMC_F_IDENTITY && o->f != MLMC_F_ABS_STEP) return fail(MLMC_ERR_INVALID_ARG, "unknown f %d", o->f);
    if (o->f != MLMC_F_IDENTITY && o->precision == MLMC_FP8_E4M3)
        return fail(MLMC_ERR_UNSUPPORTED, "a targeted function other than the identity needs FP64, FP32 or BF16");
    if (o->adaptive_L != 0 && o->adaptive_L != 1) return fail(MLMC_ERR_INVALID_ARG, "adaptive_L must be 0 or 1");
    if (o->sampling != MLMC_XI_UNIFORM && o->sampling != MLMC_XI_OPTIMAL)
        return fail(MLMC_ERR_INVALID_ARG, "unknown sampling law %d", o->sampling);
    if (o->sampling != MLMC_XI_UNIFORM && o->precision == MLMC_FP8_E4M3)
        return fail(MLMC_ERR_UNSUPPORTED, "the xi** sampling law needs FP64, FP32 or BF16");
    for (int32_t q = 0; q < nprob; ++q) {
        const mlmc_problem& pr = problems[q];
        const int L = pr.L >= 0 ? pr.L : o->L;
        if (L < 0 || L >= MLMC_MAX_LEVELS) return fail(MLMC_ERR_INVALID_ARG, "problem %d: L=%d out of range", q, L);
        int64_t c = o->c0;
        for (int l = 0; l < L; ++l) {
            c *= o->ratio;
            if (c > kMaxCl) return fail(MLMC_ERR_INVALID_ARG, "problem %d: c_L exceeds 2^30", q);
        }
        if (pr.m < 1 || pr.m > 65536 || pr.p < 1 || pr.p > 65536)
            return fail(MLMC_ERR_INVALID_ARG, "problem %d: m, p must be in [1, 65536]", q);
        if (pr.n < 1 || pr.n >= (int64_t(1) << 31)) return fail(MLMC_ERR_INVALID_ARG, "problem %d: n must be in [1, 2^31)", q);
        if (pr.ldA < pr.n || pr.ldB < pr.p) return fail(MLMC_ERR_INVALID_ARG, "problem %d: leading dimension too small", q);
        if (!pr.M_dev || !pr.S_dev || !pr.Mp_dev || !pr.Sp_dev)
            return fail(MLMC_ERR_INVALID_ARG, "problem %d: null parameter pointer", q);
        if (pr.dtype != MLMC_DTYPE_F64 && pr.dtype != MLMC_DTYPE_F32)
            return fail(MLMC_ERR_INVALID_ARG, "problem %d: unknown dtype %d", q, pr.dtype);
    }
    return MLMC_OK;
}

void free_plan(mlmc_plan_t* plan)
{
    for (auto& ps : plan->probs) {
        cudaFree(ps.PAB);
        cudaFree(ps.sum);
        cudaFree(ps.M2);
        cudaFree(ps.xi_q);
        cudaFree(ps.xi_Q);
        cudaFree(ps.xi_G);
    }
    if (plan->merge_stream) {
        cudaStreamSynchronize(plan->merge_stream);
        cudaStreamDestroy(plan->merge_stream);
    }
    for (int set = 0; set < 2; ++set) {
        cudaFree(plan->partial_sum[set]);
        cudaFree(plan->partial_q[set]);
        if (plan->produced[set]) cudaEventDestroy(plan->produced[set]);
        if (plan->merged[set]) cudaEventDestroy(plan->merged[set]);
    }
    cudaFree(plan->dbg_sum);
    cudaFree(plan->dbg_M2);
    cudaFree(plan->chan);
    cudaFree(plan->ext_q);
    cudaFree(plan->batch_chan);
    cudaFree(plan->err_flag);
    cudaFree(plan->adj_buf);
    for (void* q : plan->owned) cudaFree(q);
    plan->owned.clear();
    cudaFree(plan->yhat_dev);
    cudaFree(plan->batch_partial);
    cudaFree(plan->batch_q);
    cudaFree(plan->batch_dev);
    if (plan->batch_host) cudaFreeHost(plan->batch_host);
    if (plan->batch_copied) cudaEventDestroy(plan->batch_copied);
    if (plan->batch_exec) cudaGraphExecDestroy(plan->batch_exec);
    if (plan->capture_stream) cudaStreamDestroy(plan->capture_stream);
}

bool tensor_core_precision(int precision) { return precision == MLMC_BF16 || precision == MLMC_FP8_E4M3; }

// Operand format of the tensor-core kernel: 0 = bfloat16, 1 = FP8 E4M3 block-scaled.
int tc_format(const mlmc_options& o) { return o.precision == MLMC_FP8_E4M3 ? 1 : 0; }

// Chunks per launch of the persistent tensor-core kernels in whole rounds.  A launch's items
// (chunks x output tiles, or x tile pairs) are dealt round-robin to the CTAs (or CTA pairs) that
// fit on the GPU at once, so a count that is not a multiple of those units leaves some idle in
// the last round: 1024 chunks of one tile pair on 76 pairs take 14 rounds for 13.5 rounds of
// work (4 % idle).  Where the budget's count loses more than 1 %, it is rounded (up while the
// merge's limit allows, else down) to a multiple of the units of every tile the problem's levels
// use, so full launches keep every unit busy.
void round_to_waves(ProblemState& ps, int q, int num_sms)
{
    auto tiles_per_chunk = [](const TcTile& t, int tiles_m, int tiles_p) {
        return t.pair ? int64_t((tiles_m + 1) / 2) * tiles_p : int64_t(tiles_m) * tiles_p;
    };
    // chunk-count step that makes the items a multiple of the units, and the busy fraction now
    auto fit = [&](const TcTile& t, int tiles_m, int tiles_p, int64_t* step, double* busy) {
        const int64_t units = tc_batch_grid(t, q, num_sms);
        const int64_t per_chunk = tiles_per_chunk(t, tiles_m, tiles_p);
        if (units <= 0 || per_chunk <= 0) return false;
        *step = units / std::gcd(units, per_chunk);
        const int64_t items = int64_t(ps.max_chunks) * per_chunk;
        *busy = double(items) / double((items + units - 1) / units * units);
        return true;
    };
    int64_t step = 1;
    double busy = 1.0;
    if (!fit(ps.tile, ps.tiles_m, ps.tiles_p, &step, &busy)) return;
    if (ps.tile_wide.mh) {
        int64_t sw = 1;
        double bw = 1.0;
        if (fit(ps.tile_wide, ps.tiles_m_wide, ps.tiles_p_wide, &sw, &bw)) {
            step = std::lcm(step, sw);
            busy = std::min(busy, bw);
        }
    }
    if (busy >= 0.99 || step > ps.max_chunks) return;
    const int64_t up = (int64_t(ps.max_chunks) + step - 1) / step * step;
    ps.max_chunks = int(up <= kMaxChunksPerLaunch ? up : int64_t(ps.max_chunks) / step * step);
}

// Read the kernels' error word (synchronises the stream).
mlmc_status check_device_flag(mlmc_plan_t* plan)
{
    int flag = 0;
    cudaError_t err = cudaMemcpyAsync(&flag, plan->err_flag, sizeof(int), cudaMemcpyDeviceToHost, plan->stream);
    if (err == cudaSuccess) err = cudaStreamSynchronize(plan->stream);
    if (check_cuda(plan, err, "read device error flag") != MLMC_OK) return plan->sticky;
    if (flag != 0)
        return set_sticky(plan, fail(static_cast<mlmc_status>(flag), "a device-side wait gave up (status %d)", flag));
    return MLMC_OK;
}

mlmc_status check_prob_level(mlmc_plan_t* plan, int32_t prob, int32_t level)
{
    if (prob < 0 || prob >= int32_t(plan->probs.size()))
        return fail(MLMC_ERR_INVALID_ARG, "problem %d out of range", prob);
    if (level < 0 || level > plan->probs[prob].L)
        return fail(MLMC_ERR_INVALID_ARG, "level %d out of range for problem %d", level, prob);
    return MLMC_OK;
}

// Evaluate samples [s0, s0+count) of one level and fold them into (sum, M2), which hold the
// statistics of n_before samples.
mlmc_status run_level(mlmc_plan_t* plan, ProblemState& ps, int level, uint64_t s0, uint64_t count, double* sum,
                      double* M2, uint64_t n_before)
{
    if (count == 0) return MLMC_OK;
    const mlmc_options& o = plan->opt;
    const int64_t c = level_c(o, level);
    LevelParams prm{};
    prm.PA = ps.PAB;
    prm.PB = static_cast<const unsigned char*>(ps.PAB) + size_t(2 * ps.m_pad) * plan->elem;
    prm.ldPA = ps.ld;
    prm.ldPB = ps.ld;
    prm.n = ps.n;
    prm.m = int(ps.m);
    prm.p = int(ps.p);
    prm.m_pad = int(ps.m_pad);
    prm.p_pad = int(ps.p_pad);
    prm.l = level;
    prm.c = int(c);
    prm.R = o.ratio;
    prm.w_fine = double(ps.n) / double(c);
    prm.w_coarse = level > 0 ? double(ps.n) / double(c) - double(ps.n) / double(c / o.ratio) : 0.0;
    prm.keyA = key(ps.desc.seed_A, ps.desc.problem_id);
    prm.keyB = key(ps.desc.seed_B, ps.desc.problem_id);
    prm.keyI = key(ps.desc.seed_idx, ps.desc.problem_id);
    prm.rkA = philox_round_keys(prm.keyA);
    prm.rkB = philox_round_keys(prm.keyB);
    // the tile of this level (BF16 pairs: the single-CTA 256 x 256 tile from c_wide on)
    const bool wide = ps.tile_wide.mh != 0 && c >= ps.c_wide;
    const TcTile& tile = wide ? ps.tile_wide : ps.tile;
    prm.tiles_m = wide ? ps.tiles_m_wide : ps.tiles_m;
    prm.tiles_p = wide ? ps.tiles_p_wide : ps.tiles_p;
    prm.cc_tile = ps.cc_tile;
    prm.xi_q = ps.xi_q;
    prm.xi_Q = ps.xi_Q;
    prm.xi_Qtot = ps.xi_Qtot;
    prm.xi_G = ps.xi_G;
    const uint64_t s_end = s0 + count;
    const uint64_t ch = uint64_t(chunk_samples(c));
    prm.chunk = int(ch);
    if (fault_is("launch"))
        return set_sticky(plan, fail(MLMC_ERR_CUDA, "injected fault: level kernel launch refused"));
    // one NVTX range per level call, named after the level (visible in profiler timelines)
    char range[32];
    std::snprintf(range, sizeof(range), "mlmc level %d", level);
    nvtxRangePushA(range);
    struct PopRange {
        ~PopRange() { nvtxRangePop(); }
    } pop_range;
    const uint64_t chunk_first = s0 / ch;
    const uint64_t chunk_last = (s_end - 1) / ch;
    // Batches alternate between the two sets of partials; the merges of batch i (in order on
    // merge_stream) overlap the level kernel of batch i + 1, and batch i + 2 waits for them.
    int batch = 0;
    struct JoinOnExit {   // an early return still orders the plan's stream after every merge enqueued
        mlmc_plan_t* plan;
        const int& batch;
        bool armed = true;
        ~JoinOnExit()
        {
            if (armed && batch > 0) cudaStreamWaitEvent(plan->stream, plan->merged[(batch - 1) & 1], 0);
        }
    } join_on_exit{plan, batch};
    for (uint64_t cb = chunk_first; cb <= chunk_last; cb += uint64_t(ps.max_chunks), ++batch) {
        const int nb = int(std::min<uint64_t>(uint64_t(ps.max_chunks), chunk_last - cb + 1));
        const int set = batch & 1;
        if (batch >= 2 &&
            check_cuda(plan, cudaStreamWaitEvent(plan->stream, plan->merged[set], 0), "merge wait") != MLMC_OK)
            return plan->sticky;
        prm.partial_sum = plan->partial_sum[set];
        prm.partial_q = plan->partial_q[set];
        prm.chunk0 = cb;
        prm.nchunks = nb;
        prm.s_begin = std::max<uint64_t>(s0, cb * ch);
        prm.s_end = std::min<uint64_t>(s_end, (cb + nb) * ch);
        cudaError_t err;
        if (tensor_core_precision(o.precision)) {
            prm.maps = wide ? ps.maps_wide : ps.maps;
            TcLaunch tl{plan->err_flag, plan->timeout_ns, static_cast<float>(double(ps.n) / double(c)), plan->num_sms};
            if (o.f != MLMC_F_IDENTITY) {
                // the targeted function: fine and coarse sums apart, Welford at every level
                prm.pack = 0;
                prm.welford = 1;
                err = launch_level_tc_f(prm, tile, o.f, tl, plan->stream);
            } else if (ps.xi_Q) {
                // xi**: per-slot weights; the level means are zero for l >= 1 too
                prm.pack = tc_pack(tile, tc_format(o), ps.m, c) ? 1 : 0;
                prm.welford = level == 0 ? 1 : 0;
                err = launch_level_tc(prm, tile, tc_format(o), tl, plan->stream);
            } else {
                prm.pack = tc_pack(tile, tc_format(o), ps.m, c) ? 1 : 0;
                // f = identity: for l >= 1 the fine and coarse estimates of one realisation have the
                // same expectation, E[D_l] = 0, so only level 0 needs Welford
                prm.welford = level == 0 ? 1 : 0;
                err = launch_level_tc(prm, tile, tc_format(o), tl, plan->stream);
            }
        } else if (ps.m == 1 && ps.p == 1 && !ps.xi_Q) {
            err = launch_level_inner(prm, plan->f64, plan->opt.f, plan->stream);   // Sec. 2's inner product
        } else {
            err = plan->f64 ? launch_level_cuda_core_f64(prm, plan->opt.f, plan->stream)
                            : launch_level_cuda_core_f32(prm, plan->opt.f, plan->stream);
        }
        if (check_cuda(plan, err, "level kernel launch") != MLMC_OK) return plan->sticky;
        plan->launches += 3;  // level kernel, merge of the sums, merge of the M2
        const ChunkRun run{prm.s_begin, prm.s_end, cb, ch, n_before, nb};
        err = cudaEventRecord(plan->produced[set], plan->stream);
        if (err == cudaSuccess) err = cudaStreamWaitEvent(plan->merge_stream, plan->produced[set], 0);
        if (err == cudaSuccess)
            err = launch_merge_partials(plan->partial_sum[set], plan->f64, plan->partial_q[set],
                                        prm.tiles_m * prm.tiles_p, ps.m * ps.p, run, sum, M2, plan->chan,
                                        plan->merge_stream);
        if (err == cudaSuccess) err = cudaEventRecord(plan->merged[set], plan->merge_stream);
        if (check_cuda(plan, err, "merge kernel launch") != MLMC_OK) return plan->sticky;
        n_before += prm.s_end - prm.s_begin;
    }
    // join: later work on the plan's stream sees the merged level state
    join_on_exit.armed = false;
    if (batch > 0 &&
        check_cuda(plan, cudaStreamWaitEvent(plan->stream, plan->merged[(batch - 1) & 1], 0), "merge join") != MLMC_OK)
        return plan->sticky;
    return MLMC_OK;
}

// ---- batched form ---------------------------------------------------------------------

constexpr size_t kBatchPartialBytes = size_t(4) << 30;  // FP32 chunk partials of one wave
constexpr int kBatchMaxJobs = 4096;                     // jobs (problem, level, chunk run) per wave
constexpr int kBatchMaxItems = 1 << 20;                 // (job, chunk, tile) units per wave
constexpr int kBatchMaxWaves = 4;                       // waves per graph launch
constexpr int kBatchMaxGrid = 4096;
constexpr int kMergeMaxChunks = 4096;
// between-chunk terms of one wave's merges: one per kMergeGroup entries of each job (the partials
// of a wave hold at most kBatchPartialBytes / 4 entries), plus one per job for the rounding up
constexpr size_t kBatchChanEntries = kBatchPartialBytes / 4 / kMergeGroup + kBatchMaxJobs;

struct BatchRange {
    int prob, level;
    uint64_t s0, count;
};

struct BatchWave {
    std::vector<LevelParams> jobs;
    std::vector<MergeJob> merges;
    std::vector<std::pair<double, uint64_t>> items;   // (cost, packed item)
    std::vector<uint64_t> packed;                      // items grouped by CTA
    std::vector<int> cta_begin;                        // grid + 1
    int64_t units = 0;                                 // (chunk, tile) pairs: entries of the q partials
};

// Byte layout of one wave's device tables.
struct WaveLayout {
    size_t jobs, merges, njobs, cta, items, stride;
    WaveLayout()
    {
        jobs = 0;
        merges = jobs + sizeof(LevelParams) * kBatchMaxJobs;
        njobs = merges + sizeof(MergeJob) * kBatchMaxJobs;
        cta = njobs + 256;
        items = cta + ((sizeof(int) * (kBatchMaxGrid + 1) + 255) & ~size_t(255));
        stride = items + sizeof(uint64_t) * kBatchMaxItems;
    }
};

LevelParams base_params(const mlmc_plan_t* plan, const ProblemState& ps, int level)
{
    const mlmc_options& o = plan->opt;
    const int64_t c = level_c(o, level);
    LevelParams prm{};
    prm.PA = ps.PAB;
    prm.PB = static_cast<const unsigned char*>(ps.PAB) + size_t(2 * ps.m_pad) * plan->elem;
    prm.ldPA = ps.ld;
    prm.ldPB = ps.ld;
    prm.n = ps.n;
    prm.m = int(ps.m);
    prm.p = int(ps.p);
    prm.m_pad = int(ps.m_pad);
    prm.p_pad = int(ps.p_pad);
    prm.l = level;
    prm.c = int(c);
    prm.R = o.ratio;
    prm.w_fine = double(ps.n) / double(c);
    prm.w_coarse = level > 0 ? double(ps.n) / double(c) - double(ps.n) / double(c / o.ratio) : 0.0;
    prm.keyA = key(ps.desc.seed_A, ps.desc.problem_id);
    prm.keyB = key(ps.desc.seed_B, ps.desc.problem_id);
    prm.keyI = key(ps.desc.seed_idx, ps.desc.problem_id);
    prm.rkA = philox_round_keys(prm.keyA);
    prm.rkB = philox_round_keys(prm.keyB);
    prm.chunk = chunk_samples(c);
    return prm;
}

// Cut the ranges into waves of (problem, level, chunk run) jobs and their (chunk, tile) items,
// then balance each wave's items over `grid` persistent CTAs, longest first.
mlmc_status build_waves(mlmc_plan_t* plan, const std::vector<BatchRange>& ranges, const TcTile& tile, int grid,
                        std::vector<BatchWave>& waves)
{
    waves.clear();
    size_t part_off = 0, q_off = 0, chan_off = 0;
    std::vector<int64_t> in_wave;   // prob * MLMC_MAX_LEVELS + level of the open wave's jobs
    // samples each (problem, level) will hold before its next job runs (jobs run in build order)
    std::vector<std::pair<int64_t, uint64_t>> held;
    auto held_before = [&](int64_t lvkey, const ProblemState& ps, int level) -> uint64_t& {
        for (auto& h : held)
            if (h.first == lvkey) return h.second;
        held.emplace_back(lvkey, ps.N.v[level]);
        return held.back().second;
    };
    auto open_wave = [&]() {
        waves.emplace_back();
        part_off = q_off = chan_off = 0;
        in_wave.clear();
    };
    open_wave();
    for (const BatchRange& r : ranges) {
        if (r.count == 0) continue;
        ProblemState& ps = plan->probs[size_t(r.prob)];
        const int64_t mp = ps.m * ps.p;
        const int tm = int((ps.m + tile.rows - 1) / tile.rows), tp = int((ps.p + tile.bn - 1) / tile.bn);
        const int tiles = tm * tp;
        // the CTA pair's items cover two row tiles of 128 (a row tile beyond m holds no outputs)
        const int item_tiles = tile.pair ? ((tm + 1) / 2) * tp : tiles;
        if (size_t(mp) * 4 > kBatchPartialBytes || tiles > 65535)
            return fail(MLMC_ERR_UNSUPPORTED, "problem %d is too large for the batched launch", r.prob);
        LevelParams base = base_params(plan, ps, r.level);
        base.tiles_m = tm;
        base.tiles_p = tp;
        base.pack = tc_pack(tile, tc_format(plan->opt), ps.m, base.c) ? 1 : 0;
        base.welford = r.level == 0 ? 1 : 0;   // E[D_l] = 0 for l >= 1 (f = identity)
        if (ps.batch_maps_tile != encode_tile(tile)) {
            tc_encode_maps(&ps.batch_maps, ps.PAB, ps.n, ps.ld, tc_stage_width_a(tile), tc_stage_width_b(tile));
            ps.batch_maps_tile = encode_tile(tile);
        }
        base.maps = ps.batch_maps;
        const uint64_t ch = uint64_t(base.chunk);
        const uint64_t s_end = r.s0 + r.count;
        uint64_t cb = r.s0 / ch;
        const uint64_t last = (s_end - 1) / ch;
        const int nsub = (base.c + 15) / 16;
        const double per_sample = double(nsub) * 16.0 * double(tile.rows + tile.bn) + double(tile.rows) * tile.bn / 4.0;
        const int64_t lvkey = int64_t(r.prob) * MLMC_MAX_LEVELS + r.level;
        while (cb <= last) {
            BatchWave* w = &waves.back();
            if (std::find(in_wave.begin(), in_wave.end(), lvkey) != in_wave.end() ||
                int(w->jobs.size()) >= kBatchMaxJobs) {
                open_wave();
                continue;
            }
            const size_t cap = kBatchPartialBytes / 4;
            const uint64_t by_part = part_off < cap ? (cap - part_off) / uint64_t(mp) : 0;
            const uint64_t by_items = uint64_t(kBatchMaxItems - w->units) / uint64_t(tiles);
            const uint64_t room = std::min<uint64_t>({by_part, by_items, uint64_t(kMergeMaxChunks)});
            if (room == 0) {
                if (w->jobs.empty()) return fail(MLMC_ERR_UNSUPPORTED, "batched wave cannot hold one chunk");
                open_wave();
                continue;
            }
            const uint64_t nb = std::min<uint64_t>(room, last - cb + 1);
            const size_t groups = size_t(merge_groups(mp));
            if (chan_off + groups > kBatchChanEntries) {
                if (w->jobs.empty()) return fail(MLMC_ERR_UNSUPPORTED, "batched wave cannot hold one merge");
                open_wave();
                continue;
            }
            LevelParams prm = base;
            prm.chunk0 = cb;
            prm.nchunks = int(nb);
            prm.s_begin = std::max<uint64_t>(r.s0, cb * ch);
            prm.s_end = std::min<uint64_t>(s_end, (cb + nb) * ch);
            prm.partial_sum = plan->batch_partial + part_off;
            prm.partial_q = plan->batch_q + q_off;
            const int job = int(w->jobs.size());
            w->jobs.push_back(prm);
            uint64_t& before = held_before(lvkey, ps, r.level);
            const ChunkRun chunks{prm.s_begin, prm.s_end, cb, ch, before, int(nb)};
            before += prm.s_end - prm.s_begin;
            MergeJob mj{plan->batch_partial + part_off, plan->batch_q + q_off, ps.sum + int64_t(r.level) * mp,
                        ps.M2 + r.level, plan->batch_chan + chan_off, mp, chunks, tiles};
            w->merges.push_back(mj);
            chan_off += groups;
            // items: runs of up to `run` chunks of one tile (fewer, larger items on long ranges)
            const uint64_t run = std::clamp<uint64_t>(nb / 64, 1, 255);
            for (uint64_t cy = 0; cy < nb; cy += run) {
                const uint64_t len = std::min<uint64_t>(run, nb - cy);
                const uint64_t a = std::max<uint64_t>(prm.s_begin, (cb + cy) * ch);
                const uint64_t b = std::min<uint64_t>(prm.s_end, (cb + cy + len) * ch);
                const double cost = double(b - a) * per_sample;
                for (int t = 0; t < item_tiles; ++t)
                    w->items.emplace_back(cost, uint64_t(job) | (cy << 16) | (len << 40) | (uint64_t(t) << 48));
            }
            w->units += int64_t(nb) * tiles;
            // every job's partials start on a 256-byte boundary: the drain stores float4 vectors
            part_off = (part_off + size_t(nb) * size_t(mp) + 63) & ~size_t(63);
            q_off += size_t(nb) * size_t(tiles);
            in_wave.push_back(lvkey);
            cb += nb;
        }
    }
    if (waves.back().jobs.empty()) waves.pop_back();
    // longest processing time first onto the least loaded CTA
    for (BatchWave& w : waves) {
        std::stable_sort(w.items.begin(), w.items.end(),
                         [](const auto& x, const auto& y) { return x.first > y.first; });
        std::vector<std::vector<uint64_t>> per(static_cast<size_t>(grid));
        std::vector<std::pair<double, int>> heap;
        for (int b = 0; b < grid; ++b) heap.emplace_back(0.0, b);
        auto cmp = [](const std::pair<double, int>& x, const std::pair<double, int>& y) {
            return x.first > y.first || (x.first == y.first && x.second > y.second);
        };
        std::make_heap(heap.begin(), heap.end(), cmp);
        for (const auto& it : w.items) {
            std::pop_heap(heap.begin(), heap.end(), cmp);
            auto& top = heap.back();
            per[size_t(top.second)].push_back(it.second);
            top.first += it.first;
            std::push_heap(heap.begin(), heap.end(), cmp);
        }
        w.packed.clear();
        w.cta_begin.assign(size_t(grid) + 1, 0);
        for (int b = 0; b < grid; ++b) {
            w.cta_begin[size_t(b)] = int(w.packed.size());
            w.packed.insert(w.packed.end(), per[size_t(b)].begin(), per[size_t(b)].end());
        }
        w.cta_begin[size_t(grid)] = int(w.packed.size());
    }
    return MLMC_OK;
}

mlmc_status batch_setup(mlmc_plan_t* plan)
{
    if (plan->batch_dev) return MLMC_OK;
    cudaError_t err = cudaMalloc(reinterpret_cast<void**>(&plan->batch_partial), kBatchPartialBytes + 256);
    if (err == cudaSuccess) err = cudaMalloc(reinterpret_cast<void**>(&plan->batch_q), sizeof(double) * kBatchMaxItems);
    if (err == cudaSuccess)
        err = cudaMalloc(reinterpret_cast<void**>(&plan->batch_chan), sizeof(double) * kBatchChanEntries);
    const size_t bytes = WaveLayout().stride * kBatchMaxWaves;
    if (err == cudaSuccess) err = cudaMalloc(reinterpret_cast<void**>(&plan->batch_dev), bytes);
    if (err == cudaSuccess) err = cudaMallocHost(reinterpret_cast<void**>(&plan->batch_host), bytes);
    if (err == cudaSuccess) err = cudaEventCreateWithFlags(&plan->batch_copied, cudaEventDisableTiming);
    if (err == cudaSuccess) err = cudaStreamCreateWithFlags(&plan->capture_stream, cudaStreamNonBlocking);
    return check_cuda(plan, err, "batched-launch setup");
}

// Stage waves [first, first + count) into table slots 0.. and upload them on the plan's stream.
mlmc_status upload_waves(mlmc_plan_t* plan, const std::vector<BatchWave>& waves, size_t first, size_t count)
{
    const WaveLayout L;
    cudaError_t err = cudaEventSynchronize(plan->batch_copied);   // the pinned slots are free again
    if (check_cuda(plan, err, "batched table staging") != MLMC_OK) return plan->sticky;
    for (size_t i = 0; i < count; ++i) {
        const BatchWave& w = waves[first + i];
        unsigned char* h = plan->batch_host + i * L.stride;
        unsigned char* d = plan->batch_dev + i * L.stride;
        const int nj = int(w.jobs.size());
        std::memcpy(h + L.jobs, w.jobs.data(), sizeof(LevelParams) * size_t(nj));
        std::memcpy(h + L.merges, w.merges.data(), sizeof(MergeJob) * size_t(nj));
        std::memcpy(h + L.njobs, &nj, sizeof(int));
        std::memcpy(h + L.cta, w.cta_begin.data(), sizeof(int) * w.cta_begin.size());
        std::memcpy(h + L.items, w.packed.data(), sizeof(uint64_t) * w.packed.size());
        // one copy per table region actually used
        const std::pair<size_t, size_t> parts[] = {{L.jobs, sizeof(LevelParams) * size_t(nj)},
                                                   {L.merges, sizeof(MergeJob) * size_t(nj)},
                                                   {L.njobs, sizeof(int)},
                                                   {L.cta, sizeof(int) * w.cta_begin.size()},
                                                   {L.items, sizeof(uint64_t) * w.packed.size()}};
        for (const auto& pr : parts) {
            if (pr.second == 0) continue;
            err = cudaMemcpyAsync(d + pr.first, h + pr.first, pr.second, cudaMemcpyHostToDevice, plan->stream);
            if (check_cuda(plan, err, "batched table upload") != MLMC_OK) return plan->sticky;
        }
    }
    err = cudaEventRecord(plan->batch_copied, plan->stream);
    return check_cuda(plan, err, "batched table upload");
}

TcBatch wave_tables(const mlmc_plan_t* plan, size_t slot)
{
    const WaveLayout L;
    unsigned char* d = plan->batch_dev + slot * L.stride;
    return TcBatch{reinterpret_cast<const LevelParams*>(d + L.jobs), reinterpret_cast<const uint64_t*>(d + L.items),
                   reinterpret_cast<const int*>(d + L.cta)};
}

// Kernel launches of `count` staged waves on stream `st` (captured into the graph).
cudaError_t enqueue_waves(mlmc_plan_t* plan, size_t count, bool merge, cudaStream_t st)
{
    const WaveLayout L;
    TcLaunch tl{plan->err_flag, plan->timeout_ns, 0.0f, plan->num_sms};
    for (size_t i = 0; i < count; ++i) {
        cudaError_t err = launch_level_tc_batch(wave_tables(plan, i), plan->batch_tile, tc_format(plan->opt),
                                                plan->batch_grid, tl, st);
        if (err != cudaSuccess) return err;
        if (merge) {
            unsigned char* d = plan->batch_dev + i * L.stride;
            err = launch_merge_batch(reinterpret_cast<const MergeJob*>(d + L.merges),
                                     reinterpret_cast<const int*>(d + L.njobs), st);
            if (err != cudaSuccess) return err;
        }
    }
    return cudaSuccess;
}

// Autotuner: time every candidate tile on the first chunk of each range and keep the fastest.
mlmc_status autotune_batch_tile(mlmc_plan_t* plan, const std::vector<BatchRange>& ranges)
{
    int64_t mmax = 1, pmax = 1;
    for (const auto& ps : plan->probs) {
        mmax = std::max(mmax, ps.m);
        pmax = std::max(pmax, ps.p);
    }
    std::vector<BatchRange> probe;
    for (const BatchRange& r : ranges) {
        if (r.count == 0) continue;
        const uint64_t ch = uint64_t(chunk_samples(level_c(plan->opt, r.level)));
        const uint64_t end = std::min<uint64_t>(r.s0 + r.count, (r.s0 / ch + 1) * ch);
        probe.push_back(BatchRange{r.prob, r.level, r.s0, end - r.s0});
    }
    cudaEvent_t e0 = nullptr, e1 = nullptr;
    cudaError_t err = cudaEventCreate(&e0);
    if (err == cudaSuccess) err = cudaEventCreate(&e1);
    if (check_cuda(plan, err, "autotuner events") != MLMC_OK) return plan->sticky;
    double best = 1e300;
    TcTile best_tile = tc_tile_for(mmax, pmax, tc_format(plan->opt), false);
    mlmc_status st = MLMC_OK;
    for (int c = 0; c < 9 && st == MLMC_OK; ++c) {
        const TcTile t = decode_tile(kTileIds[c]);
        plan->tune_ms[c] = -1.0;
        // skip tiles far wider or taller than every problem (the pair: 256 x 256 per cluster)
        if ((t.mh == 2 && mmax <= 128) || (t.bn > 32 && pmax <= t.bn / 2) || (t.pair && mmax <= 128)) continue;
        if (!tc_tile_valid(t, tc_format(plan->opt))) continue;
        const int grid = std::min(tc_batch_grid(t, tc_format(plan->opt), plan->num_sms), kBatchMaxGrid);
        if (grid <= 0) continue;
        std::vector<BatchWave> waves;
        if ((st = build_waves(plan, probe, t, grid, waves)) != MLMC_OK) break;
        if (waves.empty()) break;
        if ((st = upload_waves(plan, waves, 0, 1)) != MLMC_OK) break;
        plan->batch_tile = t;
        plan->batch_grid = grid;
        float ms = 0.0f;
        err = enqueue_waves(plan, 1, false, plan->stream);   // warm-up (partials only, no merge)
        if (err == cudaSuccess) err = cudaEventRecord(e0, plan->stream);
        if (err == cudaSuccess) err = enqueue_waves(plan, 1, false, plan->stream);
        if (err == cudaSuccess) err = cudaEventRecord(e1, plan->stream);
        if (err == cudaSuccess) err = cudaEventSynchronize(e1);
        if (err == cudaSuccess) err = cudaEventElapsedTime(&ms, e0, e1);
        if ((st = check_cuda(plan, err, "autotuner launch")) != MLMC_OK) break;
        if ((st = check_device_flag(plan)) != MLMC_OK) break;
        plan->launches += 2;
        plan->tune_ms[c] = ms;
        if (ms < best) {
            best = ms;
            best_tile = t;
        }
    }
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    if (st != MLMC_OK) return st;
    plan->batch_tile = best_tile;
    plan->batch_grid = std::min(tc_batch_grid(best_tile, tc_format(plan->opt), plan->num_sms), kBatchMaxGrid);
    return plan->batch_grid > 0 ? MLMC_OK : set_sticky(plan, fail(MLMC_ERR_CUDA, "batched grid query failed"));
}

mlmc_status run_batch(mlmc_plan_t* plan, const std::vector<BatchRange>& ranges)
{
    if (fault_is("launch"))
        return set_sticky(plan, fail(MLMC_ERR_CUDA, "injected fault: batched launch refused"));
    nvtxRangePushA("mlmc batched levels");
    struct PopRange {
        ~PopRange() { nvtxRangePop(); }
    } pop_range;
    mlmc_status st = batch_setup(plan);
    if (st != MLMC_OK) return st;
    if (plan->batch_tile.mh == 0) {
        if (plan->opt.tile_override) {
            if (decode_tile(plan->opt.tile_override).pair == 2)
                return fail(MLMC_ERR_UNSUPPORTED, "tile 4256 (16-warp CTA pairs) serves single-problem launches only");
            plan->batch_tile = decode_tile(plan->opt.tile_override);
            plan->batch_grid =
                std::min(tc_batch_grid(plan->batch_tile, tc_format(plan->opt), plan->num_sms), kBatchMaxGrid);
            if (plan->batch_grid <= 0) return set_sticky(plan, fail(MLMC_ERR_CUDA, "batched grid query failed"));
        } else if ((st = autotune_batch_tile(plan, ranges)) != MLMC_OK) {
            return st;
        }
    }
    std::vector<BatchWave> waves;
    if ((st = build_waves(plan, ranges, plan->batch_tile, plan->batch_grid, waves)) != MLMC_OK) return st;
    for (size_t w0 = 0; w0 < waves.size(); w0 += kBatchMaxWaves) {
        const size_t cnt = std::min<size_t>(kBatchMaxWaves, waves.size() - w0);
        if ((st = upload_waves(plan, waves, w0, cnt)) != MLMC_OK) return st;
        // the graph depends only on the tile, the grid and the number of waves
        const std::vector<int64_t> key = {encode_tile(plan->batch_tile), plan->batch_grid, int64_t(cnt)};
        if (!plan->batch_exec || key != plan->batch_key) {
            if (plan->batch_exec) {
                cudaGraphExecDestroy(plan->batch_exec);
                plan->batch_exec = nullptr;
            }
            cudaGraph_t graph = nullptr;
            cudaError_t err = cudaStreamBeginCapture(plan->capture_stream, cudaStreamCaptureModeThreadLocal);
            if (err == cudaSuccess) {
                const cudaError_t lerr = enqueue_waves(plan, cnt, true, plan->capture_stream);
                err = cudaStreamEndCapture(plan->capture_stream, &graph);
                if (lerr != cudaSuccess) err = lerr;
            }
            if (err == cudaSuccess) err = cudaGraphInstantiate(&plan->batch_exec, graph, 0);
            if (graph) cudaGraphDestroy(graph);
            if (check_cuda(plan, err, "batched graph capture") != MLMC_OK) return plan->sticky;
            plan->batch_key = key;
        }
        cudaError_t err = cudaGraphLaunch(plan->batch_exec, plan->stream);
        if (check_cuda(plan, err, "batched graph launch") != MLMC_OK) return plan->sticky;
        plan->launches += 3 * cnt;   // per wave: level kernel and the two merges
    }
    for (const BatchRange& r : ranges) {
        if (r.count == 0) continue;
        ProblemState& ps = plan->probs[size_t(r.prob)];
        ps.prefix[r.level] = ps.prefix[r.level] && r.s0 == ps.N.v[r.level];
        ps.N.v[r.level] += r.count;
    }
    return MLMC_OK;
}

// M2 of levels [first, first + count) of a problem into a host array (synchronises).
mlmc_status level_M2(mlmc_plan_t* plan, ProblemState& ps, int first, int count, double* M2_host)
{
    cudaError_t err = cudaMemcpyAsync(M2_host, ps.M2 + first, sizeof(double) * size_t(count), cudaMemcpyDeviceToHost,
                                      plan->stream);
    if (check_cuda(plan, err, "copy M2") != MLMC_OK) return plan->sticky;
    err = cudaStreamSynchronize(plan->stream);
    if (check_cuda(plan, err, "stream synchronize") != MLMC_OK) return plan->sticky;
    return check_device_flag(plan);
}

// ||Y_l||_F: the norm of level l's mean, read back from its FP64 sum (synchronises).
mlmc_status level_mean_norm(mlmc_plan_t* plan, const ProblemState& ps, int l, double* out)
{
    const int64_t mp = ps.m * ps.p;
    std::vector<double> sums(static_cast<size_t>(mp));
    cudaError_t err = cudaMemcpyAsync(sums.data(), ps.sum + int64_t(l) * mp, sizeof(double) * size_t(mp),
                                      cudaMemcpyDeviceToHost, plan->stream);
    if (err == cudaSuccess) err = cudaStreamSynchronize(plan->stream);
    if (check_cuda(plan, err, "read level mean") != MLMC_OK) return plan->sticky;
    double nrm = 0.0;
    for (double v : sums) nrm += v * v;
    *out = ps.N.v[l] > 0 ? std::sqrt(nrm) / double(ps.N.v[l]) : 0.0;
    return MLMC_OK;
}

// Remark 3.6 over levels 0..L of one problem: V_l = M2_l / (N_l - 1), C_0 = c_0,
// C_l = c_l + c_{l-1}, N_l = max(pilot, ceil(nl_scale 2 eps^-2 sqrt(V_l / C_l) sum_j sqrt(V_j C_j))).
mlmc_status allocation(mlmc_plan_t* plan, ProblemState& ps, int q, int L, double eps, int64_t* Nl)
{
    const mlmc_options& o = plan->opt;
    for (int l = 0; l <= L; ++l)
        if (ps.N.v[l] < 2) return fail(MLMC_ERR_STATE, "problem %d level %d holds fewer than 2 samples", q, l);
    double M2[MLMC_MAX_LEVELS], V[MLMC_MAX_LEVELS], C[MLMC_MAX_LEVELS], root_sum = 0.0;
    mlmc_status st = level_M2(plan, ps, 0, L + 1, M2);
    if (st != MLMC_OK) return st;
    for (int l = 0; l <= L; ++l) {
        V[l] = std::max(0.0, M2[l] / double(ps.N.v[l] - 1));
        C[l] = level_cost(o, l);
        if (!std::isfinite(V[l])) return fail(MLMC_ERR_NUMERIC, "problem %d level %d: V_l not finite", q, l);
        root_sum += std::sqrt(V[l] * C[l]);
    }
    for (int l = 0; l <= L; ++l) {
        const double target = o.nl_scale * 2.0 / (eps * eps) * std::sqrt(V[l] / C[l]) * root_sum;
        if (!(target < 9.0e18)) return fail(MLMC_ERR_NUMERIC, "allocated N_l overflows");
        Nl[l] = std::max<int64_t>(int64_t(std::ceil(target)), o.pilot_n);
    }
    return MLMC_OK;
}

// Remark 3.5 as Alg. 2 uses it: level L (>= 2) meets the bias bound when
// ||Y_L||_F < (sqrt(R) + 1) eps / sqrt(2).
mlmc_status bias_test(mlmc_plan_t* plan, ProblemState& ps, int L, double eps, bool* met, double* norm)
{
    double nrm = 0.0;
    mlmc_status st = level_mean_norm(plan, ps, L, &nrm);
    if (st != MLMC_OK) return st;
    *norm = nrm;
    *met = L >= 2 && nrm < (std::sqrt(double(plan->opt.ratio)) + 1.0) * eps / std::sqrt(2.0);
    return MLMC_OK;
}

}  // namespace

extern "C" {

const char* mlmc_last_error(void) { return g_last_error.c_str(); }

mlmc_status mlmc_plan(const mlmc_problem* problems, int32_t nprob, const mlmc_options* options, void* stream,
                      mlmc_plan_t** plan_out)
{
    if (!plan_out) return fail(MLMC_ERR_INVALID_ARG, "null plan_out");
    *plan_out = nullptr;
    mlmc_status st = validate(problems, nprob, options);
    if (st != MLMC_OK) return st;
    if (fault_is("alloc")) return fail(MLMC_ERR_OOM, "injected fault: device allocation of the plan failed");
    mlmc_plan_t* plan = new (std::nothrow) mlmc_plan_s();
    if (!plan) return fail(MLMC_ERR_OOM, "host allocation failed");
    if (cudaGetDevice(&plan->device) != cudaSuccess) {
        delete plan;
        return fail(MLMC_ERR_CUDA, "no CUDA device available");
    }
    plan->stream = static_cast<cudaStream_t>(stream);
    plan->opt = *options;
    plan->f64 = options->precision == MLMC_FP64;
    plan->elem = plan->f64 ? 8 : 4;
    plan->probs.resize(size_t(nprob));

    if (cudaDeviceGetAttribute(&plan->num_sms, cudaDevAttrMultiProcessorCount, plan->device) != cudaSuccess)
        plan->num_sms = 1;
    size_t max_partial = 0, max_q = 0, max_mp = 0;
    auto oom = [&](const char* what) {
        free_plan(plan);
        delete plan;
        return fail(MLMC_ERR_OOM, "cudaMalloc of %s failed", what);
    };
    for (int32_t q = 0; q < nprob; ++q) {
        ProblemState& ps = plan->probs[size_t(q)];
        ps.desc = problems[q];
        ps.L = problems[q].L >= 0 ? problems[q].L : options->L;
        ps.m = problems[q].m;
        ps.n = problems[q].n;
        ps.p = problems[q].p;
        ps.m_pad = (ps.m + 3) / 4 * 4;
        ps.p_pad = (ps.p + 3) / 4 * 4;
        if (tensor_core_precision(options->precision)) {
            const TcTile tile = options->tile_override ? decode_tile(options->tile_override)
                                : options->f != MLMC_F_IDENTITY      ? tc_tile_for_f(ps.p)
                                : options->sampling == MLMC_XI_OPTIMAL ? tc_tile_for_xi(ps.m, ps.p)
                                    : tc_tile_for(ps.m, ps.p, options->precision == MLMC_FP8_E4M3 ? 1 : 0, true);
            ps.tile = tile;
            ps.tiles_m = int((ps.m + tile.rows - 1) / tile.rows);
            ps.tiles_p = int((ps.p + tile.bn - 1) / tile.bn);
            const TcTile wide = decode_tile(2256);
            if (!options->tile_override && options->precision == MLMC_BF16 && options->f == MLMC_F_IDENTITY &&
                options->sampling == MLMC_XI_UNIFORM && tile.pair == 1 && tc_tile_valid(wide, 0)) {
                ps.tile_wide = wide;
                ps.tiles_m_wide = int((ps.m + wide.rows - 1) / wide.rows);
                ps.tiles_p_wide = int((ps.p + wide.bn - 1) / wide.bn);
                ps.c_wide = kWideTileFromC;
            }
        } else {
            ps.cc_tile = options->tile_override ? options->tile_override
                                                : cuda_core_default_tile(options->precision, options->f, ps.m);
            const CudaCoreTile tile = cuda_core_tile(ps.cc_tile);
            ps.tiles_m = int((ps.m + tile.tm - 1) / tile.tm);
            ps.tiles_p = int((ps.p + tile.tp - 1) / tile.tp);
        }
        const size_t mp = size_t(ps.m * ps.p);
        const size_t per_chunk = mp * plan->elem;
        const size_t budget = tensor_core_precision(options->precision) ? kPartialBudgetTc : kPartialBudget;
        ps.max_chunks = int(std::clamp<size_t>(budget / per_chunk, 1, kMaxChunksPerLaunch));
        if (tensor_core_precision(options->precision)) round_to_waves(ps, tc_format(*options), plan->num_sms);
        max_partial = std::max(max_partial, per_chunk * size_t(ps.max_chunks));
        max_q = std::max(max_q, size_t(ps.max_chunks) *
                                    size_t(std::max(ps.tiles_m * ps.tiles_p, ps.tiles_m_wide * ps.tiles_p_wide)));
        max_mp = std::max(max_mp, mp);
        // one row per inner index k holds both gathered vectors, so a sampled index is one
        // contiguous read of 2 (m_pad + p_pad) elements
        ps.ld = 2 * (ps.m_pad + ps.p_pad);
        if (cudaMalloc(&ps.PAB, size_t(ps.n) * size_t(ps.ld) * plan->elem) != cudaSuccess) return oom("parameters");
        if (cudaMalloc(&ps.sum, sizeof(double) * mp * size_t(ps.L + 1)) != cudaSuccess) return oom("level sums");
        if (cudaMalloc(&ps.M2, sizeof(double) * size_t(ps.L + 1)) != cudaSuccess) return oom("level M2");
        cudaMemsetAsync(ps.sum, 0, sizeof(double) * mp * size_t(ps.L + 1), plan->stream);
        cudaMemsetAsync(ps.M2, 0, sizeof(double) * size_t(ps.L + 1), plan->stream);
        cudaError_t err = launch_layout_A(ps.desc.M_dev, ps.desc.S_dev, ps.desc.dtype, ps.desc.ldA, ps.m, ps.n,
                                          ps.m_pad, ps.PAB, ps.ld, plan->f64, plan->stream);
        if (err == cudaSuccess)
            err = launch_layout_B(ps.desc.Mp_dev, ps.desc.Sp_dev, ps.desc.dtype, ps.desc.ldB, ps.n, ps.p, ps.p_pad,
                                  static_cast<unsigned char*>(ps.PAB) + size_t(2 * ps.m_pad) * plan->elem, ps.ld,
                                  plan->f64, plan->stream);
        if (err != cudaSuccess) {
            free_plan(plan);
            delete plan;
            return fail(MLMC_ERR_CUDA, "layout kernel: %s", cudaGetErrorString(err));
        }
        if (tensor_core_precision(options->precision))
            tc_encode_maps(&ps.maps, ps.PAB, ps.n, ps.ld, tc_stage_width_a(ps.tile), tc_stage_width_b(ps.tile));
        if (ps.tile_wide.mh)
            tc_encode_maps(&ps.maps_wide, ps.PAB, ps.n, ps.ld, tc_stage_width_a(ps.tile_wide),
                           tc_stage_width_b(ps.tile_wide));
        if (options->sampling == MLMC_XI_OPTIMAL) {
            // xi** (Thm 3.1) from the laid-out parameters; its total must be a positive number
            if (cudaMalloc(reinterpret_cast<void**>(&ps.xi_q), sizeof(double) * size_t(ps.n)) != cudaSuccess ||
                cudaMalloc(reinterpret_cast<void**>(&ps.xi_Q), sizeof(double) * size_t(ps.n)) != cudaSuccess ||
                cudaMalloc(reinterpret_cast<void**>(&ps.xi_G), sizeof(int) * size_t(ps.n)) != cudaSuccess)
                return oom("xi** tables");
            err = launch_xi_optimal(ps.PAB, plan->f64, ps.ld, ps.m, ps.m_pad, ps.n, ps.p, ps.xi_q, ps.xi_Q, ps.xi_G,
                                    plan->stream);
            if (err == cudaSuccess)
                err = cudaMemcpyAsync(&ps.xi_Qtot, ps.xi_Q + (ps.n - 1), sizeof(double), cudaMemcpyDeviceToHost,
                                      plan->stream);
            if (err == cudaSuccess) err = cudaStreamSynchronize(plan->stream);
            if (err != cudaSuccess) {
                free_plan(plan);
                delete plan;
                return fail(MLMC_ERR_CUDA, "xi** tables: %s", cudaGetErrorString(err));
            }
            if (!(ps.xi_Qtot > 0.0) || !std::isfinite(ps.xi_Qtot)) {
                free_plan(plan);
                delete plan;
                return fail(MLMC_ERR_NUMERIC, "xi**: the column weights of a problem sum to %g", ps.xi_Qtot);
            }
        }
    }
    for (int set = 0; set < 2; ++set) {
        if (cudaMalloc(&plan->partial_sum[set], max_partial) != cudaSuccess) return oom("chunk partials");
        if (cudaMalloc(reinterpret_cast<void**>(&plan->partial_q[set]), sizeof(double) * max_q) != cudaSuccess)
            return oom("chunk sums of squares");
        if (cudaEventCreateWithFlags(&plan->produced[set], cudaEventDisableTiming) != cudaSuccess ||
            cudaEventCreateWithFlags(&plan->merged[set], cudaEventDisableTiming) != cudaSuccess)
            return oom("merge events");
    }
    {
        // the merges run beside the next batch's level kernel: the highest priority, so that
        // their few small blocks start as soon as an SM has room
        int lo = 0, hi = 0;
        cudaDeviceGetStreamPriorityRange(&lo, &hi);
        if (cudaStreamCreateWithPriority(&plan->merge_stream, cudaStreamNonBlocking, hi) != cudaSuccess)
            return oom("merge stream");
    }
    if (cudaMalloc(reinterpret_cast<void**>(&plan->dbg_sum), sizeof(double) * max_mp) != cudaSuccess)
        return oom("debug state");
    if (cudaMalloc(reinterpret_cast<void**>(&plan->dbg_M2), sizeof(double)) != cudaSuccess) return oom("debug state");
    if (cudaMalloc(reinterpret_cast<void**>(&plan->chan), sizeof(double) * size_t(merge_groups(int64_t(max_mp)))) !=
        cudaSuccess)
        return oom("merge scratch");
    if (cudaMalloc(reinterpret_cast<void**>(&plan->ext_q), sizeof(double)) != cudaSuccess) return oom("merge scratch");
    if (cudaMalloc(reinterpret_cast<void**>(&plan->err_flag), sizeof(int)) != cudaSuccess) return oom("error flag");
    cudaMemsetAsync(plan->err_flag, 0, sizeof(int), plan->stream);
    if (options->timeout_ns > 0) plan->timeout_ns = uint64_t(options->timeout_ns);
    cudaError_t err = cudaGetLastError();
    if (err != cudaSuccess) {
        free_plan(plan);
        delete plan;
        return fail(MLMC_ERR_CUDA, "plan setup: %s", cudaGetErrorString(err));
    }
    *plan_out = plan;
    return MLMC_OK;
}

mlmc_status mlmc_plan_destroy(mlmc_plan_t* plan)
{
    if (!plan) return MLMC_OK;
    DeviceGuard g(plan->device);
    cudaStreamSynchronize(plan->stream);
    free_plan(plan);
    delete plan;
    return MLMC_OK;
}

mlmc_status mlmc_synchronize(mlmc_plan_t* plan)
{
    mlmc_status st = enter(plan);
    if (st != MLMC_OK) return st;
    DeviceGuard g(plan->device);
    if (check_cuda(plan, cudaStreamSynchronize(plan->stream), "stream synchronize") != MLMC_OK) return plan->sticky;
    return check_device_flag(plan);
}

mlmc_status mlmc_level_stats(mlmc_plan_t* plan, int32_t prob, int32_t level, uint64_t sample_begin, uint64_t count)
{
    mlmc_status st = enter(plan);
    if (st != MLMC_OK) return st;
    if ((st = check_prob_level(plan, prob, level)) != MLMC_OK) return st;
    if (count == 0) return MLMC_OK;
    if (sample_begin + count < sample_begin || sample_begin + count > (uint64_t(1) << 56))
        return fail(MLMC_ERR_INVALID_ARG, "sample ids must stay below 2^56");
    DeviceGuard g(plan->device);
    ProblemState& ps = plan->probs[size_t(prob)];
    const int64_t mp = ps.m * ps.p;
    const bool continues = sample_begin == ps.N.v[level];
    st = run_level(plan, ps, level, sample_begin, count, ps.sum + int64_t(level) * mp, ps.M2 + level, ps.N.v[level]);
    if (st == MLMC_OK) {
        ps.N.v[level] += count;
        ps.prefix[level] = ps.prefix[level] && continues;
    }
    return st;
}

mlmc_status mlmc_level_stats_batch(mlmc_plan_t* plan, const mlmc_range* ranges, int32_t count)
{
    mlmc_status st = enter(plan);
    if (st != MLMC_OK) return st;
    if (count < 0 || (count > 0 && !ranges)) return fail(MLMC_ERR_INVALID_ARG, "bad range list");
    std::vector<BatchRange> rs;
    for (int32_t i = 0; i < count; ++i) {
        const mlmc_range& r = ranges[i];
        if ((st = check_prob_level(plan, r.prob, r.level)) != MLMC_OK) return st;
        if (r.sample_begin + r.count < r.sample_begin || r.sample_begin + r.count > (uint64_t(1) << 56))
            return fail(MLMC_ERR_INVALID_ARG, "range %d: sample ids must stay below 2^56", i);
        if (r.count > 0) rs.push_back(BatchRange{r.prob, r.level, r.sample_begin, r.count});
    }
    if (rs.empty()) return MLMC_OK;
    DeviceGuard g(plan->device);
    // the batched persistent launch is the identity's under the uniform law; other forms evaluate
    // the ranges in turn
    if (!tensor_core_precision(plan->opt.precision) || plan->opt.f != MLMC_F_IDENTITY ||
        plan->opt.sampling != MLMC_XI_UNIFORM) {
        for (const BatchRange& r : rs) {
            ProblemState& ps = plan->probs[size_t(r.prob)];
            const int64_t mp = ps.m * ps.p;
            const bool continues = r.s0 == ps.N.v[r.level];
            st = run_level(plan, ps, r.level, r.s0, r.count, ps.sum + int64_t(r.level) * mp, ps.M2 + r.level,
                           ps.N.v[r.level]);
            if (st != MLMC_OK) return st;
            ps.N.v[r.level] += r.count;
            ps.prefix[r.level] = ps.prefix[r.level] && continues;
        }
        return MLMC_OK;
    }
    return run_batch(plan, rs);
}

mlmc_status mlmc_get_batch_tile(const mlmc_plan_t* plan, int32_t* tile_id, double* timings_ms)
{
    if (!plan || !tile_id) return fail(MLMC_ERR_INVALID_ARG, "null argument");
    *tile_id = encode_tile(plan->batch_tile);
    if (timings_ms)
        for (int c = 0; c < 9; ++c) timings_ms[c] = plan->tune_ms[c];
    return MLMC_OK;
}

mlmc_status mlmc_get_level_stats(mlmc_plan_t* plan, int32_t prob, int32_t level, uint64_t* N, double* mean_dev,
                                 double* M2)
{
    mlmc_status st = enter(plan);
    if (st != MLMC_OK) return st;
    if ((st = check_prob_level(plan, prob, level)) != MLMC_OK) return st;
    DeviceGuard g(plan->device);
    ProblemState& ps = plan->probs[size_t(prob)];
    const int64_t mp = ps.m * ps.p;
    if (mean_dev) {
        cudaError_t err = launch_finalize(ps.sum + int64_t(level) * mp, ps.N, level, 1, mp, mean_dev, plan->stream);
        if (check_cuda(plan, err, "finalize launch") != MLMC_OK) return plan->sticky;
        plan->launches += 1;
    }
    double m2 = 0.0;
    if ((st = level_M2(plan, ps, level, 1, &m2)) != MLMC_OK) return st;
    if (N) *N = ps.N.v[level];
    if (M2) *M2 = m2;
    if (!std::isfinite(m2)) return fail(MLMC_ERR_NUMERIC, "level %d: non-finite second moment", level);
    return MLMC_OK;
}

mlmc_status mlmc_get_level_state(mlmc_plan_t* plan, int32_t prob, int32_t level, uint64_t* N, double* sum_dev,
                                 double* M2)
{
    mlmc_status st = enter(plan);
    if (st != MLMC_OK) return st;
    if ((st = check_prob_level(plan, prob, level)) != MLMC_OK) return st;
    DeviceGuard g(plan->device);
    ProblemState& ps = plan->probs[size_t(prob)];
    const int64_t mp = ps.m * ps.p;
    cudaError_t err = cudaSuccess;
    if (sum_dev)
        err = cudaMemcpyAsync(sum_dev, ps.sum + int64_t(level) * mp, sizeof(double) * size_t(mp),
                              cudaMemcpyDeviceToDevice, plan->stream);
    double q = 0.0;
    if (err == cudaSuccess)
        err = cudaMemcpyAsync(&q, ps.M2 + level, sizeof(double), cudaMemcpyDeviceToHost, plan->stream);
    if (err == cudaSuccess) err = cudaStreamSynchronize(plan->stream);
    if (check_cuda(plan, err, "read level state") != MLMC_OK) return plan->sticky;
    if ((st = check_device_flag(plan)) != MLMC_OK) return st;
    if (N) *N = ps.N.v[level];
    if (M2) *M2 = q;
    return MLMC_OK;
}

mlmc_status mlmc_set_level_state(mlmc_plan_t* plan, int32_t prob, int32_t level, uint64_t N, const double* sum_dev,
                                 double M2)
{
    mlmc_status st = enter(plan);
    if (st != MLMC_OK) return st;
    if ((st = check_prob_level(plan, prob, level)) != MLMC_OK) return st;
    if (!sum_dev) return fail(MLMC_ERR_INVALID_ARG, "null sum_dev");
    if (!(M2 >= 0.0) || !std::isfinite(M2)) return fail(MLMC_ERR_INVALID_ARG, "M2 must be finite and >= 0");
    DeviceGuard g(plan->device);
    ProblemState& ps = plan->probs[size_t(prob)];
    const int64_t mp = ps.m * ps.p;
    cudaError_t err = cudaMemcpyAsync(ps.sum + int64_t(level) * mp, sum_dev, sizeof(double) * size_t(mp),
                                      cudaMemcpyDeviceToDevice, plan->stream);
    if (err == cudaSuccess)
        err = cudaMemcpyAsync(ps.M2 + level, &M2, sizeof(double), cudaMemcpyHostToDevice, plan->stream);
    if (err == cudaSuccess) err = cudaStreamSynchronize(plan->stream);
    if (check_cuda(plan, err, "write level state") != MLMC_OK) return plan->sticky;
    ps.N.v[level] = N;
    ps.prefix[level] = true;
    ps.has_estimate = false;
    return MLMC_OK;
}

mlmc_status mlmc_merge_level_state(mlmc_plan_t* plan, int32_t prob, int32_t level, uint64_t N, const double* sum_dev,
                                   double M2)
{
    mlmc_status st = enter(plan);
    if (st != MLMC_OK) return st;
    if ((st = check_prob_level(plan, prob, level)) != MLMC_OK) return st;
    if (N == 0) return MLMC_OK;
    if (!sum_dev) return fail(MLMC_ERR_INVALID_ARG, "null sum_dev");
    if (!(M2 >= 0.0) || !std::isfinite(M2)) return fail(MLMC_ERR_INVALID_ARG, "M2 must be finite and >= 0");
    DeviceGuard g(plan->device);
    ProblemState& ps = plan->probs[size_t(prob)];
    const int64_t mp = ps.m * ps.p;
    if (ps.N.v[level] + N < N) return fail(MLMC_ERR_INVALID_ARG, "sample count overflows");
    // the other state is one chunk of N samples with its own sum and M2: the merge of the level
    // kernels' chunks, with FP64 partials
    cudaError_t err = cudaMemcpyAsync(plan->ext_q, &M2, sizeof(double), cudaMemcpyHostToDevice, plan->stream);
    const ChunkRun run{0, N, 0, N, ps.N.v[level], 1};
    if (err == cudaSuccess)
        err = launch_merge_partials(sum_dev, true, plan->ext_q, 1, mp, run, ps.sum + int64_t(level) * mp,
                                    ps.M2 + level, plan->chan, plan->stream);
    if (err == cudaSuccess) err = cudaStreamSynchronize(plan->stream);
    if (check_cuda(plan, err, "merge level state") != MLMC_OK) return plan->sticky;
    plan->launches += 2;
    ps.N.v[level] += N;
    ps.has_estimate = false;
    return MLMC_OK;
}

mlmc_status mlmc_reset_level_stats(mlmc_plan_t* plan, int32_t prob, int32_t level)
{
    mlmc_status st = enter(plan);
    if (st != MLMC_OK) return st;
    if (prob < 0 || prob >= int32_t(plan->probs.size())) return fail(MLMC_ERR_INVALID_ARG, "problem out of range");
    ProblemState& ps = plan->probs[size_t(prob)];
    if (level > ps.L) return fail(MLMC_ERR_INVALID_ARG, "level out of range");
    DeviceGuard g(plan->device);
    const int64_t mp = ps.m * ps.p;
    const int first = level < 0 ? 0 : level;
    const int cnt = level < 0 ? ps.L + 1 : 1;
    cudaError_t err = cudaMemsetAsync(ps.sum + int64_t(first) * mp, 0, sizeof(double) * size_t(mp) * size_t(cnt),
                                      plan->stream);
    if (err == cudaSuccess) err = cudaMemsetAsync(ps.M2 + first, 0, sizeof(double) * size_t(cnt), plan->stream);
    if (check_cuda(plan, err, "reset level state") != MLMC_OK) return plan->sticky;
    for (int l = first; l < first + cnt; ++l) {
        ps.N.v[l] = 0;
        ps.prefix[l] = true;
    }
    ps.has_estimate = false;
    return MLMC_OK;
}

mlmc_status mlmc_plan_host(const mlmc_problem* problems, int32_t nprob, const mlmc_options* options, void* stream,
                           mlmc_plan_t** plan_out)
{
    if (!plan_out) return fail(MLMC_ERR_INVALID_ARG, "null plan_out");
    *plan_out = nullptr;
    mlmc_status st = validate(problems, nprob, options);
    if (st != MLMC_OK) return st;
    if (fault_is("alloc")) return fail(MLMC_ERR_OOM, "injected fault: device allocation of the plan failed");
    cudaStream_t cs = static_cast<cudaStream_t>(stream);
    std::vector<mlmc_problem> dev(problems, problems + nprob);
    std::vector<void*> owned;
    auto release = [&]() {
        cudaStreamSynchronize(cs);
        for (void* q : owned) cudaFree(q);
    };
    for (int32_t q = 0; q < nprob; ++q) {
        const mlmc_problem& pr = problems[q];
        const size_t elem = pr.dtype == MLMC_DTYPE_F64 ? 8 : 4;
        // row-major with the caller's leading dimensions: m rows of ldA, n rows of ldB
        const size_t bytes_a = size_t(pr.m - 1) * size_t(pr.ldA) * elem + size_t(pr.n) * elem;
        const size_t bytes_b = size_t(pr.n - 1) * size_t(pr.ldB) * elem + size_t(pr.p) * elem;
        const void* src[4] = {pr.M_dev, pr.S_dev, pr.Mp_dev, pr.Sp_dev};
        void* dst[4] = {nullptr, nullptr, nullptr, nullptr};
        for (int i = 0; i < 4; ++i) {
            const size_t b = i < 2 ? bytes_a : bytes_b;
            if (cudaMalloc(&dst[i], b) != cudaSuccess) {
                release();
                return fail(MLMC_ERR_OOM, "cudaMalloc of the device copy of problem %d's parameters failed", q);
            }
            owned.push_back(dst[i]);
            if (cudaMemcpyAsync(dst[i], src[i], b, cudaMemcpyHostToDevice, cs) != cudaSuccess) {
                release();
                return fail(MLMC_ERR_CUDA, "copy of problem %d's parameters to the device failed", q);
            }
        }
        dev[size_t(q)].M_dev = dst[0];
        dev[size_t(q)].S_dev = dst[1];
        dev[size_t(q)].Mp_dev = dst[2];
        dev[size_t(q)].Sp_dev = dst[3];
    }
    mlmc_plan_t* plan = nullptr;
    st = mlmc_plan(dev.data(), nprob, options, stream, &plan);
    if (st != MLMC_OK) {
        release();
        return st;
    }
    size_t total = 0;
    for (int32_t q = 0; q < nprob; ++q) total += size_t(problems[q].m) * size_t(problems[q].p);
    if (cudaMalloc(reinterpret_cast<void**>(&plan->yhat_dev), sizeof(double) * total) != cudaSuccess) {
        release();
        mlmc_plan_destroy(plan);
        return fail(MLMC_ERR_OOM, "cudaMalloc of the estimate buffer failed");
    }
    plan->owned = std::move(owned);
    *plan_out = plan;
    return MLMC_OK;
}

mlmc_status mlmc_telescoping_sum_host(mlmc_plan_t* plan, double* yhat_host)
{
    mlmc_status st = enter(plan);
    if (st != MLMC_OK) return st;
    if (!yhat_host) return fail(MLMC_ERR_INVALID_ARG, "null yhat_host");
    if (!plan->yhat_dev) return fail(MLMC_ERR_STATE, "the plan was not made by mlmc_plan_host");
    if ((st = mlmc_telescoping_sum(plan, plan->yhat_dev)) != MLMC_OK) return st;
    DeviceGuard g(plan->device);
    size_t total = 0;
    for (const auto& ps : plan->probs) total += size_t(ps.m) * size_t(ps.p);
    cudaError_t err = cudaMemcpyAsync(yhat_host, plan->yhat_dev, sizeof(double) * total, cudaMemcpyDeviceToHost,
                                      plan->stream);
    if (err == cudaSuccess) err = cudaStreamSynchronize(plan->stream);
    if (check_cuda(plan, err, "copy of the estimate to the host") != MLMC_OK) return plan->sticky;
    return check_device_flag(plan);
}

mlmc_status mlmc_telescoping_sum(mlmc_plan_t* plan, double* yhat_dev)
{
    mlmc_status st = enter(plan);
    if (st != MLMC_OK) return st;
    if (!yhat_dev) return fail(MLMC_ERR_INVALID_ARG, "null yhat_dev");
    DeviceGuard g(plan->device);
    int64_t off = 0;
    for (auto& ps : plan->probs) {
        const int64_t mp = ps.m * ps.p;
        cudaError_t err = launch_telescoping(ps.sum, ps.N, ps.L + 1, mp, yhat_dev + off, plan->stream);
        if (check_cuda(plan, err, "telescoping launch") != MLMC_OK) return plan->sticky;
        plan->launches += 1;
        off += mp;
    }
    return MLMC_OK;
}

mlmc_status mlmc_allocate(mlmc_plan_t* plan, const double* eps_abs, int64_t* Nl)
{
    mlmc_status st = enter(plan);
    if (st != MLMC_OK) return st;
    if (!eps_abs || !Nl) return fail(MLMC_ERR_INVALID_ARG, "null eps_abs or Nl");
    DeviceGuard g(plan->device);
    for (size_t q = 0; q < plan->probs.size(); ++q) {
        ProblemState& ps = plan->probs[q];
        if (!(eps_abs[q] > 0.0) || !std::isfinite(eps_abs[q]))
            return fail(MLMC_ERR_INVALID_ARG, "eps_abs[%zu] must be finite and > 0", q);
        int64_t* row = Nl + q * MLMC_MAX_LEVELS;
        std::fill(row, row + MLMC_MAX_LEVELS, int64_t(0));
        if ((st = allocation(plan, ps, int(q), ps.L, eps_abs[q], row)) != MLMC_OK) return st;
    }
    return MLMC_OK;
}

mlmc_status mlmc_allocate_levels(mlmc_plan_t* plan, int32_t prob, int32_t L, double eps_abs, int64_t* Nl)
{
    mlmc_status st = enter(plan);
    if (st != MLMC_OK) return st;
    if (!Nl) return fail(MLMC_ERR_INVALID_ARG, "null Nl");
    if ((st = check_prob_level(plan, prob, L)) != MLMC_OK) return st;
    if (!(eps_abs > 0.0) || !std::isfinite(eps_abs)) return fail(MLMC_ERR_INVALID_ARG, "eps_abs must be finite and > 0");
    DeviceGuard g(plan->device);
    return allocation(plan, plan->probs[size_t(prob)], prob, L, eps_abs, Nl);
}

mlmc_status mlmc_bias_test(mlmc_plan_t* plan, int32_t prob, int32_t L, double eps_abs, int32_t* met,
                           double* mean_norm)
{
    mlmc_status st = enter(plan);
    if (st != MLMC_OK) return st;
    if (!met) return fail(MLMC_ERR_INVALID_ARG, "null met");
    if ((st = check_prob_level(plan, prob, L)) != MLMC_OK) return st;
    if (!(eps_abs > 0.0) || !std::isfinite(eps_abs)) return fail(MLMC_ERR_INVALID_ARG, "eps_abs must be finite and > 0");
    DeviceGuard g(plan->device);
    bool ok = false;
    double nrm = 0.0;
    if ((st = bias_test(plan, plan->probs[size_t(prob)], L, eps_abs, &ok, &nrm)) != MLMC_OK) return st;
    *met = ok ? 1 : 0;
    if (mean_norm) *mean_norm = nrm;
    return MLMC_OK;
}

mlmc_status mlmc_launch_count(const mlmc_plan_t* plan, uint64_t* count)
{
    if (!plan || !count) return fail(MLMC_ERR_INVALID_ARG, "null argument");
    *count = plan->launches;
    return MLMC_OK;
}

mlmc_status mlmc_estimate(mlmc_plan_t* plan, const double* eps_abs, double* yhat_dev, mlmc_report* reports)
{
    mlmc_status st = enter(plan);
    if (st != MLMC_OK) return st;
    if (!eps_abs || !yhat_dev) return fail(MLMC_ERR_INVALID_ARG, "null eps_abs or yhat_dev");
    for (size_t q = 0; q < plan->probs.size(); ++q)
        if (!(eps_abs[q] > 0.0) || !std::isfinite(eps_abs[q]))
            return fail(MLMC_ERR_INVALID_ARG, "eps_abs[%zu] must be finite and > 0", q);
    DeviceGuard g(plan->device);
    const mlmc_options& o = plan->opt;
    const uint64_t pilot = uint64_t(o.pilot_n);
    // several problems in BF16 go through the batched persistent launch
    const bool batched = tensor_core_precision(o.precision) && plan->probs.size() > 1;
    auto run_ranges = [&](const std::vector<BatchRange>& rs) -> mlmc_status {
        if (batched) return run_batch(plan, rs);
        for (const BatchRange& r : rs) {
            ProblemState& ps = plan->probs[size_t(r.prob)];
            const int64_t mp = ps.m * ps.p;
            const bool continues = r.s0 == ps.N.v[r.level];
            mlmc_status s2 = run_level(plan, ps, r.level, r.s0, r.count, ps.sum + int64_t(r.level) * mp,
                                       ps.M2 + r.level, ps.N.v[r.level]);
            if (s2 != MLMC_OK) return s2;
            ps.N.v[r.level] += r.count;
            ps.prefix[r.level] = ps.prefix[r.level] && continues;
        }
        return MLMC_OK;
    };
    // Alg. 2 in rounds.  Fixed L: one round on levels 0..L.  adaptive_L: rounds on levels 0..Lc
    // for Lc = 0, 1, ...; a problem stops after the first round with Lc >= 2 whose finest mean
    // satisfies ||Y_Lc||_F < (sqrt(R) + 1) eps / sqrt(2) (Remark 3.5), or at its own L.  Every
    // round pilots the levels that lack it, re-allocates from the variances of all samples held
    // and tops up from the next unused sample id (samples are never discarded).
    const size_t np = plan->probs.size();
    std::vector<int> Lc(np), running(np, 1), unmet(np, 0);
    for (size_t q = 0; q < np; ++q) Lc[q] = o.adaptive_L ? 0 : plan->probs[q].L;
    for (;;) {
        std::vector<BatchRange> todo;
        for (size_t q = 0; q < np; ++q) {
            if (!running[q]) continue;
            const ProblemState& ps = plan->probs[q];
            for (int l = 0; l <= Lc[q]; ++l)
                if (ps.N.v[l] < pilot) todo.push_back(BatchRange{int(q), l, ps.N.v[l], pilot - ps.N.v[l]});
        }
        if ((st = run_ranges(todo)) != MLMC_OK) return st;
        // allocation from the variances held, then top-ups from the next unused sample id
        todo.clear();
        for (size_t q = 0; q < np; ++q) {
            if (!running[q]) continue;
            ProblemState& ps = plan->probs[q];
            const int L = Lc[q];
            int64_t Nl[MLMC_MAX_LEVELS];
            if ((st = allocation(plan, ps, int(q), L, eps_abs[q], Nl)) != MLMC_OK) return set_sticky(plan, st);
            for (int l = 0; l <= L; ++l) {
                const uint64_t nl = uint64_t(Nl[l]);
                ps.Nl_est[l] = int64_t(std::max<uint64_t>(nl, ps.N.v[l]));
                if (nl > ps.N.v[l]) todo.push_back(BatchRange{int(q), l, ps.N.v[l], nl - ps.N.v[l]});
            }
        }
        if ((st = run_ranges(todo)) != MLMC_OK) return st;
        bool more = false;
        for (size_t q = 0; q < np; ++q) {
            if (!running[q]) continue;
            ProblemState& ps = plan->probs[q];
            if (!o.adaptive_L) {
                running[q] = 0;
                continue;
            }
            bool met = false;
            double nrm = 0.0;
            if (Lc[q] >= 2 && (st = bias_test(plan, ps, Lc[q], eps_abs[q], &met, &nrm)) != MLMC_OK) return st;
            if (met) {
                running[q] = 0;
            } else if (Lc[q] == ps.L) {
                running[q] = 0;
                unmet[q] = 1;
            } else {
                Lc[q] += 1;
                more = true;
            }
        }
        if (!more) break;
    }
    // telescoping sum and report
    int64_t off = 0;
    for (size_t q = 0; q < plan->probs.size(); ++q) {
        ProblemState& ps = plan->probs[q];
        const int64_t mp = ps.m * ps.p;
        const int L = Lc[q];
        cudaError_t err = launch_telescoping(ps.sum, ps.N, L + 1, mp, yhat_dev + off, plan->stream);
        if (check_cuda(plan, err, "telescoping launch") != MLMC_OK) return plan->sticky;
        plan->launches += 1;
        off += mp;
        ps.has_estimate = true;
        if (reports) {
            mlmc_report& r = reports[q];
            std::memset(&r, 0, sizeof(r));
            double M2[MLMC_MAX_LEVELS];
            if ((st = level_M2(plan, ps, 0, L + 1, M2)) != MLMC_OK) return st;
            r.L = L;
            r.bias_unmet = unmet[q];
            r.eps_abs = eps_abs[q];
            double var = 0.0;
            std::vector<double> sums(static_cast<size_t>(mp));
            for (int l = 0; l <= L; ++l) {
                r.N[l] = int64_t(ps.N.v[l]);
                r.V[l] = M2[l] / double(ps.N.v[l] - 1);
                r.cost[l] = level_cost(o, l);
                var += r.V[l] / double(ps.N.v[l]);
                r.outer_products += double(ps.N.v[l]) * double(level_c(o, l));
                err = cudaMemcpy(sums.data(), ps.sum + int64_t(l) * mp, sizeof(double) * size_t(mp),
                                 cudaMemcpyDeviceToHost);
                if (check_cuda(plan, err, "read level mean") != MLMC_OK) return plan->sticky;
                double nrm = 0.0;
                for (double v : sums) nrm += v * v;
                r.mean_norm[l] = std::sqrt(nrm) / double(ps.N.v[l]);
            }
            r.rmse_pred = std::sqrt(var);
        }
    }
    return MLMC_OK;
}

namespace {

constexpr int64_t kAdjRecordBudget = int64_t(1) << 26;   // default records per replay batch (512 MiB)
constexpr int kAdjMaxKin32 = 1584, kAdjMaxKin64 = 696;   // largest m, p the adjoint accepts (FP32, FP64)

size_t align256(size_t b) { return (b + 255) & ~size_t(255); }

// Grow the plan's adjoint scratch to at least `bytes`.
mlmc_status adj_reserve(mlmc_plan_t* plan, size_t bytes)
{
    if (bytes <= plan->adj_bytes) return MLMC_OK;
    cudaError_t err = cudaStreamSynchronize(plan->stream);
    if (check_cuda(plan, err, "adjoint scratch") != MLMC_OK) return plan->sticky;
    cudaFree(plan->adj_buf);
    plan->adj_buf = nullptr;
    plan->adj_bytes = 0;
    err = cudaMalloc(&plan->adj_buf, bytes);
    if (err != cudaSuccess) return check_cuda(plan, err, "adjoint scratch");
    plan->adj_bytes = bytes;
    return MLMC_OK;
}

// Replay of one problem: batches of (level, sample range) entries whose records fit the budget.
mlmc_status backward_problem(mlmc_plan_t* plan, ProblemState& ps, const double* G, void* dM, void* dS, void* dMp,
                             void* dSp)
{
    const mlmc_options& o = plan->opt;
    const bool f64 = plan->f64;
    int64_t cmax = 1;
    for (int l = 0; l <= ps.L; ++l) cmax = std::max(cmax, level_c(o, l));
    const int64_t want = o.adjoint_batch_log2 > 0 ? int64_t(1) << o.adjoint_batch_log2 : kAdjRecordBudget;
    const int64_t budget = std::max(want, cmax + 1);
    // scratch layout
    const int64_t n = ps.n, m = ps.m, p = ps.p;
    size_t off = 0;
    const size_t o_counts = off;  off = align256(off + sizeof(int) * size_t(n));
    const size_t o_offsets = off; off = align256(off + sizeof(int64_t) * size_t(n));
    const size_t o_cursor = off;  off = align256(off + sizeof(int64_t) * size_t(n));
    const size_t o_scan = off;    off = align256(off + sizeof(int64_t) * size_t(adjoint_scan_scratch(n)));
    const size_t o_rec = off;     off = align256(off + sizeof(uint64_t) * size_t(budget));
    const size_t o_stage = off;   off = align256(off + sizeof(double) * size_t(2 * n * m + 2 * n * p));
    mlmc_status st = adj_reserve(plan, off);
    if (st != MLMC_OK) return st;
    unsigned char* base = static_cast<unsigned char*>(plan->adj_buf);
    int* counts = reinterpret_cast<int*>(base + o_counts);
    int64_t* offsets = reinterpret_cast<int64_t*>(base + o_offsets);
    int64_t* cursor = reinterpret_cast<int64_t*>(base + o_cursor);
    int64_t* scan = reinterpret_cast<int64_t*>(base + o_scan);
    uint64_t* records = reinterpret_cast<uint64_t*>(base + o_rec);
    double* stage = reinterpret_cast<double*>(base + o_stage);

    AdjSegmentParams sp{};
    sp.PAB = ps.PAB;
    sp.ld = ps.ld;
    sp.m = int(m);
    sp.p = int(p);
    sp.m_pad = int(ps.m_pad);
    sp.n = n;
    sp.rkA = philox_round_keys(key(ps.desc.seed_A, ps.desc.problem_id));
    sp.rkB = philox_round_keys(key(ps.desc.seed_B, ps.desc.problem_id));
    sp.G = G;
    sp.offsets = offsets;
    sp.records = records;
    sp.bf16 = o.precision == MLMC_BF16 ? 1 : 0;
    sp.gM_t = stage;
    sp.gS_t = stage + n * m;
    sp.gMp = stage + 2 * n * m;
    sp.gSp = stage + 2 * n * m + n * p;
    for (int l = 0; l <= ps.L; ++l) {
        const double c = double(level_c(o, l));
        sp.w_fine[l] = double(n) / c;
        sp.w_coarse_extra[l] = l > 0 ? -double(n) / double(level_c(o, l - 1)) : 0.0;
        sp.inv_N[l] = ps.N.v[l] > 0 ? 1.0 / double(ps.N.v[l]) : 0.0;
    }
    const uint2 keyI = key(ps.desc.seed_idx, ps.desc.problem_id);
    cudaError_t err = cudaMemsetAsync(stage, 0, sizeof(double) * size_t(2 * n * m + 2 * n * p), plan->stream);
    if (check_cuda(plan, err, "adjoint staging") != MLMC_OK) return plan->sticky;

    int l = 0;
    uint64_t s_next = 0;
    for (;;) {
        // next batch
        AdjLevels lv{};
        int64_t recs = 0;
        while (l <= ps.L && lv.count < MLMC_MAX_LEVELS) {
            if (s_next >= ps.N.v[l]) {
                ++l;
                s_next = 0;
                continue;
            }
            const int64_t c = level_c(o, l);
            const uint64_t room = uint64_t((budget - recs) / c);
            if (room == 0) break;
            const uint64_t take = std::min<uint64_t>(room, ps.N.v[l] - s_next);
            lv.lev[lv.count] = l;
            lv.c[lv.count] = c;
            lv.s0[lv.count] = s_next;
            lv.pair_begin[lv.count] = lv.total_pairs;
            lv.total_pairs += int64_t(take) * ((c + 1) / 2);
            lv.count += 1;
            recs += int64_t(take) * c;
            s_next += take;
        }
        if (lv.count == 0) break;
        err = cudaMemsetAsync(counts, 0, sizeof(int) * size_t(n), plan->stream);
        if (err == cudaSuccess) err = adjoint_count(lv, keyI, n, o.ratio, counts, plan->stream);
        if (err == cudaSuccess) err = adjoint_scan(counts, n, offsets, scan, plan->stream);
        if (err == cudaSuccess)
            err = cudaMemcpyAsync(cursor, offsets, sizeof(int64_t) * size_t(n), cudaMemcpyDeviceToDevice, plan->stream);
        if (err == cudaSuccess) err = adjoint_scatter(lv, keyI, n, o.ratio, cursor, records, plan->stream);
        sp.total = recs;
        for (int side = 0; side < 2 && err == cudaSuccess; ++side) {
            const int kin = side == 0 ? int(p) : int(m);
            if (o.precision == MLMC_BF16 && adjoint_tc_supported(kin)) {
                // bfloat16 vectors: the contraction with G runs on the tensor cores
                TcLaunch tl{plan->err_flag, plan->timeout_ns, 0.0f, plan->num_sms};
                err = adjoint_segments_tc(sp, side, tl, plan->stream);
            } else {
                sp.ob = adjoint_output_block(kin, f64);
                err = adjoint_segments(sp, f64, side, plan->num_sms, plan->stream);
            }
        }
        if (check_cuda(plan, err, "adjoint batch") != MLMC_OK) return plan->sticky;
        plan->launches += 9;   // count, five scan passes, scatter, two segment reductions
    }
    err = adjoint_write_A(sp.gM_t, n, m, dM, ps.desc.ldA, ps.desc.dtype, plan->stream);
    if (err == cudaSuccess) err = adjoint_write_A(sp.gS_t, n, m, dS, ps.desc.ldA, ps.desc.dtype, plan->stream);
    if (err == cudaSuccess) err = adjoint_write_B(sp.gMp, n, p, dMp, ps.desc.ldB, ps.desc.dtype, plan->stream);
    if (err == cudaSuccess) err = adjoint_write_B(sp.gSp, n, p, dSp, ps.desc.ldB, ps.desc.dtype, plan->stream);
    if (check_cuda(plan, err, "adjoint write-out") != MLMC_OK) return plan->sticky;
    plan->launches += 4;
    return MLMC_OK;
}

}  // namespace

mlmc_status mlmc_backward(mlmc_plan_t* plan, const double* G_dev, void* const* dM_dev, void* const* dS_dev,
                          void* const* dMp_dev, void* const* dSp_dev)
{
    mlmc_status st = enter(plan);
    if (st != MLMC_OK) return st;
    if (!G_dev || !dM_dev || !dS_dev || !dMp_dev || !dSp_dev) return fail(MLMC_ERR_INVALID_ARG, "null argument");
    if (plan->opt.f != MLMC_F_IDENTITY)
        return fail(MLMC_ERR_UNSUPPORTED, "mlmc_backward: the replay is the adjoint of the linear estimator (f = x)");
    if (plan->opt.sampling != MLMC_XI_UNIFORM)
        return fail(MLMC_ERR_UNSUPPORTED, "mlmc_backward: the replay weights slots uniformly (xi^u)");
    if (plan->opt.precision == MLMC_FP8_E4M3)
        return fail(MLMC_ERR_UNSUPPORTED, "mlmc_backward: the E4M3 block scales couple the slots of a sample; "
                    "use an FP32 or BF16 plan for gradients");
    for (size_t q = 0; q < plan->probs.size(); ++q) {
        const ProblemState& ps = plan->probs[q];
        if (!dM_dev[q] || !dS_dev[q] || !dMp_dev[q] || !dSp_dev[q])
            return fail(MLMC_ERR_INVALID_ARG, "problem %zu: null gradient pointer", q);
        uint64_t total = 0;
        for (int l = 0; l <= ps.L; ++l) {
            if (!ps.prefix[l])
                return fail(MLMC_ERR_STATE, "problem %zu level %d: held samples are not the ids 0 .. N_l - 1", q, l);
            total += ps.N.v[l];
        }
        if (total == 0) return fail(MLMC_ERR_STATE, "mlmc_backward: problem %zu holds no samples", q);
        for (int side = 0; side < 2; ++side) {
            const int kin = int(side == 0 ? ps.p : ps.m);
            if (adjoint_output_block(kin, plan->f64) == 0)
                return fail(MLMC_ERR_UNSUPPORTED, "problem %zu: the adjoint keeps a block of G with all %d %s on chip; "
                            "at most %d fit", q, kin, side == 0 ? "columns" : "rows", plan->f64 ? kAdjMaxKin64 : kAdjMaxKin32);
        }
        if (ps.n > (int64_t(1) << 30)) return fail(MLMC_ERR_UNSUPPORTED, "problem %zu: the adjoint needs n <= 2^30", q);
    }
    DeviceGuard g(plan->device);
    int64_t goff = 0;
    for (size_t q = 0; q < plan->probs.size(); ++q) {
        ProblemState& ps = plan->probs[q];
        st = backward_problem(plan, ps, G_dev + goff, dM_dev[q], dS_dev[q], dMp_dev[q], dSp_dev[q]);
        if (st != MLMC_OK) return st;
        goff += ps.m * ps.p;
    }
    return MLMC_OK;
}

mlmc_status mlmc_debug_philox(const uint32_t* ctr_dev, const uint32_t* key_dev, int64_t count, uint32_t* out_dev,
                              void* stream)
{
    if (count < 0 || (count > 0 && (!ctr_dev || !key_dev || !out_dev))) return fail(MLMC_ERR_INVALID_ARG, "bad arguments");
    cudaError_t err = launch_debug_philox(ctr_dev, key_dev, count, out_dev, static_cast<cudaStream_t>(stream));
    if (err != cudaSuccess) return fail(MLMC_ERR_CUDA, "debug_philox: %s", cudaGetErrorString(err));
    return MLMC_OK;
}

mlmc_status mlmc_debug_indices(mlmc_plan_t* plan, int32_t prob, int32_t level, uint64_t sample, int64_t t0,
                               int64_t count, int64_t* idx_dev)
{
    mlmc_status st = enter(plan);
    if (st != MLMC_OK) return st;
    if ((st = check_prob_level(plan, prob, level)) != MLMC_OK) return st;
    if (t0 < 0 || count < 0 || (count > 0 && !idx_dev)) return fail(MLMC_ERR_INVALID_ARG, "bad slot range");
    DeviceGuard g(plan->device);
    ProblemState& ps = plan->probs[size_t(prob)];
    cudaError_t err = ps.xi_Q ? launch_debug_indices_xi(key(ps.desc.seed_idx, ps.desc.problem_id), level, sample, ps.n, t0,
                                                        count, ps.xi_Q, ps.xi_q, ps.xi_G, idx_dev, plan->stream)
                              : launch_debug_indices(key(ps.desc.seed_idx, ps.desc.problem_id), level, sample, ps.n, t0,
                                                     count, idx_dev, plan->stream);
    return check_cuda(plan, err, "debug_indices");
}

mlmc_status mlmc_debug_normals(mlmc_plan_t* plan, int32_t prob, int32_t which, int32_t level, uint64_t sample,
                               int64_t k, int64_t row0, int64_t count, double* z_dev)
{
    mlmc_status st = enter(plan);
    if (st != MLMC_OK) return st;
    if ((st = check_prob_level(plan, prob, level)) != MLMC_OK) return st;
    if ((which != 0 && which != 1) || row0 < 0 || count < 0 || k < 0 || (count > 0 && !z_dev))
        return fail(MLMC_ERR_INVALID_ARG, "bad arguments");
    DeviceGuard g(plan->device);
    ProblemState& ps = plan->probs[size_t(prob)];
    const uint2 kk = key(which == 0 ? ps.desc.seed_A : ps.desc.seed_B, ps.desc.problem_id);
    cudaError_t err = launch_debug_normals(kk, plan->f64, level, sample, k, row0, count, z_dev, plan->stream);
    return check_cuda(plan, err, "debug_normals");
}

mlmc_status mlmc_debug_sample(mlmc_plan_t* plan, int32_t prob, int32_t level, uint64_t sample, double* D_dev)
{
    mlmc_status st = enter(plan);
    if (st != MLMC_OK) return st;
    if ((st = check_prob_level(plan, prob, level)) != MLMC_OK) return st;
    if (!D_dev) return fail(MLMC_ERR_INVALID_ARG, "null D_dev");
    DeviceGuard g(plan->device);
    ProblemState& ps = plan->probs[size_t(prob)];
    const int64_t mp = ps.m * ps.p;
    cudaError_t err = cudaMemsetAsync(plan->dbg_sum, 0, sizeof(double) * size_t(mp), plan->stream);
    if (err == cudaSuccess) err = cudaMemsetAsync(plan->dbg_M2, 0, sizeof(double), plan->stream);
    if (check_cuda(plan, err, "debug state reset") != MLMC_OK) return plan->sticky;
    st = run_level(plan, ps, level, sample, 1, plan->dbg_sum, plan->dbg_M2, 0);
    if (st != MLMC_OK) return st;
    err = cudaMemcpyAsync(D_dev, plan->dbg_sum, sizeof(double) * size_t(mp), cudaMemcpyDeviceToDevice, plan->stream);
    return check_cuda(plan, err, "debug sample copy");
}

mlmc_status mlmc_measure_generation_rate(void* cuda_stream, double* entries_per_s)
{
    if (!entries_per_s) return fail(MLMC_ERR_INVALID_ARG, "mlmc_measure_generation_rate: null output");
    int dev = 0, sms = 0;
    cudaError_t err = cudaGetDevice(&dev);
    if (err == cudaSuccess) err = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    if (err == cudaSuccess) err = measure_generation_rate(static_cast<cudaStream_t>(cuda_stream), sms, entries_per_s);
    if (err != cudaSuccess)
        return fail(MLMC_ERR_CUDA, "mlmc_measure_generation_rate: %s", cudaGetErrorString(err));
    return MLMC_OK;
}

mlmc_status mlmc_measure_peaks(void* cuda_stream, double* ops_per_s)
{
    if (!ops_per_s) return fail(MLMC_ERR_INVALID_ARG, "mlmc_measure_peaks: null output");
    int dev = 0, sms = 0;
    cudaError_t err = cudaGetDevice(&dev);
    if (err == cudaSuccess) err = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    if (err == cudaSuccess) err = measure_peaks(static_cast<cudaStream_t>(cuda_stream), sms, ops_per_s);
    if (err != cudaSuccess) return fail(MLMC_ERR_CUDA, "mlmc_measure_peaks: %s", cudaGetErrorString(err));
    return MLMC_OK;
}

mlmc_status mlmc_debug_bounded_wait(mlmc_plan_t* plan, int64_t timeout_ns)
{
    mlmc_status st = enter(plan);
    if (st != MLMC_OK) return st;
    if (timeout_ns <= 0 || timeout_ns > int64_t(10000000000)) return fail(MLMC_ERR_INVALID_ARG, "timeout_ns must be in (0, 10 s]");
    DeviceGuard g(plan->device);
    cudaError_t err = launch_bounded_wait_probe(plan->err_flag, uint64_t(timeout_ns), plan->stream);
    if (check_cuda(plan, err, "bounded-wait probe launch") != MLMC_OK) return plan->sticky;
    plan->launches += 1;
    return MLMC_OK;
}

}  // extern "C"
