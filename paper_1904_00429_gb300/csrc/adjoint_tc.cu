// adjoint_tc.cu -- segment reduction of the adjoint on the tensor cores (BF16 plans).
//
// For a BF16 plan the replayed entries are bfloat16 values (the forward rounded them, and the
// straight-through gradient differentiates the rounded entries), so the contraction of one output
// block with the records of a chunk is a dense product: for the A side
//     U[o, j] = sum_x G[o, x] b_j[x],   o in the CTA's 128 outputs, j in the chunk's 64 records,
// (B side: G^T and the vectors a_j).  G is split into bfloat16 parts G = G_hi + G_lo + O(2^-17 |G|)
// once per CTA; each chunk runs M = 128, N = 64, K = 16 tcgen05 MMAs over both parts into one FP32
// accumulator in tensor memory.  The epilogue reads U (one output row per lane) and folds
//     gM[k, o] += sum_j omega_j U[o, j],   gS[k, o] += sum_j omega_j z_j[o] U[o, j]
// in FP32 per chunk and FP64 across chunks, exactly as the CUDA-core segment kernel does.
// A CTA walks the chunks of its segments as one stream with two accumulators (128 TMEM columns)
// and two vector buffers: while the MMAs of chunk c run, the threads fold chunk c - 1 (regenerating
// its output-side normals) and build the vectors of chunk c + 1.
// Records, segments, weights and the regeneration of the vectors (Philox, the special-function-unit
// Box-Muller of the forward kernel, bfloat16 rounding) follow adjoint.cu.  Waits are bounded.
#include <algorithm>

#include <cuda_bf16.h>
#include <cuda_runtime.h>

#include "internal.h"
#include "rng.cuh"
#include "tc_ptx.cuh"

namespace mlmc {
namespace {

constexpr int kTcThreads = 512;
constexpr int kTcWarps = kTcThreads / 32;
constexpr int kTcGroups = kTcThreads / 128;   // record groups of the epilogue (4 warps each)
constexpr int kTcRec = 64;                    // records per chunk = MMA N
constexpr int kGroupRec = kTcRec / kTcGroups;
constexpr int kTcOut = 128;                   // outputs per CTA = MMA M
constexpr int kTcMaxAtoms = 4;                // contracted entries up to 4 x 64 (resident G block)
static_assert(kGroupRec == 16, "one 16-column TMEM load per warp and chunk");

// Shared memory, bytes from the 1024-aligned base.  Vectors, records and weights are double
// buffered: the MMA of chunk c runs while the epilogue of chunk c - 1 and the vectors of chunk
// c + 1 are computed.
struct TcAdjSmem {
    size_t g_hi, g_lo, v, zslab, row, rec, omega, red, bar, total;
    __host__ __device__ explicit TcAdjSmem(int atoms)
    {
        g_hi = 0;
        g_lo = g_hi + static_cast<size_t>(atoms) * kTcOut * 128;
        v = g_lo + static_cast<size_t>(atoms) * kTcOut * 128;                 // [2][atoms][64 rows][128 B]
        zslab = v + 2 * static_cast<size_t>(atoms) * kTcRec * 128;           // [warp][4 records][32 outputs]
        row = zslab + static_cast<size_t>(kTcWarps) * 4 * 32 * 4;            // (M, S) pairs of the segment's row
        rec = row + static_cast<size_t>(atoms) * 64 * 8;                      // [2][kTcRec]
        omega = rec + 2 * kTcRec * 8;                                         // [2][kTcRec]
        red = omega + 2 * kTcRec * 4;                                         // [group][M, S][outputs]
        bar = red + static_cast<size_t>(2 * kTcGroups) * kTcOut * 8;          // 2 mbarriers, tmem address, flag
        total = bar + 32;
    }
};

struct Chunk {
    int64_t k;    // segment (contracted row of the parameters)
    int64_t c0;   // first record
    int nc;       // records (1..64)
    bool last;    // last chunk of the segment
};

template <int side, int ATOMS>
__global__ void __launch_bounds__(kTcThreads, 1) segment_tc_kernel(const AdjSegmentParams prm, const TcLaunch tl)
{
    extern __shared__ unsigned char smem_raw[];
    unsigned char* smem = reinterpret_cast<unsigned char*>((reinterpret_cast<uintptr_t>(smem_raw) + 1023) &
                                                           ~static_cast<uintptr_t>(1023));
    constexpr int kG8 = ATOMS * 8;   // 16-byte chunks (8 entries) per contracted vector
    const int kin = side == 0 ? prm.p : prm.m;
    const int kout = side == 0 ? prm.m : prm.p;
    const int o0 = blockIdx.y * kTcOut;
    const int ob = min(kTcOut, kout - o0);
    const TcAdjSmem L(ATOMS);
    unsigned char* g_hi = smem + L.g_hi;
    unsigned char* g_lo = smem + L.g_lo;
    unsigned char* vt = smem + L.v;
    float* zslab = reinterpret_cast<float*>(smem + L.zslab);
    float* row_s = reinterpret_cast<float*>(smem + L.row);
    uint64_t* rec_s = reinterpret_cast<uint64_t*>(smem + L.rec);
    float* omega = reinterpret_cast<float*>(smem + L.omega);
    double* red = reinterpret_cast<double*>(smem + L.red);
    uint64_t* bar = reinterpret_cast<uint64_t*>(smem + L.bar);
    uint32_t* tmem_s = reinterpret_cast<uint32_t*>(smem + L.bar + 16);
    volatile int* abort_s = reinterpret_cast<volatile int*>(smem + L.bar + 20);

    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    if (warp == 0) tc::tmem_alloc(tc::smem_addr(tmem_s), 2 * kTcRec);
    if (tid == 0) {
        tc::mbar_init(tc::smem_addr(&bar[0]), 1);
        tc::mbar_init(tc::smem_addr(&bar[1]), 1);
        tc::mbar_init_fence();
        *abort_s = 0;
    }
    // the CTA's block of G as bfloat16 hi and lo parts, K-major (K = contracted index), 128-byte swizzle
    for (int e = tid; e < kTcOut * ATOMS * 64; e += kTcThreads) {
        const int r = e / (ATOMS * 64), x = e % (ATOMS * 64);
        double g = 0.0;
        if (r < ob && x < kin)
            g = side == 0 ? prm.G[static_cast<int64_t>(o0 + r) * prm.p + x] : prm.G[static_cast<int64_t>(x) * prm.p + o0 + r];
        const float gf = static_cast<float>(g);
        const __nv_bfloat16 hi = __float2bfloat16_rn(gf);
        const __nv_bfloat16 lo = __float2bfloat16_rn(gf - __bfloat162float(hi));
        const uint32_t off = static_cast<uint32_t>((x >> 6) * kTcOut * 128) + tc::sw128_offset(r, (x & 63) >> 3) +
                             2u * static_cast<uint32_t>(x & 7);
        *reinterpret_cast<__nv_bfloat16*>(g_hi + off) = hi;
        *reinterpret_cast<__nv_bfloat16*>(g_lo + off) = lo;
    }
    tc::fence_proxy_async_smem();
    tc::tc_fence_before_sync();
    __syncthreads();
    tc::tc_fence_after_sync();
    const uint32_t tmem = *tmem_s;

    const float* P = static_cast<const float*>(prm.PAB);
    const int64_t in_off = side == 0 ? 2 * static_cast<int64_t>(prm.m_pad) : 0;
    const PhiloxRoundKeys& rk_in = side == 0 ? prm.rkB : prm.rkA;
    const PhiloxRoundKeys& rk_out = side == 0 ? prm.rkA : prm.rkB;
    constexpr uint32_t idesc = tc::idesc_bf16_f32(kTcOut, kTcRec);
    const int quarter = warp & 3;   // TMEM lanes (outputs) 32 * quarter ..
    const int group = warp >> 2;    // records kGroupRec * group ..
    const int o_loc = quarter * 32 + lane;
    float* zw = zslab + warp * 128;
    const uint64_t desc_hi = tc::sw128_kmajor_desc(tc::smem_addr(g_hi));
    const uint64_t desc_lo = tc::sw128_kmajor_desc(tc::smem_addr(g_lo));
    const uint64_t desc_v0 = tc::sw128_kmajor_desc(tc::smem_addr(vt));

    // chunks of this CTA's segments k = blockIdx.x + i gridDim.x, in order (uniform across the CTA)
    int64_t k_it = blockIdx.x, c_next = 0, seg_end = 0;
    bool started = false;
    auto advance = [&](Chunk& ch) -> bool {
        while (c_next >= seg_end) {
            if (started) k_it += gridDim.x;
            started = true;
            if (k_it >= prm.n) return false;
            c_next = prm.offsets[k_it];
            seg_end = k_it + 1 < prm.n ? prm.offsets[k_it + 1] : prm.total;
        }
        ch.k = k_it;
        ch.c0 = c_next;
        ch.nc = static_cast<int>(seg_end - c_next < kTcRec ? seg_end - c_next : kTcRec);
        c_next += kTcRec;
        ch.last = c_next >= seg_end;
        return true;
    };

    uint32_t phase = 0;   // bit b: parity of the next completion of bar[b]
    int last_b = -1;      // buffer of the most recent commit (thread 0)
    uint32_t last_par = 0;
    bool have_prev = false, aborted = false;
    Chunk prev{0, 0, 0, false};
    int64_t row_k = -1;
    double accM = 0.0, accS = 0.0;

    for (int it = 0;; ++it) {
        Chunk cur;
        const bool have = advance(cur);
        tc::tc_fence_before_sync();
        __syncthreads();   // the epilogue of the previous chunk is done with its buffers
        if (*abort_s) {
            aborted = true;
            break;
        }
        const int buf = it & 1;
        if (have) {
            if (tid < kTcRec) {
                uint64_t rec = 0;
                float om = 0.0f;
                if (tid < cur.nc) {
                    rec = prm.records[cur.c0 + tid];
                    const int l = static_cast<int>(rec & 31);
                    const bool coarse = (rec >> 5) & 1;
                    om = static_cast<float>((prm.w_fine[l] + (coarse ? prm.w_coarse_extra[l] : 0.0)) * prm.inv_N[l]);
                }
                rec_s[buf * kTcRec + tid] = rec;
                omega[buf * kTcRec + tid] = om;
            }
            if (cur.k != row_k) {
                const float* row = P + cur.k * prm.ld + in_off;
                for (int e = tid; e < 2 * ATOMS * 64; e += kTcThreads) row_s[e] = e < 2 * kin ? row[e] : 0.0f;
                row_k = cur.k;
            }
            __syncthreads();
            // the chunk's contracted vectors, bfloat16, as the K-major B operand (one row per record);
            // a thread builds one 16-byte swizzle chunk (8 entries, two Philox blocks) at a time
            unsigned char* vb = vt + buf * (ATOMS * kTcRec * 128);
            const uint64_t* rb = rec_s + buf * kTcRec;
#pragma unroll 1
            for (int e = tid; e < kTcRec * kG8; e += kTcThreads) {
                const int j = e / kG8, c8 = e % kG8;
                const int x = 8 * c8;
                uint4 packed = make_uint4(0u, 0u, 0u, 0u);
                if (j < cur.nc) {
                    const uint64_t rec = rb[j];
                    const uint64_t s = rec >> 6;
                    const uint32_t lsw = level_sample_word(static_cast<int>(rec & 31), s);
                    const uint4 w0 = philox4x32_10_rk(
                        make_uint4(static_cast<uint32_t>(2 * c8), static_cast<uint32_t>(cur.k), static_cast<uint32_t>(s), lsw),
                        rk_in);
                    const uint4 w1 = philox4x32_10_rk(
                        make_uint4(static_cast<uint32_t>(2 * c8 + 1), static_cast<uint32_t>(cur.k), static_cast<uint32_t>(s), lsw),
                        rk_in);
                    float z[8];
                    normals4_mufu(w0, z);
                    normals4_mufu(w1, z + 4);
                    const float4* rp = reinterpret_cast<const float4*>(row_s) + 4 * c8;
                    float v[8];
#pragma unroll
                    for (int q = 0; q < 4; ++q) {
                        const float4 pq = rp[q];   // (M, S) of entries x + 2q, x + 2q + 1
                        v[2 * q] = x + 2 * q < kin ? fmaf(pq.y, z[2 * q], pq.x) : 0.0f;
                        v[2 * q + 1] = x + 2 * q + 1 < kin ? fmaf(pq.w, z[2 * q + 1], pq.z) : 0.0f;
                    }
                    const __nv_bfloat162 b0 = __floats2bfloat162_rn(v[0], v[1]);
                    const __nv_bfloat162 b1 = __floats2bfloat162_rn(v[2], v[3]);
                    const __nv_bfloat162 b2 = __floats2bfloat162_rn(v[4], v[5]);
                    const __nv_bfloat162 b3 = __floats2bfloat162_rn(v[6], v[7]);
                    packed = make_uint4(*reinterpret_cast<const uint32_t*>(&b0), *reinterpret_cast<const uint32_t*>(&b1),
                                        *reinterpret_cast<const uint32_t*>(&b2), *reinterpret_cast<const uint32_t*>(&b3));
                }
                *reinterpret_cast<uint4*>(vb + (x >> 6) * (kTcRec * 128) + tc::sw128_offset(j, (x & 63) >> 3)) = packed;
            }
            tc::fence_proxy_async_smem();
            tc::tc_fence_before_sync();
            __syncthreads();
            if (tid == 0) {
                tc::tc_fence_after_sync();
                const uint32_t d = tmem + static_cast<uint32_t>(buf * kTcRec);
                // descriptors advance by (byte offset >> 4) in their start-address field
                const uint64_t bdesc0 = desc_v0 + static_cast<uint64_t>((buf * ATOMS * kTcRec * 128) >> 4);
#pragma unroll
                for (int part = 0; part < 2; ++part) {
#pragma unroll
                    for (int ks = 0; ks < ATOMS * 4; ++ks) {
                        const uint64_t adesc = (part ? desc_lo : desc_hi) +
                                               static_cast<uint64_t>(((ks >> 2) * kTcOut * 128 + 32 * (ks & 3)) >> 4);
                        const uint64_t bdesc = bdesc0 + static_cast<uint64_t>(((ks >> 2) * kTcRec * 128 + 32 * (ks & 3)) >> 4);
                        tc::mma_bf16(d, adesc, bdesc, idesc, (part > 0 || ks > 0) ? 1u : 0u);
                    }
                }
                tc::mma_commit(tc::smem_addr(&bar[buf]));
                last_b = buf;
                last_par = (phase >> buf) & 1u;
            }
        }
        if (have_prev) {
            // epilogue of the previous chunk while this chunk's MMAs run
            const int pb = buf ^ 1;
            if (!tc::mbar_wait_bounded(tc::smem_addr(&bar[pb]), (phase >> pb) & 1u, tc::globaltimer() + tl.timeout_ns)) {
                *abort_s = 1;
                atomicExch(tl.err_flag, MLMC_ERR_TIMEOUT);
            }
            phase ^= 1u << pb;
            __syncwarp();
            tc::tc_fence_after_sync();
            float u[kGroupRec];
            tc::tmem_ld_32x32b_x16_nowait(tmem + (static_cast<uint32_t>(quarter * 32) << 16) +
                                              static_cast<uint32_t>(pb * kTcRec + group * kGroupRec),
                                          u);
            tc::tmem_ld_wait();
            const uint64_t* rb = rec_s + pb * kTcRec;
            const float* wb = omega + pb * kTcRec;
            float sm = 0.0f, ss = 0.0f;
            if (group * kGroupRec < prev.nc) {   // uniform per warp; records past nc have omega = 0
                // normals of outputs o0 + 32 quarter + 4 (lane & 7) .. + 3 for records 4 r + lane / 8 of the
                // group, passed through the warp's slab so that lane L reads output 32 quarter + L
                const int oq = quarter * 32 + 4 * (lane & 7);
                float z[kGroupRec / 4][4];
#pragma unroll
                for (int r = 0; r < kGroupRec / 4; ++r) {
                    const uint64_t rec = rb[group * kGroupRec + 4 * r + (lane >> 3)];
                    const uint64_t s = rec >> 6;
                    const uint4 w = philox4x32_10_rk(
                        make_uint4(static_cast<uint32_t>((o0 + oq) >> 2), static_cast<uint32_t>(prev.k),
                                   static_cast<uint32_t>(s), level_sample_word(static_cast<int>(rec & 31), s)),
                        rk_out);
                    normals4_mufu(w, z[r]);
                }
#pragma unroll
                for (int r = 0; r < kGroupRec / 4; ++r) {
                    reinterpret_cast<float4*>(zw)[lane] = make_float4(z[r][0], z[r][1], z[r][2], z[r][3]);
                    __syncwarp();
#pragma unroll
                    for (int t = 0; t < 4; ++t) {
                        const int jj = 4 * r + t;
                        const float wu = wb[group * kGroupRec + jj] * u[jj];
                        sm += wu;
                        ss = fmaf(wu, zw[t * 32 + lane], ss);
                    }
                    __syncwarp();
                }
            }
            accM += static_cast<double>(sm);
            accS += static_cast<double>(ss);
            if (prev.last) {
                // the record groups of every output, summed in a fixed order
                red[(group * 2 + 0) * kTcOut + o_loc] = accM;
                red[(group * 2 + 1) * kTcOut + o_loc] = accS;
                accM = accS = 0.0;
                __syncthreads();
                if (tid < ob) {
                    double tm = 0.0, ts = 0.0;
#pragma unroll
                    for (int g = 0; g < kTcGroups; ++g) {
                        tm += red[(2 * g) * kTcOut + tid];
                        ts += red[(2 * g + 1) * kTcOut + tid];
                    }
                    const int o = o0 + tid;
                    if (side == 0) {
                        prm.gM_t[prev.k * prm.m + o] += tm;
                        prm.gS_t[prev.k * prm.m + o] += ts;
                    } else {
                        prm.gMp[prev.k * prm.p + o] += tm;
                        prm.gSp[prev.k * prm.p + o] += ts;
                    }
                }
            }
        }
        if (!have) break;
        prev = cur;
        have_prev = true;
    }
    if (aborted && tid == 0 && last_b >= 0) {
        // no MMA may still write tensor memory when it is freed: the last commit covers every
        // earlier MMA of this thread
        tc::mbar_wait_bounded(tc::smem_addr(&bar[last_b]), last_par, tc::globaltimer() + 100000000ull);
    }
    tc::tc_fence_before_sync();
    __syncthreads();
    if (warp == 0) tc::tmem_dealloc(tmem, 2 * kTcRec);
}

template <int side, int ATOMS>
cudaError_t launch_side(const AdjSegmentParams& prm, const TcLaunch& tl, cudaStream_t st)
{
    const int kout = side == 0 ? prm.m : prm.p;
    const size_t smem = TcAdjSmem(ATOMS).total + 1024;
    cudaError_t e = cudaFuncSetAttribute(segment_tc_kernel<side, ATOMS>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                         static_cast<int>(smem));
    if (e != cudaSuccess) return e;
    const int oblocks = (kout + kTcOut - 1) / kTcOut;
    const int64_t want = (static_cast<int64_t>(tl.num_sms) + oblocks - 1) / oblocks;
    const unsigned batches = static_cast<unsigned>(std::max<int64_t>(1, std::min<int64_t>(prm.n, want)));
    segment_tc_kernel<side, ATOMS><<<dim3(batches, static_cast<unsigned>(oblocks)), kTcThreads, smem, st>>>(prm, tl);
    return cudaGetLastError();
}

template <int side>
cudaError_t launch_atoms(const AdjSegmentParams& prm, int atoms, const TcLaunch& tl, cudaStream_t st)
{
    switch (atoms) {
    case 1: return launch_side<side, 1>(prm, tl, st);
    case 2: return launch_side<side, 2>(prm, tl, st);
    case 3: return launch_side<side, 3>(prm, tl, st);
    case 4: return launch_side<side, 4>(prm, tl, st);
    default: return cudaErrorInvalidValue;
    }
}

}  // namespace

bool adjoint_tc_supported(int kin)
{
    return kin >= 1 && kin <= 64 * kTcMaxAtoms && TcAdjSmem(kTcMaxAtoms).total + 1024 <= 227 * 1024;
}

cudaError_t adjoint_segments_tc(const AdjSegmentParams& prm, int side, const TcLaunch& tl, cudaStream_t st)
{
    const int kin = side == 0 ? prm.p : prm.m;
    if (!adjoint_tc_supported(kin)) return cudaErrorInvalidValue;
    const int atoms = (kin + 63) / 64;
    return side == 0 ? launch_atoms<0>(prm, atoms, tl, st) : launch_atoms<1>(prm, atoms, tl, st);
}

}  // namespace mlmc
