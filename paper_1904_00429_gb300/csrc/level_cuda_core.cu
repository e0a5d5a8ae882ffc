// level_cuda_core.cu -- fused level kernel on the CUDA cores (FP64 and FP32).
//
// One CTA owns one TM x TP tile of the m x p output and one chunk of up to
// prm.chunk samples of one level.  For every sample s it evaluates
//     D_s = sum_t w_t A[:, r_t] B[r_t, :],   w_t = n/c_l - [t coarse] n/c_{l-1},
// which is P_l - P_{l-1} of Alg. 1 written as one weighted sum: the coarse
// estimate reuses the draws r_{jR} (0-based slots t = jR - 1) of the fine one,
// so those slots carry both weights (Sec. 3.1).  Slots are processed in
// chunks of TK: the CTA draws the TK indices, gathers the sampled (M, S)
// pairs of its TM rows and (M', S') pairs of its TP columns (each gathered
// column/row is contiguous in the plan's layout), generates the entries
// A = M + S Z and w B = w (M' + S' Z') from Philox into shared memory, and
// accumulates the outer products in a register tile.  After each sample the
// tile is added to a running per-chunk sum and the chunk's M2 (sum of squared
// deviations from the chunk mean, Welford's update) grows in a running FP64
// scalar; at the end of the chunk both are written as partials, which the
// merge kernel folds into the level in chunk order.
// With a targeted function f (F != 0) the fine and coarse estimates are kept apart,
//     P_l = (n/c_l) sum_t A[:, r_t] B[r_t, :],   P_{l-1} = (n/c_{l-1}) sum_{t coarse} ...,
// in two register tiles, and D_s = f(P_l) - f(P_{l-1}) entrywise (f(P_0) at level 0).
#include <cuda_runtime.h>

#include "internal.h"
#include "rng.cuh"

namespace mlmc {
namespace {

template <typename T>
struct Pair4;  // four (M, S) pairs: 8 consecutive values

template <>
struct Pair4<float> {
    float v[8];
    static __device__ __forceinline__ Pair4 load(const float* p)
    {
        Pair4 r;
        const float4 a = __ldg(reinterpret_cast<const float4*>(p));
        const float4 b = __ldg(reinterpret_cast<const float4*>(p) + 1);
        r.v[0] = a.x; r.v[1] = a.y; r.v[2] = a.z; r.v[3] = a.w;
        r.v[4] = b.x; r.v[5] = b.y; r.v[6] = b.z; r.v[7] = b.w;
        return r;
    }
};

template <>
struct Pair4<double> {
    double v[8];
    static __device__ __forceinline__ Pair4 load(const double* p)
    {
        Pair4 r;
#pragma unroll
        for (int h = 0; h < 4; ++h) {
            const double2 a = __ldg(reinterpret_cast<const double2*>(p) + h);
            r.v[2 * h] = a.x;
            r.v[2 * h + 1] = a.y;
        }
        return r;
    }
};

// The targeted functions of mlmc_function: F = 1 is |x| H(2 - x) with H(0) = 1.
template <int F, typename T>
__device__ __forceinline__ T targeted(T x)
{
    if constexpr (F == 1) return (T(2) - x >= T(0)) ? fabs(x) : T(0);
    return x;
}

template <typename T, int TM, int TP, int TK, int RM, int RP, int F, bool XI>
__global__ void __launch_bounds__((TM / RM) * (TP / RP))
level_cuda_core_kernel(const LevelParams prm)
{
    constexpr int NT = (TM / RM) * (TP / RP);
    constexpr int TXN = TP / RP;
    static_assert(TK % 2 == 0 && TM % 4 == 0 && TP % 4 == 0, "tile shape");

    __shared__ __align__(16) T As[TK][TM];
    __shared__ __align__(16) T Bs[TK][TP];
    __shared__ int idx_s[TK];
    __shared__ T w_s[TK];   // F = 0: the slot's weight; F != 0: 1 on coarse slots, else 0
    __shared__ T g_s[TK];   // F != 0 under xi**: the slot's 1 / xi_{r_t} (folded into B)
    // xi**: a sample's draws (c_l <= kXiPre) are made up front by every thread (each needs a few
    // dependent table reads) instead of by TK / 2 threads per chunk of slots
    constexpr int kXiPre = 1024;
    __shared__ int idx_pre[XI ? kXiPre : 1];
    __shared__ double g_pre[XI ? kXiPre : 1];
    __shared__ double red_s[NT / 32];

    const int tid = threadIdx.x;
    const int tile = blockIdx.x;
    const int tm0 = (tile / prm.tiles_p) * TM;
    const int tp0 = (tile % prm.tiles_p) * TP;
    const int tx = tid % TXN;
    const int ty = tid / TXN;

    const uint64_t chunk = prm.chunk0 + blockIdx.y;
    const uint64_t sa = max(prm.s_begin, chunk * static_cast<uint64_t>(prm.chunk));
    const uint64_t sb = min(prm.s_end, (chunk + 1) * static_cast<uint64_t>(prm.chunk));

    const T* PA = static_cast<const T*>(prm.PA);
    const T* PB = static_cast<const T*>(prm.PB);
    const T wf = static_cast<T>(prm.w_fine);
    const T wc = static_cast<T>(prm.w_coarse);
    const T wcn = static_cast<T>(prm.w_fine - prm.w_coarse);   // n / c_{l-1}
    // xi** (Thm 3.1): per-slot weights 1 / xi_{r_t} = Q[n-1] / q[r_t], estimates scaled by 1 / c
    constexpr bool xi = XI;   // prm.xi_Q is set
    const double inv_c = 1.0 / static_cast<double>(prm.c);
    const double inv_cc = prm.l > 0 ? 1.0 / static_cast<double>(prm.c / prm.R) : 0.0;
    const T sf = xi ? static_cast<T>(inv_c) : wf;     // F != 0: scale of the fine estimate
    const T sc = xi ? static_cast<T>(inv_cc) : wcn;   // and of the coarse one

    T sum[RM][RP];
#pragma unroll
    for (int i = 0; i < RM; ++i)
#pragma unroll
        for (int j = 0; j < RP; ++j) sum[i][j] = T(0);
    T qw = T(0);   // the chunk's M2 (Welford terms)

    for (uint64_t s = sa; s < sb; ++s) {
        const uint32_t lsw = level_sample_word(prm.l, s);
        const uint32_t s_lo = static_cast<uint32_t>(s);
        T acc[RM][RP];
        T accc[RM][RP];   // F != 0: the coarse estimate's sum
#pragma unroll
        for (int i = 0; i < RM; ++i)
#pragma unroll
            for (int j = 0; j < RP; ++j) acc[i][j] = accc[i][j] = T(0);

        const bool pre = XI && prm.c <= kXiPre;
        if constexpr (XI) {
            if (pre) {
                for (int h = tid; 2 * h < prm.c; h += NT) {
                    uint64_t w0, w1;
                    index_words(prm.keyI, lsw, s_lo, h, w0, w1);
                    const int64_t r0 = index_from_cdf(w0, prm.xi_Q, prm.xi_q, prm.xi_G, prm.n);
                    idx_pre[2 * h] = static_cast<int>(r0);
                    g_pre[2 * h] = __ddiv_rn(prm.xi_Qtot, prm.xi_q[r0]);
                    if (2 * h + 1 < prm.c) {
                        const int64_t r1 = index_from_cdf(w1, prm.xi_Q, prm.xi_q, prm.xi_G, prm.n);
                        idx_pre[2 * h + 1] = static_cast<int>(r1);
                        g_pre[2 * h + 1] = __ddiv_rn(prm.xi_Qtot, prm.xi_q[r1]);
                    }
                }
                __syncthreads();
            }
        }
        for (int k0 = 0; k0 < prm.c; k0 += TK) {
            // 1. indices and weights of slots k0 .. k0 + TK - 1
            for (int h = tid; h < TK / 2; h += NT) {
                const int t = k0 + 2 * h;
                if (t < prm.c) {
                    int64_t r0, r1;
                    double g[2] = {1.0, 1.0};
                    if constexpr (xi) {
                        if (pre) {
                            r0 = idx_pre[t];
                            g[0] = g_pre[t];
                            r1 = t + 1 < prm.c ? idx_pre[t + 1] : 0;
                            g[1] = t + 1 < prm.c ? g_pre[t + 1] : 0.0;
                        } else {
                            uint64_t w0, w1;
                            index_words(prm.keyI, lsw, s_lo, t >> 1, w0, w1);
                            r0 = index_from_cdf(w0, prm.xi_Q, prm.xi_q, prm.xi_G, prm.n);
                            r1 = index_from_cdf(w1, prm.xi_Q, prm.xi_q, prm.xi_G, prm.n);
                            g[0] = __ddiv_rn(prm.xi_Qtot, prm.xi_q[r0]);
                            g[1] = __ddiv_rn(prm.xi_Qtot, prm.xi_q[r1]);
                        }
                    } else {
                        index_pair(prm.keyI, lsw, s_lo, t >> 1, static_cast<uint64_t>(prm.n), r0, r1);
                    }
#pragma unroll
                    for (int e = 0; e < 2; ++e) {
                        const int te = t + e;
                        const bool valid = te < prm.c;
                        const bool coarse = prm.l > 0 && (te % prm.R) == prm.R - 1;
                        idx_s[2 * h + e] = valid ? static_cast<int>(e ? r1 : r0) : -1;
                        if constexpr (F == 0) {
                            if constexpr (xi)
                                w_s[2 * h + e] = valid ? static_cast<T>(g[e] * (coarse ? inv_c - inv_cc : inv_c)) : T(0);
                            else
                                w_s[2 * h + e] = valid ? (coarse ? wc : wf) : T(0);
                        } else {
                            w_s[2 * h + e] = (valid && coarse) ? T(1) : T(0);
                            g_s[2 * h + e] = valid ? static_cast<T>(g[e]) : T(0);
                        }
                    }
                } else {
                    idx_s[2 * h] = idx_s[2 * h + 1] = -1;
                    w_s[2 * h] = w_s[2 * h + 1] = T(0);
                }
            }
            __syncthreads();

            // 2. sampled entries of A: TK slots x TM rows, four rows per Philox block
            for (int it = tid; it < TK * (TM / 4); it += NT) {
                const int tt = it / (TM / 4);
                const int q4 = it % (TM / 4);
                const int i = tm0 + 4 * q4;
                const int k = idx_s[tt];
                T a[4] = {T(0), T(0), T(0), T(0)};
                if (k >= 0 && i < prm.m) {
                    const uint4 w = philox4x32_10(make_uint4(static_cast<uint32_t>(i >> 2),
                                                             static_cast<uint32_t>(k), s_lo, lsw),
                                                  prm.keyA);
                    T z[4];
                    Normals<T>::four(w, z);
                    const Pair4<T> ms = Pair4<T>::load(PA + static_cast<int64_t>(k) * prm.ldPA + 2 * i);
#pragma unroll
                    for (int r = 0; r < 4; ++r) a[r] = fma(ms.v[2 * r + 1], z[r], ms.v[2 * r]);
                }
#pragma unroll
                for (int r = 0; r < 4; ++r) As[tt][4 * q4 + r] = a[r];
            }
            // 3. sampled entries of B, weight folded in: TK slots x TP columns
            for (int it = tid; it < TK * (TP / 4); it += NT) {
                const int tt = it / (TP / 4);
                const int q4 = it % (TP / 4);
                const int j = tp0 + 4 * q4;
                const int k = idx_s[tt];
                T b[4] = {T(0), T(0), T(0), T(0)};
                if (k >= 0 && j < prm.p) {
                    const uint4 w = philox4x32_10(make_uint4(static_cast<uint32_t>(j >> 2),
                                                             static_cast<uint32_t>(k), s_lo, lsw),
                                                  prm.keyB);
                    T z[4];
                    Normals<T>::four(w, z);
                    const Pair4<T> ms = Pair4<T>::load(PB + static_cast<int64_t>(k) * prm.ldPB + 2 * j);
                    // F != 0: the per-estimate scales are applied at the end; xi** folds 1 / xi here
                    const T wt = F == 0 ? w_s[tt] : (xi ? g_s[tt] : T(1));
#pragma unroll
                    for (int r = 0; r < 4; ++r) b[r] = wt * fma(ms.v[2 * r + 1], z[r], ms.v[2 * r]);
                }
#pragma unroll
                for (int r = 0; r < 4; ++r) Bs[tt][4 * q4 + r] = b[r];
            }
            __syncthreads();

            // 4. rank-TK update of the register tile
            const int kt = min(TK, prm.c - k0);
            for (int tt = 0; tt < kt; ++tt) {
                T av[RM], bv[RP];
#pragma unroll
                for (int i = 0; i < RM; ++i) av[i] = As[tt][ty * RM + i];
#pragma unroll
                for (int j = 0; j < RP; ++j) bv[j] = Bs[tt][tx * RP + j];
#pragma unroll
                for (int i = 0; i < RM; ++i)
#pragma unroll
                    for (int j = 0; j < RP; ++j) acc[i][j] = fma(av[i], bv[j], acc[i][j]);
                if constexpr (F != 0) {
                    if (w_s[tt] != T(0)) {   // coarse slot (uniform across the CTA)
#pragma unroll
                        for (int i = 0; i < RM; ++i)
#pragma unroll
                            for (int j = 0; j < RP; ++j) accc[i][j] = fma(av[i], bv[j], accc[i][j]);
                    }
                }
            }
            __syncthreads();
        }

        if constexpr (F != 0) {
            // D = f(P_l) - f(P_{l-1}) entrywise; f(P_0) at level 0
#pragma unroll
            for (int i = 0; i < RM; ++i)
#pragma unroll
                for (int j = 0; j < RP; ++j)
                    acc[i][j] = prm.l > 0 ? targeted<F>(sf * acc[i][j]) - targeted<F>(sc * accc[i][j])
                                          : targeted<F>(sf * acc[i][j]);
        }
        // per-sample statistics: the chunk's running sum of D and its M2 by Welford's update;
        // with k samples before, k (D - mean_k) = k D - sum_k is one fused rounding and
        // M2 += ||k D - sum_k||^2 / (k (k + 1))
        const int kprev = static_cast<int>(s - sa);
        if (kprev > 0) {
            // in T (FP64 runs at 1/64 of the FP32 rate on this GPU: FP32 plans stay in FP32)
            const T kf = static_cast<T>(kprev);
            T qs = T(0);
#pragma unroll
            for (int i = 0; i < RM; ++i)
#pragma unroll
                for (int j = 0; j < RP; ++j) {
                    const T dk = fma(kf, acc[i][j], -sum[i][j]);
                    qs = fma(dk, dk, qs);
                }
            qw = fma(qs, T(1) / static_cast<T>(kprev * (kprev + 1)), qw);
        }
#pragma unroll
        for (int i = 0; i < RM; ++i)
#pragma unroll
            for (int j = 0; j < RP; ++j) sum[i][j] += acc[i][j];
    }

    // chunk partials: the tile's sum of D (rows/cols inside the problem only)
    T* out = static_cast<T*>(prm.partial_sum) + static_cast<int64_t>(blockIdx.y) * prm.m * prm.p;
#pragma unroll
    for (int i = 0; i < RM; ++i) {
        const int gi = tm0 + ty * RM + i;
        if (gi >= prm.m) continue;
#pragma unroll
        for (int j = 0; j < RP; ++j) {
            const int gj = tp0 + tx * RP + j;
            if (gj < prm.p) out[static_cast<int64_t>(gi) * prm.p + gj] = sum[i][j];
        }
    }
    // and its M2, reduced over the CTA in a fixed order
    double q = static_cast<double>(qw);
#pragma unroll
    for (int off = 16; off > 0; off >>= 1) q += __shfl_xor_sync(0xffffffffu, q, off);
    if ((tid & 31) == 0) red_s[tid >> 5] = q;
    __syncthreads();
    if (tid == 0) {
        double t = 0.0;
        for (int w = 0; w < NT / 32; ++w) t += red_s[w];
        prm.partial_q[static_cast<int64_t>(blockIdx.y) * prm.tiles_m * prm.tiles_p + tile] = t;
    }
}

template <typename T, int TM, int TP, int TK, int RM, int RP, bool kIdentityOnly = false>
cudaError_t launch(const LevelParams& prm, int f, cudaStream_t st)
{
    constexpr int NT = (TM / RM) * (TP / RP);
    dim3 grid(prm.tiles_m * prm.tiles_p, prm.nchunks);
    const bool xi = prm.xi_Q != nullptr;
    if constexpr (kIdentityOnly) {
        if (f != 0) return cudaErrorInvalidValue;
        if (xi)
            level_cuda_core_kernel<T, TM, TP, TK, RM, RP, 0, true><<<grid, NT, 0, st>>>(prm);
        else
            level_cuda_core_kernel<T, TM, TP, TK, RM, RP, 0, false><<<grid, NT, 0, st>>>(prm);
        return cudaGetLastError();
    } else {
        switch (f * 2 + (xi ? 1 : 0)) {
        case 0: level_cuda_core_kernel<T, TM, TP, TK, RM, RP, 0, false><<<grid, NT, 0, st>>>(prm); break;
        case 1: level_cuda_core_kernel<T, TM, TP, TK, RM, RP, 0, true><<<grid, NT, 0, st>>>(prm); break;
        case 2: level_cuda_core_kernel<T, TM, TP, TK, RM, RP, 1, false><<<grid, NT, 0, st>>>(prm); break;
        case 3: level_cuda_core_kernel<T, TM, TP, TK, RM, RP, 1, true><<<grid, NT, 0, st>>>(prm); break;
        default: return cudaErrorInvalidValue;
        }
        return cudaGetLastError();
    }
}

}  // namespace

// Output tiles (id 1000 rows + columns): 64 x 64 (4 x 4 registers per thread); FP32 with
// f = identity also 128 x 64 (8 x 4) and 128 x 128 (8 x 8), which generate each sampled entry of
// A for fewer output tiles at the price of occupancy.  Measured on a GB300 at 256 x 65536 x 256:
// 128 x 64 (two CTAs per SM) 8 % faster than 64 x 64 (three), 128 x 128 (one) 11 % slower; so FP32
// outputs of more than 64 rows take 128 x 64.
int cuda_core_default_tile(int precision, int f, int64_t m)
{
    return (precision == MLMC_FP32 && f == MLMC_F_IDENTITY && m > 64) ? 128064 : 64064;
}

bool cuda_core_tile_valid(int precision, int f, int id)
{
    if (id == 64064) return true;
    return precision == MLMC_FP32 && f == MLMC_F_IDENTITY && (id == 128064 || id == 128128);
}

CudaCoreTile cuda_core_tile(int id)
{
    if (id == 128064) return CudaCoreTile{128, 64};
    if (id == 128128) return CudaCoreTile{128, 128};
    return CudaCoreTile{64, 64};
}

cudaError_t launch_level_cuda_core_f64(const LevelParams& prm, int f, cudaStream_t st)
{
    return launch<double, 64, 64, 32, 4, 4>(prm, f, st);
}

cudaError_t launch_level_cuda_core_f32(const LevelParams& prm, int f, cudaStream_t st)
{
    if (prm.cc_tile == 128128) return launch<float, 128, 128, 32, 8, 8, true>(prm, f, st);
    if (prm.cc_tile == 128064) return launch<float, 128, 64, 32, 8, 4, true>(prm, f, st);
    return launch<float, 64, 64, 32, 4, 4>(prm, f, st);
}

}  // namespace mlmc
