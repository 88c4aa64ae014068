// amg_bsr.cuh -- 2x2-block CSR operator application shared by the V-cycle of
// one hierarchy (amg_solve.cu) and of a stack of hierarchies (amg_stack.cu):
// scalar traits, block loads, the lane-parallel SpMV kernels with fused
// epilogues, their launcher and the lanes-per-row rule.
#pragma once

#include <algorithm>

#include "amg_internal.cuh"

namespace bd {

// ------------------------------------------------------------------ scalar traits
template <class S> struct V2;
template <> struct V2<double> {
    using T = double2;
    static __device__ __forceinline__ double2 mk(double a, double b) { return make_double2(a, b); }
};
template <> struct V2<float> {
    using T = float2;
    static __device__ __forceinline__ float2 mk(float a, float b) { return make_float2(a, b); }
};
template <class S> using v2 = typename V2<S>::T;

template <class S> struct BlkS {
    S a00, a01, a10, a11;
};
static __device__ __forceinline__ BlkS<double> load_blk(const double *__restrict__ v, size_t t)
{
    const double2 p = ((const double2 *)v)[2 * t], q = ((const double2 *)v)[2 * t + 1];
    return {p.x, p.y, q.x, q.y};
}
static __device__ __forceinline__ BlkS<float> load_blk(const float *__restrict__ v, size_t t)
{
    const float4 p = ((const float4 *)v)[t];
    return {p.x, p.y, p.z, p.w};
}

// ------------------------------------------------------------------ lane sums
// Sums of y0 and y1 over the T lanes of a group, left in the group's first
// lane (the other lanes hold partial values).  The lower half of the group
// reduces y0 and the upper half y1, each in the tree an xor butterfly uses
// (IEEE addition is commutative, so the results carry the butterfly's bits),
// then y1 moves to the first lane: log2(T) adds per lane instead of 2 log2(T),
// and FP64 adds are scarce on this part.
template <int T, class S>
static __device__ __forceinline__ void group_sum2(S &y0, S &y1)
{
    if constexpr (T > 1) {
        const bool hi = (threadIdx.x & (T - 1)) >= T / 2;
        S mine = hi ? y1 : y0;
        mine += __shfl_xor_sync(0xffffffffu, hi ? y0 : y1, T / 2, T);
#pragma unroll
        for (int o = T / 4; o > 0; o >>= 1) mine += __shfl_xor_sync(0xffffffffu, mine, o, T);
        y0 = mine;
        y1 = __shfl_down_sync(0xffffffffu, mine, T / 2, T);
    }
}

// ------------------------------------------------------------------ block-CSR SpMV
// T lanes cooperate on one 2x2 block row (T = 1: one thread per row, no
// reduction).  The row loop is warp-uniform so every lane reaches the shuffles.
template <int T, class S, class G, class E>
static __global__ void __launch_bounds__(256) k_bsr(int N, const int *__restrict__ rp,
                                              const int *__restrict__ ci, const S *__restrict__ v,
                                              G gather, E epi)
{
    const int lane = threadIdx.x & (T - 1);
    const int groups = (gridDim.x * blockDim.x) / T;
    const int warp_first = ((blockIdx.x * blockDim.x + threadIdx.x) & ~31) / T;
    const int g_in_warp = (threadIdx.x & 31) / T;
    for (int pw = warp_first; pw < N; pw += groups) {
        const int p = pw + g_in_warp;
        const bool act = p < N;
        S y0 = 0, y1 = 0;
        const int e = act ? rp[p + 1] : 0;
#pragma unroll 4
        for (int t = act ? rp[p] + lane : 0; t < e; t += T) {
            const int q = ci[t];
            const BlkS<S> a = load_blk(v, (size_t)t);
            const v2<S> x = gather(q);
            y0 = fma(a.a00, x.x, fma(a.a01, x.y, y0));
            y1 = fma(a.a10, x.x, fma(a.a11, x.y, y1));
        }
        group_sum2<T>(y0, y1);
        if (act && lane == 0) epi(p, y0, y1);
    }
}

// The same rows in equal contiguous shares, one thread block per SM (rows
// [N b / G, N (b + 1) / G) for block b of G): for operators whose row groups
// fit one wave, so that no SM runs a block more than the others.
template <int T, class S, class G, class E>
static __global__ void __launch_bounds__(1024, 1) k_bsr_eq(int N, const int *__restrict__ rp,
                                                  const int *__restrict__ ci, const S *__restrict__ v,
                                                  G gather, E epi)
{
    const int r0 = (int)((long long)N * blockIdx.x / gridDim.x);
    const int r1 = (int)((long long)N * (blockIdx.x + 1) / gridDim.x);
    const int lane = threadIdx.x & (T - 1);
    const int groups = blockDim.x / T;
    const int warp_first = (threadIdx.x & ~31) / T;
    const int g_in_warp = (threadIdx.x & 31) / T;
    for (int pw = r0 + warp_first; pw < r1; pw += groups) {
        const int p = pw + g_in_warp;
        const bool act = p < r1;
        S y0 = 0, y1 = 0;
        const int e = act ? rp[p + 1] : 0;
#pragma unroll 4
        for (int t = act ? rp[p] + lane : 0; t < e; t += T) {
            const int q = ci[t];
            const BlkS<S> a = load_blk(v, (size_t)t);
            const v2<S> x = gather(q);
            y0 = fma(a.a00, x.x, fma(a.a01, x.y, y0));
            y1 = fma(a.a10, x.x, fma(a.a11, x.y, y1));
        }
        group_sum2<T>(y0, y1);
        if (act && lane == 0) epi(p, y0, y1);
    }
}

// Long rows on small levels (few hundred to a few thousand block rows of
// hundreds of blocks): a whole thread block of TB threads per row, so that each
// thread walks only a few blocks; warp shuffles then shared memory reduce.
// The launch bound asks for 1024 resident threads per SM, not 2048, so that
// the FP64 instantiations get 64 registers (at 32 they spill).
template <int TB, class S, class G, class E>
static __global__ void __launch_bounds__(TB, 1024 / TB) k_bsr_wide(int N, const int *__restrict__ rp,
                                                  const int *__restrict__ ci,
                                                  const S *__restrict__ v, G gather, E epi)
{
    __shared__ S red[2][TB / 32];
    for (int p = blockIdx.x; p < N; p += gridDim.x) {
        S y0 = 0, y1 = 0;
        const int e = rp[p + 1];
#pragma unroll 4
        for (int t = rp[p] + threadIdx.x; t < e; t += TB) {
            const int q = ci[t];
            const BlkS<S> a = load_blk(v, (size_t)t);
            const v2<S> x = gather(q);
            y0 = fma(a.a00, x.x, fma(a.a01, x.y, y0));
            y1 = fma(a.a10, x.x, fma(a.a11, x.y, y1));
        }
        group_sum2<32>(y0, y1);
        const int w = threadIdx.x >> 5;
        if ((threadIdx.x & 31) == 0) {
            red[0][w] = y0;
            red[1][w] = y1;
        }
        __syncthreads();
        if (threadIdx.x == 0) {
            S a0 = 0, a1 = 0;
#pragma unroll
            for (int i = 0; i < TB / 32; i++) {
                a0 += red[0][i];
                a1 += red[1][i];
            }
            epi(p, a0, a1);
        }
        __syncthreads();
    }
}

// Rows [0, N) of a block-CSR operator given by its arrays (a prefix of the
// rows of a larger operator is a valid argument).
template <class S, class G, class E>
static int launch_bsr_rows(int N, const int *rp, const int *ci, const S *vals, int T, G g, E e, cudaStream_t s)
{
    if (N <= 0) return BD_OK;
    const int threads = 256;
    long long groups_per_block = T >= 64 ? 1 : threads / T;
    int grid = (int)std::min<long long>((N + groups_per_block - 1) / groups_per_block, (long long)kSM * 16);
    if (T >= 64) {
        int gw = (int)std::min<long long>(N, (long long)kSM * 32);
        switch (T) {
        case 64: k_bsr_wide<64, S><<<gw, 64, 0, s>>>(N, rp, ci, vals, g, e); ::bd::note_launch(); break;
        case 128: k_bsr_wide<128, S><<<gw, 128, 0, s>>>(N, rp, ci, vals, g, e); ::bd::note_launch(); break;
        default: k_bsr_wide<256, S><<<gw, 256, 0, s>>>(N, rp, ci, vals, g, e); ::bd::note_launch(); break;
        }
        BD_LAUNCH_CHECK();
        return BD_OK;
    }
    if ((long long)N * T <= (long long)kSM * 1024) {
        // one block per SM, equal shares of the rows
        const long long per = ((long long)N + kSM - 1) / kSM * T;
        const int tb = (int)std::min<long long>(1024, std::max<long long>(32, (per + 31) / 32 * 32));
        const int gb = (int)std::min<long long>(kSM, N);
        switch (T) {
        case 1: k_bsr_eq<1, S><<<gb, tb, 0, s>>>(N, rp, ci, vals, g, e); break;
        case 2: k_bsr_eq<2, S><<<gb, tb, 0, s>>>(N, rp, ci, vals, g, e); break;
        case 4: k_bsr_eq<4, S><<<gb, tb, 0, s>>>(N, rp, ci, vals, g, e); break;
        case 8: k_bsr_eq<8, S><<<gb, tb, 0, s>>>(N, rp, ci, vals, g, e); break;
        case 16: k_bsr_eq<16, S><<<gb, tb, 0, s>>>(N, rp, ci, vals, g, e); break;
        default: k_bsr_eq<32, S><<<gb, tb, 0, s>>>(N, rp, ci, vals, g, e); break;
        }
        ::bd::note_launch();
        BD_LAUNCH_CHECK();
        return BD_OK;
    }
    switch (T) {
    case 1: k_bsr<1, S><<<grid, threads, 0, s>>>(N, rp, ci, vals, g, e); ::bd::note_launch(); break;
    case 2: k_bsr<2, S><<<grid, threads, 0, s>>>(N, rp, ci, vals, g, e); ::bd::note_launch(); break;
    case 4: k_bsr<4, S><<<grid, threads, 0, s>>>(N, rp, ci, vals, g, e); ::bd::note_launch(); break;
    case 8: k_bsr<8, S><<<grid, threads, 0, s>>>(N, rp, ci, vals, g, e); ::bd::note_launch(); break;
    case 16: k_bsr<16, S><<<grid, threads, 0, s>>>(N, rp, ci, vals, g, e); ::bd::note_launch(); break;
    default: k_bsr<32, S><<<grid, threads, 0, s>>>(N, rp, ci, vals, g, e); ::bd::note_launch(); break;
    }
    BD_LAUNCH_CHECK();
    return BD_OK;
}

template <class S, class G, class E>
static int launch_bsr(const BSR &A, const S *vals, int T, G g, E e, cudaStream_t s)
{
    return launch_bsr_rows<S>(A.nbr, A.rp.p, A.ci.p, vals, T, g, e, s);
}

// Lanes per block row, from per-operator timings inside the V-cycle on the
// 128x128x32 slab's levels.  Every lane-level reduction step costs adds,
// which are scarce in FP64 on this part, so FP64 rows use as few lanes as
// their length allows; FP32 adds are cheap, so FP32 rows use more lanes to
// shorten each thread's chain of dependent loads.  Small levels get more lanes
// so the grid still fills the GPU.  Levels with few, long rows (the dense-ish
// coarse levels): a warp per row in FP64 (a thread block's extra reduction
// steps cost more FP64 adds than its extra lanes save), a thread block per
// row in FP32.
static int lanes_for(const BSR &A, bool fp32)
{
    const double avg = A.nbr > 0 ? (double)A.nb / A.nbr : 1.0;
    int T;
    if (fp32) T = avg <= 3 ? 1 : (avg <= 12 ? 2 : (avg <= 48 ? 4 : (avg <= 100 ? 8 : (avg <= 160 ? 16 : 32))));
    else T = avg <= 40 ? 1 : (avg <= 160 ? 4 : (avg <= 640 ? 8 : 16));
    while (T < 32 && (long long)A.nbr * T < 65536) T <<= 1;
    if ((long long)A.nbr * 32 < 131072 && avg > 96) {  // few long rows
        if (!fp32) return A.nbr >= 2048 ? 32 : (avg <= 600 ? 64 : 128);
        T = 64;
        while (T < 256 && T * 3 < avg) T <<= 1;
    }
    return T;
}

}  // namespace bd
