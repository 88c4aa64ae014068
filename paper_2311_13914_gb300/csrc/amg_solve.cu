// amg_solve.cu -- a10/a11: V-cycle (Algorithm 2) with Chebyshev-Jacobi
// smoothing (Appendix A) and the projected PCG of Section 2.2 on the device.
//
// Every operator application is one pass of an SpMV kernel whose epilogue
// fuses the vector work of the step around it (Chebyshev recurrence, residual,
// correction), so each level streams its matrix four times per cycle and its
// vectors a few times.  The V-cycle is written once over the storage scalar S:
// S = double is the plain FP64 form; S = float keeps FP32 copies of every
// level's values and vectors (half the bytes, none of the FP64 pipe) and runs
// inside an FP64 flexible CG, with the coarsest solve, the outer residual, the
// dot products and the null-space projection in FP64.  Reductions are
// deterministic: fixed grid, per-block partial sums, one finishing block.
#include <algorithm>
#include <cmath>
#include <cstdlib>
#include <new>
#include <type_traits>

#include "amg_internal.cuh"
#include "amg_bsr.cuh"

namespace bd {

// ------------------------------------------------------------------ sliced block operator
// FP64 values sit in two planes, (a00, a01) then (a10, a11), so each half of a
// group is one contiguous 512-byte warp load; FP32 values are one float4.
__device__ __forceinline__ BlkS<double> load_sliced(const double *__restrict__ v, size_t idx, size_t plane)
{
    const double2 p = ((const double2 *)v)[idx], q = ((const double2 *)v)[plane + idx];
    return {p.x, p.y, q.x, q.y};
}
__device__ __forceinline__ BlkS<float> load_sliced(const float *__restrict__ v, size_t idx, size_t)
{
    const float4 p = ((const float4 *)v)[idx];
    return {p.x, p.y, p.z, p.w};
}

// One warp per slice of 32/K rows with K lanes each; warp w takes slices
// [wsl[w], wsl[w+1]), which split the groups evenly over the warps.  Lane k of
// a row sums entries k, k+K, ... and the K partial sums meet in the lane-sum
// tree k_bsr<K> uses (group_sum2), so both forms give the same bits.  Rows sorted by
// length leave few padded positions, and every FP64 instruction of the loop
// and the epilogue works on 32 lanes (the FP64 pipe, not HBM, bounds the
// coarse levels in FP64).
template <int K, class S, class G, class E, int MINB, int TPB = 256>
__global__ void __launch_bounds__(TPB, MINB) k_bsell(const int *__restrict__ sptr, const int *__restrict__ wsl,
                                                    const int *__restrict__ order, const int *__restrict__ col,
                                                    const S *__restrict__ v, size_t plane, G gather, E epi)
{
    const int w = blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5);
    const int lane = threadIdx.x & 31;
    const int s1 = wsl[w + 1];
    for (int sl = wsl[w]; sl < s1; sl++) {
        const int j1 = sptr[sl + 1];
        S y0 = 0, y1 = 0;
#pragma unroll 4
        for (int j = sptr[sl]; j < j1; j++) {
            const size_t idx = (size_t)j * 32 + lane;
            const int q = col[idx];
            const BlkS<S> a = load_sliced(v, idx, plane);
            const v2<S> x = gather(q);
            y0 = fma(a.a00, x.x, fma(a.a01, x.y, y0));
            y1 = fma(a.a10, x.x, fma(a.a11, x.y, y1));
        }
        group_sum2<K>(y0, y1);
        if ((lane & (K - 1)) == 0) {
            const int r = order[sl * (32 / K) + lane / K];
            if (r >= 0) epi(r, y0, y1);
        }
    }
}

// Sorted position of every row of a window: by block count, descending, ties
// by row (a stable, deterministic order).  One thread block per window.
__global__ void k_slice_order(int rows, const int *__restrict__ rp, int *__restrict__ order)
{
    __shared__ int len[kSliceWindow];
    const int w0 = blockIdx.x * kSliceWindow;
    const int n = min(kSliceWindow, rows - w0);
    for (int i = threadIdx.x; i < n; i += blockDim.x) len[i] = rp[w0 + i + 1] - rp[w0 + i];
    __syncthreads();
    for (int i = threadIdx.x; i < n; i += blockDim.x) {
        const int li = len[i];
        int rank = 0;
        for (int j = 0; j < n; j++) {
            const int lj = len[j];
            rank += (lj > li) || (lj == li && j < i);
        }
        order[w0 + rank] = w0 + i;
    }
}

// groups of slice sl: its longest row's block count over K, rounded up
__global__ void k_slice_groups(int nsl, int K, const int *__restrict__ rp, const int *__restrict__ order,
                               int *__restrict__ cnt)
{
    const int sl = blockIdx.x * blockDim.x + threadIdx.x;
    if (sl >= nsl) return;
    const int H = 32 / K;
    int mx = 0;
    for (int i = 0; i < H; i++) {
        const int r = order[sl * H + i];
        if (r >= 0) mx = max(mx, rp[r + 1] - rp[r]);
    }
    cnt[sl] = (mx + K - 1) / K;
}

__device__ __forceinline__ void store_sliced(double *v, size_t idx, size_t plane, const double *a, bool in)
{
    ((double2 *)v)[idx] = in ? make_double2(a[0], a[1]) : make_double2(0.0, 0.0);
    ((double2 *)v)[plane + idx] = in ? make_double2(a[2], a[3]) : make_double2(0.0, 0.0);
}
__device__ __forceinline__ void store_sliced(float *v, size_t idx, size_t, const double *a, bool in)
{
    ((float4 *)v)[idx] = in ? make_float4((float)a[0], (float)a[1], (float)a[2], (float)a[3])
                            : make_float4(0.0f, 0.0f, 0.0f, 0.0f);
}

// one thread per (slice, lane): the entries of its row it owns, group by group
template <class S>
__global__ void k_slice_fill(int nsl, int K, const int *__restrict__ rp, const int *__restrict__ ci,
                             const double *__restrict__ bv, const int *__restrict__ order,
                             const int *__restrict__ sptr, int *__restrict__ col, S *__restrict__ v, size_t plane)
{
    const long long t = blockIdx.x * (long long)blockDim.x + threadIdx.x;
    if (t >= (long long)nsl * 32) return;
    const int sl = (int)(t >> 5), lane = (int)(t & 31);
    const int r = order[sl * (32 / K) + lane / K], k = lane % K;
    const int b = r >= 0 ? rp[r] : 0, len = r >= 0 ? rp[r + 1] - b : 0;
    const int g0 = sptr[sl], g1 = sptr[sl + 1];
    for (int g = g0; g < g1; g++) {
        const int j = (g - g0) * K + k;
        const size_t idx = (size_t)g * 32 + lane;
        const bool in = j < len;
        col[idx] = in ? ci[b + j] : 0;
        store_sliced(v, idx, plane, bv + 4 * (size_t)(in ? b + j : 0), in);
    }
}

// first slice of every warp: the lower bound of w * groups / warps in sptr
__global__ void k_slice_warps(int nsl, long long groups, int warps, const int *__restrict__ sptr,
                              int *__restrict__ wsl)
{
    const int w = blockIdx.x * blockDim.x + threadIdx.x;
    if (w > warps) return;
    if (w == warps) {
        wsl[w] = nsl;
        return;
    }
    const long long g = groups * w / warps;
    int lo = 0, hi = nsl;
    while (lo < hi) {
        const int m = (lo + hi) >> 1;
        if (sptr[m] < g) lo = m + 1;
        else hi = m;
    }
    wsl[w] = lo;
}

// Threads per block of the FP64 finest-level kernels: one block of 32 warps
// per SM (measured against four blocks of 8 warps: 2-4 us shorter launches,
// with the same warps resident and a quarter of the blocks to start and end),
// where every SM then gets at least a slice per warp.  Smaller levels keep
// blocks of 8 warps, so that small solves running side by side (graph branches,
// served requests) share the SMs instead of each block holding one.  The FP32
// kernels keep 8 blocks of 8 warps per SM (two blocks of 32 measured the same).
constexpr int kFineTPB = 1024;
static bool fine_wide(long long N) { return (N + 31) / 32 >= (long long)kSM * (kFineTPB / 32); }

// ------------------------------------------------------------------ finest level, sliced ELL
// Block b's share [share_lo(n), share_hi(n)) of n rows or nodes: the grid
// splits the 32-row slices in equal contiguous parts, so with one resident
// wave of blocks every SM gets the same work (a grid-stride loop leaves the
// SMs whose blocks drew one row fewer per thread idle for part of the launch).
__device__ __forceinline__ int share_lo(int n)
{
    return (int)((((long long)n + 31) >> 5) * blockIdx.x / gridDim.x) * 32;
}
__device__ __forceinline__ int share_hi(int n)
{
    return min(n, (int)((((long long)n + 31) >> 5) * (blockIdx.x + 1) / gridDim.x) * 32);
}

// Neighbour offsets of the 27-point stencil of a structured slab, passed by
// value and staged in shared memory (a warp's lanes index it divergently).
struct Stencil {
    int off[27];
};
__device__ __forceinline__ void stage_stencil(const Stencil &st, int *off)
{
    if (threadIdx.x == 0) {
#pragma unroll
        for (int i = 0; i < 27; i++) off[i] = st.off[i];  // constant indices: no local copy
    }
    __syncthreads();
}

// One thread per row; slot j of slice s holds entry j of its 32 rows
// contiguously, so every slot is one coalesced (Ki, Ke) load and one column
// load per warp.  FP32 (HBM-bound) reads 1-byte stencil codes (the
// neighbour's position in the 27-point stencil) instead of 4-byte columns:
// 9 instead of 12 bytes per node pair; FP64 (bound by its FP64 pipe as much
// as by HBM) keeps the columns, which spare it the shared-memory lookup.  Per node pair: s = v_q + u_q, a += Ki s, b += Ke u_q;
// then y_v = c M_p v_p + a, y_u = a + b.  SU: the gathered vector is stored as
// (v + u, u), which saves the add per node pair (two FP64 operations instead
// of three where the FP64 pipe is the limit).
template <class S, class G, bool SU, int UNROLL>
__device__ __forceinline__ void sell_row(int p, int lane, const int *__restrict__ sptr,
                                         const int *__restrict__ col, const unsigned char *__restrict__ code,
                                         const int *off, const v2<S> *__restrict__ kk,
                                         const S *__restrict__ cm, const G &gather, S &y0, S &y1)
{
    constexpr bool CODED = sizeof(S) == 4;
    const int sl = p >> 5;
    const int j1 = sptr[sl + 1];
    S a = 0, b = 0;
#pragma unroll (UNROLL)
    for (int j = sptr[sl]; j < j1; j++) {
        const size_t idx = (size_t)j * 32 + lane;
        const int q = CODED ? p + off[code[idx]] : col[idx];
        const v2<S> k = kk[idx];
        const v2<S> x = gather(q);
        a = fma(k.x, SU ? x.x : x.x + x.y, a);
        b = fma(k.y, x.y, b);
    }
    const v2<S> xp = gather(p);
    y0 = fma(cm[p], SU ? xp.x - xp.y : xp.x, a);
    y1 = a + b;
}

template <class S, class G, class E, bool SU = false, int MINB = 8, int TPB = 256>
__global__ void __launch_bounds__(TPB, MINB) k_sell(int N, const int *__restrict__ sptr,
                                               const int *__restrict__ col,
                                               const unsigned char *__restrict__ code, Stencil st,
                                               const v2<S> *__restrict__ kk,
                                               const S *__restrict__ cm, G gather, E epi)
{
    __shared__ int off[27];
    if (sizeof(S) == 4) stage_stencil(st, off);
    const int lane = threadIdx.x & 31, e = share_hi(N);
    for (int p = share_lo(N) + threadIdx.x; p < e; p += blockDim.x) {
        S y0, y1;
        sell_row<S, G, SU, (MINB >= 8 ? 4 : 8)>(p, lane, sptr, col, code, off, kk, cm, gather, y0, y1);
        epi(p, y0, y1);
    }
}

// ------------------------------------------------------------------ fused epilogues
template <class S> struct GatherVec {
    const v2<S> *__restrict__ x;
    __device__ __forceinline__ v2<S> operator()(int q) const { return x[q]; }
};

// Vectors a finest-level sliced-ELL operator gathers may be kept in the
// (v + u, u) form (SU); these convert at the epilogue, once per node.
template <class S, bool SU> __device__ __forceinline__ v2<S> from_su(v2<S> a)
{
    return SU ? V2<S>::mk(a.x - a.y, a.y) : a;
}
template <class S, bool SU> __device__ __forceinline__ v2<S> to_su(S v, S u)
{
    return V2<S>::mk(SU ? v + u : v, u);
}

// pre-smoothing, degree 2 from zero, d0 = D^{-1} f / theta precomputed:
// x1 = d0, r1 = f - A d0, d1 = c1 d0 + c2 D^{-1} r1, u = x1 + d1
template <class S, bool SU = false> struct EpiPre {
    const v2<S> *__restrict__ f;
    const v2<S> *__restrict__ invd;
    const v2<S> *__restrict__ d0;
    v2<S> *__restrict__ u;
    S c1, c2;
    __device__ __forceinline__ void operator()(int p, S y0, S y1) const {
        const v2<S> fp = f[p], id = invd[p], dp = from_su<S, SU>(d0[p]);
        const S r0 = fp.x - y0, r1 = fp.y - y1;
        u[p] = to_su<S, SU>(dp.x + (c1 * dp.x + c2 * id.x * r0), dp.y + (c1 * dp.y + c2 * id.y * r1));
    }
};

// restriction output f_c = R r together with d0_c = D_c^{-1} f_c / theta_c
template <class S> struct EpiStoreD0 {
    v2<S> *__restrict__ f;
    v2<S> *__restrict__ d0;
    const v2<S> *__restrict__ invd;
    S it;
    __device__ __forceinline__ void operator()(int p, S y0, S y1) const {
        f[p] = V2<S>::mk(y0, y1);
        const v2<S> id = invd[p];
        d0[p] = V2<S>::mk(y0 * id.x * it, y1 * id.y * it);
    }
};

template <class S> struct EpiResid {  // r = f - A u
    const v2<S> *__restrict__ f;
    v2<S> *__restrict__ r;
    __device__ __forceinline__ void operator()(int p, S y0, S y1) const {
        const v2<S> fp = f[p];
        r[p] = V2<S>::mk(fp.x - y0, fp.y - y1);
    }
};

template <class S, bool SU = false> struct EpiAdd {  // u += P e_c
    v2<S> *__restrict__ u;
    __device__ __forceinline__ void operator()(int p, S y0, S y1) const {
        const v2<S> a = u[p];
        u[p] = V2<S>::mk(a.x + (SU ? y0 + y1 : y0), a.y + y1);
    }
};

// post-smoothing, first half: r0 = f - A u, d0 = D^{-1} r0 / theta, w = u + d0
template <class S, bool SU = false> struct EpiPost1 {
    const v2<S> *__restrict__ f;
    const v2<S> *__restrict__ invd;
    const v2<S> *__restrict__ u;
    v2<S> *__restrict__ r;
    v2<S> *__restrict__ d;
    v2<S> *__restrict__ w;
    S it;
    __device__ __forceinline__ void operator()(int p, S y0, S y1) const {
        const v2<S> fp = f[p], id = invd[p], up = from_su<S, SU>(u[p]);
        const S r0 = fp.x - y0, r1 = fp.y - y1;
        const S d0 = r0 * id.x * it, d1 = r1 * id.y * it;
        r[p] = V2<S>::mk(r0, r1);
        d[p] = to_su<S, SU>(d0, d1);
        w[p] = V2<S>::mk(up.x + d0, up.y + d1);
    }
};

// post-smoothing, second half: r1 = r0 - A d0, d1 = c1 d0 + c2 D^{-1} r1, u = w + d1
template <class S, bool SU = false> struct EpiPost2 {
    const v2<S> *__restrict__ r;
    const v2<S> *__restrict__ d;
    const v2<S> *__restrict__ invd;
    const v2<S> *__restrict__ w;
    v2<S> *__restrict__ u;
    S c1, c2;
    __device__ __forceinline__ v2<S> value(int p, S y0, S y1) const {
        const v2<S> rp_ = r[p], dp = from_su<S, SU>(d[p]), id = invd[p], wp = w[p];
        const S r0 = rp_.x - y0, r1 = rp_.y - y1;
        return V2<S>::mk(wp.x + (c1 * dp.x + c2 * id.x * r0), wp.y + (c1 * dp.y + c2 * id.y * r1));
    }
    __device__ __forceinline__ void operator()(int p, S y0, S y1) const { u[p] = value(p, y0, y1); }
};

// The Chebyshev steps of the FP64 finest level written in the (v + u, u) form
// of the vectors they gather, with the inverse diagonal scaled per level
// (idc2 = c2 D^{-1}, idt = D^{-1}/theta): fewer FP64 operations per node on a
// level bound by the FP64 pipe.  For u = d0 + (c1 d0 + c2 D^{-1} r) with
// m = idc2 r: u_s = (1 + c1) d0_s + (m_v + m_u), u_u = (1 + c1) d0_u + m_u.
struct EpiPreX {
    const double2 *__restrict__ f;
    const double2 *__restrict__ idc2;
    const double2 *__restrict__ d0;  // (v + u, u)
    double2 *__restrict__ u;         // (v + u, u)
    double c1p;                      // 1 + c1
    __device__ __forceinline__ void operator()(int p, double y0, double y1) const
    {
        const double2 fp = f[p], k = idc2[p], dp = d0[p];
        const double m0 = k.x * (fp.x - y0), m1 = k.y * (fp.y - y1);
        u[p] = make_double2(fma(c1p, dp.x, m0 + m1), fma(c1p, dp.y, m1));
    }
};
// r = f - A u, d = D^{-1} r / theta, w = u + d: r plain, d and w in (v + u, u)
struct EpiPost1X {
    const double2 *__restrict__ f;
    const double2 *__restrict__ idt;
    const double2 *__restrict__ u;  // (v + u, u)
    double2 *__restrict__ r;
    double2 *__restrict__ d;
    double2 *__restrict__ w;
    __device__ __forceinline__ void operator()(int p, double y0, double y1) const
    {
        const double2 fp = f[p], k = idt[p], up = u[p];
        const double r0 = fp.x - y0, r1 = fp.y - y1;
        const double d1 = r1 * k.y, ds = r0 * k.x + d1;
        r[p] = make_double2(r0, r1);
        d[p] = make_double2(ds, d1);
        w[p] = make_double2(up.x + ds, up.y + d1);
    }
};
// u = w + (c1 d + c2 D^{-1} (r - A d)) in plain (v, u) form from w and d in
// (v + u, u) form
struct EpiPost2X {
    const double2 *__restrict__ r;
    const double2 *__restrict__ d;     // (v + u, u)
    const double2 *__restrict__ idc2;
    const double2 *__restrict__ w;     // (v + u, u)
    double2 *__restrict__ u;
    double c1;
    __device__ __forceinline__ double2 value(int p, double y0, double y1) const
    {
        const double2 rp_ = r[p], dp = d[p], k = idc2[p], wp = w[p];
        const double m0 = k.x * (rp_.x - y0), m1 = k.y * (rp_.y - y1);
        const double uu = wp.y + fma(c1, dp.y, m1);
        const double us = wp.x + fma(c1, dp.x, m0 + m1);
        return make_double2(us - uu, uu);
    }
    __device__ __forceinline__ void operator()(int p, double y0, double y1) const { u[p] = value(p, y0, y1); }
};

// ------------------------------------------------------------------ per-level views
// Value and vector pointers of one level in precision S (index arrays are shared).
template <class S> struct LV {
    const S *Av, *Pv, *Rv;
    const v2<S> *invd;
    v2<S> *f, *u, *r, *d, *w;
    const v2<S> *kk;  // finest level, sliced ELL
    const S *cm;
};

template <class S> static LV<S> view(amg_hierarchy *h, int l);

// The smoothing epilogues of a level: the (v + u, u)-form ones with scaled
// inverse diagonals on the FP64 sliced-ELL finest level (SU), the plain ones
// elsewhere.
template <class S, bool SU>
static auto epi_pre(const Level &L, const LV<S> &lv, const v2<S> *f, v2<S> *d0, v2<S> *u)
{
    if constexpr (SU && std::is_same<S, double>::value)
        return EpiPreX{f, (const double2 *)L.idc2.p, d0, u, 1.0 + L.ch_c1};
    else
        return EpiPre<S, SU>{f, lv.invd, d0, u, (S)L.ch_c1, (S)L.ch_c2};
}
template <class S, bool SU>
static auto epi_post1(const Level &L, const LV<S> &lv, const v2<S> *f, v2<S> *u)
{
    if constexpr (SU && std::is_same<S, double>::value)
        return EpiPost1X{f, (const double2 *)L.idt.p, u, lv.r, lv.d, lv.w};
    else
        return EpiPost1<S, SU>{f, lv.invd, u, lv.r, lv.d, lv.w, (S)L.ch_inv_theta};
}
template <class S, bool SU>
static auto epi_post2(const Level &L, const LV<S> &lv, v2<S> *u)
{
    if constexpr (SU && std::is_same<S, double>::value)
        return EpiPost2X{lv.r, lv.d, (const double2 *)L.idc2.p, lv.w, u, L.ch_c1};
    else
        return EpiPost2<S, SU>{lv.r, lv.d, lv.invd, lv.w, u, (S)L.ch_c1, (S)L.ch_c2};
}
template <> LV<double> view<double>(amg_hierarchy *h, int l)
{
    Level &L = h->lev[l];
    LV<double> v;
    v.Av = L.A.v.p;
    v.Pv = L.P.v.p;
    v.Rv = L.R.v.p;
    v.invd = (const double2 *)L.invdiag.p;
    v.f = (double2 *)L.f.p;
    v.u = (double2 *)L.u.p;
    v.r = (double2 *)L.r.p;
    v.d = (double2 *)L.d.p;
    v.w = (double2 *)L.w.p;
    v.kk = (const double2 *)h->sell.kk.p;
    v.cm = h->sell.cm.p;
    return v;
}
template <> LV<float> view<float>(amg_hierarchy *h, int l)
{
    Level &L = h->lev[l];
    LV<float> v;
    v.Av = L.A32.p;
    v.Pv = L.P32.p;
    v.Rv = L.R32.p;
    v.invd = (const float2 *)L.invdiag32.p;
    v.f = (float2 *)L.f32.p;
    v.u = (float2 *)L.u32.p;
    v.r = (float2 *)L.r32.p;
    v.d = (float2 *)L.d32.p;
    v.w = (float2 *)L.w32.p;
    v.kk = (const float2 *)h->sell.kk32.p;
    v.cm = h->sell.cm32.p;
    return v;
}

template <class S> static const S *sliced_vals(const SlicedOp &o);
template <> const double *sliced_vals<double>(const SlicedOp &o) { return o.v.p; }
template <> const float *sliced_vals<float>(const SlicedOp &o) { return o.v32.p; }

template <class S, class G, class E>
static int launch_sliced(const SlicedOp &o, int K, G g, E e, cudaStream_t s)
{
    if (o.K != K || !sliced_vals<S>(o)) return BD_ESTATE;
    constexpr int MB = sizeof(S) == 8 ? 4 : 8;  // as the finest level's sliced ELL
    const S *v = sliced_vals<S>(o);
    const size_t plane = (size_t)o.groups * 32;
    // FP64 operators whose warps fill one wave: one 1024-thread block per SM,
    // the same warps and slices as 256-thread blocks (the finest R and P:
    // 1.3-1.8 us shorter launches, measured)
    if (sizeof(S) == 8 && o.warps == kSM * 32) {
        switch (K) {
        case 1: k_bsell<1, S, G, E, 1, 1024><<<kSM, 1024, 0, s>>>(o.sptr.p, o.wsl.p, o.order.p, o.col.p, v, plane, g, e); break;
        case 2: k_bsell<2, S, G, E, 1, 1024><<<kSM, 1024, 0, s>>>(o.sptr.p, o.wsl.p, o.order.p, o.col.p, v, plane, g, e); break;
        case 4: k_bsell<4, S, G, E, 1, 1024><<<kSM, 1024, 0, s>>>(o.sptr.p, o.wsl.p, o.order.p, o.col.p, v, plane, g, e); break;
        default: k_bsell<8, S, G, E, 1, 1024><<<kSM, 1024, 0, s>>>(o.sptr.p, o.wsl.p, o.order.p, o.col.p, v, plane, g, e); break;
        }
        ::bd::note_launch();
        BD_LAUNCH_CHECK();
        return BD_OK;
    }
    const int grid = o.warps / 8;
    switch (K) {
    case 1: k_bsell<1, S, G, E, MB><<<grid, 256, 0, s>>>(o.sptr.p, o.wsl.p, o.order.p, o.col.p, v, plane, g, e); break;
    case 2: k_bsell<2, S, G, E, MB><<<grid, 256, 0, s>>>(o.sptr.p, o.wsl.p, o.order.p, o.col.p, v, plane, g, e); break;
    case 4: k_bsell<4, S, G, E, MB><<<grid, 256, 0, s>>>(o.sptr.p, o.wsl.p, o.order.p, o.col.p, v, plane, g, e); break;
    default: k_bsell<8, S, G, E, MB><<<grid, 256, 0, s>>>(o.sptr.p, o.wsl.p, o.order.p, o.col.p, v, plane, g, e); break;
    }
    ::bd::note_launch();
    BD_LAUNCH_CHECK();
    return BD_OK;
}

static bool sliced_k_ok(int K) { return K == 1 || K == 2 || K == 4 || K == 8; }

// Build M's sliced form with K lanes per row in the V-cycle's precision (the
// sorted row order is kept across rebuilds of the same operator, and buffers
// large enough already are reused).  Stream-ordered on s.
template <class T> static int ensure(DBuf<T> &b, size_t n)
{
    return b.p && b.n >= n ? BD_OK : b.alloc(n);
}

static int build_sliced(const BSR &M, int K, bool fp32, SlicedOp &o, cudaStream_t s)
{
    if (M.nbr <= 0 || M.nb <= 0 || !sliced_k_ok(K)) return BD_EINVAL;
    const int rows = M.nbr, H = 32 / K;
    o.K = 0;
    if (o.rows != rows || !o.order.p) {
        const size_t padded = ((size_t)rows + 31) / 32 * 32;
        BD_TRY(o.order.alloc(padded));
        BD_CUDA(cudaMemsetAsync(o.order.p, 0xff, sizeof(int) * padded, s));  // -1 past the last row
        k_slice_order<<<(rows + kSliceWindow - 1) / kSliceWindow, 256, 0, s>>>(rows, M.rp.p, o.order.p);
        ::bd::note_launch();
        BD_LAUNCH_CHECK();
        o.rows = rows;
    }
    o.nsl = (rows + H - 1) / H;
    BD_TRY(ensure(o.cnt, (size_t)o.nsl));
    BD_TRY(ensure(o.sptr, (size_t)o.nsl + 1));
    k_slice_groups<<<(o.nsl + 255) / 256, 256, 0, s>>>(o.nsl, K, M.rp.p, o.order.p, o.cnt.p);
    ::bd::note_launch();
    BD_LAUNCH_CHECK();
    BD_TRY(exclusive_scan(o.cnt.p, o.sptr.p, o.nsl, &o.groups, s));
    const size_t ent = (size_t)o.groups * 32;
    BD_TRY(ensure(o.col, ent));
    const long long fill_threads = (long long)o.nsl * 32;
    const int fill_grid = (int)((fill_threads + 255) / 256);
    if (fp32) {
        o.v.release();
        BD_TRY(ensure(o.v32, 4 * ent));
        k_slice_fill<float><<<fill_grid, 256, 0, s>>>(o.nsl, K, M.rp.p, M.ci.p, M.v.p, o.order.p, o.sptr.p,
                                                     o.col.p, o.v32.p, ent);
    } else {
        o.v32.release();
        BD_TRY(ensure(o.v, 4 * ent));
        k_slice_fill<double><<<fill_grid, 256, 0, s>>>(o.nsl, K, M.rp.p, M.ci.p, M.v.p, o.order.p, o.sptr.p,
                                                      o.col.p, o.v.p, ent);
    }
    ::bd::note_launch();
    BD_LAUNCH_CHECK();
    const int MB = fp32 ? 8 : 4;
    const long long cap = (long long)kSM * MB * 8;  // one resident wave of 256-thread blocks
    o.warps = (int)std::min<long long>(cap, ((long long)o.nsl + 7) / 8 * 8);
    BD_TRY(ensure(o.wsl, (size_t)o.warps + 1));
    k_slice_warps<<<(o.warps + 256) / 256, 256, 0, s>>>(o.nsl, o.groups, o.warps, o.sptr.p, o.wsl.p);
    ::bd::note_launch();
    BD_LAUNCH_CHECK();
    o.K = K;
    return BD_OK;
}

static void drop_sliced(SlicedOp &o)
{
    o.K = 0;
    o.cnt.release();
    o.col.release();
    o.v.release();
    o.v32.release();
    o.sptr.release();
    o.wsl.release();
}

// Operator op (0: A, 1: R, 2: P) of level L in the form its lanes entry names.
template <class S, class G, class E>
static int apply_op(const Level &L, int op, const S *csr_vals, G g, E e, cudaStream_t s)
{
    const int T = L.lanes[op];
    if (T < 0) return launch_sliced<S>(L.sl[op], -T, g, e, s);
    return launch_bsr<S>(op == 0 ? L.A : (op == 1 ? L.R : L.P), csr_vals, T, g, e, s);
}

// The sliced form (FP64 only: in FP32 block-CSR with more lanes was as fast
// or faster on every level) where it beat block-CSR inside the V-cycle: many
// short, ragged rows (the prolongators of levels of 65536 rows and more:
// sorted rows leave few idle lanes, one lane per row needs no reduction), many
// long rows (restrictions, 8 lanes per row) and, on levels of 65536 rows and
// more, rows in between (4 lanes; the autotuner's choices on the 256x256x64
// slab's second level, while block-CSR with 4 lanes won on the 31542 rows of
// the 128x128x32 slab's).  Elsewhere the block-CSR rule.
constexpr int kSlicedMinRows = 8192;
static int lanes_rule(const BSR &A, bool fp32, bool sliced_ok)
{
    const double avg = A.nbr > 0 ? (double)A.nb / A.nbr : 1.0;
    if (sliced_ok && !fp32 && A.nbr >= kSlicedMinRows) {
        if (A.nbr >= 65536 && avg <= 24.0) return -1;
        if (avg >= 96.0) return -8;
        if (A.nbr >= 65536) return -4;  // middle-length rows of a big level
    }
    return lanes_for(A, fp32);
}

__global__ void k_sell_width(int N, const int *__restrict__ rp, int *__restrict__ w, int nslices)
{
    int sl = blockIdx.x * blockDim.x + threadIdx.x;
    if (sl >= nslices) return;
    int mx = 0;
    for (int p = sl * 32; p < sl * 32 + 32 && p < N; p++) mx = max(mx, rp[p + 1] - rp[p]);
    w[sl] = mx;
}

// Node k = i + X (j + Y l) (X = nx+1, Y = ny+1); the neighbour q of p sits
// at stencil position 9 (lq - lp + 1) + 3 (jq - jp + 1) + (iq - ip + 1).
__global__ void k_sell_fill(int N, int X, int Y, const int *__restrict__ rp, const int *__restrict__ ci,
                            const double *__restrict__ Ki, const double *__restrict__ Ke,
                            const double *__restrict__ M, double c, const int *__restrict__ sptr,
                            int *__restrict__ col, unsigned char *__restrict__ code, double2 *__restrict__ kk,
                            double *__restrict__ cm, int *__restrict__ bad)
{
    int p = blockIdx.x * blockDim.x + threadIdx.x;
    if (p >= N) return;
    int sl = p >> 5, lane = p & 31;
    int j0 = sptr[sl], width = sptr[sl + 1] - j0, b = rp[p], len = rp[p + 1] - b;
    const int ip = p % X, jp = (p / X) % Y, lp = p / (X * Y);
    for (int j = 0; j < width; j++) {
        size_t idx = (size_t)(j0 + j) * 32 + lane;
        if (j < len) {
            const int q = ci[b + j];
            const int di = q % X - ip, dj = (q / X) % Y - jp, dl = q / (X * Y) - lp;
            if (di < -1 || di > 1 || dj < -1 || dj > 1 || dl < -1 || dl > 1) {
                atomicOr(bad, 1);
                col[idx] = p;
                code[idx] = 13;
                kk[idx] = make_double2(0.0, 0.0);
                continue;
            }
            col[idx] = q;
            code[idx] = (unsigned char)(9 * (dl + 1) + 3 * (dj + 1) + (di + 1));
            kk[idx] = make_double2(Ki[b + j], Ke[b + j]);
        } else {
            col[idx] = p;
            code[idx] = 13;  // the row itself, with zero weights
            kk[idx] = make_double2(0.0, 0.0);
        }
    }
    cm[p] = c * M[p];
}

int build_fine_sell(amg_hierarchy *h, const bd_system *sys, cudaStream_t s)
{
    FineSell &F = h->sell;
    const int N = sys->N;
    F.nslices = (N + 31) / 32;
    DBuf<int> w;
    BD_TRY(w.alloc((size_t)F.nslices + 1));
    BD_TRY(F.sptr.alloc((size_t)F.nslices + 1));
    k_sell_width<<<(F.nslices + 255) / 256, 256, 0, s>>>(N, sys->A.rp.p, w.p, F.nslices); ::bd::note_launch();
    BD_LAUNCH_CHECK();
    long long slots = 0;
    BD_TRY(exclusive_scan(w.p, F.sptr.p, F.nslices, &slots, s));
    F.slots = slots;
    BD_TRY(F.col.alloc((size_t)slots * 32));
    BD_TRY(F.code.alloc((size_t)slots * 32));
    BD_TRY(F.kk.alloc((size_t)slots * 64));
    BD_TRY(F.cm.alloc((size_t)N));
    DBuf<int> bad;
    BD_TRY(bad.alloc(1));
    BD_CUDA(cudaMemsetAsync(bad.p, 0, sizeof(int), s));
    const int X = sys->mesh.nx + 1, Y = sys->mesh.ny + 1;
    for (int dl = 0; dl < 3; dl++)
        for (int dj = 0; dj < 3; dj++)
            for (int di = 0; di < 3; di++)
                F.off[9 * dl + 3 * dj + di] = (dl - 1) * X * Y + (dj - 1) * X + (di - 1);
    const bd_params &P = sys->params;
    k_sell_fill<<<(N + 255) / 256, 256, 0, s>>>(N, X, Y, sys->A.rp.p, sys->A.ci.p, sys->Ki.p, sys->Ke.p,
                                                sys->M.p, (P.chi * P.cm) / P.dt, F.sptr.p, F.col.p, F.code.p,
                                                (double2 *)F.kk.p, F.cm.p, bad.p); ::bd::note_launch();
    BD_LAUNCH_CHECK();
    int hbad = 0;
    BD_CUDA(cudaMemcpyAsync(&hbad, bad.p, sizeof(int), cudaMemcpyDeviceToHost, s));
    BD_CUDA(cudaStreamSynchronize(s));
    if (hbad) return BD_EINVAL;  // not a 27-point pattern: the assembled system was corrupted
    F.valid = true;
    return BD_OK;
}

static Stencil stencil_of(const FineSell &F)
{
    Stencil st;
    for (int i = 0; i < 27; i++) st.off[i] = F.off[i];
    return st;
}

// operator application of level l in precision S: sliced ELL on the finest
// level when available, 2x2-block CSR otherwise.  SU (sliced ELL only): the
// gathered vector is in (v + u, u) form.
template <bool SU = false, class S, class G, class E>
static int apply_level(amg_hierarchy *h, int l, const LV<S> &lv, G g, E e, cudaStream_t s)
{
    const Level &L = h->lev[l];
    if (l == 0 && h->sell.valid) {
        const FineSell &F = h->sell;
        const long long slices = ((long long)L.N + 31) / 32;
        if (sizeof(S) == 8 && fine_wide(L.N)) {
            k_sell<S, G, E, SU, 1, kFineTPB><<<(int)std::min<long long>(slices, kSM), kFineTPB, 0, s>>>(
                L.N, F.sptr.p, F.col.p, F.code.p, stencil_of(F), lv.kk, lv.cm, g, e);
        } else {
            constexpr int MB = sizeof(S) == 8 ? 4 : 8;  // FP64: fewer, deeper-pipelined threads
            k_sell<S, G, E, SU, MB><<<(int)std::min<long long>(slices, (long long)kSM * MB), 256, 0, s>>>(
                L.N, F.sptr.p, F.col.p, F.code.p, stencil_of(F), lv.kk, lv.cm, g, e);
        }
        ::bd::note_launch();
        BD_LAUNCH_CHECK();
        return BD_OK;
    }
    if constexpr (SU) return BD_EINVAL;
    else return apply_op<S>(L, 0, lv.Av, g, e, s);
}

// ------------------------------------------------------------------ live kernel timing
int prof_begin(amg_hierarchy *h, cudaStream_t s, int label, bool fine)
{
    if (!h->prof || (!fine && h->prof < 2)) return -1;
    if (h->ev_used * 2 + 2 > (int)h->ev.size()) {
        if (h->ev.size() >= 8192) prof_collect(h);  // bounded pool: drain (synchronises)
        while (h->ev_used * 2 + 2 > (int)h->ev.size()) {
            cudaEvent_t e;
            if (cudaEventCreate(&e) != cudaSuccess) return -1;
            h->ev.push_back(e);
            if (h->ev.size() % 2 == 0) {
                h->ev_bytes.push_back(0.0);
                h->ev_flops.push_back(0.0);
                h->ev_ops.push_back(0.0);
                h->ev_label.push_back(-1);
            }
        }
    }
    int slot = h->ev_used++;
    h->ev_bytes[slot] = 0.0;
    h->ev_flops[slot] = 0.0;
    h->ev_ops[slot] = 0.0;
    h->ev_label[slot] = label;
    cudaEventRecord(h->ev[2 * slot], s);
    return slot;
}

// bytes/flops > 0 mark a finest-operator application (amg_kernel_profile sums)
void prof_end(amg_hierarchy *h, int slot, double bytes, double flops, cudaStream_t s, double ops)
{
    if (slot < 0) return;
    cudaEventRecord(h->ev[2 * slot + 1], s);
    h->ev_bytes[slot] = bytes;
    h->ev_flops[slot] = flops;
    h->ev_ops[slot] = ops;
}

void prof_collect(amg_hierarchy *h)
{
    for (int i = 0; i < h->ev_used; i++) {
        cudaEventSynchronize(h->ev[2 * i + 1]);
        float ms = 0.0f;
        if (cudaEventElapsedTime(&ms, h->ev[2 * i], h->ev[2 * i + 1]) != cudaSuccess) continue;
        if (h->ev_bytes[i] > 0.0) {
            h->prof_sum.launches++;
            h->prof_sum.total_ms += ms;
            h->prof_sum.bytes += h->ev_bytes[i];
            h->prof_sum.flops += h->ev_flops[i];
            h->prof_sum.fp64_ops += h->ev_ops[i];
        }
        const int lab = h->ev_label[i];
        if (h->prof >= 2 && lab >= 0 && lab < 256) {
            h->trace_ms[lab] += ms;
            h->trace_n[lab]++;
        }
    }
    h->ev_used = 0;
}

// Algorithmic bytes of one finest-level operator application in precision S:
// the stored matrix once (sliced ELL: Ki, Ke and a 4-byte column (FP64) or a
// 1-byte stencil code (FP32) per slot incl. padding, slice offsets, c M;
// block CSR: four values and a column per block, row offsets) and `vec`
// per-node vector streams of two S each.
template <class S>
static double fine_bytes(const amg_hierarchy *h, const Level &L, int vec)
{
    const double sz = (double)sizeof(S);
    double mat = h->sell.valid ? (2 * sz + (sz == 4 ? 1.0 : 4.0)) * 32.0 * (double)h->sell.slots +
                                     4.0 * (h->sell.nslices + 1) + sz * L.N
                               : (4 * sz + 4.0) * (double)L.A.nb + 4.0 * (L.N + 1);
    return mat + 2 * sz * vec * (double)L.N;
}
// Flops one finest-level launch executes (an FMA counts 2): sliced ELL 2 FMA
// per stored slot with the gathered vector in (v + u, u) form, 2 FMA and an
// add otherwise; block CSR 4 FMA per 2x2 block.  The epilogue's few flops per
// node are not counted.
static double fine_flops(const amg_hierarchy *h, const Level &L, bool su)
{
    if (h->sell.valid) return (su ? 4.0 : 5.0) * 32.0 * (double)h->sell.slots;
    return 8.0 * (double)L.A.nb;
}
// FP64 pipe operations (a fused multiply-add, an add and a multiply count one
// each: what the pipe issues) of one finest-level launch of the FP64 V-cycle
// or of the PCG's A p: per stored slot the 2 FMA of the (v + u, u) form, per
// node the row tail (c M v + a, a + b, and v = (v + u) - u) and the fused
// step as its epilogue issues it: pre-smoother 6, residual 2, first
// post-smoothing half 6, second half 10 (14 with the PCG's z statistics),
// A p with p.Ap 2.  The FP32 V-cycle's launches issue FP64 operations only
// for the z statistics (conversions and sums, 10 per node).  Block-CSR finest
// levels: 4 FMA per 2x2 block, epilogues not counted.
enum FineRole { FR_PRE, FR_RESID, FR_POST1, FR_POST2, FR_POST2Z, FR_AP };
template <class S>
static double fine_ops(const amg_hierarchy *h, const Level &L, int role)
{
    if (!h->sell.valid) return sizeof(S) == 8 || role == FR_AP ? 4.0 * (double)L.A.nb : 0.0;
    if (sizeof(S) == 4 && role != FR_AP) return role == FR_POST2Z ? 10.0 * L.N : 0.0;
    static const double epi[] = {6.0, 2.0, 6.0, 10.0, 14.0, 2.0};
    return 2.0 * 32.0 * (double)h->sell.slots + (3.0 + epi[role]) * (double)L.N;
}

// ------------------------------------------------------------------ coarsest level
// x = Cinv (r - (z.r / z.z) z) in FP64 whatever the storage precision; one
// block, one warp per output row.
template <class S>
__global__ void k_coarse_solve(int n, const double *__restrict__ cinv, const double *__restrict__ z,
                               double zz, const S *__restrict__ r, S *__restrict__ x)
{
    extern __shared__ double rs[];
    __shared__ double red[32];
    double part = 0.0;
    for (int i = threadIdx.x; i < n; i += blockDim.x) part += z[i] * (double)r[i];
    for (int o = 16; o; o >>= 1) part += __shfl_xor_sync(0xffffffffu, part, o);
    if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = part;
    __syncthreads();
    if (threadIdx.x < 32) {
        double v = threadIdx.x < (blockDim.x >> 5) ? red[threadIdx.x] : 0.0;
        for (int o = 16; o; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
        if (threadIdx.x == 0) red[0] = v;
    }
    __syncthreads();
    double a = zz > 0.0 ? red[0] / zz : 0.0;
    for (int i = threadIdx.x; i < n; i += blockDim.x) rs[i] = (double)r[i] - a * z[i];
    __syncthreads();
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nw = blockDim.x >> 5;
    for (int i = warp; i < n; i += nw) {
        const double *row = cinv + (size_t)i * n;
        double sacc = 0.0;
        for (int j = lane; j < n; j += 32) sacc += row[j] * rs[j];
        for (int o = 16; o; o >>= 1) sacc += __shfl_xor_sync(0xffffffffu, sacc, o);
        if (lane == 0) x[i] = (S)sacc;
    }
}

// The same for larger coarsest levels, over the whole GPU: every block forms
// z.r and the projected right-hand side r - (z.r/z.z) z in shared memory
// itself (same order in each block, so all agree), then one warp per row: one
// FP64 FMA per matrix entry.
template <class S>
__global__ void __launch_bounds__(256) k_coarse_solve_wide(int n, const double *__restrict__ cinv,
                                                           const double *__restrict__ z, double zz,
                                                           const S *__restrict__ r, S *__restrict__ x)
{
    extern __shared__ double rs[];
    __shared__ double red[8];
    __shared__ double alpha;
    double part = 0.0;
    for (int i = threadIdx.x; i < n; i += blockDim.x) part += z[i] * (double)r[i];
    for (int o = 16; o; o >>= 1) part += __shfl_xor_sync(0xffffffffu, part, o);
    if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = part;
    __syncthreads();
    if (threadIdx.x == 0) {
        double v = 0.0;
        for (int w = 0; w < (int)(blockDim.x >> 5); w++) v += red[w];
        alpha = zz > 0.0 ? v / zz : 0.0;
    }
    __syncthreads();
    const double a = alpha;
    for (int i = threadIdx.x; i < n; i += blockDim.x) rs[i] = (double)r[i] - a * z[i];
    __syncthreads();
    const int lane = threadIdx.x & 31;
    const int warp = blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5);
    const int nw = gridDim.x * (blockDim.x >> 5);
    for (int i = warp; i < n; i += nw) {
        const double *row = cinv + (size_t)i * n;
        double sacc = 0.0;
        for (int j = lane; j < n; j += 32) sacc = fma(row[j], rs[j], sacc);
        for (int o = 16; o; o >>= 1) sacc += __shfl_xor_sync(0xffffffffu, sacc, o);
        if (lane == 0) x[i] = (S)sacc;
    }
}

template <class S>
__global__ void k_copy2(int N, const v2<S> *__restrict__ a, v2<S> *__restrict__ b)
{
    for (int i = share_lo(N) + threadIdx.x, e = share_hi(N); i < e; i += blockDim.x) b[i] = a[i];
}

template <class S, bool SU = false>
__global__ void k_scale_d0(int N, const v2<S> *__restrict__ f, const v2<S> *__restrict__ invd, S it,
                           v2<S> *__restrict__ d0)
{
    for (int i = share_lo(N) + threadIdx.x, e = share_hi(N); i < e; i += blockDim.x) {
        const v2<S> a = f[i], b = invd[i];
        d0[i] = to_su<S, SU>(a.x * b.x * it, a.y * b.y * it);
    }
}

// FP64 residual in, FP32 right-hand side and d0 of the finest level out
__global__ void k_in32(int N, const double2 *__restrict__ r, const float2 *__restrict__ invd, float it,
                       float2 *__restrict__ f, float2 *__restrict__ d0)
{
    for (int i = share_lo(N) + threadIdx.x, e = share_hi(N); i < e; i += blockDim.x) {
        const double2 a = r[i];
        const float2 b = invd[i];
        const float f0 = (float)a.x, f1 = (float)a.y;
        f[i] = make_float2(f0, f1);
        d0[i] = make_float2(f0 * b.x * it, f1 * b.y * it);
    }
}

__global__ void k_out64(int N, const float2 *__restrict__ u, double2 *__restrict__ z)
{
    for (int i = share_lo(N) + threadIdx.x, e = share_hi(N); i < e; i += blockDim.x) {
        const float2 a = u[i];
        z[i] = make_double2((double)a.x, (double)a.y);
    }
}

__global__ void k_scale_vec(long long n, const double *__restrict__ a, double c, double *__restrict__ b)
{
    for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n;
         i += (long long)gridDim.x * blockDim.x)
        b[i] = c * a[i];
}

__global__ void k_to_f32(long long n, const double *__restrict__ a, float *__restrict__ b)
{
    for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n;
         i += (long long)gridDim.x * blockDim.x)
        b[i] = (float)a[i];
}

// The PCG's z statistics computed by the V-cycle's last finest-level kernel
// (defined with the PCG reductions below).
struct ZOut;
static int zo_streams(const ZOut *zo);
template <class S, bool SU, class E2>
static int launch_sell_z(amg_hierarchy *h, const LV<S> &lv, const E2 &epi, const ZOut &zo, cudaStream_t s);
// FP32 V-cycle output to the PCG's z (FP64) with the z statistics in one pass
static int launch_z_from32(amg_hierarchy *h, const float2 *u, const ZOut &zo, cudaStream_t s);

// One V-cycle in precision S; f0/u0 are the finest level's right-hand side and
// output (d0 of the finest level must already be in lev[0]'s d vector).  SU0:
// the finest level's gathered vectors (d0, the iterate u until the last
// smoothing step, the post-smoother's d) are kept in (v + u, u) form; the
// output u0 is in (v, u) form either way.  zo (PCG only): the last
// post-smoothing step on a sliced-ELL finest level writes the FP64 result to
// zo->z and sums the z statistics (*zdone set); u0 is then not written.
template <class S, bool SU0>
static int vcycle_impl(amg_hierarchy *h, const v2<S> *f0, v2<S> *u0, cudaStream_t s, const ZOut *zo = nullptr,
                       bool *zdone = nullptr)
{
    const int nl = h->nlev;
    const bool deg2 = h->opts.cheb_degree == 2;
    auto down = [&](int l, auto su) -> int {
        constexpr bool SU = decltype(su)::value;
        Level &L = h->lev[l];
        const LV<S> lv = view<S>(h, l);
        const v2<S> *f = l == 0 ? f0 : lv.f;
        v2<S> *u = l == 0 ? u0 : lv.u;
        v2<S> *d0 = lv.d;
        if (deg2) {
            int sl = prof_begin(h, s, 16 * l + R_PRE, l == 0);
            BD_TRY(apply_level<SU>(h, l, lv, GatherVec<S>{d0}, epi_pre<S, SU>(L, lv, f, d0, u), s));
            prof_end(h, sl, l == 0 ? fine_bytes<S>(h, L, 4) : 0.0, fine_flops(h, L, SU), s, fine_ops<S>(h, L, FR_PRE));
        } else {
            int sl = prof_begin(h, s, 16 * l + R_PRE, false);
            k_copy2<S><<<grid_for(L.N, 256), 256, 0, s>>>(L.N, d0, u); ::bd::note_launch();
            BD_LAUNCH_CHECK();
            prof_end(h, sl, 0.0, 0.0, s);
        }
        int sr = prof_begin(h, s, 16 * l + R_RESID, l == 0);
        BD_TRY(apply_level<SU>(h, l, lv, GatherVec<S>{u}, EpiResid<S>{f, lv.r}, s));
        prof_end(h, sr, l == 0 ? fine_bytes<S>(h, L, 3) : 0.0, fine_flops(h, L, SU), s, fine_ops<S>(h, L, FR_RESID));
        const Level &C = h->lev[l + 1];
        const LV<S> cv = view<S>(h, l + 1);
        int sx = prof_begin(h, s, 16 * l + R_RESTRICT, false);
        BD_TRY(apply_op<S>(L, 1, lv.Rv, GatherVec<S>{lv.r},
                             EpiStoreD0<S>{cv.f, cv.d, cv.invd, (S)C.ch_inv_theta}, s));
        prof_end(h, sx, 0.0, 0.0, s);
        return BD_OK;
    };
    auto up = [&](int l, auto su) -> int {
        constexpr bool SU = decltype(su)::value;
        Level &L = h->lev[l];
        const LV<S> lv = view<S>(h, l);
        const v2<S> *f = l == 0 ? f0 : lv.f;
        v2<S> *u = l == 0 ? u0 : lv.u;
        const LV<S> cv = view<S>(h, l + 1);
        int sp = prof_begin(h, s, 16 * l + R_PROLONG, false);
        BD_TRY(apply_op<S>(L, 2, lv.Pv, GatherVec<S>{cv.u},
                             EpiAdd<S, SU>{u}, s));
        prof_end(h, sp, 0.0, 0.0, s);
        int s1 = prof_begin(h, s, 16 * l + R_POST1, l == 0);
        BD_TRY(apply_level<SU>(h, l, lv, GatherVec<S>{u}, epi_post1<S, SU>(L, lv, f, u), s));
        prof_end(h, s1, l == 0 ? fine_bytes<S>(h, L, 6) : 0.0, fine_flops(h, L, SU), s, fine_ops<S>(h, L, FR_POST1));
        if (deg2) {
            int s2 = prof_begin(h, s, 16 * l + R_POST2, l == 0);
            const auto epi = epi_post2<S, SU>(L, lv, u);
            double bytes = l == 0 ? fine_bytes<S>(h, L, 5) : 0.0;
            // FP64: the post-smoother's last kernel carries the PCG's z statistics;
            // FP32: the plain kernel, then one pass that converts u to z and sums
            // the statistics (faster than carrying the FP64 work in the
            // HBM-bound FP32 kernel, measured)
            const bool fuse_z = l == 0 && zo && h->sell.valid && sizeof(S) == 8;
            if (fuse_z) {
                BD_TRY((launch_sell_z<S, SU>(h, lv, epi, *zo, s)));
                if (zdone) *zdone = true;
                // u is not stored; z written and the PCG's r (and z_old) read in FP64
                bytes = fine_bytes<S>(h, L, 4) + 16.0 * L.N * (zo_streams(zo));
            } else {
                BD_TRY(apply_level<SU>(h, l, lv, GatherVec<S>{lv.d}, epi, s));
            }
            prof_end(h, s2, bytes, fine_flops(h, L, SU), s, fine_ops<S>(h, L, fuse_z ? FR_POST2Z : FR_POST2));
            if (l == 0 && zo && sizeof(S) == 4) {
                int sz = prof_begin(h, s, R_ZSTATS, false);
                BD_TRY(launch_z_from32(h, (const float2 *)u, *zo, s));
                prof_end(h, sz, 0.0, 0.0, s);
                if (zdone) *zdone = true;
            }
        } else {
            int s2 = prof_begin(h, s, 16 * l + R_POST2, false);
            k_copy2<S><<<grid_for(L.N, 256), 256, 0, s>>>(L.N, lv.w, u); ::bd::note_launch();
            BD_LAUNCH_CHECK();
            prof_end(h, s2, 0.0, 0.0, s);
        }
        return BD_OK;
    };
    for (int l = 0; l < nl - 1; l++)
        BD_TRY(l == 0 ? down(l, std::integral_constant<bool, SU0>{}) : down(l, std::false_type{}));
    {
        const LV<S> cv = view<S>(h, nl - 1);
        const S *f = (const S *)(nl == 1 ? f0 : cv.f);
        S *u = (S *)(nl == 1 ? u0 : cv.u);
        size_t smem = sizeof(double) * (size_t)h->nc;
        int sc = prof_begin(h, s, R_COARSE, false);
        if (h->nc <= 256) {
            k_coarse_solve<S><<<1, 1024, smem, s>>>(h->nc, h->cinv.p, h->zc.p, h->zz, f, u); ::bd::note_launch();
        } else {
            k_coarse_solve_wide<S><<<(h->nc + 7) / 8, 256, smem, s>>>(h->nc, h->cinv.p, h->zc.p, h->zz, f, u);
            ::bd::note_launch();
        }
        BD_LAUNCH_CHECK();
        prof_end(h, sc, 0.0, 0.0, s);
    }
    for (int l = nl - 2; l >= 0; l--)
        BD_TRY(l == 0 ? up(l, std::integral_constant<bool, SU0>{}) : up(l, std::false_type{}));
    return BD_OK;
}

// z = B r with FP64 vectors at the boundary, in the hierarchy's precision.
// d0_ready: the producer of r already wrote the finest level's input (D0Out);
// zo, zdone: as vcycle_impl (z is written to z_dev either way).
static int vcycle_run(amg_hierarchy *h, const double *r_dev, double *z_dev, cudaStream_t s, bool d0_ready,
                      const ZOut *zo, bool *zdone)
{
    Level &L0 = h->lev[0];
    if (zdone) *zdone = false;
    if (h->prec32) {
        const LV<float> v0 = view<float>(h, 0);
        if (!d0_ready) {
            int si = prof_begin(h, s, R_VIN, false);
            k_in32<<<grid_for(L0.N, 256), 256, 0, s>>>(L0.N, (const double2 *)r_dev, v0.invd,
                                                       (float)L0.ch_inv_theta, v0.f, v0.d); ::bd::note_launch();
            BD_LAUNCH_CHECK();
            prof_end(h, si, 0.0, 0.0, s);
        }
        bool zd = false;
        BD_TRY((vcycle_impl<float, false>(h, v0.f, v0.u, s, zo, &zd)));
        if (!zd) {
            int so = prof_begin(h, s, R_VOUT, false);
            k_out64<<<grid_for(L0.N, 256), 256, 0, s>>>(L0.N, v0.u, (double2 *)z_dev); ::bd::note_launch();
            BD_LAUNCH_CHECK();
            prof_end(h, so, 0.0, 0.0, s);
        }
        if (zdone) *zdone = zd;
        return BD_OK;
    }
    // FP64 sliced ELL: the finest level's gathered vectors in (v + u, u) form
    const LV<double> v0 = view<double>(h, 0);
    const bool su = h->sell.valid;
    if (h->nlev > 1 && !d0_ready) {
        int si = prof_begin(h, s, R_VIN, false);
        if (su)
            k_scale_d0<double, true><<<grid_for(L0.N, 256), 256, 0, s>>>(L0.N, (const double2 *)r_dev, v0.invd,
                                                                         L0.ch_inv_theta, v0.d);
        else
            k_scale_d0<double, false><<<grid_for(L0.N, 256), 256, 0, s>>>(L0.N, (const double2 *)r_dev, v0.invd,
                                                                          L0.ch_inv_theta, v0.d);
        ::bd::note_launch();
        BD_LAUNCH_CHECK();
        prof_end(h, si, 0.0, 0.0, s);
    }
    return su ? vcycle_impl<double, true>(h, (const double2 *)r_dev, (double2 *)z_dev, s, zo, zdone)
              : vcycle_impl<double, false>(h, (const double2 *)r_dev, (double2 *)z_dev, s, zo, zdone);
}

int vcycle_device(amg_hierarchy *h, const double *r_dev, double *z_dev, cudaStream_t s)
{
    return vcycle_run(h, r_dev, z_dev, s, false, nullptr, nullptr);
}

// ------------------------------------------------------------------ PCG reductions
// scal[] slots of the device scalars
enum {
    S_SUMFU = 0, S_FF, S_NF2, S_RR, S_RZ, S_PQ, S_ALPHA, S_BETA, S_MEANZ,
    S_BREAK, S_MEANF, S_TRR, S_MEANX,
    // device-side loop control of the graph form
    S_RTOL, S_MAXIT, S_WARM, S_IT, S_STATUS,
    S_NSLOTS
};
constexpr int kPart = 4;  // partial sums per block
// Grid of the PCG vector kernels: one resident wave of fewer, larger blocks
// than kRedBlocks, so the last block's reduction of the partials is shorter.
constexpr int kVecBlocks = 608, kVecThreads = 512;
constexpr int kMaxBlockThreads = 512;  // largest block of a reduction kernel

// What the last block of a reduction kernel does with the totals.
// first < 0: "first iteration" is read from the device iteration counter
// (graph form).  Stages 6 and 7 are the graph form's loop control: 6 opens
// the loop after the initial residual, 7 closes an iteration; both set the
// WHILE node's condition.
struct Fin {
    double *scal;
    double *partial;
    unsigned int *counter;
    int stage, N, first, flex;
    cudaGraphConditionalHandle cond;
};

__device__ void finish_stage(const Fin &f, double a, double b, double c, double d)
{
    double *scal = f.scal;
    const int N = f.N;
    const int first = f.first < 0 ? (scal[S_IT] == 0.0) : f.first;
    switch (f.stage) {
    case 0:  // f statistics: sum f_u, ||f||^2
        scal[S_SUMFU] = a;
        scal[S_FF] = b;
        scal[S_MEANF] = a / N;
        break;
    case 1:  // ||fp||^2
        scal[S_NF2] = a;
        break;
    case 2:  // ||r||^2
        scal[S_RR] = a;
        break;
    case 3: {  // z statistics: sum z_u, sum r_u, r.z, r.z_old
        double mz = a / N;
        double rz = c - mz * b;  // r . (z projected)
        scal[S_MEANZ] = mz;
        // standard CG: beta = rz_new / rz_old; flexible (Polak-Ribiere):
        // beta = (r.z_new - r.z_old) / rz_old with z_old the previous projected z
        double num = f.flex ? rz - d : rz;
        scal[S_BETA] = first ? 0.0 : num / scal[S_RZ];
        scal[S_RZ] = rz;
        break;
    }
    case 4:  // p.q
        scal[S_PQ] = a;
        if (!(a > 0.0) || !isfinite(a) || !isfinite(scal[S_RZ])) scal[S_BREAK] = 1.0;
        scal[S_ALPHA] = scal[S_RZ] / a;
        break;
    case 5:  // true residual and mean of x_u
        scal[S_TRR] = a;
        scal[S_MEANX] = b / N;
        break;
    case 6: {  // initial ||r||^2; open the loop unless already converged
        scal[S_RR] = a;
        const double nf = sqrt(scal[S_NF2]);
        const bool go = nf > 0.0 && !(sqrt(a) <= scal[S_RTOL] * nf) && scal[S_MAXIT] > 0.0;
        scal[S_IT] = 0.0;
        scal[S_STATUS] = go ? (double)BD_ENOTCONV : (double)BD_OK;
        cudaGraphSetConditional(f.cond, go ? 1u : 0u);
        break;
    }
    case 7: {  // ||r||^2 after the update; close or continue the loop
        scal[S_RR] = a;
        const double it = scal[S_IT] + 1.0;
        scal[S_IT] = it;
        const double nf = sqrt(scal[S_NF2]), rr = sqrt(a);
        bool go = true;
        if (scal[S_BREAK] != 0.0 || !isfinite(rr)) {
            scal[S_STATUS] = (double)BD_EBREAKDOWN;
            go = false;
        } else if (rr <= scal[S_RTOL] * nf) {
            scal[S_STATUS] = (double)BD_OK;
            go = false;
        } else if (it >= scal[S_MAXIT]) {
            go = false;  // status stays BD_ENOTCONV
        }
        cudaGraphSetConditional(f.cond, go ? 1u : 0u);
        break;
    }
    }
}

// Block sums of the first NV of a thread's values, in a fixed order: every
// thread stores its values, then warp k adds column k (the entries of lanes
// l, l + 32, ... in index order) and folds its 32 lane sums by shuffles into
// tot[k].  That is 12 FP64 warp additions per value and block for 256 threads
// (36 for 1024), where a shuffle tree in every warp costs 45 for 256.
template <int NV, int BT>
__device__ __forceinline__ void block_sum(const double (&v)[4], double (*buf)[BT], double *tot)
{
#pragma unroll
    for (int k = 0; k < NV; k++) buf[k][threadIdx.x] = v[k];
    __syncthreads();
    const int w = threadIdx.x >> 5, l = threadIdx.x & 31;
    if (w < NV) {
        double t = buf[w][l];
        for (int i = l + 32; i < (int)blockDim.x; i += 32) t += buf[w][i];
        for (int o = 16; o; o >>= 1) t += __shfl_xor_sync(0xffffffffu, t, o);
        if (l == 0) tot[w] = t;
    }
    __syncthreads();
}

// Block sums -> partial[blockIdx]; the last block to arrive reduces all
// partials in a fixed order (independent of which block is last, so the
// result is reproducible) and applies the stage.  No waiting: blocks that are
// not last simply exit.  NV of (a, b, c, d) are live; the stage sees zeros for
// the rest.  Needs blockDim.x <= BT and a multiple of 32 (the shared buffer
// holds BT values per sum: kernels of 256 threads keep the rest of shared
// memory for L1).
template <int NV, int BT = kMaxBlockThreads>
__device__ void block_finish(double a, double b, double c, double d, const Fin &f)
{
    __shared__ double buf[NV][BT];
    __shared__ double tot[4];
    __shared__ bool last;
    double v[4] = {a, b, c, d};
    block_sum<NV, BT>(v, buf, tot);
    if (threadIdx.x == 0) {
        double *o = f.partial + kPart * blockIdx.x;
#pragma unroll
        for (int k = 0; k < NV; k++) o[k] = tot[k];
        __threadfence();
        const unsigned int ticket = atomicAdd(f.counter, 1u);
        last = ticket == gridDim.x - 1;
    }
    __syncthreads();
    if (!last) return;
    __threadfence();
#pragma unroll
    for (int k = 0; k < 4; k++) v[k] = 0.0;
    // L2 loads (the partials were published by the other blocks' fences and
    // tickets), not volatile ones, so that the unrolled loads of several
    // partials are in flight together: the last block's serial tail
#pragma unroll 4
    for (int i = threadIdx.x; i < (int)gridDim.x; i += blockDim.x) {
        const double *q = f.partial + kPart * i;
#pragma unroll
        for (int k = 0; k < NV; k++) v[k] += __ldcg(q + k);
    }
    block_sum<NV, BT>(v, buf, tot);
    if (threadIdx.x == 0) {
        finish_stage(f, tot[0], NV > 1 ? tot[1] : 0.0, NV > 2 ? tot[2] : 0.0, NV > 3 ? tot[3] : 0.0);
        *f.counter = 0u;
    }
}

__global__ void k_f_stats(int N, const double2 *__restrict__ f, Fin fin)
{
    double a = 0.0, b = 0.0;
    for (int i = share_lo(N) + threadIdx.x, e = share_hi(N); i < e; i += blockDim.x) {
        double2 v = f[i];
        a += v.y;
        b += v.x * v.x + v.y * v.y;
    }
    block_finish<2>(a, b, 0.0, 0.0, fin);
}

__global__ void k_project_f(int N, const double2 *__restrict__ f, double2 *__restrict__ fp, Fin fin)
{
    const double m = fin.scal[S_MEANF];
    double a = 0.0;
    for (int i = share_lo(N) + threadIdx.x, e = share_hi(N); i < e; i += blockDim.x) {
        double2 v = f[i];
        v.y -= m;
        fp[i] = v;
        a += v.x * v.x + v.y * v.y;
    }
    block_finish<1>(a, 0.0, 0.0, 0.0, fin);
}

__global__ void k_zero2(int N, double2 *x)
{
    for (int i = share_lo(N) + threadIdx.x, e = share_hi(N); i < e; i += blockDim.x)
        x[i] = make_double2(0.0, 0.0);
}

// x = 0 when (mode 0) the solve is cold, or (mode 1) the right-hand side is zero
__global__ void k_zero_if(int N, double2 *__restrict__ x, const double *__restrict__ scal, int mode)
{
    const bool z = mode == 0 ? scal[S_WARM] == 0.0 : scal[S_NF2] == 0.0;
    if (!z) return;
    for (int i = share_lo(N) + threadIdx.x, e = share_hi(N); i < e; i += blockDim.x)
        x[i] = make_double2(0.0, 0.0);
}

// The next V-cycle's finest-level input, written by the kernel that forms the
// PCG residual r, so that the V-cycle needs no pass of its own over r.  FP64:
// d0 = D^{-1} r / theta, in (v + u, u) form for a sliced-ELL finest level
// (mode 1) or in (v, u) form (mode 2); FP32 V-cycle (mode 3): f = (float) r
// and d0 = D^{-1} f / theta in FP32.  The same arithmetic as k_scale_d0 and
// k_in32.
struct D0Out {
    int mode = 0;  // 0: nothing to write
    double2 *d64 = nullptr;
    const double2 *invd64 = nullptr;
    double it = 0.0;
    float2 *f32 = nullptr, *d32 = nullptr;
    const float2 *invd32 = nullptr;
    float it32 = 0.0f;
    __device__ __forceinline__ void operator()(int p, double r0, double r1) const
    {
        if (mode == 1 || mode == 2) {
            const double2 b = invd64[p];
            const double v = r0 * b.x * it, u = r1 * b.y * it;
            d64[p] = mode == 1 ? make_double2(v + u, u) : make_double2(v, u);
        } else if (mode == 3) {
            const float2 b = invd32[p];
            const float f0 = (float)r0, f1 = (float)r1;
            f32[p] = make_float2(f0, f1);
            d32[p] = make_float2(f0 * b.x * it32, f1 * b.y * it32);
        }
    }
};

// FP64 finest-level operator with a reduction epilogue (block CSR form, T lanes).
// MODE 0: out = A x, partial x.(A x).  MODE 1: out = f - A x (if out), partials
// ||f - A x||^2 and sum of x_u.  x is in (v, u) form.
template <int T, int MODE>
__global__ void __launch_bounds__(256) k_bsr_reduce(int N, const int *__restrict__ rp,
                                                     const int *__restrict__ ci,
                                                     const double *__restrict__ v,
                                                     const double2 *__restrict__ x,
                                                     const double2 *__restrict__ f,
                                                     double2 *__restrict__ out, Fin fin, D0Out d0)
{
    const int lane = threadIdx.x & (T - 1);
    const int groups = (gridDim.x * blockDim.x) / T;
    const int warp_first = ((blockIdx.x * blockDim.x + threadIdx.x) & ~31) / T;
    const int g_in_warp = (threadIdx.x & 31) / T;
    double acc = 0.0, xs = 0.0;
    for (int pw = warp_first; pw < N; pw += groups) {
        const int p = pw + g_in_warp;
        const bool act = p < N;
        double y0 = 0.0, y1 = 0.0;
        const int e = act ? rp[p + 1] : 0;
        for (int t = act ? rp[p] + lane : 0; t < e; t += T) {
            const int q = ci[t];
            const BlkS<double> a = load_blk(v, (size_t)t);
            const double2 xq = x[q];
            y0 = fma(a.a00, xq.x, fma(a.a01, xq.y, y0));
            y1 = fma(a.a10, xq.x, fma(a.a11, xq.y, y1));
        }
        group_sum2<T>(y0, y1);
        if (act && lane == 0) {
            const double2 xp = x[p];
            if (MODE == 0) {
                out[p] = make_double2(y0, y1);
                acc += xp.x * y0 + xp.y * y1;
            } else {
                const double2 fp = f[p];
                const double r0 = fp.x - y0, r1 = fp.y - y1;
                if (out) out[p] = make_double2(r0, r1);
                d0(p, r0, r1);
                acc += r0 * r0 + r1 * r1;
                xs += xp.y;
            }
        }
    }
    block_finish<MODE == 0 ? 1 : 2, 256>(acc, xs, 0.0, 0.0, fin);
}

// Same with the sliced-ELL finest level.  SU: x is stored as (v + u, u), so a
// node pair costs two FP64 FMAs (a += Ki s, b += Ke u) instead of three.
template <int MODE, bool SU, int TPB = 256>
__global__ void __launch_bounds__(TPB, 1024 / TPB) k_sell_reduce(int N, const int *__restrict__ sptr,
                                                      const int *__restrict__ col,
                                                      const double2 *__restrict__ kk,
                                                      const double *__restrict__ cm,
                                                      const double2 *__restrict__ x,
                                                      const double2 *__restrict__ f,
                                                      double2 *__restrict__ out, Fin fin, D0Out d0)
{
    double acc = 0.0, xs = 0.0;
    const int lane = threadIdx.x & 31, e = share_hi(N);
    for (int p = share_lo(N) + threadIdx.x; p < e; p += blockDim.x) {
        const int sl = p >> 5;
        const int j1 = sptr[sl + 1];
        double a = 0.0, b = 0.0;
#pragma unroll 8
        for (int j = sptr[sl]; j < j1; j++) {
            const size_t idx = (size_t)j * 32 + lane;
            const int q = col[idx];
            const double2 k = kk[idx];
            const double2 xq = x[q];
            a = fma(k.x, SU ? xq.x : xq.x + xq.y, a);
            b = fma(k.y, xq.y, b);
        }
        const double2 xs2 = x[p];
        const double vp = SU ? xs2.x - xs2.y : xs2.x, up = xs2.y;
        const double y0 = fma(cm[p], vp, a), y1 = a + b;
        if (MODE == 0) {
            out[p] = make_double2(y0, y1);
            acc = fma(vp, y0, fma(up, y1, acc));
        } else {
            const double2 fp = f[p];
            const double r0 = fp.x - y0, r1 = fp.y - y1;
            if (out) out[p] = make_double2(r0, r1);
            d0(p, r0, r1);
            acc += r0 * r0 + r1 * r1;
            xs += up;
        }
    }
    block_finish<MODE == 0 ? 1 : 2, TPB>(acc, xs, 0.0, 0.0, fin);
}

// MODE 0 applies A to the search direction (in (v+u, u) form when the finest
// level is sliced ELL); MODE 1 forms f - A x for an iterate in (v, u) form.
template <int MODE>
static void fine_reduce(const amg_hierarchy *h, const double2 *x, const double2 *f, double2 *out,
                        const Fin &fin, cudaStream_t s, const D0Out &d0 = D0Out{})
{
    const Level &L0 = h->lev[0];
    if (h->sell.valid) {
        const FineSell &F = h->sell;
        if (fine_wide(L0.N))
            k_sell_reduce<MODE, MODE == 0, kFineTPB><<<kSM, kFineTPB, 0, s>>>(
                L0.N, F.sptr.p, F.col.p, (const double2 *)F.kk.p, F.cm.p, x, f, out, fin, d0);
        else
            k_sell_reduce<MODE, MODE == 0><<<kSM * 4, 256, 0, s>>>(L0.N, F.sptr.p, F.col.p,
                                                                  (const double2 *)F.kk.p, F.cm.p, x, f, out, fin, d0);
        ::bd::note_launch();
        return;
    }
    const BSR &A = L0.A;
    switch (std::min(lanes_for(A, false), 32)) {
    case 1: k_bsr_reduce<1, MODE><<<kRedBlocks, 256, 0, s>>>(A.nbr, A.rp.p, A.ci.p, A.v.p, x, f, out, fin, d0); ::bd::note_launch(); break;
    case 2: k_bsr_reduce<2, MODE><<<kRedBlocks, 256, 0, s>>>(A.nbr, A.rp.p, A.ci.p, A.v.p, x, f, out, fin, d0); ::bd::note_launch(); break;
    case 4: k_bsr_reduce<4, MODE><<<kRedBlocks, 256, 0, s>>>(A.nbr, A.rp.p, A.ci.p, A.v.p, x, f, out, fin, d0); ::bd::note_launch(); break;
    case 8: k_bsr_reduce<8, MODE><<<kRedBlocks, 256, 0, s>>>(A.nbr, A.rp.p, A.ci.p, A.v.p, x, f, out, fin, d0); ::bd::note_launch(); break;
    case 16: k_bsr_reduce<16, MODE><<<kRedBlocks, 256, 0, s>>>(A.nbr, A.rp.p, A.ci.p, A.v.p, x, f, out, fin, d0); ::bd::note_launch(); break;
    default: k_bsr_reduce<32, MODE><<<kRedBlocks, 256, 0, s>>>(A.nbr, A.rp.p, A.ci.p, A.v.p, x, f, out, fin, d0); ::bd::note_launch(); break;
    }
}

// sums of z_u and r_u, r.z and (flexible form) r.z_old
__global__ void k_z_stats(int N, const double2 *__restrict__ z, const double2 *__restrict__ r,
                          const double2 *__restrict__ zold, Fin fin)
{
    double a = 0.0, b = 0.0, c = 0.0, d = 0.0;
    for (int i = share_lo(N) + threadIdx.x, e = share_hi(N); i < e; i += blockDim.x) {
        const double2 zi = z[i], ri = r[i];
        a += zi.y;
        b += ri.y;
        c += ri.x * zi.x + ri.y * zi.y;
        if (zold) {
            const double2 oi = zold[i];
            d += ri.x * oi.x + ri.y * oi.y;
        }
    }
    block_finish<4>(a, b, c, d, fin);
}

// The V-cycle's last finest-level kernel with the z statistics fused in: the
// post-smoothed iterate is the preconditioned residual z, stored in FP64, and
// the sums k_z_stats forms (z_u, r_u, r.z, r.z_old) are taken in FP64 in the
// same pass (stage 3).
struct ZOut {
    double2 *z;
    const double2 *r;
    const double2 *zold;  // flexible CG's previous projected z, or null
    Fin fin;
};

// FP64: at most 64 registers (32 warps per SM, as the other FP64 finest-level
// kernels).  FP32 V-cycle: the per-thread partial sums are FP32, the
// precision z itself comes in (the V-cycle's output, converted exactly), with
// r and z_old rounded to FP32 for the products; blocks and the grid add the
// partials in FP64.  That keeps the kernel within 32 registers, so it runs 8
// blocks per SM like the other FP32 finest-level kernels, which need every
// resident warp to keep enough bytes in flight.
template <class S, bool SU, int MINB, class E2, int TPB = 256>
__global__ void __launch_bounds__(TPB, MINB) k_sell_z(int N, const int *__restrict__ sptr,
                                                    const int *__restrict__ col,
                                                    const unsigned char *__restrict__ code, Stencil st,
                                                    const v2<S> *__restrict__ kk, const S *__restrict__ cm,
                                                    GatherVec<S> gather, E2 epi, ZOut zo)
{
    __shared__ int off[27];
    if (sizeof(S) == 4) stage_stencil(st, off);
    S a = 0, b = 0, c = 0, d = 0;
    const int lane = threadIdx.x & 31, e = share_hi(N);
    for (int p = share_lo(N) + threadIdx.x; p < e; p += blockDim.x) {
        S y0, y1;
        sell_row<S, GatherVec<S>, SU, (sizeof(S) == 8 ? 8 : 4)>(p, lane, sptr, col, code, off, kk, cm, gather, y0,
                                                                 y1);
        const v2<S> u = epi.value(p, y0, y1);
        const double2 z = make_double2((double)u.x, (double)u.y), r = zo.r[p];
        zo.z[p] = z;
        const S rx = (S)r.x, ry = (S)r.y;
        a += u.y;
        b += ry;
        c = fma(rx, u.x, fma(ry, u.y, c));
        if (zo.zold) {
            const double2 o = zo.zold[p];
            d = fma(rx, (S)o.x, fma(ry, (S)o.y, d));
        }
    }
    block_finish<4, TPB>((double)a, (double)b, (double)c, (double)d, zo.fin);
}

static int zo_streams(const ZOut *zo) { return zo->zold ? 3 : 2; }

// z = (double) u of the FP32 V-cycle, and its statistics (z_u, r_u, r.z,
// r.z_old) in FP64 (stage 3), in one pass
__global__ void k_z_from32(int N, const float2 *__restrict__ u, ZOut zo)
{
    double a = 0.0, b = 0.0, c = 0.0, d = 0.0;
    for (int i = share_lo(N) + threadIdx.x, e = share_hi(N); i < e; i += blockDim.x) {
        const float2 v = u[i];
        const double2 z = make_double2((double)v.x, (double)v.y), r = zo.r[i];
        zo.z[i] = z;
        a += z.y;
        b += r.y;
        c += r.x * z.x + r.y * z.y;
        if (zo.zold) {
            const double2 o = zo.zold[i];
            d += r.x * o.x + r.y * o.y;
        }
    }
    block_finish<4>(a, b, c, d, zo.fin);
}

static int launch_z_from32(amg_hierarchy *h, const float2 *u, const ZOut &zo, cudaStream_t s)
{
    k_z_from32<<<kVecBlocks, kVecThreads, 0, s>>>(h->lev[0].N, u, zo);
    ::bd::note_launch();
    BD_LAUNCH_CHECK();
    return BD_OK;
}

template <class S, bool SU, class E2>
static int launch_sell_z(amg_hierarchy *h, const LV<S> &lv, const E2 &epi, const ZOut &zo, cudaStream_t s)
{
    const FineSell &F = h->sell;
    const int N = h->lev[0].N;
    const long long slices = ((long long)N + 31) / 32;
    if (sizeof(S) == 8 && fine_wide(N)) {
        k_sell_z<S, SU, 1, E2, kFineTPB><<<(int)std::min<long long>(slices, kSM), kFineTPB, 0, s>>>(
            N, F.sptr.p, F.col.p, F.code.p, stencil_of(F), lv.kk, lv.cm, GatherVec<S>{lv.d}, epi, zo);
    } else {
        constexpr int MB = sizeof(S) == 8 ? 4 : 8;
        k_sell_z<S, SU, MB, E2><<<(int)std::min<long long>(slices, (long long)kSM * MB), 256, 0, s>>>(
            N, F.sptr.p, F.col.p, F.code.p, stencil_of(F), lv.kk, lv.cm, GatherVec<S>{lv.d}, epi, zo);
    }
    ::bd::note_launch();
    BD_LAUNCH_CHECK();
    return BD_OK;
}

// z <- z - mean(z_u) e_u; p = z (first iteration) or z + beta p, stored in
// (v+u, u) form when SU; keeps the projected z for the next flexible beta
// when zold is given.
template <bool SU>
__global__ void k_p_update(int N, double2 *__restrict__ z, double2 *__restrict__ p,
                           double2 *__restrict__ zold, const double *__restrict__ scal, int first)
{
    const double mz = scal[S_MEANZ], beta = scal[S_BETA];
    if (first < 0) first = scal[S_IT] == 0.0;
    for (int i = share_lo(N) + threadIdx.x, e = share_hi(N); i < e; i += blockDim.x) {
        double2 zi = z[i];
        zi.y -= mz;
        z[i] = zi;
        if (zold) zold[i] = zi;
        const double2 zs = SU ? make_double2(zi.x + zi.y, zi.y) : zi;
        if (first) {
            p[i] = zs;
        } else {
            const double2 pi = p[i];
            p[i] = make_double2(zs.x + beta * pi.x, zs.y + beta * pi.y);
        }
    }
}

template <bool SU>
__global__ void k_xr_update(int N, double2 *__restrict__ x, double2 *__restrict__ r,
                            const double2 *__restrict__ p, const double2 *__restrict__ q, Fin fin, D0Out d0)
{
    const double alpha = fin.scal[S_ALPHA];
    double acc = 0.0;
    for (int i = share_lo(N) + threadIdx.x, e = share_hi(N); i < e; i += blockDim.x) {
        double2 xi = x[i], ri = r[i];
        const double2 pi = p[i], qi = q[i];
        const double pv = SU ? pi.x - pi.y : pi.x;
        xi.x += alpha * pv;
        xi.y += alpha * pi.y;
        ri.x -= alpha * qi.x;
        ri.y -= alpha * qi.y;
        x[i] = xi;
        r[i] = ri;
        d0(i, ri.x, ri.y);
        acc += ri.x * ri.x + ri.y * ri.y;
    }
    block_finish<1>(acc, 0.0, 0.0, 0.0, fin);
}

__global__ void k_project_x(int N, double2 *__restrict__ x, const double *__restrict__ scal)
{
    const double m = scal[S_MEANX];
    for (int i = share_lo(N) + threadIdx.x, e = share_hi(N); i < e; i += blockDim.x) x[i].y -= m;
}

static void p_update(const amg_hierarchy *h, int N, double2 *z, double2 *p, double2 *zold, double *scal,
                     int first, cudaStream_t s)
{
    if (h->sell.valid) k_p_update<true><<<kVecBlocks, kVecThreads, 0, s>>>(N, z, p, zold, scal, first);
    else k_p_update<false><<<kVecBlocks, kVecThreads, 0, s>>>(N, z, p, zold, scal, first);
    note_launch();
}

static void xr_update(const amg_hierarchy *h, int N, double2 *x, double2 *r, const double2 *p,
                      const double2 *q, const Fin &fin, cudaStream_t s, const D0Out &d0)
{
    if (h->sell.valid) k_xr_update<true><<<kVecBlocks, kVecThreads, 0, s>>>(N, x, r, p, q, fin, d0);
    else k_xr_update<false><<<kVecBlocks, kVecThreads, 0, s>>>(N, x, r, p, q, fin, d0);
    note_launch();
}

// What the producer of the PCG residual writes for the next V-cycle (see
// D0Out); mode 0 where the V-cycle has no smoothing level and is FP64.
static D0Out d0_out(amg_hierarchy *h)
{
    D0Out d;
    Level &L0 = h->lev[0];
    if (h->prec32) {
        d.mode = 3;
        d.f32 = (float2 *)L0.f32.p;
        d.d32 = (float2 *)L0.d32.p;
        d.invd32 = (const float2 *)L0.invdiag32.p;
        d.it32 = (float)L0.ch_inv_theta;
    } else if (h->nlev > 1) {
        d.mode = h->sell.valid ? 1 : 2;
        d.d64 = (double2 *)L0.d.p;
        d.invd64 = (const double2 *)L0.invdiag.p;
        d.it = L0.ch_inv_theta;
    }
    return d;
}

// ------------------------------------------------------------------ lane autotuning
// Candidates: block-CSR with powers of two from (average blocks per row)/16
// lanes per row to 4x the average, 64/128/256 meaning a thread block per row
// (rows of 32 blocks and more only), and, where the operator may take it, the
// sliced form with 1, 2, 4 and 8 lanes per row (FP64, operators of 8192 rows
// and more).  Each runs once untimed, then three times back to back, and the
// median counts (the V-cycle applies a level's operator several times in a
// row: smoother, residual).  Single launches do not rank every operator as the
// V-cycle does: on the 128x128x32 slab they put the sliced form first for the
// middle level's A, which inside the V-cycle is 5 % slower than block-CSR with
// 4 lanes, warm or after an L2 flush; the row-length rule holds the choices
// measured inside the V-cycle.  The launches of all block-CSR candidates are
// queued with their events and read after one synchronisation; each sliced
// candidate is built, timed and synchronised in turn (the next one reuses its
// buffers).
constexpr int kLaneCands = 13, kLaneReps = 3;
constexpr long long kTuneMinBlocks = 20000;  // smaller operators keep the rule

template <class S>
static int tune_operator(Level &L, int op, bool sliced_ok, const v2<S> *x, const v2<S> *f, v2<S> *out,
                         const S *vals, cudaEvent_t (*ev)[kLaneReps][2], cudaStream_t s)
{
    const BSR &M = op == 0 ? L.A : (op == 1 ? L.R : L.P);
    const bool fp32 = sizeof(S) == 4;
    const double avg = M.nbr > 0 ? (double)M.nb / M.nbr : 1.0;
    const EpiResid<S> epi{f, out};
    int Tlo = 1, Thi = 256;
    while (Tlo * 16 < avg && Tlo < 32) Tlo <<= 1;
    while (Thi > 1 && Thi > 4.0 * avg) Thi >>= 1;
    if (avg < 32.0) Thi = std::min(Thi, 32);
    Thi = std::max(Thi, Tlo);
    int cand[kLaneCands], nc = 0;
    for (int T = Tlo; T <= Thi && nc < kLaneCands - 4; T <<= 1) cand[nc++] = T;
    const int ncsr = nc;
    if (sliced_ok && !fp32 && M.nbr >= kSlicedMinRows)
        for (int K = 1; K <= 8; K <<= 1) cand[nc++] = -K;
    const int rule = L.lanes[op];
    for (int c = 0; c < nc; c++) {
        if (cand[c] < 0) BD_TRY(build_sliced(M, -cand[c], fp32, L.sl[op], s));
        L.lanes[op] = cand[c];
        BD_TRY(apply_op<S>(L, op, vals, GatherVec<S>{x}, epi, s));
        for (int k = 0; k < kLaneReps; k++) {
            BD_CUDA(cudaEventRecord(ev[c][k][0], s));
            BD_TRY(apply_op<S>(L, op, vals, GatherVec<S>{x}, epi, s));
            BD_CUDA(cudaEventRecord(ev[c][k][1], s));
        }
        if (cand[c] < 0 || c + 1 == ncsr) BD_CUDA(cudaStreamSynchronize(s));
    }
    BD_CUDA(cudaStreamSynchronize(s));
    // the fastest median wins unless the rule's choice (when among the
    // candidates) is within 3 % of it: near-ties then resolve the same way
    // on every run
    float best = 0.0f, t_rule = -1.0f;
    int bestT = rule;
    for (int c = 0; c < nc; c++) {
        float t[kLaneReps];
        for (int k = 0; k < kLaneReps; k++) BD_CUDA(cudaEventElapsedTime(&t[k], ev[c][k][0], ev[c][k][1]));
        const float med = std::max(std::min(t[0], t[1]), std::min(std::max(t[0], t[1]), t[2]));
        if (cand[c] == rule) t_rule = med;
        if (c == 0 || med < best) {
            best = med;
            bestT = cand[c];
        }
    }
    const int pick = (t_rule >= 0.0f && t_rule <= 1.03f * best) ? rule : bestT;
    L.lanes[op] = pick;
    if (pick > 0) drop_sliced(L.sl[op]);
    else if (L.sl[op].K != -pick) BD_TRY(build_sliced(M, -pick, fp32, L.sl[op], s));
    return BD_OK;
}

// Time the candidate forms of every block operator the V-cycle applies (A
// below the finest level, or on it where it is not sliced ELL; R and P) on
// this GPU and keep the fastest.  The workspace vectors serve as operands;
// their contents do not matter.  The form changes the order of a row's sum,
// so the choice is fixed per hierarchy: every solve with it is reproducible.
template <class S>
static int autotune_lanes(amg_hierarchy *h, cudaStream_t s)
{
    cudaEvent_t ev[kLaneCands][kLaneReps][2] = {};
    int st = BD_OK;
    for (auto &c : ev)
        for (auto &r : c)
            for (cudaEvent_t &e : r)
                if (st == BD_OK && cudaEventCreate(&e) != cudaSuccess) st = BD_ECUDA;
    for (int l = 0; l < h->nlev - 1 && st == BD_OK; l++) {
        Level &L = h->lev[l];
        const LV<S> lv = view<S>(h, l), cv = view<S>(h, l + 1);
        for (int op = 0; op < 3 && st == BD_OK; op++) {
            if (op == 0 && l == 0 && h->sell.valid) continue;
            const BSR &M = op == 0 ? L.A : (op == 1 ? L.R : L.P);
            if (M.nb < kTuneMinBlocks) continue;
            const S *vals = op == 0 ? lv.Av : (op == 1 ? lv.Rv : lv.Pv);
            const v2<S> *x = op == 0 ? lv.u : (op == 1 ? lv.r : cv.u);
            const v2<S> *f = op == 1 ? cv.f : lv.f;
            v2<S> *out = op == 0 ? lv.r : (op == 1 ? cv.r : lv.w);
            st = tune_operator<S>(L, op, op > 0 || l > 0, x, f, out, vals, ev, s);
        }
    }
    for (auto &c : ev)
        for (auto &r : c)
            for (cudaEvent_t e : r)
                if (e) cudaEventDestroy(e);
    return st;
}

// ------------------------------------------------------------------ workspace
int prepare_solve(amg_hierarchy *h, cudaStream_t s)
{
    const bool p32 = h->prec32;
    for (int l = 0; l < h->nlev; l++) {
        Level &L = h->lev[l];
        size_t n = 2 * (size_t)L.N;
        if (p32) {
            BD_TRY(L.f32.alloc(n));
            BD_TRY(L.u32.alloc(n));
            BD_TRY(L.r32.alloc(n));
            BD_TRY(L.d32.alloc(n));
            BD_TRY(L.w32.alloc(n));
            BD_TRY(L.invdiag32.alloc(n));
            BD_TRY(L.A32.alloc(4 * (size_t)L.A.nb));
            k_to_f32<<<grid_for(n, 256), 256, 0, s>>>((long long)n, L.invdiag.p, L.invdiag32.p); ::bd::note_launch();
            k_to_f32<<<grid_for(4 * L.A.nb, 256), 256, 0, s>>>(4 * L.A.nb, L.A.v.p, L.A32.p); ::bd::note_launch();
            if (l < h->nlev - 1) {
                BD_TRY(L.P32.alloc(4 * (size_t)L.P.nb));
                BD_TRY(L.R32.alloc(4 * (size_t)L.R.nb));
                k_to_f32<<<grid_for(4 * L.P.nb, 256), 256, 0, s>>>(4 * L.P.nb, L.P.v.p, L.P32.p); ::bd::note_launch();
                k_to_f32<<<grid_for(4 * L.R.nb, 256), 256, 0, s>>>(4 * L.R.nb, L.R.v.p, L.R32.p); ::bd::note_launch();
            }
            BD_LAUNCH_CHECK();
        } else {
            BD_TRY(L.f.alloc(n));
            BD_TRY(L.u.alloc(n));
            BD_TRY(L.r.alloc(n));
            BD_TRY(L.d.alloc(n));
            BD_TRY(L.w.alloc(n));
        }
        if (l < h->nlev - 1) {
            double lo = h->opts.eig_lo * L.lam, hi = h->opts.eig_hi * L.lam;
            double theta = 0.5 * (hi + lo), delta = 0.5 * (hi - lo);
            double sigma = theta / delta, rho0 = 1.0 / sigma;
            double rho1 = 1.0 / (2.0 * sigma - rho0);
            L.ch_inv_theta = 1.0 / theta;
            L.ch_c1 = rho1 * rho0;
            L.ch_c2 = 2.0 * rho1 / delta;
            if (l == 0 && !p32 && h->sell.valid) {
                // the FP64 finest level's scaled inverse diagonals (EpiPreX and kin)
                BD_TRY(L.idc2.alloc(n));
                BD_TRY(L.idt.alloc(n));
                k_scale_vec<<<grid_for(n, 256), 256, 0, s>>>((long long)n, L.invdiag.p, L.ch_c2, L.idc2.p);
                ::bd::note_launch();
                k_scale_vec<<<grid_for(n, 256), 256, 0, s>>>((long long)n, L.invdiag.p, L.ch_inv_theta, L.idt.p);
                ::bd::note_launch();
                BD_LAUNCH_CHECK();
            }
        }
    }
    if (p32 && h->sell.valid) {
        FineSell &F = h->sell;
        size_t nk = 64 * (size_t)F.slots;
        BD_TRY(F.kk32.alloc(nk));
        BD_TRY(F.cm32.alloc((size_t)h->lev[0].N));
        k_to_f32<<<grid_for(nk, 256), 256, 0, s>>>((long long)nk, F.kk.p, F.kk32.p); ::bd::note_launch();
        k_to_f32<<<grid_for(h->lev[0].N, 256), 256, 0, s>>>(h->lev[0].N, F.cm.p, F.cm32.p); ::bd::note_launch();
        BD_LAUNCH_CHECK();
    }
    size_t n0 = 2 * (size_t)h->lev[0].N;
    BD_TRY(h->x.alloc(n0));
    BD_TRY(h->r.alloc(n0));
    BD_TRY(h->z.alloc(n0));
    BD_TRY(h->p.alloc(n0));
    BD_TRY(h->q.alloc(n0));
    BD_TRY(h->fp.alloc(n0));
    BD_TRY(h->fin.alloc(n0));
    if (p32) {
        BD_TRY(h->zold.alloc(n0));
        BD_CUDA(cudaMemsetAsync(h->zold.p, 0, h->zold.bytes(), s));
    }
    BD_TRY(h->partial.alloc(kPart * (size_t)kRedBlocks));
    BD_TRY(h->counter.alloc(1));
    BD_CUDA(cudaMemsetAsync(h->counter.p, 0, sizeof(unsigned int), s));
    BD_TRY(h->scal.alloc(S_NSLOTS));
    if (!h->host_scal) BD_CUDA(cudaMallocHost((void **)&h->host_scal, sizeof(double) * S_NSLOTS));
    if (!h->host_init) BD_CUDA(cudaMallocHost((void **)&h->host_init, sizeof(double) * S_NSLOTS));
    // lanes per block row of the V-cycle's block-CSR operators
    // (the sliced form for A only below the finest level: the PCG's fused
    // A p and residual reductions on a non-sliced-ELL finest level use
    // block-CSR; nothing on the coarsest level, which is solved densely)
    for (int l = 0; l < h->nlev; l++) {
        Level &L = h->lev[l];
        const bool last = l == h->nlev - 1;
        L.lanes[0] = lanes_rule(L.A, p32, l > 0 && !last);
        L.lanes[1] = last ? 0 : lanes_rule(L.R, p32, true);
        L.lanes[2] = last ? 0 : lanes_rule(L.P, p32, true);
        for (int op = 0; op < 3; op++) {
            if (L.lanes[op] < 0)
                BD_TRY(build_sliced(op == 0 ? L.A : (op == 1 ? L.R : L.P), -L.lanes[op], p32, L.sl[op], s));
            else drop_sliced(L.sl[op]);
        }
    }
    if (h->opts.autotune) BD_TRY(p32 ? autotune_lanes<float>(h, s) : autotune_lanes<double>(h, s));
    BD_CUDA(cudaStreamSynchronize(s));
    return BD_OK;
}

static int read_scal(amg_hierarchy *h, cudaStream_t s)
{
    BD_CUDA(cudaMemcpyAsync(h->host_scal, h->scal.p, sizeof(double) * S_NSLOTS, cudaMemcpyDeviceToHost, s));
    BD_CUDA(cudaStreamSynchronize(s));
    return BD_OK;
}

static Fin make_fin(amg_hierarchy *h, int stage, int first, cudaGraphConditionalHandle cond = 0)
{
    Fin f;
    f.scal = h->scal.p;
    f.partial = h->partial.p;
    f.counter = h->counter.p;
    f.stage = stage;
    f.N = h->lev[0].N;
    f.first = first;
    f.flex = h->prec32 ? 1 : 0;
    f.cond = cond;
    return f;
}

// Projected PCG on device vectors (f_dev, x_dev: 2N doubles each), host-driven
// loop: one residual read-back per iteration.  With an FP32 V-cycle the
// preconditioner is not exactly symmetric, so beta takes the flexible
// (Polak-Ribiere) form.
static int pcg_solve_loop(amg_hierarchy *h, const double *f_dev, double *x_dev, int warm,
                          const solve_options *o, cudaStream_t s, solve_info *info)
{
    Level &L0 = h->lev[0];
    const int N = L0.N;
    const bool flex = h->prec32;
    double2 *x = (double2 *)x_dev, *r = (double2 *)h->r.p, *z = (double2 *)h->z.p;
    double2 *p = (double2 *)h->p.p, *q = (double2 *)h->q.p, *fp = (double2 *)h->fp.p;
    double2 *zold = flex ? (double2 *)h->zold.p : nullptr;
    double *scal = h->scal.p;
    cudaEvent_t e0 = nullptr, e1 = nullptr;
    BD_CUDA(cudaEventCreate(&e0));
    BD_CUDA(cudaEventCreate(&e1));
    BD_CUDA(cudaEventRecord(e0, s));
    BD_CUDA(cudaMemsetAsync(scal, 0, sizeof(double) * S_NSLOTS, s));
    k_f_stats<<<kVecBlocks, kVecThreads, 0, s>>>(N, (const double2 *)f_dev, make_fin(h, 0, 0)); ::bd::note_launch();
    k_project_f<<<kVecBlocks, kVecThreads, 0, s>>>(N, (const double2 *)f_dev, fp, make_fin(h, 1, 0)); ::bd::note_launch();
    if (!warm) {
        k_zero2<<<kVecBlocks, kVecThreads, 0, s>>>(N, x); ::bd::note_launch();
    }
    const D0Out d0 = d0_out(h);
    fine_reduce<1>(h, x, fp, r, make_fin(h, 2, 0), s, d0);
    BD_LAUNCH_CHECK();
    BD_TRY(read_scal(h, s));
    double ff = h->host_scal[S_FF], sumfu = h->host_scal[S_SUMFU];
    double nf = sqrt(h->host_scal[S_NF2]);
    double rr = sqrt(h->host_scal[S_RR]);
    int status = BD_OK, it = 0;
    if (o->strict && ff > 0.0) {
        double null_part = fabs(sumfu) / sqrt((double)N);
        if (null_part > 1e-8 * sqrt(ff)) status = BD_EINCONSISTENT;
    }
    if (status == BD_OK && nf == 0.0) {
        k_zero2<<<kVecBlocks, kVecThreads, 0, s>>>(N, x); ::bd::note_launch();
        BD_LAUNCH_CHECK();
        rr = 0.0;
    } else if (status == BD_OK && !(rr <= o->rtol * nf)) {
        status = BD_ENOTCONV;
        while (it < o->max_it) {
            const ZOut zo{z, r, it == 0 ? nullptr : zold, make_fin(h, 3, it == 0)};
            bool zd = false;
            BD_TRY(vcycle_run(h, (const double *)r, (double *)z, s, true, &zo, &zd));
            if (!zd) {
                int sz = prof_begin(h, s, R_ZSTATS, false);
                k_z_stats<<<kVecBlocks, kVecThreads, 0, s>>>(N, z, r, zo.zold, zo.fin); ::bd::note_launch();
                prof_end(h, sz, 0.0, 0.0, s);
            }
            int su = prof_begin(h, s, R_PUPDATE, false);
            p_update(h, N, z, p, zold, scal, it == 0, s);
            prof_end(h, su, 0.0, 0.0, s);
            // the FP64 PCG operator counts among the finest-operator launches
            // when the V-cycle is FP64 too (one kernel family per profile)
            int sq = prof_begin(h, s, R_AP, !h->prec32);
            fine_reduce<0>(h, p, nullptr, q, make_fin(h, 4, 0), s);
            prof_end(h, sq, h->prec32 ? 0.0 : fine_bytes<double>(h, L0, 2), fine_flops(h, L0, true), s,
                     fine_ops<double>(h, L0, FR_AP));
            int sx = prof_begin(h, s, R_XRUPDATE, false);
            xr_update(h, N, x, r, p, q, make_fin(h, 2, 0), s, d0);
            prof_end(h, sx, 0.0, 0.0, s);
            BD_LAUNCH_CHECK();
            BD_TRY(read_scal(h, s));
            it++;
            if (h->host_scal[S_BREAK] != 0.0) {
                status = BD_EBREAKDOWN;
                break;
            }
            rr = sqrt(h->host_scal[S_RR]);
            if (!std::isfinite(rr)) {
                status = BD_EBREAKDOWN;
                break;
            }
            if (rr <= o->rtol * nf) {
                status = BD_OK;
                break;
            }
        }
    }
    // true residual and projection of x
    fine_reduce<1>(h, x, fp, nullptr, make_fin(h, 5, 0), s);
    k_project_x<<<kVecBlocks, kVecThreads, 0, s>>>(N, x, scal); ::bd::note_launch();
    BD_LAUNCH_CHECK();
    BD_CUDA(cudaEventRecord(e1, s));
    BD_TRY(read_scal(h, s));
    prof_collect(h);
    float ms = 0.0f;
    cudaEventElapsedTime(&ms, e0, e1);
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    if (info) {
        info->status = status;
        info->iters = it;
        info->rel_res = nf > 0.0 ? rr / nf : 0.0;
        info->true_rel_res = nf > 0.0 ? sqrt(h->host_scal[S_TRR]) / nf : 0.0;
        info->solve_ms = ms;
    }
    return status;
}

// ------------------------------------------------------------------ graph form
// The whole solve as one CUDA graph: the pre-loop kernels, a WHILE node whose
// body is one PCG iteration (V-cycle included), the post-loop kernels.  The
// body's last reduction decides convergence, breakdown or max_it on the device
// and sets the node's condition, so a solve costs one graph launch and one
// host synchronisation.  The loop is bounded by max_it.  The graph works on the
// hierarchy's own buffers (right-hand side in `fin`, iterate in `x`).
static void end_capture_quietly(cudaStream_t s)
{
    cudaStreamCaptureStatus cs;
    if (cudaStreamIsCapturing(s, &cs) == cudaSuccess && cs != cudaStreamCaptureStatusNone) {
        cudaGraph_t g = nullptr;
        cudaStreamEndCapture(s, &g);
        if (g) cudaGraphDestroy(g);
    }
    cudaGetLastError();
}

// Capture one whole solve of h into the graph being captured on stream s:
// pre-loop kernels, a WHILE node whose body (captured on s2) is one PCG
// iteration and whose condition the device sets, post-loop kernels.  Operates
// on h's own buffers (f in h->fin, x in h->x, scalars in h->scal).
static int capture_solve(amg_hierarchy *h, cudaStream_t s, cudaStream_t s2)
{
    Level &L0 = h->lev[0];
    const int N = L0.N;
    const bool flex = h->prec32;
    double2 *x = (double2 *)h->x.p, *r = (double2 *)h->r.p, *z = (double2 *)h->z.p;
    double2 *p = (double2 *)h->p.p, *q = (double2 *)h->q.p, *fp = (double2 *)h->fp.p;
    double2 *zold = flex ? (double2 *)h->zold.p : nullptr;
    const double2 *fin = (const double2 *)h->fin.p;
    double *scal = h->scal.p;
    // kernel-node counts per section (the launch counter counts executions, so
    // the increments made while capturing are taken back below)
    const long long c0 = launch_count();
    k_f_stats<<<kVecBlocks, kVecThreads, 0, s>>>(N, fin, make_fin(h, 0, 0)); ::bd::note_launch();
    k_project_f<<<kVecBlocks, kVecThreads, 0, s>>>(N, fin, fp, make_fin(h, 1, 0)); ::bd::note_launch();
    k_zero_if<<<kVecBlocks, kVecThreads, 0, s>>>(N, x, scal, 0); ::bd::note_launch();
    BD_LAUNCH_CHECK();
    cudaStreamCaptureStatus cs;
    cudaGraph_t g = nullptr;
    const cudaGraphNode_t *deps = nullptr;
    size_t nd = 0;
    BD_CUDA(cudaStreamGetCaptureInfo(s, &cs, nullptr, &g, &deps, nullptr, &nd));
    cudaGraphConditionalHandle cond;
    BD_CUDA(cudaGraphConditionalHandleCreate(&cond, g, 0, 0));
    const D0Out d0 = d0_out(h);
    fine_reduce<1>(h, x, fp, r, make_fin(h, 6, 0, cond), s, d0);
    BD_LAUNCH_CHECK();
    BD_CUDA(cudaStreamGetCaptureInfo(s, &cs, nullptr, &g, &deps, nullptr, &nd));
    cudaGraphNodeParams np = {};
    np.type = cudaGraphNodeTypeConditional;
    np.conditional.handle = cond;
    np.conditional.type = cudaGraphCondTypeWhile;
    np.conditional.size = 1;
    cudaGraphNode_t wnode;
    BD_CUDA(cudaGraphAddNode(&wnode, g, deps, nullptr, nd, &np));
    cudaGraph_t body = np.conditional.phGraph_out[0];
    const long long c1 = launch_count();
    BD_CUDA(cudaStreamBeginCaptureToGraph(s2, body, nullptr, nullptr, 0, cudaStreamCaptureModeThreadLocal));
    const ZOut zo{z, r, zold, make_fin(h, 3, -1)};
    bool zd = false;
    BD_TRY(vcycle_run(h, (const double *)r, (double *)z, s2, true, &zo, &zd));
    if (!zd) {
        k_z_stats<<<kVecBlocks, kVecThreads, 0, s2>>>(N, z, r, zold, zo.fin); ::bd::note_launch();
    }
    p_update(h, N, z, p, zold, scal, -1, s2);
    fine_reduce<0>(h, p, nullptr, q, make_fin(h, 4, 0), s2);
    xr_update(h, N, x, r, p, q, make_fin(h, 7, 0, cond), s2, d0);
    BD_LAUNCH_CHECK();
    cudaGraph_t body_out = nullptr;
    BD_CUDA(cudaStreamEndCapture(s2, &body_out));
    const long long c2 = launch_count();
    BD_CUDA(cudaStreamUpdateCaptureDependencies(s, &wnode, nullptr, 1, cudaStreamSetCaptureDependencies));
    k_zero_if<<<kVecBlocks, kVecThreads, 0, s>>>(N, x, scal, 1); ::bd::note_launch();
    fine_reduce<1>(h, x, fp, nullptr, make_fin(h, 5, 0), s);
    k_project_x<<<kVecBlocks, kVecThreads, 0, s>>>(N, x, scal); ::bd::note_launch();
    BD_LAUNCH_CHECK();
    const long long c3 = launch_count();
    h->graph_pre = c1 - c0;
    h->graph_body = c2 - c1;
    h->graph_post = c3 - c2;
    note_launches(-(c3 - c0));
    return BD_OK;
}

static int capture_graph(amg_hierarchy *h)
{
    BD_CUDA(cudaStreamBeginCapture(h->cap_stream, cudaStreamCaptureModeThreadLocal));
    BD_TRY(capture_solve(h, h->cap_stream, h->cap_stream2));
    BD_CUDA(cudaStreamEndCapture(h->cap_stream, &h->graph));
    BD_CUDA(cudaGraphInstantiate(&h->graph_exec, h->graph, 0));
    return BD_OK;
}

static int build_graph(amg_hierarchy *h)
{
    if (!h->cap_stream) BD_CUDA(cudaStreamCreateWithFlags(&h->cap_stream, cudaStreamNonBlocking));
    if (!h->cap_stream2) BD_CUDA(cudaStreamCreateWithFlags(&h->cap_stream2, cudaStreamNonBlocking));
    int st = capture_graph(h);
    if (st != BD_OK) {
        end_capture_quietly(h->cap_stream2);
        end_capture_quietly(h->cap_stream);
        if (h->graph_exec) cudaGraphExecDestroy(h->graph_exec);
        if (h->graph) cudaGraphDestroy(h->graph);
        h->graph_exec = nullptr;
        h->graph = nullptr;
    }
    return st;
}

// Enqueue one graph-form solve on `s` (inputs copied in, the graph, the
// iterate copied out, the device scalars copied to the pinned host block);
// pcg_graph_finish waits for it.  Only one solve per hierarchy may be in flight.
static int report_from_scal(amg_hierarchy *h, const double *sc, float ms, solve_info *info);

static int pcg_graph_launch(amg_hierarchy *h, const double *f_dev, double *x_dev, int warm,
                            const solve_options *o, cudaStream_t s)
{
    const size_t bytes = sizeof(double) * 2 * (size_t)h->lev[0].N;
    if (!h->ev_solve[0]) {
        BD_CUDA(cudaEventCreate(&h->ev_solve[0]));
        BD_CUDA(cudaEventCreate(&h->ev_solve[1]));
    }
    BD_CUDA(cudaEventRecord(h->ev_solve[0], s));
    if (f_dev != h->fin.p) BD_CUDA(cudaMemcpyAsync(h->fin.p, f_dev, bytes, cudaMemcpyDeviceToDevice, s));
    if (warm && x_dev != h->x.p) BD_CUDA(cudaMemcpyAsync(h->x.p, x_dev, bytes, cudaMemcpyDeviceToDevice, s));
    for (int i = 0; i < S_NSLOTS; i++) h->host_init[i] = 0.0;
    h->host_init[S_RTOL] = o->rtol;
    h->host_init[S_MAXIT] = (double)o->max_it;
    h->host_init[S_WARM] = warm ? 1.0 : 0.0;
    BD_CUDA(cudaMemcpyAsync(h->scal.p, h->host_init, sizeof(double) * S_NSLOTS, cudaMemcpyHostToDevice, s));
    BD_CUDA(cudaGraphLaunch(h->graph_exec, s));
    if (x_dev != h->x.p) BD_CUDA(cudaMemcpyAsync(x_dev, h->x.p, bytes, cudaMemcpyDeviceToDevice, s));
    BD_CUDA(cudaEventRecord(h->ev_solve[1], s));
    BD_CUDA(cudaMemcpyAsync(h->host_scal, h->scal.p, sizeof(double) * S_NSLOTS, cudaMemcpyDeviceToHost, s));
    return BD_OK;
}

static int pcg_graph_finish(amg_hierarchy *h, cudaStream_t s, solve_info *info)
{
    BD_CUDA(cudaStreamSynchronize(s));
    float ms = 0.0f;
    cudaEventElapsedTime(&ms, h->ev_solve[0], h->ev_solve[1]);
    return report_from_scal(h, h->host_scal, ms, info);
}

static int pcg_solve_graph(amg_hierarchy *h, const double *f_dev, double *x_dev, int warm,
                           const solve_options *o, cudaStream_t s, solve_info *info)
{
    BD_TRY(pcg_graph_launch(h, f_dev, x_dev, warm, o, s));
    return pcg_graph_finish(h, s, info);
}

static bool graph_form(amg_hierarchy *h, const solve_options *o)
{
    static const bool graph_off = [] {
        const char *e = getenv("BD_SOLVE_GRAPH");
        return e && e[0] == '0';
    }();
    if (h->prof || o->strict || h->graph_failed || graph_off) return false;
    if (!h->graph_exec && build_graph(h) != BD_OK) h->graph_failed = true;
    return h->graph_exec != nullptr;
}

// Split form for callers that overlap several hierarchies' solves: begin
// enqueues the solve (graph form) or runs it to completion (host-driven loop),
// end waits and reports.
int pcg_solve_begin(amg_hierarchy *h, const double *f_dev, double *x_dev, int warm,
                    const solve_options *o, cudaStream_t s, solve_info *info, bool *pending)
{
    if (graph_form(h, o)) {
        *pending = true;
        return pcg_graph_launch(h, f_dev, x_dev, warm, o, s);
    }
    *pending = false;
    return pcg_solve_loop(h, f_dev, x_dev, warm, o, s, info);
}

int pcg_solve_end(amg_hierarchy *h, cudaStream_t s, solve_info *info) { return pcg_graph_finish(h, s, info); }

// The graph form unless live kernel timing is on (its CUDA events bracket
// single launches), strict mode is requested (checked on the host before the
// loop), the graph could not be built, or BD_SOLVE_GRAPH=0 is set.
int pcg_solve_device(amg_hierarchy *h, const double *f_dev, double *x_dev, int warm,
                     const solve_options *o, cudaStream_t s, solve_info *info)
{
    if (graph_form(h, o)) return pcg_solve_graph(h, f_dev, x_dev, warm, o, s, info);
    return pcg_solve_loop(h, f_dev, x_dev, warm, o, s, info);
}

// Report of one solve from its scalar block (graph form): status, iterations,
// residuals; counts its kernel executions.
static int report_from_scal(amg_hierarchy *h, const double *sc, float ms, solve_info *info)
{
    const double nf = sqrt(sc[S_NF2]);
    const int status = (int)sc[S_STATUS];
    note_launches(h->graph_pre + h->graph_post + (long long)sc[S_IT] * h->graph_body);
    if (info) {
        info->status = status;
        info->iters = (int)sc[S_IT];
        info->rel_res = nf > 0.0 ? sqrt(sc[S_RR]) / nf : 0.0;
        info->true_rel_res = nf > 0.0 ? sqrt(sc[S_TRR]) / nf : 0.0;
        info->solve_ms = ms;
    }
    return status;
}

// ------------------------------------------------------------------ batched solves
// Many independent solves as one CUDA graph: branch k copies f_k and x_k into
// hierarchy k's buffers, runs its whole solve (capture_solve) and copies x and
// the scalar block back; the branches have no edges between them, so one
// launch runs all of them concurrently on the GPU.
struct BatchGraph {
    std::vector<amg_hierarchy *> h;
    std::vector<const double *> f;
    std::vector<double *> x;
    std::vector<cudaStream_t> st;
    std::vector<cudaEvent_t> join;
    cudaStream_t origin = nullptr, body = nullptr;
    cudaEvent_t fork = nullptr, ev[2] = {nullptr, nullptr};
    cudaGraph_t graph = nullptr;
    cudaGraphExec_t exec = nullptr;
    DBuf<double> init_dev;          // count x S_NSLOTS initial scalar blocks
    double *host_init = nullptr;    // pinned, count x S_NSLOTS
    double *host_scal = nullptr;    // pinned, count x S_NSLOTS (results)

    void drop_graph()
    {
        if (exec) cudaGraphExecDestroy(exec);
        if (graph) cudaGraphDestroy(graph);
        exec = nullptr;
        graph = nullptr;
    }
    ~BatchGraph()
    {
        drop_graph();
        for (cudaStream_t q : st) cudaStreamDestroy(q);
        for (cudaEvent_t e : join) cudaEventDestroy(e);
        if (origin) cudaStreamDestroy(origin);
        if (body) cudaStreamDestroy(body);
        if (fork) cudaEventDestroy(fork);
        if (ev[0]) cudaEventDestroy(ev[0]);
        if (ev[1]) cudaEventDestroy(ev[1]);
        if (host_init) cudaFreeHost(host_init);
        if (host_scal) cudaFreeHost(host_scal);
    }
};

static int batch_capture(BatchGraph &b)
{
    const int count = (int)b.h.size();
    BD_CUDA(cudaStreamBeginCapture(b.origin, cudaStreamCaptureModeThreadLocal));
    BD_CUDA(cudaEventRecord(b.fork, b.origin));
    for (int k = 0; k < count; k++) {
        amg_hierarchy *h = b.h[k];
        cudaStream_t s = b.st[k];
        const size_t bytes = sizeof(double) * 2 * (size_t)h->lev[0].N;
        BD_CUDA(cudaStreamWaitEvent(s, b.fork, 0));
        BD_CUDA(cudaMemcpyAsync(h->scal.p, b.init_dev.p + (size_t)k * S_NSLOTS, sizeof(double) * S_NSLOTS,
                                cudaMemcpyDeviceToDevice, s));
        BD_CUDA(cudaMemcpyAsync(h->fin.p, b.f[k], bytes, cudaMemcpyDeviceToDevice, s));
        BD_CUDA(cudaMemcpyAsync(h->x.p, b.x[k], bytes, cudaMemcpyDeviceToDevice, s));
        BD_TRY(capture_solve(h, s, b.body));
        BD_CUDA(cudaMemcpyAsync(b.x[k], h->x.p, bytes, cudaMemcpyDeviceToDevice, s));
        BD_CUDA(cudaMemcpyAsync(b.host_scal + (size_t)k * S_NSLOTS, h->scal.p, sizeof(double) * S_NSLOTS,
                                cudaMemcpyDeviceToHost, s));
        BD_CUDA(cudaEventRecord(b.join[k], s));
        BD_CUDA(cudaStreamWaitEvent(b.origin, b.join[k], 0));
    }
    BD_CUDA(cudaStreamEndCapture(b.origin, &b.graph));
    BD_CUDA(cudaGraphInstantiate(&b.exec, b.graph, 0));
    return BD_OK;
}

}  // namespace bd

using namespace bd;

struct amg_batch {
    bd::BatchGraph g;
};

extern "C" int amg_batch_create(amg_hierarchy *const *h, int count, amg_batch **out)
{
    if (!out) return BD_EINVAL;
    *out = nullptr;
    if (!h || count < 1) return BD_EINVAL;
    for (int k = 0; k < count; k++) {
        if (!h[k]) return BD_EINVAL;
        for (int j = 0; j < k; j++)
            if (h[j] == h[k]) return BD_EINVAL;  // one hierarchy's buffers serve one branch
    }
    amg_batch *b = new (std::nothrow) amg_batch();
    if (!b) return BD_ENOMEM;
    BatchGraph &g = b->g;
    g.h.assign(h, h + count);
    int st = BD_OK;
    auto ok = [&](cudaError_t e) {
        if (e != cudaSuccess && st == BD_OK) st = BD_ECUDA;
    };
    ok(cudaStreamCreateWithFlags(&g.origin, cudaStreamNonBlocking));
    ok(cudaStreamCreateWithFlags(&g.body, cudaStreamNonBlocking));
    ok(cudaEventCreateWithFlags(&g.fork, cudaEventDisableTiming));
    ok(cudaEventCreate(&g.ev[0]));
    ok(cudaEventCreate(&g.ev[1]));
    g.st.assign(count, nullptr);
    g.join.assign(count, nullptr);
    for (int k = 0; k < count && st == BD_OK; k++) {
        ok(cudaStreamCreateWithFlags(&g.st[k], cudaStreamNonBlocking));
        ok(cudaEventCreateWithFlags(&g.join[k], cudaEventDisableTiming));
    }
    const size_t nsc = (size_t)count * S_NSLOTS;
    if (st == BD_OK) st = g.init_dev.alloc(nsc);
    if (st == BD_OK) ok(cudaMallocHost((void **)&g.host_init, sizeof(double) * nsc));
    if (st == BD_OK) ok(cudaMallocHost((void **)&g.host_scal, sizeof(double) * nsc));
    if (st != BD_OK) {
        delete b;
        return st;
    }
    for (amg_hierarchy *hk : g.h) hk->batch_refs++;
    *out = b;
    return BD_OK;
}

extern "C" int amg_batch_solve(amg_batch *b, const double *const *f, double *const *x, const solve_options *opts,
                               void *stream, solve_info *info)
{
    if (!b || !f || !x) return BD_EINVAL;
    BatchGraph &g = b->g;
    const int count = (int)g.h.size();
    solve_options o;
    solve_options_default(&o);
    if (opts) o = *opts;
    if (!(o.rtol > 0.0) || o.max_it < 0 || o.strict) return BD_EINVAL;
    for (int k = 0; k < count; k++)
        if (!f[k] || !x[k]) return BD_EINVAL;
    // the graph is tied to the vectors it copies from and to
    bool same = g.exec != nullptr;
    for (int k = 0; k < count && same; k++) same = g.f[k] == f[k] && g.x[k] == x[k];
    if (!same) {
        g.drop_graph();
        g.f.assign(f, f + count);
        g.x.assign(x, x + count);
        const int st = batch_capture(g);
        if (st != BD_OK) {
            end_capture_quietly(g.body);
            for (cudaStream_t q : g.st) end_capture_quietly(q);
            end_capture_quietly(g.origin);
            g.drop_graph();
            return st;
        }
    }
    cudaStream_t s = (cudaStream_t)stream;
    for (int k = 0; k < count; k++) {
        double *hi = g.host_init + (size_t)k * S_NSLOTS;
        for (int i = 0; i < S_NSLOTS; i++) hi[i] = 0.0;
        hi[S_RTOL] = o.rtol;
        hi[S_MAXIT] = (double)o.max_it;
        hi[S_WARM] = o.warm_start ? 1.0 : 0.0;
    }
    BD_CUDA(cudaMemcpyAsync(g.init_dev.p, g.host_init, sizeof(double) * count * S_NSLOTS,
                            cudaMemcpyHostToDevice, s));
    BD_CUDA(cudaEventRecord(g.ev[0], s));
    BD_CUDA(cudaGraphLaunch(g.exec, s));
    BD_CUDA(cudaEventRecord(g.ev[1], s));
    BD_CUDA(cudaStreamSynchronize(s));
    float ms = 0.0f;
    cudaEventElapsedTime(&ms, g.ev[0], g.ev[1]);
    int worst = BD_OK;
    for (int k = 0; k < count; k++) {
        const int stk = report_from_scal(g.h[k], g.host_scal + (size_t)k * S_NSLOTS, ms, info ? info + k : nullptr);
        if (stk != BD_OK && worst == BD_OK) worst = stk;
    }
    return worst;
}

extern "C" void amg_batch_destroy(amg_batch *b)
{
    if (!b) return;
    for (amg_hierarchy *hk : b->g.h) hk->batch_refs--;
    delete b;
}

extern "C" int amg_set_level_lanes(amg_hierarchy *h, int level, const int lanes[3], void *stream)
{
    if (!h || !lanes || level < 0 || level >= h->nlev) return BD_EINVAL;
    if (h->batch_refs > 0) return BD_ESTATE;
    Level &L = h->lev[level];
    const bool last = level == h->nlev - 1;
    for (int op = 0; op < 3; op++) {
        const int T = lanes[op];
        if (T == 0) continue;
        const bool applied = !last && !(op == 0 && level == 0 && h->sell.valid);
        const bool csr_ok = T > 0 && T <= 256 && (T & (T - 1)) == 0;
        const bool sliced_ok = T < 0 && sliced_k_ok(-T) && !(op == 0 && level == 0);
        if (!applied || !(csr_ok || sliced_ok)) return BD_EINVAL;
    }
    cudaStream_t s = (cudaStream_t)stream;
    BD_CUDA(cudaStreamSynchronize(s));
    // The captured whole-solve graph holds the old launches and buffers: drop
    // it before any buffer changes, so that no error return below leaves a
    // graph that reads freed or rebuilt memory (the next solve captures anew).
    if (h->graph_exec) cudaGraphExecDestroy(h->graph_exec);
    if (h->graph) cudaGraphDestroy(h->graph);
    h->graph_exec = nullptr;
    h->graph = nullptr;
    h->graph_failed = false;
    for (int op = 0; op < 3; op++) {
        const int T = lanes[op];
        if (T == 0) continue;
        const BSR &M = op == 0 ? L.A : (op == 1 ? L.R : L.P);
        if (T < 0) {
            const int rc = build_sliced(M, -T, h->prec32, L.sl[op], s);
            if (rc != BD_OK) {
                // a half-built sliced form is unusable: fall back to the
                // block-CSR form the rule gives, which needs no extra buffers
                drop_sliced(L.sl[op]);
                L.lanes[op] = lanes_for(M, h->prec32);
                return rc;
            }
        } else {
            drop_sliced(L.sl[op]);
        }
        L.lanes[op] = T;
    }
    return BD_OK;
}

extern "C" int amg_vcycle(amg_hierarchy *h, const double *r, double *z, int on_device, void *stream)
{
    if (!h || !r || !z) return BD_EINVAL;
    cudaStream_t s = (cudaStream_t)stream;
    size_t bytes = sizeof(double) * 2 * (size_t)h->lev[0].N;
    if (on_device) {
        BD_TRY(vcycle_device(h, r, z, s));
        BD_CUDA(cudaStreamSynchronize(s));
        prof_collect(h);
        return BD_OK;
    }
    BD_TRY(copy_in(h->r.p, r, bytes, 0, s));
    BD_TRY(vcycle_device(h, h->r.p, h->z.p, s));
    BD_TRY(copy_out(z, h->z.p, bytes, 0, s));
    BD_CUDA(cudaStreamSynchronize(s));
    prof_collect(h);
    return BD_OK;
}

extern "C" int amg_profile_enable(amg_hierarchy *h, int enable)
{
    if (!h || enable < 0 || enable > 2) return BD_EINVAL;
    prof_collect(h);
    if (enable && !h->prof) {  // fresh sums when switched on
        h->prof_sum = amg_kernel_profile{};
        for (int i = 0; i < 256; i++) {
            h->trace_ms[i] = 0.0;
            h->trace_n[i] = 0;
        }
    }
    h->prof = enable;
    return BD_OK;
}

extern "C" int amg_profile_breakdown(const amg_hierarchy *h, double *ms, long long *count)
{
    if (!h || !ms || !count) return BD_EINVAL;
    for (int i = 0; i < 256; i++) {
        ms[i] = h->trace_ms[i];
        count[i] = h->trace_n[i];
    }
    return BD_OK;
}

extern "C" int amg_profile_read(const amg_hierarchy *h, amg_kernel_profile *out)
{
    if (!h || !out) return BD_EINVAL;
    *out = h->prof_sum;
    out->precision = h->prec32 ? 1 : 0;
    return BD_OK;
}

extern "C" int amg_solve(amg_hierarchy *h, const double *f, double *x, int on_device,
                         const solve_options *opts, void *stream, solve_info *info)
{
    if (!h || !f || !x) return BD_EINVAL;
    solve_options o;
    solve_options_default(&o);
    if (opts) o = *opts;
    if (!(o.rtol > 0.0) || o.max_it < 0) return BD_EINVAL;
    cudaStream_t s = (cudaStream_t)stream;
    size_t bytes = sizeof(double) * 2 * (size_t)h->lev[0].N;
    if (on_device) return pcg_solve_device(h, f, x, o.warm_start, &o, s, info);
    // host arrays: f and x are staged in device buffers
    DBuf<double> fdev;
    BD_TRY(fdev.alloc(2 * (size_t)h->lev[0].N));
    BD_TRY(copy_in(fdev.p, f, bytes, 0, s));
    if (o.warm_start) BD_TRY(copy_in(h->x.p, x, bytes, 0, s));
    int st = pcg_solve_device(h, fdev.p, h->x.p, o.warm_start, &o, s, info);
    BD_TRY(copy_out(x, h->x.p, bytes, 0, s));
    BD_CUDA(cudaStreamSynchronize(s));
    return st;
}
