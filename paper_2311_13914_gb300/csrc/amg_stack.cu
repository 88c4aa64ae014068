// amg_stack.cu -- the stacked batch (many hierarchies solved together).
//
// Level l of a stack holds level l of every member hierarchy that has one,
// the members' operators placed block-diagonally and their vectors end to
// end, so each step of the V-cycle (Algorithm 2: Chebyshev pre-smoothing,
// residual, restriction, coarsest solve, prolongation, post-smoothing) is one
// kernel launch over all members instead of one launch per member.  Within a
// level the members that smooth there come first (rows [0, Ns)), the members
// whose coarsest level it is follow; their dense solves run together in one
// launch (one thread block per member).  The projected PCG of Section 2.2
// keeps its scalars per member (null-space means, alpha, beta, residual norm,
// the stopping test): every reduction runs over chunks of at most kStChunk
// nodes that never span two members, and the last block to finish adds each
// member's chunk sums in chunk order, so the result does not depend on
// scheduling.  One CUDA graph per batch solve: the iteration body under a
// WHILE node whose condition the last reduction of an iteration sets on the
// device (some member still iterating); members that have converged, broken
// down or reached max_it keep their iterate.
#include <algorithm>
#include <cmath>
#include <new>
#include <type_traits>
#include <vector>

#include "amg_bsr.cuh"
#include "amg_internal.cuh"

namespace bd {
namespace {

constexpr int kStChunk = 1024;   // nodes per reduction chunk
constexpr int kStThreads = 256;  // threads of the reduction and vector kernels

// per-member device scalars
enum {
    T_MEANF = 0, T_NF2, T_RR, T_RZ, T_PQ, T_ALPHA, T_BETA, T_MEANZ, T_BREAK, T_IT, T_STATUS,
    T_ACTIVE, T_TRR, T_MEANX, T_RTOL, T_MAXIT, T_WARM, T_NSLOTS
};

// node -> member, and each member's Chebyshev coefficients on one level:
// coef[4k] = 1/theta, coef[4k+1] = c1, coef[4k+2] = c2, coef[4k+3] = 1 + c1
struct StCoef {
    const int *__restrict__ mem;
    const double *__restrict__ coef;
    __device__ __forceinline__ const double *at(int p) const { return coef + 4 * mem[p]; }
};

template <class S> struct StGather {
    const v2<S> *__restrict__ x;
    __device__ __forceinline__ v2<S> operator()(int q) const { return x[q]; }
};

// Epilogues of the stacked V-cycle: the single-hierarchy Chebyshev steps
// (Saad, Alg. 12.1 on D^{-1}A, degree 2) with the coefficients of the row's
// member.
template <class S> struct StPre {  // from zero: u = d0 + (c1 d0 + c2 D^{-1} (f - A d0))
    const v2<S> *__restrict__ f;
    const v2<S> *__restrict__ invd;
    const v2<S> *__restrict__ d0;
    v2<S> *__restrict__ u;
    StCoef c;
    __device__ __forceinline__ void operator()(int p, S y0, S y1) const
    {
        const double *k = c.at(p);
        const S c1 = (S)k[1], c2 = (S)k[2];
        const v2<S> fp = f[p], id = invd[p], dp = d0[p];
        const S r0 = fp.x - y0, r1 = fp.y - y1;
        u[p] = V2<S>::mk(dp.x + (c1 * dp.x + c2 * id.x * r0), dp.y + (c1 * dp.y + c2 * id.y * r1));
    }
};
template <class S> struct StResid {  // r = f - A u
    const v2<S> *__restrict__ f;
    v2<S> *__restrict__ r;
    __device__ __forceinline__ void operator()(int p, S y0, S y1) const
    {
        const v2<S> fp = f[p];
        r[p] = V2<S>::mk(fp.x - y0, fp.y - y1);
    }
};
template <class S> struct StStoreD0 {  // f_c = R r and d0_c = D_c^{-1} f_c / theta_c
    v2<S> *__restrict__ f;
    v2<S> *__restrict__ d0;
    const v2<S> *__restrict__ invd;
    StCoef c;
    __device__ __forceinline__ void operator()(int p, S y0, S y1) const
    {
        const S it = (S)c.at(p)[0];
        const v2<S> id = invd[p];
        f[p] = V2<S>::mk(y0, y1);
        d0[p] = V2<S>::mk(y0 * id.x * it, y1 * id.y * it);
    }
};
template <class S> struct StAdd {  // u += P e_c
    v2<S> *__restrict__ u;
    __device__ __forceinline__ void operator()(int p, S y0, S y1) const
    {
        const v2<S> a = u[p];
        u[p] = V2<S>::mk(a.x + y0, a.y + y1);
    }
};
template <class S> struct StPost1 {  // r = f - A u, d = D^{-1} r / theta, w = u + d
    const v2<S> *__restrict__ f;
    const v2<S> *__restrict__ invd;
    const v2<S> *__restrict__ u;
    v2<S> *__restrict__ r;
    v2<S> *__restrict__ d;
    v2<S> *__restrict__ w;
    StCoef c;
    __device__ __forceinline__ void operator()(int p, S y0, S y1) const
    {
        const S it = (S)c.at(p)[0];
        const v2<S> fp = f[p], id = invd[p], up = u[p];
        const S r0 = fp.x - y0, r1 = fp.y - y1;
        const S d0 = r0 * id.x * it, d1 = r1 * id.y * it;
        r[p] = V2<S>::mk(r0, r1);
        d[p] = V2<S>::mk(d0, d1);
        w[p] = V2<S>::mk(up.x + d0, up.y + d1);
    }
};
template <class S> struct StPost2 {  // u = w + (c1 d + c2 D^{-1} (r - A d))
    const v2<S> *__restrict__ r;
    const v2<S> *__restrict__ d;
    const v2<S> *__restrict__ invd;
    const v2<S> *__restrict__ w;
    v2<S> *__restrict__ u;
    StCoef c;
    __device__ __forceinline__ void operator()(int p, S y0, S y1) const
    {
        const double *k = c.at(p);
        const S c1 = (S)k[1], c2 = (S)k[2];
        const v2<S> rp_ = r[p], dp = d[p], id = invd[p], wp = w[p];
        const S r0 = rp_.x - y0, r1 = rp_.y - y1;
        u[p] = V2<S>::mk(wp.x + (c1 * dp.x + c2 * id.x * r0), wp.y + (c1 * dp.y + c2 * id.y * r1));
    }
};
struct StStore {  // q = A p (FP64, PCG)
    double2 *__restrict__ q;
    __device__ __forceinline__ void operator()(int p, double y0, double y1) const { q[p] = make_double2(y0, y1); }
};

// The FP64 finest level's steps with the vectors its operator gathers (d0, u,
// d, w) kept in (v + u, u) form and the inverse diagonal scaled per member
// (idc2 = c2 D^{-1}, idt = D^{-1} / theta), as the single hierarchy's FP64
// finest level does them: 2 FMA per stored node pair instead of 3 operations.
// Pre-smoothing from zero with m = idc2 (f - A d0): u_s = (1 + c1) d0_s + (m_v
// + m_u), u_u = (1 + c1) d0_u + m_u.
struct StPreX {
    const double2 *__restrict__ f;
    const double2 *__restrict__ idc2;
    const double2 *__restrict__ d0;  // (v + u, u)
    double2 *__restrict__ u;         // (v + u, u)
    StCoef c;
    __device__ __forceinline__ void operator()(int p, double y0, double y1) const
    {
        const double c1p = c.at(p)[3];
        const double2 fp = f[p], k = idc2[p], dp = d0[p];
        const double m0 = k.x * (fp.x - y0), m1 = k.y * (fp.y - y1);
        u[p] = make_double2(fma(c1p, dp.x, m0 + m1), fma(c1p, dp.y, m1));
    }
};
struct StAddX {  // u += P e_c with u in (v + u, u) form
    double2 *__restrict__ u;
    __device__ __forceinline__ void operator()(int p, double y0, double y1) const
    {
        const double2 a = u[p];
        u[p] = make_double2(a.x + (y0 + y1), a.y + y1);
    }
};
// r = f - A u (plain), d = D^{-1} r / theta and w = u + d in (v + u, u) form
struct StPost1X {
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
// u = w + (c1 d + c2 D^{-1} (r - A d)) in plain (v, u) form (the V-cycle's
// output) from w and d in (v + u, u) form
struct StPost2X {
    const double2 *__restrict__ r;
    const double2 *__restrict__ d;  // (v + u, u)
    const double2 *__restrict__ idc2;
    const double2 *__restrict__ w;  // (v + u, u)
    double2 *__restrict__ u;
    StCoef c;
    __device__ __forceinline__ void operator()(int p, double y0, double y1) const
    {
        const double c1 = c.at(p)[1];
        const double2 rp_ = r[p], dp = d[p], k = idc2[p], wp = w[p];
        const double m0 = k.x * (rp_.x - y0), m1 = k.y * (rp_.y - y1);
        const double uu = wp.y + fma(c1, dp.y, m1);
        const double us = wp.x + fma(c1, dp.x, m0 + m1);
        u[p] = make_double2(us - uu, uu);
    }
};

// Finest level of the stack in sliced ELL with the shared Ki/Ke pattern of
// the Bidomain operator (every member's own slices, its rows padded to whole
// 32-row slices; padded rows, member -1, are skipped): one thread per row,
// slot j of a slice holds entry j of its 32 rows; per node pair
// a += Ki (v_q + u_q), b += Ke u_q, then y_v = c M_p v_p + a, y_u = a + b.
// SU: the gathered vector is stored as (v + u, u), so a node pair costs two
// FMAs and the row's own v is recovered once.
template <class S, class E, bool SU = false>
__global__ void __launch_bounds__(256) k_st_sell(int rows, const int *__restrict__ mem, const int *__restrict__ sptr,
                                                 const int *__restrict__ col, const v2<S> *__restrict__ kk,
                                                 const S *__restrict__ cm, StGather<S> g, E epi)
{
    for (int p = blockIdx.x * blockDim.x + threadIdx.x; p < rows; p += gridDim.x * blockDim.x) {
        if (mem[p] < 0) continue;
        const int sl = p >> 5, lane = p & 31, j1 = sptr[sl + 1];
        S a = 0, b = 0;
#pragma unroll 4
        for (int j = sptr[sl]; j < j1; j++) {
            const size_t idx = (size_t)j * 32 + lane;
            const v2<S> k = kk[idx];
            const v2<S> x = g(col[idx]);
            a = fma(k.x, SU ? x.x : x.x + x.y, a);
            b = fma(k.y, x.y, b);
        }
        const v2<S> xp = g(p);
        epi(p, fma(cm[p], SU ? xp.x - xp.y : xp.x, a), a + b);
    }
}

// The same for a large FP64 level, as the single hierarchy's finest level runs
// it: one block of 1024 threads per SM, each block an equal contiguous share of
// the 32-row slices (the stack's rows are whole slices), rows unrolled deeper
// with the registers one block per SM leaves.
template <class S, class E, bool SU>
__global__ void __launch_bounds__(1024, 1) k_st_sell_wide(int rows, const int *__restrict__ mem,
                                                          const int *__restrict__ sptr, const int *__restrict__ col,
                                                          const v2<S> *__restrict__ kk, const S *__restrict__ cm,
                                                          StGather<S> g, E epi)
{
    const long long nsl = ((long long)rows + 31) >> 5;
    const int lo = (int)(nsl * blockIdx.x / gridDim.x) * 32;
    const int hi = min(rows, (int)(nsl * (blockIdx.x + 1) / gridDim.x) * 32);
    for (int p = lo + threadIdx.x; p < hi; p += blockDim.x) {
        if (mem[p] < 0) continue;
        const int sl = p >> 5, lane = p & 31, j1 = sptr[sl + 1];
        S a = 0, b = 0;
#pragma unroll 8
        for (int j = sptr[sl]; j < j1; j++) {
            const size_t idx = (size_t)j * 32 + lane;
            const v2<S> k = kk[idx];
            const v2<S> x = g(col[idx]);
            a = fma(k.x, SU ? x.x : x.x + x.y, a);
            b = fma(k.y, x.y, b);
        }
        const v2<S> xp = g(p);
        epi(p, fma(cm[p], SU ? xp.x - xp.y : xp.x, a), a + b);
    }
}

// ------------------------------------------------------------------ assembly of the stack
__global__ void k_st_shift(long long n, const int *__restrict__ src, int *__restrict__ dst, int add)
{
    for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x)
        dst[i] = src[i] + add;
}
__global__ void k_st_fill(long long n, int *__restrict__ dst, int v)
{
    for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x)
        dst[i] = v;
}
__global__ void k_st_set(int *dst, int v) { *dst = v; }

// ------------------------------------------------------------------ coarsest levels
struct StCoarseJob {
    const double *cinv;  // n x n dense inverse of the member's rank-one-fixed coarsest operator
    const double *z;     // its null vector
    double zz;           // z . z
    int n;               // unknowns
    int level;           // stack level holding the member's coarsest level
    long long off;       // first unknown of the member on that level
};
template <class S> struct StLevelPtrs {
    S *f[kMaxLevels];
    S *u[kMaxLevels];
};

// x = Cinv (r - (z.r / z.z) z) in FP64 for every member at once (block k:
// member k's coarsest level), as the single-hierarchy coarsest solve.
template <class S>
__global__ void __launch_bounds__(512) k_st_coarse(const StCoarseJob *__restrict__ jobs, StLevelPtrs<S> lp)
{
    extern __shared__ double rs[];
    __shared__ double red[32];
    const StCoarseJob J = jobs[blockIdx.x];
    const S *r = lp.f[J.level] + J.off;
    S *x = lp.u[J.level] + J.off;
    const int n = J.n;
    double part = 0.0;
    for (int i = threadIdx.x; i < n; i += blockDim.x) part += J.z[i] * (double)r[i];
    for (int o = 16; o; o >>= 1) part += __shfl_xor_sync(0xffffffffu, part, o);
    if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = part;
    __syncthreads();
    if (threadIdx.x < 32) {
        double v = threadIdx.x < (blockDim.x >> 5) ? red[threadIdx.x] : 0.0;
        for (int o = 16; o; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
        if (threadIdx.x == 0) red[0] = v;
    }
    __syncthreads();
    const double a = J.zz > 0.0 ? red[0] / J.zz : 0.0;
    for (int i = threadIdx.x; i < n; i += blockDim.x) rs[i] = (double)r[i] - a * J.z[i];
    __syncthreads();
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nw = blockDim.x >> 5;
    for (int i = warp; i < n; i += nw) {
        const double *row = J.cinv + (size_t)i * n;
        double s = 0.0;
        for (int j = lane; j < n; j += 32) s += row[j] * rs[j];
        for (int o = 16; o; o >>= 1) s += __shfl_xor_sync(0xffffffffu, s, o);
        if (lane == 0) x[i] = (S)s;
    }
}

// ------------------------------------------------------------------ PCG reductions
// Context of the per-member reductions on the finest level.
struct StRed {
    double *scal;                  // count x T_NSLOTS
    double *part;                  // chunks x 4
    unsigned int *counter;
    const int *cmem, *cbeg, *cend; // member and node range of each chunk
    const int *mc0, *mc1;          // chunk range of each member
    const int *nn;                 // finest-level nodes of each member
    int count, flex;
    cudaGraphConditionalHandle cond;
};

// Vectors of the finest level (FP64 PCG vectors in (v, u) pairs; the V-cycle's
// input f0, d0 and output u0 in its precision S).
template <class S> struct StPcg {
    const double2 *fin;
    double2 *fp, *x, *r, *z, *p, *q, *zold;
    v2<S> *f0, *d0;
    const v2<S> *u0, *invd0;
    StCoef c0;
    const int *mem;                // finest-level node -> member
    int psu;                       // p stored as (v + u, u) (sliced-ELL finest level)
    int dsu;                       // FP64 V-cycle: d0 stored as (v + u, u)
};

enum { R_FSTATS = 0, R_PROJF, R_INIT, R_ZSTATS, R_PQ, R_XR, R_TRUE };

// V-cycle input from the residual: f0 = r (FP32 copy; the FP64 V-cycle reads
// r itself) and d0 = D^{-1} r / theta.
template <class S>
__device__ __forceinline__ void st_vin(const StPcg<S> &v, int i, double2 ri)
{
    const double it = v.c0.at(i)[0];
    if (sizeof(S) == 4) v.f0[i] = V2<S>::mk((S)ri.x, (S)ri.y);
    const v2<S> id = v.invd0[i];
    const S itS = (S)it;
    const S dv = (S)ri.x * id.x * itS, du = (S)ri.y * id.y * itS;
    v.d0[i] = V2<S>::mk(v.dsu ? dv + du : dv, du);
}

// Per-member totals -> scalars (last block, one thread per member).  Returns
// whether the member keeps iterating (stages that open or close an iteration).
__device__ bool st_finish(int MODE, const StRed &R, int k, double a, double b, double c, double d)
{
    double *sc = R.scal + (size_t)k * T_NSLOTS;
    const double N = (double)R.nn[k];
    switch (MODE) {
    case R_FSTATS:
        sc[T_MEANF] = a / N;
        return false;
    case R_PROJF:
        sc[T_NF2] = a;
        return false;
    case R_INIT: {
        sc[T_RR] = a;
        const double nf = sqrt(sc[T_NF2]);
        const bool go = nf > 0.0 && !(sqrt(a) <= sc[T_RTOL] * nf) && sc[T_MAXIT] > 0.0;
        sc[T_IT] = 0.0;
        sc[T_BREAK] = 0.0;
        sc[T_STATUS] = go ? (double)BD_ENOTCONV : (double)BD_OK;
        sc[T_ACTIVE] = go ? 1.0 : 0.0;
        return go;
    }
    case R_ZSTATS: {
        if (sc[T_ACTIVE] == 0.0) return false;
        const double mz = a / N, rz = c - mz * b;  // r . (z projected)
        const double num = R.flex ? rz - d : rz;   // flexible (Polak-Ribiere) or standard beta
        sc[T_MEANZ] = mz;
        sc[T_BETA] = sc[T_IT] == 0.0 ? 0.0 : num / sc[T_RZ];
        sc[T_RZ] = rz;
        return false;
    }
    case R_PQ: {
        if (sc[T_ACTIVE] == 0.0) return false;
        sc[T_PQ] = a;
        if (!(a > 0.0) || !isfinite(a) || !isfinite(sc[T_RZ])) sc[T_BREAK] = 1.0;
        sc[T_ALPHA] = sc[T_RZ] / a;
        return false;
    }
    case R_XR: {
        if (sc[T_ACTIVE] == 0.0) return false;
        sc[T_RR] = a;
        const double it = sc[T_IT] + 1.0;
        sc[T_IT] = it;
        const double nf = sqrt(sc[T_NF2]), rr = sqrt(a);
        bool go = true;
        if (sc[T_BREAK] != 0.0 || !isfinite(rr)) {
            sc[T_STATUS] = (double)BD_EBREAKDOWN;
            go = false;
        } else if (rr <= sc[T_RTOL] * nf) {
            sc[T_STATUS] = (double)BD_OK;
            go = false;
        } else if (it >= sc[T_MAXIT]) {
            go = false;  // status stays BD_ENOTCONV
        }
        sc[T_ACTIVE] = go ? 1.0 : 0.0;
        return go;
    }
    case R_TRUE:
        sc[T_TRR] = a;
        sc[T_MEANX] = b / N;
        return false;
    }
    return false;
}

// One block per chunk: the chunk's sums (in a fixed order: every thread's
// nodes ascending, then warp k adds column k of the block's values) go to
// part[chunk]; the last block to arrive adds each member's chunks in chunk
// order and applies the stage.  Element-wise work of the stage rides along.
template <int MODE, class S>
__global__ void __launch_bounds__(kStThreads) k_st_red(StRed R, StPcg<S> v)
{
    constexpr int NV = (MODE == R_ZSTATS) ? 4 : ((MODE == R_TRUE) ? 2 : 1);
    __shared__ double buf[NV][kStThreads];
    __shared__ double tot[4];
    __shared__ bool last;
    const int c = blockIdx.x;
    const int m = R.cmem[c];
    const double *sc = R.scal + (size_t)m * T_NSLOTS;
    double acc[4] = {0.0, 0.0, 0.0, 0.0};
    const int b = R.cbeg[c], e = R.cend[c];
    if (MODE == R_FSTATS) {
        for (int i = b + threadIdx.x; i < e; i += blockDim.x) acc[0] += v.fin[i].y;
    } else if (MODE == R_PROJF) {
        const double mf = sc[T_MEANF];
        const bool warm = sc[T_WARM] != 0.0;
        for (int i = b + threadIdx.x; i < e; i += blockDim.x) {
            double2 f = v.fin[i];
            f.y -= mf;
            v.fp[i] = f;
            if (!warm) v.x[i] = make_double2(0.0, 0.0);
            acc[0] += f.x * f.x + f.y * f.y;
        }
    } else if (MODE == R_INIT) {  // q = A x already formed
        for (int i = b + threadIdx.x; i < e; i += blockDim.x) {
            const double2 f = v.fp[i], q = v.q[i];
            const double2 ri = make_double2(f.x - q.x, f.y - q.y);
            v.r[i] = ri;
            st_vin<S>(v, i, ri);
            acc[0] += ri.x * ri.x + ri.y * ri.y;
        }
    } else if (MODE == R_ZSTATS) {
        if (sc[T_ACTIVE] != 0.0) {
            for (int i = b + threadIdx.x; i < e; i += blockDim.x) {
                const v2<S> u = v.u0[i];
                const double2 zi = make_double2((double)u.x, (double)u.y), ri = v.r[i];
                v.z[i] = zi;
                acc[0] += zi.y;
                acc[1] += ri.y;
                acc[2] += ri.x * zi.x + ri.y * zi.y;
                if (R.flex) {
                    const double2 o = v.zold[i];
                    acc[3] += ri.x * o.x + ri.y * o.y;
                }
            }
        }
    } else if (MODE == R_PQ) {  // q = A p already formed
        if (sc[T_ACTIVE] != 0.0)
            for (int i = b + threadIdx.x; i < e; i += blockDim.x) {
                const double2 p = v.p[i], q = v.q[i];
                const double pv = v.psu ? p.x - p.y : p.x;
                acc[0] += pv * q.x + p.y * q.y;
            }
    } else if (MODE == R_XR) {
        if (sc[T_ACTIVE] != 0.0) {
            const double al = sc[T_ALPHA];
            for (int i = b + threadIdx.x; i < e; i += blockDim.x) {
                const double2 p = v.p[i], q = v.q[i];
                double2 xi = v.x[i], ri = v.r[i];
                xi.x += al * (v.psu ? p.x - p.y : p.x);
                xi.y += al * p.y;
                ri.x -= al * q.x;
                ri.y -= al * q.y;
                v.x[i] = xi;
                v.r[i] = ri;
                st_vin<S>(v, i, ri);
                acc[0] += ri.x * ri.x + ri.y * ri.y;
            }
        }
    } else if (MODE == R_TRUE) {  // q = A x of the final iterate
        for (int i = b + threadIdx.x; i < e; i += blockDim.x) {
            const double2 f = v.fp[i], q = v.q[i], xi = v.x[i];
            const double t0 = f.x - q.x, t1 = f.y - q.y;
            acc[0] += t0 * t0 + t1 * t1;
            acc[1] += xi.y;
        }
    }
    // block sums in a fixed order
#pragma unroll
    for (int k = 0; k < NV; k++) buf[k][threadIdx.x] = acc[k];
    __syncthreads();
    {
        const int w = threadIdx.x >> 5, l = threadIdx.x & 31;
        if (w < NV) {
            double t = buf[w][l];
            for (int i = l + 32; i < kStThreads; i += 32) t += buf[w][i];
            for (int o = 16; o; o >>= 1) t += __shfl_xor_sync(0xffffffffu, t, o);
            if (l == 0) tot[w] = t;
        }
    }
    __syncthreads();
    if (threadIdx.x == 0) {
        double *o = R.part + 4 * (size_t)c;
#pragma unroll
        for (int k = 0; k < NV; k++) o[k] = tot[k];
        __threadfence();
        const unsigned int ticket = atomicAdd(R.counter, 1u);
        last = ticket == gridDim.x - 1;
    }
    __syncthreads();
    if (!last) return;
    __threadfence();
    bool go = false;
    for (int k = threadIdx.x; k < R.count; k += blockDim.x) {
        double s[4] = {0.0, 0.0, 0.0, 0.0};
        for (int cc = R.mc0[k]; cc < R.mc1[k]; cc++) {
            const double *q = R.part + 4 * (size_t)cc;
#pragma unroll
            for (int j = 0; j < NV; j++) s[j] += __ldcg(q + j);
        }
        go |= st_finish(MODE, R, k, s[0], s[1], s[2], s[3]);
    }
    go = __syncthreads_or(go);
    if (threadIdx.x == 0) {
        if (MODE == R_INIT || MODE == R_XR) cudaGraphSetConditional(R.cond, go ? 1u : 0u);
        *R.counter = 0u;
    }
}

// z <- z - mean(z_u) e_u; p = z (first iteration) or z + beta p, stored in
// (v + u, u) form when psu; the projected z kept for the next flexible beta.
// Members no longer iterating keep p.
template <class S>
__global__ void k_st_p(int N, StPcg<S> v, const double *__restrict__ scal)
{
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < N; i += gridDim.x * blockDim.x) {
        const int m = v.mem[i];
        if (m < 0) continue;  // padding of a member's last 32-row slice
        const double *sc = scal + (size_t)m * T_NSLOTS;
        if (sc[T_ACTIVE] == 0.0) continue;
        double2 zi = v.z[i];
        zi.y -= sc[T_MEANZ];
        v.z[i] = zi;
        if (v.zold) v.zold[i] = zi;
        const double2 zs = v.psu ? make_double2(zi.x + zi.y, zi.y) : zi;
        if (sc[T_IT] == 0.0) {
            v.p[i] = zs;
        } else {
            const double beta = sc[T_BETA];
            const double2 pi = v.p[i];
            v.p[i] = make_double2(zs.x + beta * pi.x, zs.y + beta * pi.y);
        }
    }
}

// x <- x - mean(x_u) e_u (mean-zero u_e), or zero for a zero right-hand side.
__global__ void k_st_project_x(int N, double2 *__restrict__ x, const int *__restrict__ mem,
                               const double *__restrict__ scal)
{
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < N; i += gridDim.x * blockDim.x) {
        if (mem[i] < 0) continue;  // padding
        const double *sc = scal + (size_t)mem[i] * T_NSLOTS;
        double2 xi = x[i];
        if (!(sc[T_NF2] > 0.0)) xi = make_double2(0.0, 0.0);
        else xi.y -= sc[T_MEANX];
        x[i] = xi;
    }
}

}  // namespace

// ------------------------------------------------------------------ stack levels
struct StLevel {
    int N = 0;                 // nodes of the members present on this level
    int Ns = 0;                // nodes of the members that smooth here: rows [0, Ns)
    int rowsA = 0;             // rows of the stacked A (N on the finest level, Ns below)
    BSR A, R, P;               // FP64 values (A of the finest level always: the PCG's A p)
    DBuf<float> A32, R32, P32; // FP32 V-cycle values
    int lanes[3] = {0, 0, 0};
    DBuf<int> mem;             // member of each node
    DBuf<double> coef;         // 3 per member
    DBuf<double> f, u, r, d, w, invd;          // FP64 V-cycle (f unused on the finest level)
    DBuf<float> f32, u32, r32, d32, w32, invd32;
    // finest level only, when every member has its sliced-ELL finest level:
    // the members' slices end to end (columns shifted to the stack's nodes)
    bool sell = false;
    DBuf<int> ssptr, scol;
    DBuf<double> skk, scm;     // FP64 (the PCG's A p always; the FP64 V-cycle)
    DBuf<float> skk32, scm32;  // FP32 V-cycle
    // FP64 V-cycle on the sliced finest level: its gathered vectors in
    // (v + u, u) form, with the members' c2 D^{-1} and D^{-1} / theta
    bool su = false;
    DBuf<double> idc2, idt;
};

}  // namespace bd

using namespace bd;

struct amg_stack {
    int count = 0;
    bool p32 = false;
    int L = 0;                                // stack levels
    std::vector<amg_hierarchy *> h;
    StLevel lev[kMaxLevels];
    std::vector<int> nlev;                    // levels of each member
    std::vector<long long> off0;              // first node of each member on the finest level
    std::vector<int> n0;                      // finest-level nodes of each member
    DBuf<StCoarseJob> jobs;
    int max_nc = 0;
    // PCG on the finest level
    DBuf<double> fin, x, r, z, p, q, fp, zold;
    DBuf<int> cmem, cbeg, cend, mc0, mc1, nn;
    int nchunks = 0;
    DBuf<double> part, scal;
    DBuf<unsigned int> counter;
    double *host_init = nullptr, *host_scal = nullptr;
    // graph of one batch solve
    std::vector<const double *> gf;
    std::vector<double *> gx;
    cudaGraph_t graph = nullptr;
    cudaGraphExec_t exec = nullptr;
    cudaStream_t cap = nullptr, cap2 = nullptr;
    cudaEvent_t ev[2] = {nullptr, nullptr};
    long long n_pre = 0, n_body = 0, n_post = 0;

    void drop_graph()
    {
        if (exec) cudaGraphExecDestroy(exec);
        if (graph) cudaGraphDestroy(graph);
        exec = nullptr;
        graph = nullptr;
    }
    ~amg_stack()
    {
        drop_graph();
        if (cap) cudaStreamDestroy(cap);
        if (cap2) cudaStreamDestroy(cap2);
        if (ev[0]) cudaEventDestroy(ev[0]);
        if (ev[1]) cudaEventDestroy(ev[1]);
        if (host_init) cudaFreeHost(host_init);
        if (host_scal) cudaFreeHost(host_scal);
        for (amg_hierarchy *hk : h) hk->batch_refs--;
    }
};

namespace bd {
namespace {

// One member's block rows [0, nbr) of M appended to the stacked operator at
// row `row0` / block `blk0`, its columns shifted by `col0`.
int st_append(const BSR &M, int nbr, const float *v32, BSR &O, DBuf<float> *O32, int row0, long long blk0, int col0,
              bool fp64, cudaStream_t s)
{
    if (nbr <= 0) return BD_OK;
    int nb = 0;
    BD_CUDA(cudaMemcpyAsync(&nb, M.rp.p + nbr, sizeof(int), cudaMemcpyDeviceToHost, s));
    BD_CUDA(cudaStreamSynchronize(s));
    k_st_shift<<<grid_for(nbr, 256), 256, 0, s>>>(nbr, M.rp.p, O.rp.p + row0, (int)blk0); ::bd::note_launch();
    if (nb > 0) {
        k_st_shift<<<grid_for(nb, 256), 256, 0, s>>>(nb, M.ci.p, O.ci.p + blk0, col0); ::bd::note_launch();
        if (fp64) BD_CUDA(cudaMemcpyAsync(O.v.p + 4 * blk0, M.v.p, sizeof(double) * 4 * (size_t)nb,
                                          cudaMemcpyDeviceToDevice, s));
        if (O32) BD_CUDA(cudaMemcpyAsync(O32->p + 4 * blk0, v32, sizeof(float) * 4 * (size_t)nb,
                                         cudaMemcpyDeviceToDevice, s));
    }
    BD_LAUNCH_CHECK();
    return BD_OK;
}

// Stacked operator over `rows` (member list with each member's block rows,
// first node on the row level and first node on the column level).
struct StPart {
    const BSR *M;
    const float *v32;
    int nbr;
    long long row0;
    long long col0;
};
// rows: the stacked operator's rows, the parts' rows at their row0 (ascending)
// and empty rows in between (the finest level's padding to 32-row slices)
int st_build(const std::vector<StPart> &parts, long long rows, int ncols, bool fp64, bool fp32, BSR &O,
             DBuf<float> &O32, cudaStream_t s)
{
    long long blocks = 0;
    for (const StPart &pt : parts) blocks += pt.nbr > 0 ? pt.M->nb : 0;  // full operators: nbr == M->nbr
    if (rows > 2147483647LL || blocks > 2147483647LL) return BD_ERANGE;
    O.nbr = (int)rows;
    O.nbc = ncols;
    O.nb = blocks;
    BD_TRY(O.rp.alloc((size_t)rows + 1));
    BD_TRY(O.ci.alloc((size_t)std::max<long long>(blocks, 1)));
    if (fp64) BD_TRY(O.v.alloc(4 * (size_t)std::max<long long>(blocks, 1)));
    if (fp32) BD_TRY(O32.alloc(4 * (size_t)std::max<long long>(blocks, 1)));
    long long blk = 0, next = 0;
    for (const StPart &pt : parts) {
        if (pt.nbr <= 0) continue;
        if (pt.row0 > next) {  // empty rows before this part
            k_st_fill<<<grid_for(pt.row0 - next, 256), 256, 0, s>>>(pt.row0 - next, O.rp.p + next, (int)blk);
            ::bd::note_launch();
        }
        BD_TRY(st_append(*pt.M, pt.nbr, pt.v32, O, fp32 ? &O32 : nullptr, (int)pt.row0, blk, (int)pt.col0, fp64, s));
        blk += pt.M->nb;
        next = pt.row0 + pt.nbr;
    }
    k_st_fill<<<grid_for(rows + 1 - next, 256), 256, 0, s>>>(rows + 1 - next, O.rp.p + next, (int)blocks);
    ::bd::note_launch();
    BD_LAUNCH_CHECK();
    return BD_OK;
}

int st_sell_build(amg_stack *b, const std::vector<int> &order, const std::vector<long long> &off, cudaStream_t s)
{
    StLevel &S = b->lev[0];
    long long slots = 0;
    int nsl = 0;
    for (int k : order) {
        slots += b->h[k]->sell.slots;
        nsl += b->h[k]->sell.nslices;
    }
    if (slots * 32 > 2147483647LL) return BD_ERANGE;
    BD_TRY(S.ssptr.alloc((size_t)nsl + 1));
    BD_TRY(S.scol.alloc((size_t)slots * 32));
    BD_TRY(S.skk.alloc((size_t)slots * 64));
    BD_TRY(S.scm.alloc((size_t)std::max(S.N, 1)));
    BD_CUDA(cudaMemsetAsync(S.scm.p, 0, S.scm.bytes(), s));
    if (b->p32) {
        BD_TRY(S.skk32.alloc((size_t)slots * 64));
        BD_TRY(S.scm32.alloc((size_t)std::max(S.N, 1)));
        BD_CUDA(cudaMemsetAsync(S.scm32.p, 0, S.scm32.bytes(), s));
    }
    long long so = 0;
    for (int k : order) {
        const FineSell &F = b->h[k]->sell;
        const int N = b->h[k]->lev[0].N;
        const long long sl0 = off[k] / 32;  // the member's first slice (offsets are 32-aligned)
        k_st_shift<<<grid_for(F.nslices, 256), 256, 0, s>>>(F.nslices, F.sptr.p, S.ssptr.p + sl0, (int)so);
        ::bd::note_launch();
        k_st_shift<<<grid_for(F.slots * 32, 256), 256, 0, s>>>(F.slots * 32, F.col.p, S.scol.p + so * 32, (int)off[k]);
        ::bd::note_launch();
        BD_CUDA(cudaMemcpyAsync(S.skk.p + so * 64, F.kk.p, sizeof(double) * 64 * (size_t)F.slots,
                                cudaMemcpyDeviceToDevice, s));
        BD_CUDA(cudaMemcpyAsync(S.scm.p + off[k], F.cm.p, sizeof(double) * (size_t)N, cudaMemcpyDeviceToDevice, s));
        if (b->p32) {
            BD_CUDA(cudaMemcpyAsync(S.skk32.p + so * 64, F.kk32.p, sizeof(float) * 64 * (size_t)F.slots,
                                    cudaMemcpyDeviceToDevice, s));
            BD_CUDA(cudaMemcpyAsync(S.scm32.p + off[k], F.cm32.p, sizeof(float) * (size_t)N,
                                    cudaMemcpyDeviceToDevice, s));
        }
        so += F.slots;
    }
    k_st_set<<<1, 1, 0, s>>>(S.ssptr.p + nsl, (int)slots);
    ::bd::note_launch();
    BD_LAUNCH_CHECK();
    return BD_OK;
}

template <class T> int st_vec(DBuf<T> &b, long long n, cudaStream_t s)
{
    BD_TRY(b.alloc((size_t)std::max<long long>(n, 1)));
    BD_CUDA(cudaMemsetAsync(b.p, 0, b.bytes(), s));
    return BD_OK;
}

int st_create(amg_stack *b, cudaStream_t s)
{
    const int count = b->count;
    b->nlev.resize(count);
    int L = 0;
    for (int k = 0; k < count; k++) {
        b->nlev[k] = b->h[k]->nlev;
        L = std::max(L, b->nlev[k]);
    }
    b->L = L;
    bool sell0 = true;
    for (int k = 0; k < count; k++) sell0 = sell0 && b->h[k]->sell.valid;
    b->lev[0].sell = sell0;
    // member order and node offsets per level: smoothing members, then the
    // members whose coarsest level it is; on a sliced-ELL finest level every
    // member starts on a 32-row slice
    std::vector<std::vector<int>> order(L);
    std::vector<std::vector<long long>> off(L, std::vector<long long>(count, -1));
    for (int l = 0; l < L; l++) {
        long long o = 0;
        int ns = 0;
        for (int pass = 0; pass < 2; pass++)
            for (int k = 0; k < count; k++) {
                const int last = b->nlev[k] - 1;
                if ((pass == 0 && last > l) || (pass == 1 && last == l)) {
                    order[l].push_back(k);
                    off[l][k] = o;
                    const long long nk = b->h[k]->lev[l].N;
                    o += (l == 0 && sell0) ? (nk + 31) / 32 * 32 : nk;
                    if (pass == 0) ns = (int)o;
                }
            }
        if (o > 1073741823LL) return BD_ERANGE;
        b->lev[l].N = (int)o;
        b->lev[l].Ns = ns;
    }
    const bool p32 = b->p32;
    for (int l = 0; l < L; l++) {
        StLevel &S = b->lev[l];
        // A: every member on the finest level (the PCG applies it), the smoothing ones below
        std::vector<StPart> pa, pr, pp;
        for (int k : order[l]) {
            const Level &Lk = b->h[k]->lev[l];
            const bool smooth = b->nlev[k] - 1 > l;
            if ((l == 0 && !sell0) || (l > 0 && smooth))
                pa.push_back({&Lk.A, p32 ? Lk.A32.p : nullptr, Lk.A.nbr, off[l][k], off[l][k]});
            if (smooth) pp.push_back({&Lk.P, p32 ? Lk.P32.p : nullptr, Lk.P.nbr, off[l][k], off[l + 1][k]});
        }
        if (l + 1 < L)
            for (int k : order[l + 1]) {
                const Level &Lk = b->h[k]->lev[l];
                pr.push_back({&Lk.R, p32 ? Lk.R32.p : nullptr, Lk.R.nbr, off[l + 1][k], off[l][k]});
            }
        BD_TRY(st_build(pa, l == 0 ? S.N : S.Ns, S.N, l == 0 || !p32, p32, S.A, S.A32, s));
        S.rowsA = S.A.nbr;
        if (!pp.empty()) {
            BD_TRY(st_build(pp, S.Ns, b->lev[l + 1].N, !p32, p32, S.P, S.P32, s));
            BD_TRY(st_build(pr, b->lev[l + 1].N, S.N, !p32, p32, S.R, S.R32, s));
        }
        if (l == 0 && sell0) BD_TRY(st_sell_build(b, order[0], off[0], s));
        // node -> member (-1 on padding), Chebyshev coefficients, inverse diagonals
        BD_TRY(S.mem.alloc((size_t)std::max(S.N, 1)));
        BD_CUDA(cudaMemsetAsync(S.mem.p, 0xff, S.mem.bytes(), s));
        std::vector<double> coef(4 * (size_t)count, 0.0);
        for (int k : order[l]) {
            const Level &Lk = b->h[k]->lev[l];
            k_st_fill<<<grid_for(Lk.N, 256), 256, 0, s>>>(Lk.N, S.mem.p + off[l][k], k); ::bd::note_launch();
            coef[4 * k] = Lk.ch_inv_theta;
            coef[4 * k + 1] = Lk.ch_c1;
            coef[4 * k + 2] = Lk.ch_c2;
            coef[4 * k + 3] = 1.0 + Lk.ch_c1;
        }
        BD_TRY(S.coef.alloc(coef.size()));
        BD_CUDA(cudaMemcpyAsync(S.coef.p, coef.data(), sizeof(double) * coef.size(), cudaMemcpyHostToDevice, s));
        BD_CUDA(cudaStreamSynchronize(s));  // coef lives on the host stack
        const long long n2 = 2LL * S.N;
        if (p32) {
            BD_TRY(st_vec(S.invd32, n2, s));
            for (int k : order[l])
                BD_CUDA(cudaMemcpyAsync(S.invd32.p + 2 * off[l][k], b->h[k]->lev[l].invdiag32.p,
                                        sizeof(float) * 2 * b->h[k]->lev[l].N, cudaMemcpyDeviceToDevice, s));
            BD_TRY(st_vec(S.f32, n2, s));
            BD_TRY(st_vec(S.u32, n2, s));
            BD_TRY(st_vec(S.r32, n2, s));
            BD_TRY(st_vec(S.d32, n2, s));
            BD_TRY(st_vec(S.w32, n2, s));
        } else {
            BD_TRY(st_vec(S.invd, n2, s));
            for (int k : order[l])
                BD_CUDA(cudaMemcpyAsync(S.invd.p + 2 * off[l][k], b->h[k]->lev[l].invdiag.p,
                                        sizeof(double) * 2 * b->h[k]->lev[l].N, cudaMemcpyDeviceToDevice, s));
            // the (v + u, u) form on a sliced finest level whose members all carry
            // their scaled inverse diagonals (every FP64 sliced finest level does)
            // (only the members that smooth there, rows [0, Ns), use them)
            bool su = l == 0 && sell0;
            for (int k : order[l])
                if (b->nlev[k] > 1) su = su && b->h[k]->lev[0].idc2.p && b->h[k]->lev[0].idt.p;
            S.su = su;
            if (su) {
                BD_TRY(st_vec(S.idc2, n2, s));
                BD_TRY(st_vec(S.idt, n2, s));
                for (int k : order[l]) {
                    if (b->nlev[k] <= 1) continue;
                    const size_t bytes = sizeof(double) * 2 * b->h[k]->lev[0].N;
                    BD_CUDA(cudaMemcpyAsync(S.idc2.p + 2 * off[0][k], b->h[k]->lev[0].idc2.p, bytes,
                                            cudaMemcpyDeviceToDevice, s));
                    BD_CUDA(cudaMemcpyAsync(S.idt.p + 2 * off[0][k], b->h[k]->lev[0].idt.p, bytes,
                                            cudaMemcpyDeviceToDevice, s));
                }
            }
            if (l > 0) BD_TRY(st_vec(S.f, n2, s));
            BD_TRY(st_vec(S.u, n2, s));
            BD_TRY(st_vec(S.r, n2, s));
            BD_TRY(st_vec(S.d, n2, s));
            BD_TRY(st_vec(S.w, n2, s));
        }
        S.lanes[0] = lanes_for(S.A, p32);
        if (!pp.empty()) {
            S.lanes[1] = lanes_for(S.R, p32);
            S.lanes[2] = lanes_for(S.P, p32);
        }
    }
    // the finest A in FP64 for the PCG's products: lanes for its rows
    // coarsest-level jobs
    std::vector<StCoarseJob> jobs(count);
    for (int k = 0; k < count; k++) {
        const amg_hierarchy *hk = b->h[k];
        const int c = b->nlev[k] - 1;
        jobs[k] = {hk->cinv.p, hk->zc.p, hk->zz, hk->nc, c, 2 * off[c][k]};
        b->max_nc = std::max(b->max_nc, hk->nc);
    }
    BD_TRY(b->jobs.alloc(count));
    BD_CUDA(cudaMemcpyAsync(b->jobs.p, jobs.data(), sizeof(StCoarseJob) * count, cudaMemcpyHostToDevice, s));
    // PCG vectors and reduction chunks of the finest level
    const long long n2 = 2LL * b->lev[0].N;
    BD_TRY(st_vec(b->fin, n2, s));
    BD_TRY(st_vec(b->x, n2, s));
    BD_TRY(st_vec(b->r, n2, s));
    BD_TRY(st_vec(b->z, n2, s));
    BD_TRY(st_vec(b->p, n2, s));
    BD_TRY(st_vec(b->q, n2, s));
    BD_TRY(st_vec(b->fp, n2, s));
    if (p32) BD_TRY(st_vec(b->zold, n2, s));
    b->off0.assign(count, 0);
    b->n0.assign(count, 0);
    std::vector<int> cm, cb, ce, m0(count, 0), m1(count, 0), nn(count, 0);
    for (int k : order[0]) {
        const int N = b->h[k]->lev[0].N;
        b->off0[k] = off[0][k];
        b->n0[k] = N;
        nn[k] = N;
        m0[k] = (int)cm.size();
        for (int a = 0; a < N; a += kStChunk) {
            cm.push_back(k);
            cb.push_back((int)(off[0][k] + a));
            ce.push_back((int)(off[0][k] + std::min(N, a + kStChunk)));
        }
        m1[k] = (int)cm.size();
    }
    b->nchunks = (int)cm.size();
    BD_TRY(b->cmem.alloc(cm.size()));
    BD_TRY(b->cbeg.alloc(cb.size()));
    BD_TRY(b->cend.alloc(ce.size()));
    BD_TRY(b->mc0.alloc(count));
    BD_TRY(b->mc1.alloc(count));
    BD_TRY(b->nn.alloc(count));
    BD_CUDA(cudaMemcpyAsync(b->cmem.p, cm.data(), sizeof(int) * cm.size(), cudaMemcpyHostToDevice, s));
    BD_CUDA(cudaMemcpyAsync(b->cbeg.p, cb.data(), sizeof(int) * cb.size(), cudaMemcpyHostToDevice, s));
    BD_CUDA(cudaMemcpyAsync(b->cend.p, ce.data(), sizeof(int) * ce.size(), cudaMemcpyHostToDevice, s));
    BD_CUDA(cudaMemcpyAsync(b->mc0.p, m0.data(), sizeof(int) * count, cudaMemcpyHostToDevice, s));
    BD_CUDA(cudaMemcpyAsync(b->mc1.p, m1.data(), sizeof(int) * count, cudaMemcpyHostToDevice, s));
    BD_CUDA(cudaMemcpyAsync(b->nn.p, nn.data(), sizeof(int) * count, cudaMemcpyHostToDevice, s));
    BD_TRY(b->part.alloc(4 * (size_t)std::max(b->nchunks, 1)));
    BD_TRY(b->scal.alloc((size_t)count * T_NSLOTS));
    BD_TRY(b->counter.alloc(1));
    BD_CUDA(cudaMemsetAsync(b->counter.p, 0, sizeof(unsigned int), s));
    BD_CUDA(cudaMallocHost((void **)&b->host_init, sizeof(double) * count * T_NSLOTS));
    BD_CUDA(cudaMallocHost((void **)&b->host_scal, sizeof(double) * count * T_NSLOTS));
    BD_CUDA(cudaStreamCreateWithFlags(&b->cap, cudaStreamNonBlocking));
    BD_CUDA(cudaStreamCreateWithFlags(&b->cap2, cudaStreamNonBlocking));
    BD_CUDA(cudaEventCreate(&b->ev[0]));
    BD_CUDA(cudaEventCreate(&b->ev[1]));
    BD_CUDA(cudaStreamSynchronize(s));
    return BD_OK;
}

// ------------------------------------------------------------------ stacked V-cycle
template <class S> struct StView {
    const S *Av, *Rv, *Pv;
    v2<S> *f, *u, *r, *d, *w;
    const v2<S> *invd;
};
template <class S> StView<S> st_view(amg_stack *b, int l);
template <> StView<double> st_view<double>(amg_stack *b, int l)
{
    StLevel &S = b->lev[l];
    return {S.A.v.p, S.R.v.p, S.P.v.p, (double2 *)(l == 0 ? b->r.p : S.f.p), (double2 *)S.u.p,
            (double2 *)S.r.p, (double2 *)S.d.p, (double2 *)S.w.p, (const double2 *)S.invd.p};
}
template <> StView<float> st_view<float>(amg_stack *b, int l)
{
    StLevel &S = b->lev[l];
    return {S.A32.p, S.R32.p, S.P32.p, (float2 *)S.f32.p, (float2 *)S.u32.p, (float2 *)S.r32.p,
            (float2 *)S.d32.p, (float2 *)S.w32.p, (const float2 *)S.invd32.p};
}

template <class S> const v2<S> *st_kk(const StLevel &Lv);
template <> const double2 *st_kk<double>(const StLevel &Lv) { return (const double2 *)Lv.skk.p; }
template <> const float2 *st_kk<float>(const StLevel &Lv) { return (const float2 *)Lv.skk32.p; }
template <class S> const S *st_cm(const StLevel &Lv);
template <> const double *st_cm<double>(const StLevel &Lv) { return Lv.scm.p; }
template <> const float *st_cm<float>(const StLevel &Lv) { return Lv.scm32.p; }

// Operator of stack level l on rows [0, rows): the finest level's sliced ELL
// when built, block CSR otherwise.
template <class S, class E, bool SU = false>
int st_apply(const StLevel &Lv, int l, int rows, const S *vals, const v2<S> *x, E e, cudaStream_t s)
{
    if (l == 0 && Lv.sell) {
        if (rows <= 0) return BD_OK;
        // a large FP64 level: one 1024-thread block per SM on equal shares (measured
        // against the grid-stride kernel: 64 slabs 2624 -> 2666 solves/s)
        if (sizeof(S) == 8 && ((long long)rows + 31) / 32 >= (long long)kSM * 32) {
            k_st_sell_wide<S, E, SU><<<kSM, 1024, 0, s>>>(rows, Lv.mem.p, Lv.ssptr.p, Lv.scol.p, st_kk<S>(Lv),
                                                          st_cm<S>(Lv), StGather<S>{x}, e);
        } else {
            const int grid = (int)std::min<long long>(((long long)rows + 255) / 256, (long long)kSM * 8);
            k_st_sell<S, E, SU><<<grid, 256, 0, s>>>(rows, Lv.mem.p, Lv.ssptr.p, Lv.scol.p, st_kk<S>(Lv),
                                                     st_cm<S>(Lv), StGather<S>{x}, e);
        }
        ::bd::note_launch();
        BD_LAUNCH_CHECK();
        return BD_OK;
    }
    if constexpr (SU) return BD_ESTATE;  // the (v + u, u) form exists on the sliced level only
    else return launch_bsr_rows<S>(rows, Lv.A.rp.p, Lv.A.ci.p, vals, Lv.lanes[0], StGather<S>{x}, e, s);
}

template <class S>
int st_vcycle(amg_stack *b, cudaStream_t s)
{
    const int L = b->L;
    for (int l = 0; l + 1 < L; l++) {
        StLevel &Lv = b->lev[l];
        if (Lv.Ns <= 0) continue;
        const StView<S> v = st_view<S>(b, l), cv = st_view<S>(b, l + 1);
        const StCoef c{Lv.mem.p, Lv.coef.p}, cc{b->lev[l + 1].mem.p, b->lev[l + 1].coef.p};
        if constexpr (std::is_same<S, double>::value) {
            if (l == 0 && Lv.su) {
                BD_TRY((st_apply<S, StPreX, true>(Lv, l, Lv.Ns, v.Av, v.d,
                                                  StPreX{v.f, (const double2 *)Lv.idc2.p, v.d, v.u, c}, s)));
                BD_TRY((st_apply<S, StResid<S>, true>(Lv, l, Lv.Ns, v.Av, v.u, StResid<S>{v.f, v.r}, s)));
                BD_TRY(launch_bsr<S>(Lv.R, v.Rv, Lv.lanes[1], StGather<S>{v.r},
                                     StStoreD0<S>{cv.f, cv.d, cv.invd, cc}, s));
                continue;
            }
        }
        BD_TRY(st_apply<S>(Lv, l, Lv.Ns, v.Av, v.d, StPre<S>{v.f, v.invd, v.d, v.u, c}, s));
        BD_TRY(st_apply<S>(Lv, l, Lv.Ns, v.Av, v.u, StResid<S>{v.f, v.r}, s));
        BD_TRY(launch_bsr<S>(Lv.R, v.Rv, Lv.lanes[1], StGather<S>{v.r}, StStoreD0<S>{cv.f, cv.d, cv.invd, cc}, s));
    }
    StLevelPtrs<S> lp{};
    for (int l = 0; l < L; l++) {
        const StView<S> v = st_view<S>(b, l);
        lp.f[l] = (S *)v.f;
        lp.u[l] = (S *)v.u;
    }
    const size_t smem = sizeof(double) * (size_t)std::max(b->max_nc, 1);
    if (smem > 48 * 1024) BD_CUDA(cudaFuncSetAttribute(k_st_coarse<S>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                                       (int)smem));
    k_st_coarse<S><<<b->count, 512, smem, s>>>(b->jobs.p, lp); ::bd::note_launch();
    BD_LAUNCH_CHECK();
    for (int l = L - 2; l >= 0; l--) {
        StLevel &Lv = b->lev[l];
        if (Lv.Ns <= 0) continue;
        const StView<S> v = st_view<S>(b, l), cv = st_view<S>(b, l + 1);
        const StCoef c{Lv.mem.p, Lv.coef.p};
        if constexpr (std::is_same<S, double>::value) {
            if (l == 0 && Lv.su) {
                BD_TRY(launch_bsr<S>(Lv.P, v.Pv, Lv.lanes[2], StGather<S>{cv.u}, StAddX{v.u}, s));
                BD_TRY((st_apply<S, StPost1X, true>(Lv, l, Lv.Ns, v.Av, v.u,
                                                    StPost1X{v.f, (const double2 *)Lv.idt.p, v.u, v.r, v.d, v.w},
                                                    s)));
                BD_TRY((st_apply<S, StPost2X, true>(Lv, l, Lv.Ns, v.Av, v.d,
                                                    StPost2X{v.r, v.d, (const double2 *)Lv.idc2.p, v.w, v.u, c},
                                                    s)));
                continue;
            }
        }
        BD_TRY(launch_bsr<S>(Lv.P, v.Pv, Lv.lanes[2], StGather<S>{cv.u}, StAdd<S>{v.u}, s));
        BD_TRY(st_apply<S>(Lv, l, Lv.Ns, v.Av, v.u, StPost1<S>{v.f, v.invd, v.u, v.r, v.d, v.w, c}, s));
        BD_TRY(st_apply<S>(Lv, l, Lv.Ns, v.Av, v.d, StPost2<S>{v.r, v.d, v.invd, v.w, v.u, c}, s));
    }
    return BD_OK;
}

// ------------------------------------------------------------------ stacked PCG graph
template <class S>
StPcg<S> st_pcg(amg_stack *b)
{
    const StView<S> v0 = st_view<S>(b, 0);
    StPcg<S> v;
    v.fin = (const double2 *)b->fin.p;
    v.fp = (double2 *)b->fp.p;
    v.x = (double2 *)b->x.p;
    v.r = (double2 *)b->r.p;
    v.z = (double2 *)b->z.p;
    v.p = (double2 *)b->p.p;
    v.q = (double2 *)b->q.p;
    v.zold = b->p32 ? (double2 *)b->zold.p : nullptr;
    v.f0 = v0.f;
    v.d0 = v0.d;
    v.u0 = v0.u;
    v.invd0 = v0.invd;
    v.c0 = StCoef{b->lev[0].mem.p, b->lev[0].coef.p};
    v.mem = b->lev[0].mem.p;
    v.psu = b->lev[0].sell ? 1 : 0;
    v.dsu = b->lev[0].su ? 1 : 0;
    return v;
}

StRed st_red(amg_stack *b, cudaGraphConditionalHandle cond)
{
    return {b->scal.p, b->part.p, b->counter.p, b->cmem.p, b->cbeg.p, b->cend.p, b->mc0.p, b->mc1.p, b->nn.p,
            b->count, b->p32 ? 1 : 0, cond};
}

// q = A x on the finest level; su: x is stored in (v + u, u) form (the PCG's p
// on a sliced level)
int st_apply_a(amg_stack *b, const double2 *x, double2 *q, cudaStream_t s, bool su = false)
{
    StLevel &S = b->lev[0];
    if (S.sell && su) return st_apply<double, StStore, true>(S, 0, S.N, nullptr, x, StStore{q}, s);
    if (S.sell) return st_apply<double>(S, 0, S.N, nullptr, x, StStore{q}, s);
    return launch_bsr_rows<double>(S.N, S.A.rp.p, S.A.ci.p, S.A.v.p, lanes_for(S.A, false), StGather<double>{x},
                                   StStore{q}, s);
}

template <class S>
int st_capture(amg_stack *b)
{
    cudaStream_t s = b->cap, s2 = b->cap2;
    const int count = b->count, N0 = b->lev[0].N;
    const StPcg<S> v = st_pcg<S>(b);
    const int nch = b->nchunks;
    const int vg = grid_for(N0, kStThreads);
    BD_CUDA(cudaStreamBeginCapture(s, cudaStreamCaptureModeThreadLocal));
    const long long c0 = launch_count();
    BD_CUDA(cudaMemcpyAsync(b->scal.p, b->host_init, sizeof(double) * count * T_NSLOTS, cudaMemcpyHostToDevice, s));
    for (int k = 0; k < count; k++) {
        const size_t bytes = sizeof(double) * 2 * (size_t)b->n0[k];
        BD_CUDA(cudaMemcpyAsync(b->fin.p + 2 * b->off0[k], b->gf[k], bytes, cudaMemcpyDeviceToDevice, s));
        BD_CUDA(cudaMemcpyAsync(b->x.p + 2 * b->off0[k], b->gx[k], bytes, cudaMemcpyDeviceToDevice, s));
    }
    k_st_red<R_FSTATS, S><<<nch, kStThreads, 0, s>>>(st_red(b, 0), v); ::bd::note_launch();
    k_st_red<R_PROJF, S><<<nch, kStThreads, 0, s>>>(st_red(b, 0), v); ::bd::note_launch();
    BD_TRY(st_apply_a(b, v.x, v.q, s));
    BD_LAUNCH_CHECK();
    cudaStreamCaptureStatus cs;
    cudaGraph_t g = nullptr;
    const cudaGraphNode_t *deps = nullptr;
    size_t nd = 0;
    BD_CUDA(cudaStreamGetCaptureInfo(s, &cs, nullptr, &g, &deps, nullptr, &nd));
    cudaGraphConditionalHandle cond;
    BD_CUDA(cudaGraphConditionalHandleCreate(&cond, g, 0, 0));
    k_st_red<R_INIT, S><<<nch, kStThreads, 0, s>>>(st_red(b, cond), v); ::bd::note_launch();
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
    BD_TRY(st_vcycle<S>(b, s2));
    k_st_red<R_ZSTATS, S><<<nch, kStThreads, 0, s2>>>(st_red(b, 0), v); ::bd::note_launch();
    k_st_p<S><<<vg, kStThreads, 0, s2>>>(N0, v, b->scal.p); ::bd::note_launch();
    BD_TRY(st_apply_a(b, v.p, v.q, s2, v.psu != 0));
    k_st_red<R_PQ, S><<<nch, kStThreads, 0, s2>>>(st_red(b, 0), v); ::bd::note_launch();
    k_st_red<R_XR, S><<<nch, kStThreads, 0, s2>>>(st_red(b, cond), v); ::bd::note_launch();
    BD_LAUNCH_CHECK();
    cudaGraph_t body_out = nullptr;
    BD_CUDA(cudaStreamEndCapture(s2, &body_out));
    const long long c2 = launch_count();
    BD_CUDA(cudaStreamUpdateCaptureDependencies(s, &wnode, nullptr, 1, cudaStreamSetCaptureDependencies));
    BD_TRY(st_apply_a(b, v.x, v.q, s));
    k_st_red<R_TRUE, S><<<nch, kStThreads, 0, s>>>(st_red(b, 0), v); ::bd::note_launch();
    k_st_project_x<<<vg, kStThreads, 0, s>>>(N0, v.x, b->lev[0].mem.p, b->scal.p); ::bd::note_launch();
    BD_LAUNCH_CHECK();
    for (int k = 0; k < count; k++) {
        const size_t bytes = sizeof(double) * 2 * (size_t)b->n0[k];
        BD_CUDA(cudaMemcpyAsync(b->gx[k], b->x.p + 2 * b->off0[k], bytes, cudaMemcpyDeviceToDevice, s));
    }
    BD_CUDA(cudaMemcpyAsync(b->host_scal, b->scal.p, sizeof(double) * count * T_NSLOTS, cudaMemcpyDeviceToHost, s));
    const long long c3 = launch_count();
    BD_CUDA(cudaStreamEndCapture(s, &b->graph));
    BD_CUDA(cudaGraphInstantiate(&b->exec, b->graph, 0));
    b->n_pre = c1 - c0;
    b->n_body = c2 - c1;
    b->n_post = c3 - c2;
    note_launches(-(c3 - c0));
    return BD_OK;
}

void end_capture(cudaStream_t s)
{
    cudaStreamCaptureStatus cs;
    if (cudaStreamIsCapturing(s, &cs) == cudaSuccess && cs != cudaStreamCaptureStatusNone) {
        cudaGraph_t g = nullptr;
        cudaStreamEndCapture(s, &g);
        if (g) cudaGraphDestroy(g);
    }
    cudaGetLastError();
}

}  // namespace
}  // namespace bd

// ------------------------------------------------------------------ public
extern "C" int amg_stack_create(amg_hierarchy *const *h, int count, void *stream, amg_stack **out)
{
    if (!out) return BD_EINVAL;
    *out = nullptr;
    if (!h || count < 1) return BD_EINVAL;
    for (int k = 0; k < count; k++) {
        if (!h[k] || h[k]->nlev < 1) return BD_EINVAL;
        if (h[k]->prec32 != h[0]->prec32) return BD_EINVAL;     // one V-cycle precision per stack
        if (h[k]->opts.cheb_degree != 2) return BD_EINVAL;     // Appendix A's degree-2 smoother only
    }
    amg_stack *b = new (std::nothrow) amg_stack();
    if (!b) return BD_ENOMEM;
    b->count = count;
    b->p32 = h[0]->prec32;
    b->h.assign(h, h + count);
    for (amg_hierarchy *hk : b->h) hk->batch_refs++;  // their forms may not change while stacked
    const int st = bd::st_create(b, (cudaStream_t)stream);
    if (st != BD_OK) {
        delete b;
        return st;
    }
    *out = b;
    return BD_OK;
}

extern "C" int amg_stack_solve(amg_stack *b, const double *const *f, double *const *x, const solve_options *opts,
                               void *stream, solve_info *info)
{
    if (!b || !f || !x) return BD_EINVAL;
    const int count = b->count;
    solve_options o;
    solve_options_default(&o);
    if (opts) o = *opts;
    if (!(o.rtol > 0.0) || o.max_it < 0 || o.strict) return BD_EINVAL;
    for (int k = 0; k < count; k++)
        if (!f[k] || !x[k]) return BD_EINVAL;
    bool same = b->exec != nullptr;
    for (int k = 0; k < count && same; k++) same = b->gf[k] == f[k] && b->gx[k] == x[k];
    if (!same) {
        b->drop_graph();
        b->gf.assign(f, f + count);
        b->gx.assign(x, x + count);
        const int st = b->p32 ? bd::st_capture<float>(b) : bd::st_capture<double>(b);
        if (st != BD_OK) {
            bd::end_capture(b->cap2);
            bd::end_capture(b->cap);
            b->drop_graph();
            return st;
        }
    }
    for (int k = 0; k < count; k++) {
        double *hi = b->host_init + (size_t)k * bd::T_NSLOTS;
        for (int i = 0; i < bd::T_NSLOTS; i++) hi[i] = 0.0;
        hi[bd::T_RTOL] = o.rtol;
        hi[bd::T_MAXIT] = (double)o.max_it;
        hi[bd::T_WARM] = o.warm_start ? 1.0 : 0.0;
    }
    cudaStream_t s = (cudaStream_t)stream;
    BD_CUDA(cudaEventRecord(b->ev[0], s));
    BD_CUDA(cudaGraphLaunch(b->exec, s));
    BD_CUDA(cudaEventRecord(b->ev[1], s));
    BD_CUDA(cudaStreamSynchronize(s));
    float ms = 0.0f;
    cudaEventElapsedTime(&ms, b->ev[0], b->ev[1]);
    int worst = BD_OK;
    double loops = 0.0;
    for (int k = 0; k < count; k++) {
        const double *sc = b->host_scal + (size_t)k * bd::T_NSLOTS;
        loops = std::max(loops, sc[bd::T_IT]);
        const double nf = std::sqrt(sc[bd::T_NF2]);
        const int stk = (int)sc[bd::T_STATUS];
        if (info) {
            info[k].status = stk;
            info[k].iters = (int)sc[bd::T_IT];
            info[k].rel_res = nf > 0.0 ? std::sqrt(sc[bd::T_RR]) / nf : 0.0;
            info[k].true_rel_res = nf > 0.0 ? std::sqrt(sc[bd::T_TRR]) / nf : 0.0;
            info[k].solve_ms = ms;
            info[k].total_iters = (long long)sc[bd::T_IT];
        }
        if (stk != BD_OK && worst == BD_OK) worst = stk;
    }
    bd::note_launches(b->n_pre + b->n_post + (long long)loops * b->n_body);
    return worst;
}

extern "C" int amg_stack_info(const amg_stack *b, int *levels, long long *launches_per_iteration)
{
    if (!b) return BD_EINVAL;
    if (levels) *levels = b->L;
    if (launches_per_iteration) *launches_per_iteration = b->n_body;
    return BD_OK;
}

extern "C" void amg_stack_destroy(amg_stack *b) { delete b; }
