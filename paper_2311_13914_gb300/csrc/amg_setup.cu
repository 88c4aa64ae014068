// amg_setup.cu -- a1..a9: smoothed-aggregation hierarchy setup on the device
// (Algorithm 1; Section 4 for the strength graph, MIS, cluster rule and
// tentative prolongator; Appendix A for the squared graph, one prolongator
// smoothing step, the 10-step CG eigen-estimate and the coarse limit).
//
// Compiled with -fmad=false.  Every floating-point value that decides an
// integer (strength, aggregate choice) or enters the next level is formed by
// the documented sequence of rounded operations: sums over the middle index in
// ascending order, correctly rounded dot products, IEEE sqrt and division.
// Aggregates and sparsity patterns are therefore bit-identical to any
// implementation that follows the same order, whatever the thread schedule.
#include <algorithm>
#include <new>
#include <climits>
#include <cmath>

#include "amg_internal.cuh"

namespace bd {

// ------------------------------------------------------------------ hashing
__host__ __device__ __forceinline__ unsigned long long mix64(unsigned long long z)
{
    z = (z ^ (z >> 30)) * 0xbf58476d1ce4e5b9ULL;
    z = (z ^ (z >> 27)) * 0x94d049bb133111ebULL;
    return z ^ (z >> 31);
}

static unsigned long long level_key(unsigned long long seed, int level, int stream)
{
    return mix64(seed + 0x9E3779B97F4A7C15ULL * (unsigned long long)(2 * level + stream + 1));
}

__device__ __forceinline__ int find_block(const int *__restrict__ rp, const int *__restrict__ ci,
                                          int row, int col)
{
    int lo = rp[row], hi = rp[row + 1] - 1;
    while (lo <= hi) {
        int mid = (lo + hi) >> 1;
        int c = ci[mid];
        if (c == col) return mid;
        if (c < col) lo = mid + 1;
        else hi = mid - 1;
    }
    return -1;
}

// ------------------------------------------------------------------ diagonal
__global__ void k_diag(int N, const int *__restrict__ rp, const int *__restrict__ ci,
                       const double *__restrict__ v, double *__restrict__ diag, int *bad)
{
    int p = blockIdx.x * blockDim.x + threadIdx.x;
    if (p >= N) return;
    int t = find_block(rp, ci, p, p);
    double d0 = t >= 0 ? v[4 * (size_t)t] : 0.0, d1 = t >= 0 ? v[4 * (size_t)t + 3] : 0.0;
    if (!(d0 > 0.0) || !(d1 > 0.0)) *bad = 1;
    diag[2 * p] = d0;
    diag[2 * p + 1] = d1;
}

// ------------------------------------------------------------------ a1 strength
// w_pq = 0.5 (|A_u(p,q)| + |A_u(q,p)|) / sqrt(A_u(p,p) A_u(q,q)), kept if >= theta,
// A_u = the (u_e, u_e) entry of the 2x2 node block.
__device__ __forceinline__ bool strength_w(const int *rp, const int *ci, const double *v,
                                           const double *diag, int p, int t, double theta,
                                           double *w_out)
{
    int q = ci[t];
    if (q == p) return false;
    int tt = find_block(rp, ci, q, p);
    double apq = fabs(v[4 * (size_t)t + 3]);
    double aqp = tt >= 0 ? fabs(v[4 * (size_t)tt + 3]) : 0.0;
    double num = 0.5 * (apq + aqp);
    double den = sqrt(diag[2 * p + 1] * diag[2 * q + 1]);
    if (!(den > 0.0)) return false;
    double w = num / den;
    *w_out = w;
    return w >= theta;
}

// One pass forms every entry's weight (a square root and a division, costly
// on the FP64 pipe) and counts the strong ones; wt[t] keeps the weight of a
// strong entry and -1 otherwise (weights are >= 0), so the fill only compacts.
__global__ void k_strength_count(int N, const int *__restrict__ rp, const int *__restrict__ ci,
                                 const double *__restrict__ v, const double *__restrict__ diag,
                                 double theta, int *cnt, double *__restrict__ wt)
{
    int p = blockIdx.x * blockDim.x + threadIdx.x;
    if (p >= N) return;
    int c = 0;
    double w;
    for (int t = rp[p]; t < rp[p + 1]; t++) {
        const bool strong = strength_w(rp, ci, v, diag, p, t, theta, &w);
        wt[t] = strong ? w : -1.0;
        c += strong;
    }
    cnt[p] = c;
}

__global__ void k_strength_fill(int N, const int *__restrict__ rp, const int *__restrict__ ci,
                                const double *__restrict__ wt, const int *__restrict__ srp,
                                int *__restrict__ sci, double *__restrict__ sw)
{
    int p = blockIdx.x * blockDim.x + threadIdx.x;
    if (p >= N) return;
    int pos = srp[p];
    for (int t = rp[p]; t < rp[p + 1]; t++) {
        const double w = wt[t];
        if (w >= 0.0) {
            sci[pos] = ci[t];
            sw[pos] = w;
            pos++;
        }
    }
}

// ------------------------------------------------------------------ deterministic SpGEMM
// C = A B for BS x BS block CSR (BS = 1 scalar, 2 node blocks).  One thread
// block per output row; a dense accumulator indexed by output column lives in
// global scratch (one slice per resident block); touched columns are listed
// in shared memory, sorted, and emitted ascending.  Every entry is
// accumulated as acc = acc + a*b over the scalar middle index in ascending
// order (for BS = 2: middle block k ascending, then its two scalar columns).
template <int BS>
__global__ void k_spgemm_count(int nrows, const int *__restrict__ arp, const int *__restrict__ aci,
                               const int *__restrict__ brp, const int *__restrict__ bci, int ncols,
                               int *__restrict__ mark_all, int *__restrict__ cnt)
{
    __shared__ int count;
    int *mark = mark_all + (size_t)blockIdx.x * ncols;
    for (int i = blockIdx.x; i < nrows; i += gridDim.x) {
        if (threadIdx.x == 0) count = 0;
        __syncthreads();
        for (int t = arp[i]; t < arp[i + 1]; t++) {
            int k = aci[t];
            for (int s = brp[k] + threadIdx.x; s < brp[k + 1]; s += blockDim.x) {
                int j = bci[s];
                if (atomicExch(&mark[j], i) != i) atomicAdd(&count, 1);
            }
        }
        __syncthreads();
        if (threadIdx.x == 0) cnt[i] = count;
        __syncthreads();
    }
}

template <int BS>
__global__ void k_spgemm_fill(int nrows, const int *__restrict__ arp, const int *__restrict__ aci,
                              const double *__restrict__ av, const int *__restrict__ brp,
                              const int *__restrict__ bci, const double *__restrict__ bv, int ncols,
                              int *__restrict__ mark_all, double *__restrict__ acc_all,
                              const int *__restrict__ crp, int *__restrict__ cci,
                              double *__restrict__ cv, int P2)
{
    extern __shared__ int cols[];
    __shared__ int count;
    constexpr int BB = BS * BS;
    int *mark = mark_all + (size_t)blockIdx.x * ncols;
    double *acc = acc_all + (size_t)blockIdx.x * ncols * BB;
    for (int i = blockIdx.x; i < nrows; i += gridDim.x) {
        if (threadIdx.x == 0) count = 0;
        __syncthreads();
        for (int t = arp[i]; t < arp[i + 1]; t++) {
            int k = aci[t];
            double a[BB];
#pragma unroll
            for (int e = 0; e < BB; e++) a[e] = av[(size_t)t * BB + e];
            for (int s = brp[k] + threadIdx.x; s < brp[k + 1]; s += blockDim.x) {
                int j = bci[s];
                double *c = acc + (size_t)j * BB;
                if (mark[j] != i) {
                    mark[j] = i;
#pragma unroll
                    for (int e = 0; e < BB; e++) c[e] = 0.0;
                    cols[atomicAdd(&count, 1)] = j;
                }
                const double *b = bv + (size_t)s * BB;
                if (BS == 1) {
                    c[0] = c[0] + a[0] * b[0];
                } else {
                    // scalar middle index 2k then 2k+1
                    c[0] = c[0] + a[0] * b[0];
                    c[0] = c[0] + a[1] * b[2];
                    c[1] = c[1] + a[0] * b[1];
                    c[1] = c[1] + a[1] * b[3];
                    c[2] = c[2] + a[2] * b[0];
                    c[2] = c[2] + a[3] * b[2];
                    c[3] = c[3] + a[2] * b[1];
                    c[3] = c[3] + a[3] * b[3];
                }
            }
            __syncthreads();
        }
        int n = count;
        int p2 = 1;
        while (p2 < n) p2 <<= 1;
        for (int x = n + threadIdx.x; x < p2; x += blockDim.x) cols[x] = INT_MAX;
        __syncthreads();
        for (int kk = 2; kk <= p2; kk <<= 1)
            for (int jj = kk >> 1; jj > 0; jj >>= 1) {
                for (int x = threadIdx.x; x < p2; x += blockDim.x) {
                    int y = x ^ jj;
                    if (y > x) {
                        bool up = (x & kk) == 0;
                        int cx = cols[x], cy = cols[y];
                        if ((cx > cy) == up) {
                            cols[x] = cy;
                            cols[y] = cx;
                        }
                    }
                }
                __syncthreads();
            }
        int base = crp[i];
        for (int x = threadIdx.x; x < n; x += blockDim.x) {
            int j = cols[x];
            cci[base + x] = j;
#pragma unroll
            for (int e = 0; e < BB; e++) cv[(size_t)(base + x) * BB + e] = acc[(size_t)j * BB + e];
        }
        __syncthreads();
    }
    (void)P2;
}

// Dense path with the row's accumulators and column marks in shared memory
// (coarse levels: few columns), otherwise identical to k_spgemm_count /
// k_spgemm_fill: a block per output row, every entry accumulated in ascending
// middle index.  Shared memory: marks (ncols ints) for the count; marks,
// accumulators (ncols x BB doubles) and the row's column list (P2 ints) for
// the fill.
__global__ void k_spgemm_count_smem(int nrows, const int *__restrict__ arp, const int *__restrict__ aci,
                                    const int *__restrict__ brp, const int *__restrict__ bci, int ncols,
                                    int *__restrict__ cnt)
{
    extern __shared__ int smark[];
    __shared__ int count;
    for (int j = threadIdx.x; j < ncols; j += blockDim.x) smark[j] = -1;
    __syncthreads();
    for (int i = blockIdx.x; i < nrows; i += gridDim.x) {
        if (threadIdx.x == 0) count = 0;
        __syncthreads();
        for (int t = arp[i]; t < arp[i + 1]; t++) {
            int k = aci[t];
            for (int s2 = brp[k] + threadIdx.x; s2 < brp[k + 1]; s2 += blockDim.x) {
                int j = bci[s2];
                if (atomicExch(&smark[j], i) != i) atomicAdd(&count, 1);
            }
        }
        __syncthreads();
        if (threadIdx.x == 0) cnt[i] = count;
        __syncthreads();
    }
}

template <int BS>
__global__ void k_spgemm_fill_smem(int nrows, const int *__restrict__ arp, const int *__restrict__ aci,
                                   const double *__restrict__ av, const int *__restrict__ brp,
                                   const int *__restrict__ bci, const double *__restrict__ bv, int ncols,
                                   const int *__restrict__ crp, int *__restrict__ cci, double *__restrict__ cv)
{
    constexpr int BB = BS * BS;
    extern __shared__ double sacc[];
    int *mark = (int *)(sacc + (size_t)ncols * BB);
    int *cols = mark + ncols;
    __shared__ int count;
    for (int j = threadIdx.x; j < ncols; j += blockDim.x) mark[j] = -1;
    __syncthreads();
    for (int i = blockIdx.x; i < nrows; i += gridDim.x) {
        if (threadIdx.x == 0) count = 0;
        __syncthreads();
        for (int t = arp[i]; t < arp[i + 1]; t++) {
            int k = aci[t];
            double a[BB];
#pragma unroll
            for (int e = 0; e < BB; e++) a[e] = av[(size_t)t * BB + e];
            for (int s2 = brp[k] + threadIdx.x; s2 < brp[k + 1]; s2 += blockDim.x) {
                int j = bci[s2];
                double *c = sacc + (size_t)j * BB;
                if (mark[j] != i) {
                    mark[j] = i;
#pragma unroll
                    for (int e = 0; e < BB; e++) c[e] = 0.0;
                    cols[atomicAdd(&count, 1)] = j;
                }
                const double *b = bv + (size_t)s2 * BB;
                if (BS == 1) {
                    c[0] = c[0] + a[0] * b[0];
                } else {
                    // scalar middle index 2k then 2k+1
                    c[0] = c[0] + a[0] * b[0];
                    c[0] = c[0] + a[1] * b[2];
                    c[1] = c[1] + a[0] * b[1];
                    c[1] = c[1] + a[1] * b[3];
                    c[2] = c[2] + a[2] * b[0];
                    c[2] = c[2] + a[3] * b[2];
                    c[3] = c[3] + a[2] * b[1];
                    c[3] = c[3] + a[3] * b[3];
                }
            }
            __syncthreads();
        }
        int n = count;
        int p2 = 1;
        while (p2 < n) p2 <<= 1;
        for (int x = n + threadIdx.x; x < p2; x += blockDim.x) cols[x] = INT_MAX;
        __syncthreads();
        for (int kk = 2; kk <= p2; kk <<= 1)
            for (int jj = kk >> 1; jj > 0; jj >>= 1) {
                for (int x = threadIdx.x; x < p2; x += blockDim.x) {
                    int y = x ^ jj;
                    if (y > x) {
                        bool up = (x & kk) == 0;
                        int cx = cols[x], cy = cols[y];
                        if ((cx > cy) == up) {
                            cols[x] = cy;
                            cols[y] = cx;
                        }
                    }
                }
                __syncthreads();
            }
        int base = crp[i];
        for (int x = threadIdx.x; x < n; x += blockDim.x) {
            int j = cols[x];
            cci[base + x] = j;
#pragma unroll
            for (int e = 0; e < BB; e++) cv[(size_t)(base + x) * BB + e] = sacc[(size_t)j * BB + e];
        }
        __syncthreads();
    }
}

// Hash path for products with very many columns and short rows (the squared
// strength graph of a large fine level): one warp per output row, open
// addressing in shared memory, the same accumulation order.
__device__ __forceinline__ int hslot(int key, int mask) { return (int)(((unsigned)key * 2654435761u) & (unsigned)mask); }

__global__ void k_spgemm_bound(int nrows, const int *__restrict__ arp, const int *__restrict__ aci,
                               const int *__restrict__ brp, int *__restrict__ ub)
{
    int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= nrows) return;
    long long u = 0;
    for (int t = arp[i]; t < arp[i + 1]; t++) u += brp[aci[t] + 1] - brp[aci[t]];
    ub[i] = u > INT_MAX ? INT_MAX : (int)u;
}

// Hash-path SpGEMM: L lanes per output row, 32/L rows per warp (L from the
// average row length of B, so that short rows of B -- a tentative
// prolongator has one block per row -- do not leave most lanes idle: every
// FP64 instruction costs the pipe a full warp slot however few lanes are on).
// Each row has its own hash table in shared memory.
template <int L>
__device__ __forceinline__ unsigned sub_mask(int lane)
{
    return L == 32 ? 0xffffffffu : (((1u << L) - 1u) << (lane & ~(L - 1)));
}

template <int L>
__global__ void k_spgemm_count_hash(int nrows, const int *__restrict__ arp, const int *__restrict__ aci,
                                    const int *__restrict__ brp, const int *__restrict__ bci, int HC,
                                    int *__restrict__ cnt, int *overflow)
{
    constexpr int R = 32 / L;
    extern __shared__ int hk[];
    const int warps = blockDim.x >> 5, wid = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int sub = lane / L, sl = lane % L;
    int *keys = hk + ((size_t)wid * R + sub) * HC;
    for (int base = (blockIdx.x * warps + wid) * R; base < nrows; base += gridDim.x * warps * R) {
        const int i = base + sub;
        for (int x = sl; x < HC; x += L) keys[x] = -1;
        __syncwarp();
        int c = 0;
        if (i < nrows) {
            for (int t = arp[i]; t < arp[i + 1]; t++) {
                int k = aci[t];
                for (int s2 = brp[k] + sl; s2 < brp[k + 1]; s2 += L) {
                    int j = bci[s2], h = hslot(j, HC - 1), probe = 0;
                    for (; probe < HC; probe++) {
                        int old = atomicCAS(&keys[h], -1, j);
                        if (old == -1) { c++; break; }
                        if (old == j) break;
                        h = (h + 1) & (HC - 1);
                    }
                    if (probe == HC) atomicOr(overflow, 1);
                }
            }
        }
#pragma unroll
        for (int o = L / 2; o; o >>= 1) c += __shfl_xor_sync(0xffffffffu, c, o, L);
        if (i < nrows && sl == 0) cnt[i] = c;
        __syncwarp();
    }
}

template <int BS, int L>
__global__ void k_spgemm_fill_hash(int nrows, const int *__restrict__ arp, const int *__restrict__ aci,
                                   const double *__restrict__ av, const int *__restrict__ brp,
                                   const int *__restrict__ bci, const double *__restrict__ bv, int HC,
                                   const int *__restrict__ crp, int *__restrict__ cci,
                                   double *__restrict__ cv)
{
    constexpr int BB = BS * BS;
    constexpr int R = 32 / L;
    extern __shared__ double hs[];
    const int warps = blockDim.x >> 5, wid = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int sub = lane / L, sl = lane % L;
    const size_t per = (size_t)HC * BB + (size_t)(3 * HC + 1) / 2;  // in doubles
    double *acc = hs + ((size_t)wid * R + sub) * per;
    int *keys = (int *)(acc + (size_t)HC * BB);
    int *sk = keys + HC, *sp = sk + HC;
    for (int base = (blockIdx.x * warps + wid) * R; base < nrows; base += gridDim.x * warps * R) {
        const int i = base + sub;
        const bool act = i < nrows;
        for (int x = sl; x < HC; x += L) keys[x] = -1;
        __syncwarp();
        // middle indices in ascending order, all rows of the warp in step (a
        // barrier per middle index keeps each entry's additions in that order)
        const int t0 = act ? arp[i] : 0, tn = act ? arp[i + 1] - t0 : 0;
        int tmax = tn;
#pragma unroll
        for (int o = 16; o; o >>= 1) tmax = max(tmax, __shfl_xor_sync(0xffffffffu, tmax, o));
        for (int tt = 0; tt < tmax; tt++) {
            if (tt < tn) {
                const int t = t0 + tt;
                const int k = aci[t];
                double a[BB];
#pragma unroll
                for (int e = 0; e < BB; e++) a[e] = av[(size_t)t * BB + e];
                for (int s2 = brp[k] + sl; s2 < brp[k + 1]; s2 += L) {
                    int j = bci[s2], h = hslot(j, HC - 1);
                    for (int probe = 0; probe < HC; probe++) {
                        int old = atomicCAS(&keys[h], -1, j);
                        if (old == -1) {
#pragma unroll
                            for (int e = 0; e < BB; e++) acc[(size_t)h * BB + e] = 0.0;
                            break;
                        }
                        if (old == j) break;
                        h = (h + 1) & (HC - 1);
                    }
                    double *c = acc + (size_t)h * BB;
                    const double *b = bv + (size_t)s2 * BB;
                    if (BS == 1) {
                        c[0] = c[0] + a[0] * b[0];
                    } else {
                        c[0] = c[0] + a[0] * b[0];
                        c[0] = c[0] + a[1] * b[2];
                        c[1] = c[1] + a[0] * b[1];
                        c[1] = c[1] + a[1] * b[3];
                        c[2] = c[2] + a[2] * b[0];
                        c[2] = c[2] + a[3] * b[2];
                        c[3] = c[3] + a[2] * b[1];
                        c[3] = c[3] + a[3] * b[3];
                    }
                }
            }
            __syncwarp();
        }
        // compact the occupied slots, sort them by column, emit
        const unsigned smask = sub_mask<L>(lane);
        int n = 0;
        for (int x0 = 0; x0 < HC; x0 += L) {
            const int x = x0 + sl;
            const bool has = keys[x] != -1;
            const unsigned m = __ballot_sync(0xffffffffu, has) & smask;
            if (has) {
                const int pos = n + __popc(m & ((1u << lane) - 1u));
                sk[pos] = keys[x];
                sp[pos] = x;
            }
            n += __popc(m);
        }
        int p2 = 1;
        while (p2 < n) p2 <<= 1;
        int p2max = p2;
#pragma unroll
        for (int o = 16; o; o >>= 1) p2max = max(p2max, __shfl_xor_sync(0xffffffffu, p2max, o));
        for (int x = n + sl; x < p2max; x += L) {
            sk[x] = INT_MAX;
            sp[x] = 0;
        }
        __syncwarp();
        for (int kk = 2; kk <= p2max; kk <<= 1)
            for (int jj = kk >> 1; jj > 0; jj >>= 1) {
                for (int x = sl; x < p2max; x += L) {
                    int y = x ^ jj;
                    if (y > x) {
                        bool up = (x & kk) == 0;
                        int cx = sk[x], cy = sk[y];
                        if ((cx > cy) == up) {
                            sk[x] = cy;
                            sk[y] = cx;
                            int tp = sp[x];
                            sp[x] = sp[y];
                            sp[y] = tp;
                        }
                    }
                }
                __syncwarp();
            }
        if (act) {
            const int cb = crp[i];
            for (int x = sl; x < n; x += L) {
                cci[cb + x] = sk[x];
#pragma unroll
                for (int e = 0; e < BB; e++) cv[(size_t)(cb + x) * BB + e] = acc[(size_t)sp[x] * BB + e];
            }
        }
        __syncwarp();
    }
}

static int pow2_at_least(long long v)
{
    int p = 1;
    while (p < v) p <<= 1;
    return p;
}

constexpr long long kHashProducts = 4096;  // products per row up to which the hash path is used

// Lanes per output row of the hash path: the power of two nearest above the
// average row length of B (at most 32).
static int hash_lanes(double b_per_row)
{
    int L = 1;
    while (L < 32 && L < b_per_row) L <<= 1;
    return L;
}

template <int L>
static int launch_count_hash(int nrows, int HCs, const int *arp, const int *aci, const int *brp, const int *bci,
                             int *cnt, int *flag, cudaStream_t s)
{
    constexpr int R = 32 / L;
    const size_t per_warp = (size_t)R * HCs * 4;
    const int warps = std::max(1, std::min(8, (int)((192u << 10) / per_warp)));
    const size_t smem = (size_t)warps * per_warp;
    if (smem > (227u << 10)) return BD_ERANGE;
    BD_CUDA(cudaFuncSetAttribute(k_spgemm_count_hash<L>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
    const long long rows_per_block = (long long)warps * R;
    const int gb = (int)std::min<long long>(kSM * 8, std::max<long long>(1, (nrows + rows_per_block - 1) / rows_per_block));
    k_spgemm_count_hash<L><<<gb, 32 * warps, smem, s>>>(nrows, arp, aci, brp, bci, HCs, cnt, flag); ::bd::note_launch();
    BD_LAUNCH_CHECK();
    return BD_OK;
}

template <int BS, int L>
static int launch_fill_hash(int nrows, int HCn, const int *arp, const int *aci, const double *av, const int *brp,
                            const int *bci, const double *bv, const int *crp, int *cci, double *cv, cudaStream_t s)
{
    constexpr int R = 32 / L;
    const size_t per = ((size_t)HCn * BS * BS + (size_t)(3 * HCn + 1) / 2) * sizeof(double);
    const size_t per_warp = (size_t)R * per;
    if (per_warp > (200u << 10)) return BD_ERANGE;
    const int warps = std::max(1, std::min(8, (int)((200u << 10) / per_warp)));
    const size_t smem = per_warp * warps;
    BD_CUDA(cudaFuncSetAttribute(k_spgemm_fill_hash<BS, L>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
    const long long rows_per_block = (long long)warps * R;
    const int gb = (int)std::min<long long>(kSM * 8, std::max<long long>(1, (nrows + rows_per_block - 1) / rows_per_block));
    k_spgemm_fill_hash<BS, L><<<gb, 32 * warps, smem, s>>>(nrows, arp, aci, av, brp, bci, bv, HCn, crp, cci, cv);
    ::bd::note_launch();
    BD_LAUNCH_CHECK();
    return BD_OK;
}

// b_per_row: average blocks per row of B (sets the lanes per row of the hash path)
template <int BS>
static int spgemm(int nrows, int ncols, const int *arp, const int *aci, const double *av,
                  const int *brp, const int *bci, const double *bv, DBuf<int> &crp, DBuf<int> &cci,
                  DBuf<double> &cv, long long *cnnz, cudaStream_t s, double b_per_row)
{
    constexpr int BB = BS * BS;
    BD_TRY(crp.alloc((size_t)nrows + 1));
    DBuf<int> cnt;
    BD_TRY(cnt.alloc((size_t)nrows + 1));
    size_t per_block = (size_t)ncols * (sizeof(int) + BB * sizeof(double));
    long long g = kSM * 4;
    long long cap = (2LL << 30) / (long long)(per_block ? per_block : 1);
    if (g > cap) g = cap;
    bool dense = g >= kSM || g >= nrows;
    if (g > nrows) g = nrows > 0 ? nrows : 1;
    if (g < 1) g = 1;
    int grid = (int)g;
    DBuf<int> mark;
    DBuf<double> acc;
    DBuf<int> flag;  // [0] hash-table overflow, [1] largest product bound, [2] longest output row
    BD_TRY(flag.alloc(3));
    BD_CUDA(cudaMemsetAsync(flag.p, 0, 3 * sizeof(int), s));
    // Rows with few products (the fine levels' many short rows) go to the
    // warp-per-row hash path: the dense path's thread block per row then idles
    // most of its threads and synchronises once per middle index.  Both paths
    // accumulate every entry in the same order, so the choice changes no bit.
    long long mub = 1;
    if (nrows > 0) {
        k_spgemm_bound<<<(nrows + 255) / 256, 256, 0, s>>>(nrows, arp, aci, brp, cnt.p); ::bd::note_launch();
        BD_LAUNCH_CHECK();
        BD_TRY(device_max(cnt.p, nrows, flag.p + 1, s));
        int hb = 0;
        BD_CUDA(cudaMemcpyAsync(&hb, flag.p + 1, sizeof(int), cudaMemcpyDeviceToHost, s));
        BD_CUDA(cudaStreamSynchronize(s));
        mub = std::max<long long>(mub, hb);
        if (mub <= kHashProducts) dense = false;
    }
    int HCn = 0;
    const int lanes = hash_lanes(b_per_row);
    ::bd::note_spgemm_path(dense);
    // the dense path keeps a row's accumulators in shared memory when they
    // fit (with the largest column list a row can have)
    const size_t dense_smem = (size_t)ncols * (BB * sizeof(double) + sizeof(int)) +
                              (size_t)pow2_at_least(std::max(ncols, 1)) * sizeof(int);
    const bool dense_in_smem = dense && dense_smem <= (200u << 10);
    if (dense_in_smem) {
        const size_t cs = (size_t)ncols * sizeof(int);
        BD_CUDA(cudaFuncSetAttribute(k_spgemm_count_smem, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                     (int)std::max<size_t>(cs, 4)));
        const int gc = (int)std::min<long long>(nrows, (long long)kSM * 8);
        k_spgemm_count_smem<<<std::max(gc, 1), 128, std::max<size_t>(cs, 4), s>>>(nrows, arp, aci, brp, bci, ncols,
                                                                                   cnt.p);
        ::bd::note_launch();
        BD_LAUNCH_CHECK();
    } else if (dense) {
        BD_TRY(mark.alloc((size_t)grid * ncols));
        BD_TRY(acc.alloc((size_t)grid * ncols * BB));
        BD_CUDA(cudaMemsetAsync(mark.p, 0xff, mark.bytes(), s));
        k_spgemm_count<BS><<<grid, 128, 0, s>>>(nrows, arp, aci, brp, bci, ncols, mark.p, cnt.p); ::bd::note_launch();
        BD_LAUNCH_CHECK();
    } else {
        int HCs = pow2_at_least(2 * std::min<long long>(mub, kMaxSortSeg));
        if (HCs < 32) HCs = 32;
        // rows whose tables do not fit 32/lanes to a warp take more lanes each
        int Lc = lanes;
        while (Lc < 32 && (size_t)(32 / Lc) * HCs * 4 > (192u << 10)) Lc <<= 1;
        switch (Lc) {
        case 1: BD_TRY(launch_count_hash<1>(nrows, HCs, arp, aci, brp, bci, cnt.p, flag.p, s)); break;
        case 2: BD_TRY(launch_count_hash<2>(nrows, HCs, arp, aci, brp, bci, cnt.p, flag.p, s)); break;
        case 4: BD_TRY(launch_count_hash<4>(nrows, HCs, arp, aci, brp, bci, cnt.p, flag.p, s)); break;
        case 8: BD_TRY(launch_count_hash<8>(nrows, HCs, arp, aci, brp, bci, cnt.p, flag.p, s)); break;
        case 16: BD_TRY(launch_count_hash<16>(nrows, HCs, arp, aci, brp, bci, cnt.p, flag.p, s)); break;
        default: BD_TRY(launch_count_hash<32>(nrows, HCs, arp, aci, brp, bci, cnt.p, flag.p, s)); break;
        }
    }
    BD_TRY(device_max(cnt.p, nrows, flag.p + 2, s));  // cnt: the output row lengths
    long long total = 0;
    BD_TRY(exclusive_scan(cnt.p, crp.p, nrows, &total, s));
    int hf[3] = {0, 0, 0};
    BD_CUDA(cudaMemcpyAsync(hf, flag.p, sizeof(hf), cudaMemcpyDeviceToHost, s));
    BD_CUDA(cudaStreamSynchronize(s));
    if (hf[0]) return BD_ERANGE;
    const int maxrow = hf[2];
    if (maxrow > kMaxSortSeg) return BD_ERANGE;
    BD_TRY(cci.alloc((size_t)total));
    BD_TRY(cv.alloc((size_t)total * BB));
    if (dense_in_smem) {
        BD_CUDA(cudaFuncSetAttribute(k_spgemm_fill_smem<BS>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                     (int)dense_smem));
        const int per_sm = std::max(1, (int)((227u << 10) / (dense_smem + 1024)));
        const int gf = (int)std::min<long long>(nrows, (long long)kSM * per_sm);
        k_spgemm_fill_smem<BS><<<std::max(gf, 1), 256, dense_smem, s>>>(nrows, arp, aci, av, brp, bci, bv, ncols,
                                                                         crp.p, cci.p, cv.p);
        ::bd::note_launch();
        BD_LAUNCH_CHECK();
    } else if (dense) {
        int P2 = pow2_at_least(maxrow);
        BD_CUDA(cudaMemsetAsync(mark.p, 0xff, mark.bytes(), s));
        size_t smem = (size_t)P2 * sizeof(int);
        BD_CUDA(cudaFuncSetAttribute(k_spgemm_fill<BS>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                     (int)std::max<size_t>(smem, 4)));
        k_spgemm_fill<BS><<<grid, 128, smem, s>>>(nrows, arp, aci, av, brp, bci, bv, ncols, mark.p,
                                                  acc.p, crp.p, cci.p, cv.p, P2); ::bd::note_launch();
        BD_LAUNCH_CHECK();
    } else {
        HCn = pow2_at_least(2LL * std::max(maxrow, 16));
        // rows whose tables do not fit 32/lanes to a warp take more lanes each
        int Lf = lanes;
        while (Lf < 32 && (size_t)(32 / Lf) * (((size_t)HCn * BB + (size_t)(3 * HCn + 1) / 2) * sizeof(double)) >
                              (200u << 10))
            Lf <<= 1;
        switch (Lf) {
        case 1: BD_TRY((launch_fill_hash<BS, 1>(nrows, HCn, arp, aci, av, brp, bci, bv, crp.p, cci.p, cv.p, s))); break;
        case 2: BD_TRY((launch_fill_hash<BS, 2>(nrows, HCn, arp, aci, av, brp, bci, bv, crp.p, cci.p, cv.p, s))); break;
        case 4: BD_TRY((launch_fill_hash<BS, 4>(nrows, HCn, arp, aci, av, brp, bci, bv, crp.p, cci.p, cv.p, s))); break;
        case 8: BD_TRY((launch_fill_hash<BS, 8>(nrows, HCn, arp, aci, av, brp, bci, bv, crp.p, cci.p, cv.p, s))); break;
        case 16: BD_TRY((launch_fill_hash<BS, 16>(nrows, HCn, arp, aci, av, brp, bci, bv, crp.p, cci.p, cv.p, s))); break;
        default: BD_TRY((launch_fill_hash<BS, 32>(nrows, HCn, arp, aci, av, brp, bci, bv, crp.p, cci.p, cv.p, s))); break;
        }
    }
    *cnnz = total;
    return BD_OK;
}

// ------------------------------------------------------------------ squared graph
// Wh = I + W (unit diagonal inserted in order), S2 = Wh*Wh without diagonal.
__global__ void k_insert_diag(int N, const int *__restrict__ srp, const int *__restrict__ sci,
                              const double *__restrict__ sw, int *__restrict__ wrp,
                              int *__restrict__ wci, double *__restrict__ wv)
{
    int p = blockIdx.x * blockDim.x + threadIdx.x;
    if (p > N) return;
    wrp[p] = srp[p] + p;
    if (p == N) return;
    int pos = srp[p] + p;
    bool done = false;
    for (int t = srp[p]; t < srp[p + 1]; t++) {
        if (!done && sci[t] > p) {
            wci[pos] = p;
            wv[pos++] = 1.0;
            done = true;
        }
        wci[pos] = sci[t];
        wv[pos++] = sw[t];
    }
    if (!done) {
        wci[pos] = p;
        wv[pos] = 1.0;
    }
}

__global__ void k_drop_diag(int N, const int *__restrict__ qrp, const int *__restrict__ qci,
                            const double *__restrict__ qv, int *__restrict__ orp,
                            int *__restrict__ oci, double *__restrict__ ov)
{
    int p = blockIdx.x * blockDim.x + threadIdx.x;
    if (p > N) return;
    orp[p] = qrp[p] - p;  // every row of Wh*Wh holds its diagonal
    if (p == N) return;
    int pos = qrp[p] - p;
    for (int t = qrp[p]; t < qrp[p + 1]; t++) {
        if (qci[t] == p) continue;
        oci[pos] = qci[t];
        ov[pos++] = qv[t];
    }
}

// ------------------------------------------------------------------ a2 MIS (Luby rounds)
// state: 0 undecided, 1 in the set, 2 out.  Node p beats q when its priority
// (mix64(p ^ key), -p) is larger.  With fixed priorities the rounds return the
// set the sequential greedy pass builds in decreasing priority.
__device__ __forceinline__ bool beats(unsigned long long hp, int p, unsigned long long hq, int q)
{
    return hp > hq || (hp == hq && p < q);
}

__global__ void k_mis_select(int N, const int *__restrict__ srp, const int *__restrict__ sci,
                             unsigned char *state, unsigned long long key)
{
    int p = blockIdx.x * blockDim.x + threadIdx.x;
    if (p >= N || state[p] != 0) return;
    unsigned long long hp = mix64((unsigned long long)p ^ key);
    for (int t = srp[p]; t < srp[p + 1]; t++) {
        int q = sci[t];
        unsigned char sq = ((volatile unsigned char *)state)[q];
        if (sq == 1) return;
        if (sq == 0 && beats(mix64((unsigned long long)q ^ key), q, hp, p)) return;
    }
    state[p] = 1;
}

__global__ void k_mis_exclude(int N, const int *__restrict__ srp, const int *__restrict__ sci,
                              unsigned char *state, int *undecided)
{
    int p = blockIdx.x * blockDim.x + threadIdx.x;
    if (p >= N || state[p] != 0) return;
    for (int t = srp[p]; t < srp[p + 1]; t++)
        if (state[sci[t]] == 1) {
            state[p] = 2;
            return;
        }
    atomicAdd(undecided, 1);
}

// ------------------------------------------------------------------ a3 aggregation
__global__ void k_root_flags(int N, const unsigned char *state, unsigned char *mis, int *flag)
{
    int p = blockIdx.x * blockDim.x + threadIdx.x;
    if (p >= N) return;
    int r = state[p] == 1;
    mis[p] = (unsigned char)r;
    flag[p] = r;
}

__global__ void k_assign(int N, const int *__restrict__ srp, const int *__restrict__ sci,
                         const double *__restrict__ sw, const unsigned char *__restrict__ mis,
                         const int *__restrict__ root_id, int *__restrict__ agg, int *bad)
{
    int p = blockIdx.x * blockDim.x + threadIdx.x;
    if (p >= N) return;
    if (mis[p]) {
        agg[p] = root_id[p];
        return;
    }
    int best = -1;
    double bw = -1.0;
    for (int t = srp[p]; t < srp[p + 1]; t++) {
        int q = sci[t];
        if (mis[q] && sw[t] > bw) {
            bw = sw[t];
            best = q;
        }
    }
    if (best < 0) {
        *bad = 1;
        agg[p] = 0;
        return;
    }
    agg[p] = root_id[best];
}

// ------------------------------------------------------------------ a4 tentative prolongator
__global__ void k_count_members(int N, const int *agg, int *cnt)
{
    int p = blockIdx.x * blockDim.x + threadIdx.x;
    if (p < N) atomicAdd(&cnt[agg[p]], 1);
}

__global__ void k_scatter_members(int N, const int *agg, const int *off, int *fill, int *members)
{
    int p = blockIdx.x * blockDim.x + threadIdx.x;
    if (p < N) {
        int J = agg[p];
        members[off[J] + atomicAdd(&fill[J], 1)] = p;
    }
}

// Bc(2J+f) = sqrt(sum over members k ascending of B(2k+f)^2)
__global__ void k_coarse_B(int nagg, const int *__restrict__ off, const int *__restrict__ members,
                           const double *__restrict__ B, double *__restrict__ Bc)
{
    int J = blockIdx.x * blockDim.x + threadIdx.x;
    if (J >= nagg) return;
    double s0 = 0.0, s1 = 0.0;
    for (int t = off[J]; t < off[J + 1]; t++) {
        int k = members[t];
        double b0 = B[2 * k], b1 = B[2 * k + 1];
        s0 = s0 + b0 * b0;
        s1 = s1 + b1 * b1;
    }
    Bc[2 * J] = sqrt(s0);
    Bc[2 * J + 1] = sqrt(s1);
}

// Pt as 2x2-block CSR: one block per node row, diag(B(2k)/Bc(2J), B(2k+1)/Bc(2J+1)).
__global__ void k_ptent(int N, const int *__restrict__ agg, const double *__restrict__ B,
                        const double *__restrict__ Bc, int *__restrict__ rp, int *__restrict__ ci,
                        double *__restrict__ v, double *__restrict__ ptd)
{
    int p = blockIdx.x * blockDim.x + threadIdx.x;
    if (p > N) return;
    rp[p] = p;
    if (p == N) return;
    int J = agg[p];
    double a = B[2 * p] / Bc[2 * J], b = B[2 * p + 1] / Bc[2 * J + 1];
    ci[p] = J;
    v[4 * (size_t)p + 0] = a;
    v[4 * (size_t)p + 1] = 0.0;
    v[4 * (size_t)p + 2] = 0.0;
    v[4 * (size_t)p + 3] = b;
    ptd[2 * p] = a;
    ptd[2 * p + 1] = b;
}

// ------------------------------------------------------------------ a5 lambda_max (CG-Lanczos)
struct LanczosState {
    double rz, pq, rz1;
    double alpha[64], beta[64];
    int m, stop;
    double lam;
    int bad;
};

__global__ void k_lanczos_init(int n, unsigned long long key, const double *__restrict__ diag,
                               double *r, double *z, double *p)
{
    int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    unsigned long long h = mix64(key ^ (unsigned long long)i);
    double u = (double)(h >> 11) * (1.0 / 9007199254740992.0);
    double ri = 2.0 * u - 1.0;
    double zi = ri / diag[i];
    r[i] = ri;
    z[i] = zi;
    p[i] = zi;
}

// y = A x, scalar rows in ascending column order, acc = acc + a*x from 0.0
__global__ void k_spmv_ordered(int N, const int *__restrict__ rp, const int *__restrict__ ci,
                               const double *__restrict__ v, const double *__restrict__ x,
                               double *__restrict__ y)
{
    int p = blockIdx.x * blockDim.x + threadIdx.x;
    if (p >= N) return;
    double s0 = 0.0, s1 = 0.0;
    for (int t = rp[p]; t < rp[p + 1]; t++) {
        int q = ci[t];
        double x0 = x[2 * q], x1 = x[2 * q + 1];
        const double *a = v + 4 * (size_t)t;
        s0 = s0 + a[0] * x0;
        s0 = s0 + a[1] * x1;
        s1 = s1 + a[2] * x0;
        s1 = s1 + a[3] * x1;
    }
    y[2 * p] = s0;
    y[2 * p + 1] = s1;
}

__global__ void k_lanczos_alpha(LanczosState *st, int j)
{
    if (st->stop) return;
    if (!(st->pq > 0.0) || !(st->rz > 0.0)) {
        st->stop = 1;
        return;
    }
    st->alpha[j] = st->rz / st->pq;
}

__global__ void k_lanczos_update_r(int n, const LanczosState *st, int j, const double *__restrict__ q,
                                   const double *__restrict__ diag, double *r, double *z)
{
    if (st->stop) return;
    int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    double a = st->alpha[j];
    double ri = r[i] - a * q[i];
    r[i] = ri;
    z[i] = ri / diag[i];
}

__global__ void k_lanczos_beta(LanczosState *st, int j)
{
    if (st->stop) return;
    double beta = st->rz1 / st->rz;
    st->beta[j] = beta;
    st->m = j + 1;
    if (!(st->rz1 > 0.0)) {
        st->stop = 1;
        return;
    }
    st->rz = st->rz1;
}

__global__ void k_lanczos_update_p(int n, const LanczosState *st, int j, const double *__restrict__ z,
                                   double *p)
{
    if (st->stop) return;
    int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    double b = st->beta[j];
    p[i] = z[i] + b * p[i];
}

__device__ int sturm_count_below(int m, const double *d, const double *e, double x)
{
    int c = 0;
    double q = d[0] - x;
    if (q < 0.0) c++;
    for (int i = 1; i < m; i++) {
        if (q == 0.0) q = -1e-300;
        q = (d[i] - x) - (e[i - 1] * e[i - 1]) / q;
        if (q < 0.0) c++;
    }
    return c;
}

__global__ void k_lanczos_finish(LanczosState *st)
{
    int m = st->m;
    if (m == 0) {
        st->bad = 1;
        st->lam = 0.0;
        return;
    }
    double d[64], e[64];
    for (int j = 0; j < m; j++) {
        d[j] = 1.0 / st->alpha[j];
        if (j > 0) d[j] = d[j] + st->beta[j - 1] / st->alpha[j - 1];
        if (j < m - 1) e[j] = sqrt(st->beta[j]) / st->alpha[j];
    }
    double lo = 0.0, hi = 0.0;
    for (int i = 0; i < m; i++) {
        double r = 0.0;
        if (i > 0) r = r + fabs(e[i - 1]);
        if (i < m - 1) r = r + fabs(e[i]);
        double a = d[i] - r, b = d[i] + r;
        if (i == 0 || a < lo) lo = a;
        if (i == 0 || b > hi) hi = b;
    }
    for (int it = 0; it < 4096; it++) {
        double mid = 0.5 * (lo + hi);
        if (!(mid > lo && mid < hi)) break;
        if (sturm_count_below(m, d, e, mid) == m) hi = mid;
        else lo = mid;
    }
    st->lam = hi;
}

// ------------------------------------------------------------------ a6 smoothed prolongator
// P(i,j) = Pt(i,j) - s_i AP(i,j),  s_i = omega / A(i,i),  omega = 4/(3 lambda)
__global__ void k_smooth_p(int N, const int *__restrict__ rp, const int *__restrict__ ci,
                           double *__restrict__ v, const int *__restrict__ agg,
                           const double *__restrict__ ptd, const double *__restrict__ diag,
                           const LanczosState *st)
{
    int p = blockIdx.x * blockDim.x + threadIdx.x;
    if (p >= N) return;
    double omega = 4.0 / (3.0 * st->lam);
    double s0 = omega / diag[2 * p], s1 = omega / diag[2 * p + 1];
    int J = agg[p];
    for (int t = rp[p]; t < rp[p + 1]; t++) {
        bool own = ci[t] == J;
        double *b = v + 4 * (size_t)t;
        double p00 = own ? ptd[2 * p] : 0.0, p11 = own ? ptd[2 * p + 1] : 0.0;
        b[0] = p00 - s0 * b[0];
        b[1] = 0.0 - s0 * b[1];
        b[2] = 0.0 - s1 * b[2];
        b[3] = p11 - s1 * b[3];
    }
}

// ------------------------------------------------------------------ a7 transpose
__global__ void k_count_cols(long long nb, const int *ci, int *cnt)
{
    long long t = blockIdx.x * (long long)blockDim.x + threadIdx.x;
    if (t < nb) atomicAdd(&cnt[ci[t]], 1);
}

__global__ void k_scatter_t(int N, const int *__restrict__ rp, const int *__restrict__ ci,
                            const int *__restrict__ off, int *fill, int *tci, int *perm)
{
    int p = blockIdx.x * blockDim.x + threadIdx.x;
    if (p >= N) return;
    for (int t = rp[p]; t < rp[p + 1]; t++) {
        int J = ci[t];
        int pos = off[J] + atomicAdd(&fill[J], 1);
        tci[pos] = p;
        perm[pos] = t;
    }
}

__global__ void k_gather_t(long long nb, const int *__restrict__ perm, const double *__restrict__ v,
                           double *__restrict__ tv)
{
    long long t = blockIdx.x * (long long)blockDim.x + threadIdx.x;
    if (t >= nb) return;
    const double *a = v + 4 * (size_t)perm[t];
    double *b = tv + 4 * (size_t)t;
    b[0] = a[0];
    b[1] = a[2];
    b[2] = a[1];
    b[3] = a[3];
}

static int bsr_transpose(const BSR &a, BSR &t, cudaStream_t s)
{
    t.nbr = a.nbc;
    t.nbc = a.nbr;
    t.nb = a.nb;
    DBuf<int> cnt, fill, perm;
    BD_TRY(cnt.alloc((size_t)a.nbc + 2));  // counts, then the largest at [a.nbc + 1]
    BD_TRY(fill.alloc((size_t)a.nbc + 1));
    BD_TRY(perm.alloc((size_t)a.nb));
    BD_TRY(t.rp.alloc((size_t)a.nbc + 1));
    BD_TRY(t.ci.alloc((size_t)a.nb));
    BD_TRY(t.v.alloc(4 * (size_t)a.nb));
    BD_CUDA(cudaMemsetAsync(cnt.p, 0, cnt.bytes(), s));
    BD_CUDA(cudaMemsetAsync(fill.p, 0, fill.bytes(), s));
    k_count_cols<<<(int)((a.nb + 255) / 256), 256, 0, s>>>(a.nb, a.ci.p, cnt.p); ::bd::note_launch();
    BD_LAUNCH_CHECK();
    BD_TRY(device_max(cnt.p, a.nbc, cnt.p + a.nbc + 1, s));
    long long tot = 0;
    BD_TRY(exclusive_scan(cnt.p, t.rp.p, a.nbc, &tot, s));  // stream synchronised
    int mx = 0;
    BD_CUDA(cudaMemcpyAsync(&mx, cnt.p + a.nbc + 1, sizeof(int), cudaMemcpyDeviceToHost, s));
    BD_CUDA(cudaStreamSynchronize(s));
    k_scatter_t<<<(a.nbr + 255) / 256, 256, 0, s>>>(a.nbr, a.rp.p, a.ci.p, t.rp.p, fill.p, t.ci.p,
                                                    perm.p); ::bd::note_launch();
    BD_LAUNCH_CHECK();
    BD_TRY(sort_segments(t.ci.p, perm.p, t.rp.p, a.nbc, mx, s));
    k_gather_t<<<(int)((a.nb + 255) / 256), 256, 0, s>>>(a.nb, perm.p, a.v.p, t.v.p); ::bd::note_launch();
    BD_LAUNCH_CHECK();
    return BD_OK;
}

// ------------------------------------------------------------------ a9 coarsest level
__global__ void k_coarse_dense(int N, const int *__restrict__ rp, const int *__restrict__ ci,
                               const double *__restrict__ v, double *__restrict__ Ad)
{
    int p = blockIdx.x * blockDim.x + threadIdx.x;
    if (p >= N) return;
    int n = 2 * N;
    for (int t = rp[p]; t < rp[p + 1]; t++) {
        int q = ci[t];
        Ad[(size_t)(2 * p) * n + 2 * q] = v[4 * (size_t)t];
        Ad[(size_t)(2 * p) * n + 2 * q + 1] = v[4 * (size_t)t + 1];
        Ad[(size_t)(2 * p + 1) * n + 2 * q] = v[4 * (size_t)t + 2];
        Ad[(size_t)(2 * p + 1) * n + 2 * q + 1] = v[4 * (size_t)t + 3];
    }
}

// Single block: rank-one fix, Cholesky (left-looking, sums ascending), then the
// explicit inverse by forward/backward substitution of unit vectors.
__global__ void k_coarse_factor(int n, double *A, const double *__restrict__ z, double *Ainv,
                                double *zz_out, int *bad)
{
    __shared__ double smax_s, zz_s;
    if (threadIdx.x == 0) {
        double smax = 0.0, zz = 0.0;
        for (int i = 0; i < n; i++) {
            double d = A[(size_t)i * n + i];
            if (d > smax) smax = d;
            zz = zz + z[i] * z[i];
        }
        smax_s = smax;
        zz_s = zz;
        *zz_out = zz;
    }
    __syncthreads();
    double smax = smax_s, zz = zz_s;
    for (size_t e = threadIdx.x; e < (size_t)n * n; e += blockDim.x) {
        int i = (int)(e / n), j = (int)(e % n);
        A[e] = A[e] + (smax * z[i]) * z[j] / zz;
    }
    __syncthreads();
    __shared__ double dj;
    for (int j = 0; j < n; j++) {
        if (threadIdx.x == 0) {
            double sdiag = A[(size_t)j * n + j];
            for (int k = 0; k < j; k++) sdiag = sdiag - A[(size_t)j * n + k] * A[(size_t)j * n + k];
            if (!(sdiag > 0.0)) *bad = 1;
            dj = sqrt(sdiag > 0.0 ? sdiag : 1.0);
            A[(size_t)j * n + j] = dj;
        }
        __syncthreads();
        for (int i = j + 1 + threadIdx.x; i < n; i += blockDim.x) {
            double t = A[(size_t)i * n + j];
            for (int k = 0; k < j; k++) t = t - A[(size_t)i * n + k] * A[(size_t)j * n + k];
            A[(size_t)i * n + j] = t / dj;
        }
        __syncthreads();
    }
    // columns of the inverse: L y = e_c, L^T x = y
    for (int c = threadIdx.x; c < n; c += blockDim.x) {
        double *x = Ainv + (size_t)c * n;  // column c stored contiguously (inverse is symmetric)
        for (int i = 0; i < n; i++) {
            double s = (i == c) ? 1.0 : 0.0;
            for (int k = 0; k < i; k++) s = s - A[(size_t)i * n + k] * x[k];
            x[i] = s / A[(size_t)i * n + i];
        }
        for (int i = n - 1; i >= 0; i--) {
            double s = x[i];
            for (int k = i + 1; k < n; k++) s = s - A[(size_t)k * n + i] * x[k];
            x[i] = s / A[(size_t)i * n + i];
        }
    }
}

// Larger coarsest levels: the same rank-one-fixed matrix, inverted in place by
// Gauss-Jordan elimination without pivoting (the matrix is symmetric positive
// definite), in blocks of kGJ pivots (below).
__global__ void k_coarse_stats(int n, const double *__restrict__ A, const double *__restrict__ z,
                               double *__restrict__ out)
{
    if (threadIdx.x != 0 || blockIdx.x != 0) return;
    double smax = 0.0, zz = 0.0;
    for (int i = 0; i < n; i++) {
        double d = A[(size_t)i * n + i];
        if (d > smax) smax = d;
        zz = zz + z[i] * z[i];
    }
    out[0] = smax;
    out[1] = zz;
}

// one thread block per row, its threads strided over the columns
__global__ void k_coarse_rank1(int n, double *__restrict__ A, const double *__restrict__ z,
                               const double *__restrict__ st)
{
    const double smax = st[0], zz = st[1];
    const int i = blockIdx.x;
    for (int j = threadIdx.x; j < n; j += blockDim.x) {
        const size_t e = (size_t)i * n + j;
        A[e] = A[e] + (smax * z[i]) * z[j] / zz;
    }
}

// Blocked Gauss-Jordan with pivot blocks of kGJ: for the pivot rows P,
// D = A[P,P] is inverted in shared memory, W = D^-1 A[P,:], and every other row
// i takes A[i,j] -= A[i,P] W[:,j] (a rank-kGJ update, FP64-bound, 32 rows per
// thread block so each W value is reused 32 times), A[i,P] = -A[i,P] D^-1,
// while the pivot rows become W with D^-1 in the pivot columns.
constexpr int kGJ = 32;

__global__ void k_gj_pivot(int n, int K, int bb, const double *__restrict__ A, double *__restrict__ Dinv,
                           int *__restrict__ bad)
{
    __shared__ double D[kGJ][kGJ + 1];
    __shared__ double prow[kGJ], pcol[kGJ];
    __shared__ double srp;
    for (int e = threadIdx.x; e < bb * bb; e += blockDim.x) D[e / bb][e % bb] = A[(size_t)(K + e / bb) * n + K + e % bb];
    __syncthreads();
    for (int k = 0; k < bb; k++) {
        // one division per pivot, by one thread: the pivot row is scaled by its
        // reciprocal (FP64 division is a long sequence on the FP64 pipe, and one
        // thread block does all of this)
        if (threadIdx.x == 0) {
            const double piv = D[k][k];
            srp = 1.0 / piv;
            if (!(piv > 0.0)) *bad = 1;
        }
        __syncthreads();
        const double rpiv = srp;
        if (threadIdx.x < bb) {
            prow[threadIdx.x] = D[k][threadIdx.x] * rpiv;
            pcol[threadIdx.x] = D[threadIdx.x][k];
        }
        __syncthreads();
        for (int e = threadIdx.x; e < bb * bb; e += blockDim.x) {
            const int i = e / bb, j = e % bb;
            double a;
            if (i == k && j == k) a = rpiv;
            else if (i == k) a = prow[j];
            else if (j == k) a = -pcol[i] * rpiv;
            else a = D[i][j] - pcol[i] * prow[j];
            D[i][j] = a;
        }
        __syncthreads();
    }
    for (int e = threadIdx.x; e < bb * bb; e += blockDim.x) Dinv[e] = D[e / bb][e % bb];
}

// W[k][j] = sum_m Dinv[k][m] A[K+m][j] for every column j (bb x n), and a copy
// Cb of the pivot columns A[:, P] (the update overwrites them).  blockIdx.y
// takes kGJ / kGJPanelK rows k of W, so the panel spreads over the GPU.
constexpr int kGJPanelK = 4;
__global__ void k_gj_panel(int n, int K, int bb, const double *__restrict__ A, const double *__restrict__ Dinv,
                           double *__restrict__ W, double *__restrict__ Cb)
{
    __shared__ double Di[kGJPanelK][kGJ];
    const int k0 = blockIdx.y * kGJPanelK;
    for (int e = threadIdx.x; e < kGJPanelK * kGJ; e += blockDim.x) {
        const int k = k0 + e / kGJ, m = e % kGJ;
        Di[e / kGJ][m] = k < bb && m < bb ? Dinv[k * bb + m] : 0.0;
    }
    __syncthreads();
    const int j = blockIdx.x * blockDim.x + threadIdx.x;
    if (j >= n || k0 >= bb) return;
    if (blockIdx.y == 0)
        for (int m = 0; m < kGJ; m++) Cb[(size_t)j * kGJ + m] = m < bb ? A[(size_t)j * n + K + m] : 0.0;
    double col[kGJ];
#pragma unroll
    for (int m = 0; m < kGJ; m++) col[m] = m < bb ? A[(size_t)(K + m) * n + j] : 0.0;
#pragma unroll
    for (int kk = 0; kk < kGJPanelK; kk++) {
        const int k = k0 + kk;
        if (k >= bb) break;
        double w = 0.0;
#pragma unroll
        for (int m = 0; m < kGJ; m++) w = fma(Di[kk][m], col[m], w);
        W[(size_t)k * n + j] = w;
    }
}

// Column chunk blockIdx.x * blockDim.x + threadIdx.x, rows [r0, r1): an equal
// share of the n rows for each of the gridDim.y blocks of a column chunk (the
// grid is one resident wave), taken kGJ rows at a time through shared memory.
__global__ void k_gj_update(int n, int K, int bb, double *__restrict__ A, const double *__restrict__ Dinv,
                            const double *__restrict__ W, const double *__restrict__ Cb)
{
    __shared__ double C[kGJ][kGJ];  // A[i, P] of kGJ rows, from the copy
    const int r0 = (int)((long long)n * blockIdx.y / gridDim.y);
    const int r1 = (int)((long long)n * (blockIdx.y + 1) / gridDim.y);
    const int j = blockIdx.x * blockDim.x + threadIdx.x;
    const bool act = j < n;
    const bool jp = j >= K && j < K + bb;
    double w[kGJ];
#pragma unroll
    for (int m = 0; m < kGJ; m++)
        w[m] = act && m < bb ? (jp ? Dinv[m * bb + (j - K)] : W[(size_t)m * n + j]) : 0.0;
    for (int rb = r0; rb < r1; rb += kGJ) {
        const int nr = min(kGJ, r1 - rb);
        __syncthreads();
        for (int e = threadIdx.x; e < kGJ * kGJ; e += blockDim.x) {
            const int r = e / kGJ, m = e % kGJ;
            C[r][m] = r < nr ? Cb[(size_t)(rb + r) * kGJ + m] : 0.0;
        }
        __syncthreads();
        if (!act) continue;
        for (int r = 0; r < nr; r++) {
            const int i = rb + r;
            const size_t e = (size_t)i * n + j;
            if (i >= K && i < K + bb) {  // pivot row: W, with D^-1 in the pivot columns
                // (read from W and D^-1 again: a dynamic index into w would put w in
                // local memory for every multiply-add of the update)
                A[e] = jp ? Dinv[(i - K) * bb + (j - K)] : W[(size_t)(i - K) * n + j];
                continue;
            }
            double a = jp ? 0.0 : A[e];
#pragma unroll
            for (int m = 0; m < kGJ; m++) a = fma(-C[r][m], w[m], a);
            A[e] = a;
        }
    }
}

__global__ void k_null_vector(int N, const double *__restrict__ B, double *z)
{
    int p = blockIdx.x * blockDim.x + threadIdx.x;
    if (p >= N) return;
    z[2 * p] = 0.0;
    z[2 * p + 1] = B[2 * p + 1];
}

__global__ void k_invdiag(int n, const double *__restrict__ d, double *inv)
{
    int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i < n) inv[i] = 1.0 / d[i];
}

__global__ void k_fill(int n, double v, double *x)
{
    int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i < n) x[i] = v;
}

static inline int nblk(long long n, int b = 256) { return (int)((n + b - 1) / b); }

// Thread block size of the one-thread-per-row setup kernels: on coarse levels
// (few, long rows) one warp per block, so the rows spread over as many SMs as
// possible instead of crowding a handful (each row is a sequential sum).
static inline int row_block(long long rows) { return rows < (long long)kSM * 256 ? 32 : 256; }

// ------------------------------------------------------------------ one level of Algorithm 1
static int coarsen_level(amg_hierarchy *h, int l, bool &is_coarsest, cudaStream_t s)
{
    Level &L = h->lev[l];
    const amg_options &o = h->opts;
    int N = L.N, n = 2 * N;
    is_coarsest = false;
    if (n <= o.coarse_eq_limit || l == o.max_levels - 1 || l == kMaxLevels - 1) {
        is_coarsest = true;
        return BD_OK;
    }
    // a1 strength
    DBuf<double> diag;
    BD_TRY(diag.alloc((size_t)n));
    DBuf<int> bad;
    BD_TRY(bad.alloc(1));
    BD_CUDA(cudaMemsetAsync(bad.p, 0, sizeof(int), s));
    k_diag<<<nblk(N), 256, 0, s>>>(N, L.A.rp.p, L.A.ci.p, L.A.v.p, diag.p, bad.p); ::bd::note_launch();
    BD_LAUNCH_CHECK();
    CSR S;
    S.nr = S.nc = N;
    DBuf<int> cnt;
    DBuf<double> wt;
    BD_TRY(cnt.alloc((size_t)N + 1));
    BD_TRY(wt.alloc((size_t)L.A.nb));
    BD_TRY(S.rp.alloc((size_t)N + 1));
    k_strength_count<<<nblk(N, row_block(N)), row_block(N), 0, s>>>(N, L.A.rp.p, L.A.ci.p, L.A.v.p, diag.p, o.theta,
                                                                   cnt.p, wt.p); ::bd::note_launch();
    BD_LAUNCH_CHECK();
    long long snnz = 0;
    BD_TRY(exclusive_scan(cnt.p, S.rp.p, N, &snnz, s));
    S.nnz = snnz;
    BD_TRY(S.ci.alloc((size_t)snnz));
    BD_TRY(S.v.alloc((size_t)snnz));
    k_strength_fill<<<nblk(N, row_block(N)), row_block(N), 0, s>>>(N, L.A.rp.p, L.A.ci.p, wt.p, S.rp.p, S.ci.p,
                                                                  S.v.p); ::bd::note_launch();
    BD_LAUNCH_CHECK();
    int hbad = 0;
    BD_CUDA(cudaMemcpyAsync(&hbad, bad.p, sizeof(int), cudaMemcpyDeviceToHost, s));
    BD_CUDA(cudaStreamSynchronize(s));
    if (hbad) return BD_EINVAL;  // non-positive diagonal: not a semi-definite operator
    if (l < o.square_levels) {
        CSR W, Q, S2;
        BD_TRY(W.rp.alloc((size_t)N + 1));
        BD_TRY(W.ci.alloc((size_t)snnz + N));
        BD_TRY(W.v.alloc((size_t)snnz + N));
        k_insert_diag<<<nblk(N + 1), 256, 0, s>>>(N, S.rp.p, S.ci.p, S.v.p, W.rp.p, W.ci.p, W.v.p); ::bd::note_launch();
        BD_LAUNCH_CHECK();
        long long qn = 0;
        BD_TRY(spgemm<1>(N, N, W.rp.p, W.ci.p, W.v.p, W.rp.p, W.ci.p, W.v.p, Q.rp, Q.ci, Q.v, &qn, s,
                         (double)(snnz + N) / std::max(N, 1)));
        BD_TRY(S2.rp.alloc((size_t)N + 1));
        BD_TRY(S2.ci.alloc((size_t)(qn - N)));
        BD_TRY(S2.v.alloc((size_t)(qn - N)));
        k_drop_diag<<<nblk(N + 1), 256, 0, s>>>(N, Q.rp.p, Q.ci.p, Q.v.p, S2.rp.p, S2.ci.p, S2.v.p); ::bd::note_launch();
        BD_LAUNCH_CHECK();
        S.rp = std::move(S2.rp);
        S.ci = std::move(S2.ci);
        S.v = std::move(S2.v);
        S.nnz = qn - N;
    }
    // a2 MIS
    DBuf<unsigned char> state;
    BD_TRY(state.alloc((size_t)N));
    BD_CUDA(cudaMemsetAsync(state.p, 0, (size_t)N, s));
    DBuf<int> und;
    BD_TRY(und.alloc(1));
    unsigned long long key = level_key(o.seed, l, 0);
    int rounds = 0;
    for (;;) {
        BD_CUDA(cudaMemsetAsync(und.p, 0, sizeof(int), s));
        k_mis_select<<<nblk(N), 256, 0, s>>>(N, S.rp.p, S.ci.p, state.p, key); ::bd::note_launch();
        BD_LAUNCH_CHECK();
        k_mis_exclude<<<nblk(N), 256, 0, s>>>(N, S.rp.p, S.ci.p, state.p, und.p); ::bd::note_launch();
        BD_LAUNCH_CHECK();
        int hu = 0;
        BD_CUDA(cudaMemcpyAsync(&hu, und.p, sizeof(int), cudaMemcpyDeviceToHost, s));
        BD_CUDA(cudaStreamSynchronize(s));
        if (hu == 0) break;
        if (++rounds > N + 1) return BD_ETIMEOUT;  // each round settles at least one node
    }
    // a3 aggregates
    BD_TRY(L.mis.alloc((size_t)N));
    BD_TRY(L.agg.alloc((size_t)N));
    DBuf<int> flag, rid;
    BD_TRY(flag.alloc((size_t)N + 1));
    BD_TRY(rid.alloc((size_t)N + 1));
    k_root_flags<<<nblk(N), 256, 0, s>>>(N, state.p, L.mis.p, flag.p); ::bd::note_launch();
    BD_LAUNCH_CHECK();
    long long nagg = 0;
    BD_TRY(exclusive_scan(flag.p, rid.p, N, &nagg, s));
    BD_CUDA(cudaMemsetAsync(bad.p, 0, sizeof(int), s));
    k_assign<<<nblk(N), 256, 0, s>>>(N, S.rp.p, S.ci.p, S.v.p, L.mis.p, rid.p, L.agg.p, bad.p); ::bd::note_launch();
    BD_LAUNCH_CHECK();
    BD_CUDA(cudaMemcpyAsync(&hbad, bad.p, sizeof(int), cudaMemcpyDeviceToHost, s));
    BD_CUDA(cudaStreamSynchronize(s));
    if (hbad) return BD_ECUDA;  // a non-root without a root neighbour: MIS not maximal
    L.nagg = (int)nagg;
    if (2 * nagg >= n) {  // no coarsening: this level is the coarsest
        L.mis.release();
        L.agg.release();
        L.nagg = 0;
        is_coarsest = true;
        return BD_OK;
    }
    int Nc = (int)nagg;
    // a4 tentative prolongator and coarse near-null coefficients
    DBuf<int> moff, mfill, members;
    BD_TRY(moff.alloc((size_t)Nc + 1));
    BD_TRY(mfill.alloc((size_t)Nc + 2));  // counts, then the largest at [Nc + 1]
    BD_TRY(members.alloc((size_t)N));
    BD_CUDA(cudaMemsetAsync(mfill.p, 0, mfill.bytes(), s));
    k_count_members<<<nblk(N), 256, 0, s>>>(N, L.agg.p, mfill.p); ::bd::note_launch();
    BD_LAUNCH_CHECK();
    BD_TRY(device_max(mfill.p, Nc, mfill.p + Nc + 1, s));
    long long tot = 0;
    BD_TRY(exclusive_scan(mfill.p, moff.p, Nc, &tot, s));  // stream synchronised
    int mx = 0;
    BD_CUDA(cudaMemcpyAsync(&mx, mfill.p + Nc + 1, sizeof(int), cudaMemcpyDeviceToHost, s));
    BD_CUDA(cudaStreamSynchronize(s));
    BD_CUDA(cudaMemsetAsync(mfill.p, 0, mfill.bytes(), s));
    k_scatter_members<<<nblk(N), 256, 0, s>>>(N, L.agg.p, moff.p, mfill.p, members.p); ::bd::note_launch();
    BD_LAUNCH_CHECK();
    BD_TRY(sort_segments(members.p, nullptr, moff.p, Nc, mx, s));
    Level &C = h->lev[l + 1];
    C.N = Nc;
    BD_TRY(C.B.alloc(2 * (size_t)Nc));
    k_coarse_B<<<nblk(Nc), 256, 0, s>>>(Nc, moff.p, members.p, L.B.p, C.B.p); ::bd::note_launch();
    BD_LAUNCH_CHECK();
    BSR Pt;
    Pt.nbr = N;
    Pt.nbc = Nc;
    Pt.nb = N;
    DBuf<double> ptd;
    BD_TRY(Pt.rp.alloc((size_t)N + 1));
    BD_TRY(Pt.ci.alloc((size_t)N));
    BD_TRY(Pt.v.alloc(4 * (size_t)N));
    BD_TRY(ptd.alloc((size_t)n));
    k_ptent<<<nblk(N + 1), 256, 0, s>>>(N, L.agg.p, L.B.p, C.B.p, Pt.rp.p, Pt.ci.p, Pt.v.p, ptd.p); ::bd::note_launch();
    BD_LAUNCH_CHECK();
    // a5 lambda_max of D^{-1}A
    DBuf<LanczosState> lst;
    BD_TRY(lst.alloc(1));
    BD_CUDA(cudaMemsetAsync(lst.p, 0, sizeof(LanczosState), s));
    DBuf<double> vr, vz, vp, vq;
    BD_TRY(vr.alloc((size_t)n));
    BD_TRY(vz.alloc((size_t)n));
    BD_TRY(vp.alloc((size_t)n));
    BD_TRY(vq.alloc((size_t)n));
    k_lanczos_init<<<nblk(n), 256, 0, s>>>(n, level_key(o.seed, l, 1), diag.p, vr.p, vz.p, vp.p); ::bd::note_launch();
    BD_LAUNCH_CHECK();
    long long *acc = h->exact_acc.p;
    BD_TRY(exact_dot(vr.p, vz.p, n, &lst.p->rz, acc, s));
    for (int j = 0; j < o.esteig_steps; j++) {
        k_spmv_ordered<<<nblk(N, row_block(N)), row_block(N), 0, s>>>(N, L.A.rp.p, L.A.ci.p, L.A.v.p, vp.p, vq.p);
        ::bd::note_launch();
        BD_LAUNCH_CHECK();
        BD_TRY(exact_dot(vp.p, vq.p, n, &lst.p->pq, acc, s));
        k_lanczos_alpha<<<1, 1, 0, s>>>(lst.p, j); ::bd::note_launch();
        BD_LAUNCH_CHECK();
        k_lanczos_update_r<<<nblk(n), 256, 0, s>>>(n, lst.p, j, vq.p, diag.p, vr.p, vz.p); ::bd::note_launch();
        BD_LAUNCH_CHECK();
        BD_TRY(exact_dot(vr.p, vz.p, n, &lst.p->rz1, acc, s));
        k_lanczos_beta<<<1, 1, 0, s>>>(lst.p, j); ::bd::note_launch();
        BD_LAUNCH_CHECK();
        k_lanczos_update_p<<<nblk(n), 256, 0, s>>>(n, lst.p, j, vz.p, vp.p); ::bd::note_launch();
        BD_LAUNCH_CHECK();
    }
    k_lanczos_finish<<<1, 1, 0, s>>>(lst.p); ::bd::note_launch();
    BD_LAUNCH_CHECK();
    LanczosState hst;
    BD_CUDA(cudaMemcpyAsync(&hst, lst.p, sizeof(hst), cudaMemcpyDeviceToHost, s));
    BD_CUDA(cudaStreamSynchronize(s));
    if (hst.bad) return BD_EINVAL;
    L.lam = hst.lam;
    // a6 P = Pt - omega D^{-1} A Pt
    long long pnb = 0;
    L.P.nbr = N;
    L.P.nbc = Nc;
    BD_TRY(spgemm<2>(N, Nc, L.A.rp.p, L.A.ci.p, L.A.v.p, Pt.rp.p, Pt.ci.p, Pt.v.p, L.P.rp, L.P.ci,
                     L.P.v, &pnb, s, 1.0));  // one block per row of the tentative prolongator
    L.P.nb = pnb;
    k_smooth_p<<<nblk(N), 256, 0, s>>>(N, L.P.rp.p, L.P.ci.p, L.P.v.p, L.agg.p, ptd.p, diag.p, lst.p); ::bd::note_launch();
    BD_LAUNCH_CHECK();
    // a7 R = P^T
    BD_TRY(bsr_transpose(L.P, L.R, s));
    // a8 A_c = R (A P)
    BSR AP;
    long long apnb = 0;
    BD_TRY(spgemm<2>(N, Nc, L.A.rp.p, L.A.ci.p, L.A.v.p, L.P.rp.p, L.P.ci.p, L.P.v.p, AP.rp, AP.ci,
                     AP.v, &apnb, s, (double)L.P.nb / std::max(N, 1)));
    AP.nbr = N;
    AP.nbc = Nc;
    AP.nb = apnb;
    long long cnb = 0;
    C.A.nbr = C.A.nbc = Nc;
    BD_TRY(spgemm<2>(Nc, Nc, L.R.rp.p, L.R.ci.p, L.R.v.p, AP.rp.p, AP.ci.p, AP.v.p, C.A.rp, C.A.ci,
                     C.A.v, &cnb, s, (double)apnb / std::max(N, 1)));
    C.A.nb = cnb;
    BD_CUDA(cudaStreamSynchronize(s));
    return BD_OK;
}

static int finish_level_common(Level &L, cudaStream_t s)
{
    int n = 2 * L.N;
    DBuf<double> diag;
    DBuf<int> bad;
    BD_TRY(diag.alloc((size_t)n));
    BD_TRY(bad.alloc(1));
    BD_CUDA(cudaMemsetAsync(bad.p, 0, sizeof(int), s));
    k_diag<<<nblk(L.N), 256, 0, s>>>(L.N, L.A.rp.p, L.A.ci.p, L.A.v.p, diag.p, bad.p); ::bd::note_launch();
    BD_LAUNCH_CHECK();
    BD_TRY(L.invdiag.alloc((size_t)n));
    k_invdiag<<<nblk(n), 256, 0, s>>>(n, diag.p, L.invdiag.p); ::bd::note_launch();
    BD_LAUNCH_CHECK();
    int hbad = 0;
    BD_CUDA(cudaMemcpyAsync(&hbad, bad.p, sizeof(int), cudaMemcpyDeviceToHost, s));
    BD_CUDA(cudaStreamSynchronize(s));
    return hbad ? BD_EINVAL : BD_OK;
}

constexpr int kCoarseSingleBlock = 256;  // coarsest sizes factored by one thread block

static int build_coarsest(amg_hierarchy *h, int l, cudaStream_t s)
{
    Level &L = h->lev[l];
    int n = 2 * L.N;
    if (n > kMaxCoarse) return BD_ERANGE;
    h->nc = n;
    DBuf<double> Ad;
    BD_TRY(Ad.alloc((size_t)n * n));
    BD_TRY(h->cinv.alloc((size_t)n * n));
    BD_TRY(h->zc.alloc((size_t)n));
    BD_CUDA(cudaMemsetAsync(Ad.p, 0, Ad.bytes(), s));
    k_coarse_dense<<<nblk(L.N), 256, 0, s>>>(L.N, L.A.rp.p, L.A.ci.p, L.A.v.p, Ad.p); ::bd::note_launch();
    BD_LAUNCH_CHECK();
    k_null_vector<<<nblk(L.N), 256, 0, s>>>(L.N, L.B.p, h->zc.p); ::bd::note_launch();
    BD_LAUNCH_CHECK();
    DBuf<double> zz;
    DBuf<int> bad;
    BD_TRY(zz.alloc(1));
    BD_TRY(bad.alloc(1));
    BD_CUDA(cudaMemsetAsync(bad.p, 0, sizeof(int), s));
    if (n <= kCoarseSingleBlock) {
        k_coarse_factor<<<1, 256, 0, s>>>(n, Ad.p, h->zc.p, h->cinv.p, zz.p, bad.p); ::bd::note_launch();
        BD_LAUNCH_CHECK();
    } else {
        DBuf<double> st;
        BD_TRY(st.alloc(2));
        k_coarse_stats<<<1, 32, 0, s>>>(n, Ad.p, h->zc.p, st.p); ::bd::note_launch();
        k_coarse_rank1<<<n, 256, 0, s>>>(n, Ad.p, h->zc.p, st.p); ::bd::note_launch();
        DBuf<double> Dinv, W, Cb;
        BD_TRY(Dinv.alloc((size_t)kGJ * kGJ));
        BD_TRY(W.alloc((size_t)kGJ * n));
        BD_TRY(Cb.alloc((size_t)kGJ * n));
        // the update as one resident wave: column chunks x equal row shares
        int occ = 0;
        BD_CUDA(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, k_gj_update, 128, 0));
        const int gx = (n + 127) / 128;
        const int gy = std::max(1, std::min((kSM * std::max(occ, 1)) / gx, (n + kGJ - 1) / kGJ));
        const dim3 gu(gx, gy), gp(gx, kGJ / kGJPanelK);
        for (int K = 0; K < n; K += kGJ) {
            const int bb = std::min(kGJ, n - K);
            k_gj_pivot<<<1, 256, 0, s>>>(n, K, bb, Ad.p, Dinv.p, bad.p); ::bd::note_launch();
            k_gj_panel<<<gp, 128, 0, s>>>(n, K, bb, Ad.p, Dinv.p, W.p, Cb.p); ::bd::note_launch();
            k_gj_update<<<gu, 128, 0, s>>>(n, K, bb, Ad.p, Dinv.p, W.p, Cb.p); ::bd::note_launch();
        }
        BD_LAUNCH_CHECK();
        BD_CUDA(cudaMemcpyAsync(h->cinv.p, Ad.p, Ad.bytes(), cudaMemcpyDeviceToDevice, s));
        BD_CUDA(cudaMemcpyAsync(zz.p, st.p + 1, sizeof(double), cudaMemcpyDeviceToDevice, s));
        BD_CUDA(cudaStreamSynchronize(s));  // the scratch buffers are freed on return
    }
    int hbad = 0;
    BD_CUDA(cudaMemcpyAsync(&hbad, bad.p, sizeof(int), cudaMemcpyDeviceToHost, s));
    BD_CUDA(cudaMemcpyAsync(&h->zz, zz.p, sizeof(double), cudaMemcpyDeviceToHost, s));
    BD_CUDA(cudaStreamSynchronize(s));
    return hbad ? BD_EINVAL : BD_OK;
}

static int setup_from_level0(amg_hierarchy *h, cudaStream_t s)
{
    Level &L0 = h->lev[0];
    BD_TRY(h->exact_acc.alloc(kExactLimbs + 1));
    BD_TRY(L0.B.alloc(2 * (size_t)L0.N));
    k_fill<<<nblk(2LL * L0.N), 256, 0, s>>>(2 * L0.N, 1.0, L0.B.p); ::bd::note_launch();
    BD_LAUNCH_CHECK();
    int l = 0;
    for (;;) {
        BD_TRY(finish_level_common(h->lev[l], s));
        bool coarsest = false;
        BD_TRY(coarsen_level(h, l, coarsest, s));
        if (coarsest) break;
        l++;
    }
    h->nlev = l + 1;
    BD_TRY(build_coarsest(h, l, s));
    return BD_OK;
}

static int check_opts(const amg_options *o)
{
    if (!(o->theta >= 0.0) || o->coarse_eq_limit < 2 || o->max_levels < 1 ||
        o->max_levels > kMaxLevels || (o->cheb_degree != 1 && o->cheb_degree != 2) ||
        o->esteig_steps < 1 || o->esteig_steps > 64 || o->square_levels < 0 ||
        !(o->eig_lo > 0.0) || !(o->eig_hi > o->eig_lo) || (o->precision != 0 && o->precision != 1) ||
        (o->autotune != 0 && o->autotune != 1))
        return BD_EINVAL;
    return BD_OK;
}

}  // namespace bd

using namespace bd;

extern "C" int amg_setup(const bd_system *sys, const amg_options *opts, void *stream,
                         amg_hierarchy **out)
{
    if (!sys || !out) return BD_EINVAL;
    *out = nullptr;
    amg_options o;
    amg_options_default(&o);
    if (opts) o = *opts;
    BD_TRY(check_opts(&o));
    cudaStream_t s = (cudaStream_t)stream;
    amg_hierarchy *h = new (std::nothrow) amg_hierarchy();
    if (!h) return BD_ENOMEM;
    h->opts = o;
    Level &L0 = h->lev[0];
    L0.N = sys->N;
    L0.A.nbr = L0.A.nbc = sys->N;
    L0.A.nb = sys->A.nb;
    int st;
    if ((st = L0.A.rp.alloc((size_t)sys->N + 1)) || (st = L0.A.ci.alloc((size_t)sys->A.nb)) ||
        (st = L0.A.v.alloc(4 * (size_t)sys->A.nb))) {
        delete h;
        return st;
    }
    if (cudaMemcpyAsync(L0.A.rp.p, sys->A.rp.p, L0.A.rp.bytes(), cudaMemcpyDeviceToDevice, s) ||
        cudaMemcpyAsync(L0.A.ci.p, sys->A.ci.p, L0.A.ci.bytes(), cudaMemcpyDeviceToDevice, s) ||
        cudaMemcpyAsync(L0.A.v.p, sys->A.v.p, L0.A.v.bytes(), cudaMemcpyDeviceToDevice, s)) {
        delete h;
        return BD_ECUDA;
    }
    h->prec32 = o.precision == 1;
    if ((st = setup_from_level0(h, s)) || (st = build_fine_sell(h, sys, s)) ||
        (st = prepare_solve(h, s))) {
        delete h;
        return st;
    }
    *out = h;
    return BD_OK;
}

// The elliptic operator Ai + Ae of the decoupled scheme (Section 2.2, Eq. 6)
// as the block operator [I, 0; 0, Ai + Ae] on the assembled node pattern, so
// that the block hierarchy's u-field is smoothed aggregation on Ai + Ae.
__global__ void k_elliptic_values(int N, const int *__restrict__ rp, const int *__restrict__ ci,
                                  const double *__restrict__ Ki, const double *__restrict__ Ke,
                                  double *__restrict__ v)
{
    for (int p = blockIdx.x * blockDim.x + threadIdx.x; p < N; p += gridDim.x * blockDim.x)
        for (int t = rp[p]; t < rp[p + 1]; t++) {
            v[4 * (size_t)t] = ci[t] == p ? 1.0 : 0.0;
            v[4 * (size_t)t + 1] = 0.0;
            v[4 * (size_t)t + 2] = 0.0;
            v[4 * (size_t)t + 3] = Ki[t] + Ke[t];
        }
}

extern "C" int bd_elliptic_setup(const bd_system *sys, const amg_options *opts, void *stream,
                                 amg_hierarchy **out)
{
    if (!sys || !out) return BD_EINVAL;
    *out = nullptr;
    amg_options o;
    amg_options_default(&o);
    if (opts) o = *opts;
    BD_TRY(check_opts(&o));
    cudaStream_t s = (cudaStream_t)stream;
    amg_hierarchy *h = new (std::nothrow) amg_hierarchy();
    if (!h) return BD_ENOMEM;
    h->opts = o;
    h->prec32 = o.precision == 1;
    Level &L0 = h->lev[0];
    L0.N = sys->N;
    L0.A.nbr = L0.A.nbc = sys->N;
    L0.A.nb = sys->A.nb;
    int st;
    if ((st = L0.A.rp.alloc((size_t)sys->N + 1)) || (st = L0.A.ci.alloc((size_t)sys->A.nb)) ||
        (st = L0.A.v.alloc(4 * (size_t)sys->A.nb))) {
        delete h;
        return st;
    }
    if (cudaMemcpyAsync(L0.A.rp.p, sys->A.rp.p, L0.A.rp.bytes(), cudaMemcpyDeviceToDevice, s) ||
        cudaMemcpyAsync(L0.A.ci.p, sys->A.ci.p, L0.A.ci.bytes(), cudaMemcpyDeviceToDevice, s)) {
        delete h;
        return BD_ECUDA;
    }
    k_elliptic_values<<<grid_for(sys->N, 256), 256, 0, s>>>(sys->N, sys->A.rp.p, sys->A.ci.p, sys->Ki.p,
                                                            sys->Ke.p, L0.A.v.p); ::bd::note_launch();
    if (cudaGetLastError() != cudaSuccess) {
        delete h;
        return BD_ECUDA;
    }
    if ((st = setup_from_level0(h, s)) || (st = prepare_solve(h, s))) {
        delete h;
        return st;
    }
    *out = h;
    return BD_OK;
}

extern "C" int amg_setup_from_csr(int n, const int *row_ptr, const int *col, const double *val,
                                  int on_device, const amg_options *opts, void *stream,
                                  amg_hierarchy **out)
{
    if (!row_ptr || !col || !val || !out || n < 2 || (n & 1)) return BD_EINVAL;
    *out = nullptr;
    amg_options o;
    amg_options_default(&o);
    if (opts) o = *opts;
    BD_TRY(check_opts(&o));
    cudaStream_t s = (cudaStream_t)stream;
    DBuf<int> drp, dci;
    DBuf<double> dv;
    const int *prp = row_ptr, *pci = col;
    const double *pv = val;
    if (!on_device) {
        int nnz = row_ptr[n];
        if (nnz < 0) return BD_EINVAL;
        BD_TRY(drp.alloc((size_t)n + 1));
        BD_TRY(dci.alloc((size_t)nnz));
        BD_TRY(dv.alloc((size_t)nnz));
        BD_TRY(copy_in(drp.p, row_ptr, sizeof(int) * ((size_t)n + 1), 0, s));
        BD_TRY(copy_in(dci.p, col, sizeof(int) * (size_t)nnz, 0, s));
        BD_TRY(copy_in(dv.p, val, sizeof(double) * (size_t)nnz, 0, s));
        prp = drp.p;
        pci = dci.p;
        pv = dv.p;
    }
    amg_hierarchy *h = new (std::nothrow) amg_hierarchy();
    if (!h) return BD_ENOMEM;
    h->opts = o;
    h->prec32 = o.precision == 1;
    h->lev[0].N = n / 2;
    int st = bsr_from_scalar_csr(n, prp, pci, pv, h->lev[0].A, s);
    if (!st) st = setup_from_level0(h, s);
    if (!st) st = prepare_solve(h, s);
    if (st) {
        delete h;
        return st;
    }
    *out = h;
    return BD_OK;
}

extern "C" int amg_num_levels(const amg_hierarchy *h, int *nlevels)
{
    if (!h || !nlevels) return BD_EINVAL;
    *nlevels = h->nlev;
    return BD_OK;
}

extern "C" int amg_level_info(const amg_hierarchy *h, int level, int *n, long long *nnz, int *n_agg,
                              double *lambda, long long *p_nnz)
{
    if (!h || level < 0 || level >= h->nlev) return BD_EINVAL;
    const Level &L = h->lev[level];
    bool last = level == h->nlev - 1;
    if (n) *n = 2 * L.N;
    if (nnz) *nnz = 4 * L.A.nb;
    if (n_agg) *n_agg = last ? 0 : L.nagg;
    if (lambda) *lambda = last ? 0.0 : L.lam;
    if (p_nnz) *p_nnz = last ? 0 : 4 * L.P.nb;
    return BD_OK;
}

extern "C" int amg_level_lanes(const amg_hierarchy *h, int level, int lanes[3])
{
    if (!h || !lanes || level < 0 || level >= h->nlev) return BD_EINVAL;
    const Level &L = h->lev[level];
    const bool last = level == h->nlev - 1;
    lanes[0] = last || (level == 0 && h->sell.valid) ? 0 : L.lanes[0];
    lanes[1] = last ? 0 : L.lanes[1];
    lanes[2] = last ? 0 : L.lanes[2];
    return BD_OK;
}

extern "C" int amg_export_level(const amg_hierarchy *h, int level, int *a_row_ptr, int *a_col,
                                double *a_val, unsigned char *mis, int *agg, int *p_row_ptr,
                                int *p_col, double *p_val, void *stream)
{
    if (!h || level < 0 || level >= h->nlev) return BD_EINVAL;
    cudaStream_t s = (cudaStream_t)stream;
    const Level &L = h->lev[level];
    bool last = level == h->nlev - 1;
    if (a_row_ptr || a_col || a_val) BD_TRY(bsr_to_scalar_csr_host(L.A, a_row_ptr, a_col, a_val, s));
    if (!last) {
        if (mis) BD_CUDA(cudaMemcpyAsync(mis, L.mis.p, (size_t)L.N, cudaMemcpyDeviceToHost, s));
        if (agg) BD_CUDA(cudaMemcpyAsync(agg, L.agg.p, sizeof(int) * (size_t)L.N, cudaMemcpyDeviceToHost, s));
        if (p_row_ptr || p_col || p_val) BD_TRY(bsr_to_scalar_csr_host(L.P, p_row_ptr, p_col, p_val, s));
    }
    BD_CUDA(cudaStreamSynchronize(s));
    return BD_OK;
}

extern "C" void amg_destroy(amg_hierarchy *h)
{
    if (!h) return;
    if (h->host_scal) cudaFreeHost(h->host_scal);
    delete h;
}
