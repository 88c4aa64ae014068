// bd_runtime.cu -- status codes, option defaults, device utilities (prefix
// scan, segmented sort, correctly rounded dot product), copies and format
// conversion used by the other translation units.
#include <atomic>
#include <climits>
#include <cstring>
#include <mutex>

#include "bd_common.cuh"

namespace bd {

static thread_local char g_last_err[256];
static std::atomic<long long> g_launches{0};

void note_launch() { g_launches.fetch_add(1, std::memory_order_relaxed); }
void note_launches(long long n) { g_launches.fetch_add(n, std::memory_order_relaxed); }
long long launch_count() { return g_launches.load(std::memory_order_relaxed); }
static std::atomic<long long> g_spgemm_paths[2]{{0}, {0}};
void note_spgemm_path(bool dense) { g_spgemm_paths[dense ? 1 : 0].fetch_add(1, std::memory_order_relaxed); }
long long spgemm_path_count(bool dense) { return g_spgemm_paths[dense ? 1 : 0].load(std::memory_order_relaxed); }

void record_cuda_error(cudaError_t e, const char *what, const char *file, int line)
{
    snprintf(g_last_err, sizeof(g_last_err), "%s failed: %s (%s:%d)", what,
             cudaGetErrorString(e), file, line);
}

// ------------------------------------------------------------------ prefix scan
constexpr int kScanThreads = 1024;
constexpr int kScanTile = 2 * kScanThreads;

__device__ __forceinline__ long long block_exclusive_scan(long long v, long long *warp_tot,
                                                           long long *block_total)
{
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
    long long inc = v;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        long long t = __shfl_up_sync(0xffffffffu, inc, o);
        if (lane >= o) inc += t;
    }
    if (lane == 31) warp_tot[wid] = inc;
    __syncthreads();
    if (wid == 0) {
        long long w = (lane < (int)(blockDim.x >> 5)) ? warp_tot[lane] : 0;
        long long wi = w;
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            long long t = __shfl_up_sync(0xffffffffu, wi, o);
            if (lane >= o) wi += t;
        }
        warp_tot[lane] = wi - w;
        if (lane == 31) *block_total = wi;
    }
    __syncthreads();
    long long r = warp_tot[wid] + inc - v;
    __syncthreads();
    return r;
}

__global__ void k_scan_tiles(const int *__restrict__ in, int *__restrict__ out, int n,
                             long long *__restrict__ tile_sums)
{
    __shared__ long long wt[32];
    __shared__ long long tot;
    long long base = (long long)blockIdx.x * kScanTile;
    long long i0 = base + 2 * threadIdx.x;
    int a = i0 < n ? in[i0] : 0;
    int b = i0 + 1 < n ? in[i0 + 1] : 0;
    long long ex = block_exclusive_scan((long long)a + b, wt, &tot);
    if (i0 < n) out[i0] = (int)ex;  // tile-local, fits: tile sum checked below
    if (i0 + 1 < n) out[i0 + 1] = (int)(ex + a);
    if (threadIdx.x == 0) tile_sums[blockIdx.x] = tot;
}

__global__ void k_scan_sums(long long *sums, int ntiles, long long *total)
{
    __shared__ long long wt[32];
    __shared__ long long tot;
    long long carry = 0;
    for (int base = 0; base < ntiles; base += blockDim.x) {
        int i = base + threadIdx.x;
        long long v = i < ntiles ? sums[i] : 0;
        long long ex = block_exclusive_scan(v, wt, &tot);
        if (i < ntiles) sums[i] = carry + ex;
        carry += tot;
        __syncthreads();
    }
    if (threadIdx.x == 0) *total = carry;
}

__global__ void k_scan_add(int *out, int n, const long long *tile_off, const long long *total,
                           int *overflow)
{
    long long base = (long long)blockIdx.x * kScanTile;
    long long off = tile_off[blockIdx.x];
    for (int k = 0; k < 2; k++) {
        long long i = base + 2 * threadIdx.x + k;
        if (i < n) {
            long long v = off + out[i];
            if (v > INT_MAX) *overflow = 1;
            out[i] = (int)v;
        }
    }
    if (blockIdx.x == 0 && threadIdx.x == 0) {
        long long t = *total;
        if (t > INT_MAX) *overflow = 1;
        out[n] = (int)(t > INT_MAX ? INT_MAX : t);
    }
}

int exclusive_scan(const int *in, int *out, int n, long long *total, cudaStream_t s)
{
    int ntiles = (n + kScanTile - 1) / kScanTile;
    if (ntiles < 1) ntiles = 1;
    DBuf<long long> sums;
    DBuf<int> flag;
    BD_TRY(sums.alloc((size_t)ntiles + 1));
    BD_TRY(flag.alloc(1));
    BD_CUDA(cudaMemsetAsync(flag.p, 0, sizeof(int), s));
    k_scan_tiles<<<ntiles, kScanThreads, 0, s>>>(in, out, n, sums.p); ::bd::note_launch();
    BD_LAUNCH_CHECK();
    k_scan_sums<<<1, kScanThreads, 0, s>>>(sums.p, ntiles, sums.p + ntiles); ::bd::note_launch();
    BD_LAUNCH_CHECK();
    k_scan_add<<<ntiles, kScanThreads, 0, s>>>(out, n, sums.p, sums.p + ntiles, flag.p); ::bd::note_launch();
    BD_LAUNCH_CHECK();
    long long t = 0;
    int of = 0;
    BD_CUDA(cudaMemcpyAsync(&t, sums.p + ntiles, sizeof(t), cudaMemcpyDeviceToHost, s));
    BD_CUDA(cudaMemcpyAsync(&of, flag.p, sizeof(int), cudaMemcpyDeviceToHost, s));
    BD_CUDA(cudaStreamSynchronize(s));
    if (of) return BD_ERANGE;
    if (total) *total = t;
    return BD_OK;
}

// ------------------------------------------------------------------ maximum
// Warp maxima combined by atomicMax: the result does not depend on the order.
__global__ void k_max_int(const int *__restrict__ a, int n, int *out)
{
    int m = 0;
    for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n;
         i += (long long)gridDim.x * blockDim.x)
        m = max(m, a[i]);
    m = __reduce_max_sync(0xffffffffu, m);
    if ((threadIdx.x & 31) == 0 && m > 0) atomicMax(out, m);
}

int device_max(const int *a, int n, int *slot, cudaStream_t s)
{
    BD_CUDA(cudaMemsetAsync(slot, 0, sizeof(int), s));
    if (n <= 0) return BD_OK;
    k_max_int<<<grid_for(n, 256), 256, 0, s>>>(a, n, slot); ::bd::note_launch();
    BD_LAUNCH_CHECK();
    return BD_OK;
}

// ------------------------------------------------------------------ segmented sort
// One block per segment, bitonic sort in shared memory (padded to a power of 2).
__global__ void k_sort_segments(int *keys, int *payload, const int *seg, int nseg, int P)
{
    extern __shared__ int sm[];
    int *sk = sm, *sp = sm + P;
    for (int g = blockIdx.x; g < nseg; g += gridDim.x) {
        int b = seg[g], len = seg[g + 1] - b;
        if (len <= 1) continue;
        int p2 = 1;
        while (p2 < len) p2 <<= 1;
        for (int i = threadIdx.x; i < p2; i += blockDim.x) {
            sk[i] = i < len ? keys[b + i] : INT_MAX;
            if (payload) sp[i] = i < len ? payload[b + i] : 0;
        }
        __syncthreads();
        for (int k = 2; k <= p2; k <<= 1)
            for (int j = k >> 1; j > 0; j >>= 1) {
                for (int i = threadIdx.x; i < p2; i += blockDim.x) {
                    int ixj = i ^ j;
                    if (ixj > i) {
                        bool up = (i & k) == 0;
                        int ki = sk[i], kj = sk[ixj];
                        if ((ki > kj) == up) {
                            sk[i] = kj;
                            sk[ixj] = ki;
                            if (payload) {
                                int t = sp[i];
                                sp[i] = sp[ixj];
                                sp[ixj] = t;
                            }
                        }
                    }
                }
                __syncthreads();
            }
        for (int i = threadIdx.x; i < len; i += blockDim.x) {
            keys[b + i] = sk[i];
            if (payload) payload[b + i] = sp[i];
        }
        __syncthreads();
    }
}

int sort_segments(int *keys, int *payload, const int *seg, int nseg, int max_len, cudaStream_t s)
{
    if (nseg <= 0 || max_len <= 1) return BD_OK;
    if (max_len > kMaxSortSeg) return BD_ERANGE;
    int P = 1;
    while (P < max_len) P <<= 1;
    size_t smem = 2 * (size_t)P * sizeof(int);
    BD_CUDA(cudaFuncSetAttribute(k_sort_segments, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                 (int)smem));
    int threads = P >= 256 ? 256 : (P < 32 ? 32 : P);
    int grid = nseg < kSM * 16 ? nseg : kSM * 16;
    k_sort_segments<<<grid, threads, smem, s>>>(keys, payload, seg, nseg, P); ::bd::note_launch();
    BD_LAUNCH_CHECK();
    return BD_OK;
}

// ------------------------------------------------------------------ exact dot
// Long accumulator: limb i holds a signed count of units 2^(32 i - 1074).
// Each rounded product is split into three 32-bit digits and added with
// 64-bit integer atomics (associative, so the result does not depend on the
// order of the additions).

// Digits of a finite double: limb index li and three signed 32-bit digits
// (two's complement in 64 bits) such that x = sum_k d_k 2^(32 (li + k) - 1074).
// Returns false for an infinity or NaN (flag bits in *nf: 1 NaN, 2 +inf, 4 -inf).
__device__ __forceinline__ bool exact_digits(double x, int &li, unsigned long long &d0, unsigned long long &d1,
                                             unsigned long long &d2, int &nf)
{
    unsigned long long b = (unsigned long long)__double_as_longlong(x);
    int neg = (int)(b >> 63);
    int E = (int)((b >> 52) & 0x7ff);
    unsigned long long m = b & 0xFFFFFFFFFFFFFULL;
    li = 0;
    d0 = d1 = d2 = 0;
    nf = 0;
    if (E == 0x7ff) {
        nf = m ? 1 : (neg ? 4 : 2);
        return false;
    }
    int off = 0;
    if (E != 0) {
        m |= (1ULL << 52);
        off = E - 1;
    }
    if (m == 0) return true;
    li = off >> 5;
    const int sh = off & 31;
    unsigned long long t0 = (m & 0xffffffffULL) << sh;
    unsigned long long t1 = (m >> 32) << sh;
    d0 = t0 & 0xffffffffULL;
    unsigned long long u1 = (t0 >> 32) + (t1 & 0xffffffffULL);
    d1 = u1 & 0xffffffffULL;
    d2 = (u1 >> 32) + (t1 >> 32);
    if (neg) {
        d0 = 0ULL - d0;
        d1 = 0ULL - d1;
        d2 = 0ULL - d2;
    }
    return true;
}

__device__ __forceinline__ void exact_acc_digits(long long *acc, int li, unsigned long long d0,
                                                 unsigned long long d1, unsigned long long d2)
{
    unsigned long long *a = (unsigned long long *)acc;
    if (d0) atomicAdd(a + li, d0);
    if (d1) atomicAdd(a + li + 1, d1);
    if (d2) atomicAdd(a + li + 2, d2);
}

// Whole warps step through the elements.  When every nonzero finite product
// of a warp's step falls on the same limb index (the usual case: products of
// similar magnitude), the warp sums its digits exactly (32 signed 33-bit
// digits fit 64 bits) and one lane adds them; otherwise every lane adds its
// own.  Integer sums are associative, so the total is the same either way.
__global__ void k_exact_dot_partial(const double *__restrict__ x, const double *__restrict__ y,
                                    int n, long long *gacc)
{
    __shared__ long long acc[kExactLimbs];
    __shared__ int flags;
    for (int i = threadIdx.x; i < kExactLimbs; i += blockDim.x) acc[i] = 0;
    if (threadIdx.x == 0) flags = 0;
    __syncthreads();
    const int lane = threadIdx.x & 31;
    const long long stride = (long long)gridDim.x * blockDim.x;
    for (long long base = (long long)blockIdx.x * blockDim.x + (threadIdx.x & ~31); base < n; base += stride) {
        const long long i = base + lane;
        const double p = i < n ? __dmul_rn(x[i], y[i]) : 0.0;
        int li, nf;
        unsigned long long d0, d1, d2;
        const bool fin = exact_digits(p, li, d0, d1, d2, nf);
        const bool nz = fin && (d0 | d1 | d2);
        const unsigned nzm = __ballot_sync(0xffffffffu, nz);
        const bool allfin = __all_sync(0xffffffffu, fin);
        if (nzm == 0 && allfin) continue;
        const int li0 = __shfl_sync(0xffffffffu, li, __ffs(nzm ? nzm : 1u) - 1);
        if (allfin && __all_sync(0xffffffffu, !nz || li == li0)) {
#pragma unroll
            for (int o = 16; o > 0; o >>= 1) {
                d0 += __shfl_xor_sync(0xffffffffu, d0, o);
                d1 += __shfl_xor_sync(0xffffffffu, d1, o);
                d2 += __shfl_xor_sync(0xffffffffu, d2, o);
            }
            if (lane == 0) exact_acc_digits(acc, li0, d0, d1, d2);
        } else {
            if (!fin) atomicOr(&flags, nf);
            else if (nz) exact_acc_digits(acc, li, d0, d1, d2);
        }
    }
    __syncthreads();
    for (int i = threadIdx.x; i < kExactLimbs; i += blockDim.x)
        if (acc[i]) atomicAdd((unsigned long long *)&gacc[i], (unsigned long long)acc[i]);
    if (threadIdx.x == 0 && flags) atomicOr((int *)&gacc[kExactLimbs], flags);
}

// Round the exact total to the nearest double (ties to even).
__global__ void k_exact_round(long long *gacc, double *out)
{
    if (threadIdx.x != 0 || blockIdx.x != 0) return;
    int flags = (int)gacc[kExactLimbs];
    if (flags) {
        double r;
        if ((flags & 1) || ((flags & 2) && (flags & 4))) r = __longlong_as_double(0x7ff8000000000000LL);
        else if (flags & 2) r = __longlong_as_double(0x7ff0000000000000LL);
        else r = __longlong_as_double((long long)0xfff0000000000000ULL);
        *out = r;
        return;
    }
    long long l[kExactLimbs];
    for (int i = 0; i < kExactLimbs; i++) l[i] = gacc[i];
    // carry propagation into 32-bit digits, the top limb keeps the sign
    for (int i = 0; i < kExactLimbs - 1; i++) {
        long long lo = l[i] & 0xffffffffLL;
        long long c = (l[i] - lo) >> 32;  // exact: l[i]-lo is a multiple of 2^32
        l[i] = lo;
        l[i + 1] += c;
    }
    bool negative = l[kExactLimbs - 1] < 0;
    if (negative) {
        for (int i = 0; i < kExactLimbs; i++) l[i] = -l[i];
        for (int i = 0; i < kExactLimbs - 1; i++) {
            long long lo = l[i] & 0xffffffffLL;
            long long c = (l[i] - lo) >> 32;
            l[i] = lo;
            l[i + 1] += c;
        }
    }
    int top = -1;
    for (int i = kExactLimbs - 1; i >= 0; i--)
        if (l[i] != 0) {
            top = i;
            break;
        }
    double r;
    if (top < 0) {
        r = 0.0;
    } else if (l[top] >= (1LL << 32)) {
        r = __longlong_as_double(0x7ff0000000000000LL);
    } else {
        int H = 32 * top + 31 - __clz((unsigned)l[top]);
        auto bit = [&](int pos) -> unsigned long long {
            return (unsigned long long)((l[pos >> 5] >> (pos & 31)) & 1);
        };
        unsigned long long mant = 0;
        if (H < 53) {
            for (int p = H; p >= 0; p--) mant = (mant << 1) | bit(p);
            r = scalbn((double)mant, -1074);
        } else {
            for (int p = H; p >= H - 52; p--) mant = (mant << 1) | bit(p);
            unsigned long long rb = bit(H - 53);
            unsigned long long sticky = 0;
            for (int p = H - 54; p >= 0 && !sticky; p--) sticky |= bit(p);
            if (rb && (sticky || (mant & 1))) {
                mant += 1;
                if (mant == (1ULL << 53)) {
                    mant >>= 1;
                    H += 1;
                }
            }
            r = scalbn((double)mant, H - 52 - 1074);
        }
        if (negative) r = -r;
    }
    *out = r;
}

int exact_dot(const double *x, const double *y, int n, double *out, long long *acc, cudaStream_t s)
{
    BD_CUDA(cudaMemsetAsync(acc, 0, sizeof(long long) * (kExactLimbs + 1), s));
    if (n > 0) {
        int grid = grid_for(n, 256, 2);
        k_exact_dot_partial<<<grid, 256, 0, s>>>(x, y, n, acc); ::bd::note_launch();
        BD_LAUNCH_CHECK();
    }
    k_exact_round<<<1, 1, 0, s>>>(acc, out); ::bd::note_launch();
    BD_LAUNCH_CHECK();
    return BD_OK;
}

// ------------------------------------------------------------------ copies
int copy_in(void *dst_dev, const void *src, size_t bytes, int src_on_device, cudaStream_t s)
{
    if (bytes == 0) return BD_OK;
    BD_CUDA(cudaMemcpyAsync(dst_dev, src, bytes,
                            src_on_device ? cudaMemcpyDeviceToDevice : cudaMemcpyHostToDevice, s));
    return BD_OK;
}

int copy_out(void *dst, const void *src_dev, size_t bytes, int dst_on_device, cudaStream_t s)
{
    if (bytes == 0) return BD_OK;
    BD_CUDA(cudaMemcpyAsync(dst, src_dev, bytes,
                            dst_on_device ? cudaMemcpyDeviceToDevice : cudaMemcpyDeviceToHost, s));
    return BD_OK;
}

// ------------------------------------------------------------------ format conversion
__global__ void k_bsr_count(int N, const int *__restrict__ rp, const int *__restrict__ ci,
                            int *cnt, int *bad)
{
    int p = blockIdx.x * blockDim.x + threadIdx.x;
    if (p >= N) return;
    int a = rp[2 * p], b = rp[2 * p + 1], c = rp[2 * p + 2];
    int l0 = b - a, l1 = c - b;
    if (l0 != l1 || (l0 & 1) || l0 < 0) {
        *bad = 1;
        cnt[p] = 0;
        return;
    }
    int prev = -1;
    for (int t = 0; t < l0; t += 2) {
        int c0 = ci[a + t], c1 = ci[a + t + 1], e0 = ci[b + t], e1 = ci[b + t + 1];
        if ((c0 & 1) || c1 != c0 + 1 || e0 != c0 || e1 != c1 || c0 < 0 || c0 / 2 <= prev ||
            c0 / 2 >= N) {
            *bad = 1;
            break;
        }
        prev = c0 / 2;
    }
    cnt[p] = l0 / 2;
}

__global__ void k_bsr_fill(int N, const int *__restrict__ rp, const int *__restrict__ ci,
                           const double *__restrict__ v, const int *__restrict__ brp,
                           int *__restrict__ bci, double *__restrict__ bv)
{
    int p = blockIdx.x * blockDim.x + threadIdx.x;
    if (p >= N) return;
    int a = rp[2 * p], b = rp[2 * p + 1];
    int o = brp[p];
    for (int t = 0, k = 0; t < b - a; t += 2, k++) {
        bci[o + k] = ci[a + t] / 2;
        bv[4 * (size_t)(o + k) + 0] = v[a + t];
        bv[4 * (size_t)(o + k) + 1] = v[a + t + 1];
        bv[4 * (size_t)(o + k) + 2] = v[b + t];
        bv[4 * (size_t)(o + k) + 3] = v[b + t + 1];
    }
}

int bsr_from_scalar_csr(int n, const int *rp, const int *ci, const double *v, BSR &out,
                        cudaStream_t s)
{
    if (n < 2 || (n & 1)) return BD_EINVAL;
    int N = n / 2;
    DBuf<int> cnt, bad;
    BD_TRY(cnt.alloc((size_t)N + 1));
    BD_TRY(bad.alloc(1));
    BD_CUDA(cudaMemsetAsync(bad.p, 0, sizeof(int), s));
    out.nbr = out.nbc = N;
    BD_TRY(out.rp.alloc((size_t)N + 1));
    k_bsr_count<<<(N + 255) / 256, 256, 0, s>>>(N, rp, ci, cnt.p, bad.p); ::bd::note_launch();
    BD_LAUNCH_CHECK();
    int hbad = 0;
    BD_CUDA(cudaMemcpyAsync(&hbad, bad.p, sizeof(int), cudaMemcpyDeviceToHost, s));
    BD_CUDA(cudaStreamSynchronize(s));
    if (hbad) return BD_EINVAL;
    long long nb = 0;
    BD_TRY(exclusive_scan(cnt.p, out.rp.p, N, &nb, s));
    out.nb = nb;
    BD_TRY(out.ci.alloc((size_t)nb));
    BD_TRY(out.v.alloc(4 * (size_t)nb));
    k_bsr_fill<<<(N + 255) / 256, 256, 0, s>>>(N, rp, ci, v, out.rp.p, out.ci.p, out.v.p); ::bd::note_launch();
    BD_LAUNCH_CHECK();
    return BD_OK;
}

int bsr_to_scalar_csr_host(const BSR &a, int *rp, int *ci, double *v, cudaStream_t s)
{
    std::vector<int> brp((size_t)a.nbr + 1), bci((size_t)a.nb);
    std::vector<double> bv(4 * (size_t)a.nb);
    BD_CUDA(cudaMemcpyAsync(brp.data(), a.rp.p, brp.size() * sizeof(int), cudaMemcpyDeviceToHost, s));
    if (a.nb) {
        BD_CUDA(cudaMemcpyAsync(bci.data(), a.ci.p, bci.size() * sizeof(int), cudaMemcpyDeviceToHost, s));
        BD_CUDA(cudaMemcpyAsync(bv.data(), a.v.p, bv.size() * sizeof(double), cudaMemcpyDeviceToHost, s));
    }
    BD_CUDA(cudaStreamSynchronize(s));
    long long pos = 0;
    for (int p = 0; p < a.nbr; p++)
        for (int f = 0; f < 2; f++) {
            if (rp) rp[2 * p + f] = (int)pos;
            for (int t = brp[p]; t < brp[p + 1]; t++)
                for (int g = 0; g < 2; g++) {
                    if (ci) ci[pos] = 2 * bci[t] + g;
                    if (v) v[pos] = bv[4 * (size_t)t + 2 * f + g];
                    pos++;
                }
        }
    if (rp) rp[2 * a.nbr] = (int)pos;
    return BD_OK;
}

// ------------------------------------------------------------------ allocation-free dot
// Scratch of bd_dot_exact_noalloc: one long accumulator (kExactLimbs limbs and
// a flags word, 552 bytes) in device memory that every GPU loading the library
// holds until the process exits.  Host code must not use the array's name as a
// device address: the address is looked up once per device below.
static __device__ __align__(256) long long g_noalloc_dot_acc[kExactLimbs + 1];

constexpr int kNoallocMaxDevices = 64;
static std::mutex g_noalloc_mu;
static long long *g_noalloc_acc[kNoallocMaxDevices];

// Device address of g_noalloc_dot_acc for the current device (first use on a
// device performs the lookup).
static int noalloc_scratch(long long **out)
{
    int dev = 0;
    BD_CUDA(cudaGetDevice(&dev));
    if (dev < 0 || dev >= kNoallocMaxDevices) return BD_ERANGE;
    std::lock_guard<std::mutex> lock(g_noalloc_mu);
    if (!g_noalloc_acc[dev]) {
        void *p = nullptr;
        BD_CUDA(cudaGetSymbolAddress(&p, g_noalloc_dot_acc));
        g_noalloc_acc[dev] = (long long *)p;
    }
    *out = g_noalloc_acc[dev];
    return BD_OK;
}

}  // namespace bd

// ------------------------------------------------------------------ public: misc
extern "C" const char *bd_strerror(int st)
{
    switch (st) {
    case BD_OK: return "ok";
    case BD_EINVAL: return "invalid argument";
    case BD_ENOMEM: return "out of memory";
    case BD_ENOTCONV: return "PCG did not converge within max_it";
    case BD_EBREAKDOWN: return "PCG breakdown (p^T A p <= 0, NaN or Inf)";
    case BD_ETIMEOUT: return "bounded device loop timed out";
    case BD_ECUDA: return "CUDA runtime error";
    case BD_EINCONSISTENT: return "right-hand side not orthogonal to the null space";
    case BD_ERANGE: return "size exceeds a documented maximum";
    case BD_ESTATE: return "handle in the wrong state";
    default: return "unknown status";
    }
}

extern "C" long long bd_launch_count(void) { return bd::g_launches.load(); }

extern "C" int bd_spgemm_path_counts(long long *hash_calls, long long *dense_calls)
{
    if (!hash_calls || !dense_calls) return BD_EINVAL;
    *hash_calls = bd::spgemm_path_count(false);
    *dense_calls = bd::spgemm_path_count(true);
    return BD_OK;
}

extern "C" int bd_dot_exact(const double *x, const double *y, long long n, int on_device,
                            double *out, void *stream)
{
    if (!x || !y || !out || n < 0) return BD_EINVAL;
    if (n > 2147483647LL) return BD_ERANGE;
    cudaStream_t s = (cudaStream_t)stream;
    bd::DBuf<long long> acc;
    bd::DBuf<double> res, dx, dy;
    BD_TRY(acc.alloc(bd::kExactLimbs + 1));
    BD_TRY(res.alloc(1));
    const double *px = x, *py = y;
    if (!on_device && n > 0) {
        BD_TRY(dx.alloc((size_t)n));
        BD_TRY(dy.alloc((size_t)n));
        BD_TRY(bd::copy_in(dx.p, x, sizeof(double) * (size_t)n, 0, s));
        BD_TRY(bd::copy_in(dy.p, y, sizeof(double) * (size_t)n, 0, s));
        px = dx.p;
        py = dy.p;
    }
    BD_TRY(bd::exact_dot(px, py, (int)n, res.p, acc.p, s));
    BD_CUDA(cudaMemcpyAsync(out, res.p, sizeof(double), cudaMemcpyDeviceToHost, s));
    BD_CUDA(cudaStreamSynchronize(s));
    return BD_OK;
}

extern "C" int bd_dot_exact_noalloc(const double *x, const double *y, long long n, double *out,
                                    void *stream)
{
    if (!x || !y || !out || n < 0) return BD_EINVAL;
    if (n > 2147483647LL) return BD_ERANGE;
    long long *acc = nullptr;
    BD_TRY(bd::noalloc_scratch(&acc));
    // exact_dot clears the accumulator on `stream`, then launches the partial
    // and rounding kernels; nothing is allocated.
    return bd::exact_dot(x, y, (int)n, out, acc, (cudaStream_t)stream);
}

extern "C" void amg_options_default(amg_options *o)
{
    if (!o) return;
    o->theta = 0.06;
    o->coarse_eq_limit = 100;
    o->max_levels = 10;
    o->cheb_degree = 2;
    o->esteig_steps = 10;
    o->square_levels = 16;  /* every level (App. A squares the first only) */
    o->eig_lo = 0.05;
    o->eig_hi = 1.05;
    o->seed = 0;
    o->precision = 0;
    o->autotune = 0;
}

extern "C" void solve_options_default(solve_options *o)
{
    if (!o) return;
    o->rtol = 1e-8;
    o->max_it = 500;
    o->warm_start = 0;
    o->strict = 0;
}

extern "C" void bd_rm_params_default(bd_rm_params *p)
{
    if (!p) return;
    p->G = 1.5;
    p->vth = 13.0;
    p->vp = 100.0;
    p->eta1 = 4.4;
    p->eta2 = 0.012;
    p->eta3 = 1.0;
}
