// bd_common.cuh -- internal declarations shared by the CUDA translation units
// of the Bidomain SA-AMG-PCG library (not part of the public ABI).
#pragma once

#include <cuda_runtime.h>

#include <cstdint>
#include <cstdio>
#include <utility>
#include <vector>

#include "bidomain.h"

namespace bd {

// ------------------------------------------------------------------ launch counter
// Every kernel launch of the library calls note_launch(); bd_launch_count()
// reports the running total (host-side, atomic).
void note_launch();
void note_launches(long long n);  // adds n (may be negative: undo capture-time counts)
// SpGEMM calls of the setup by path (hash: warp per row; dense: block per row),
// counted process-wide for bd_spgemm_path_counts().
void note_spgemm_path(bool dense);
long long spgemm_path_count(bool dense);
long long launch_count();

// ------------------------------------------------------------------ errors
void record_cuda_error(cudaError_t e, const char *what, const char *file, int line);

#define BD_CUDA(x)                                                                   \
    do {                                                                             \
        cudaError_t e_ = (x);                                                        \
        if (e_ != cudaSuccess) {                                                     \
            ::bd::record_cuda_error(e_, #x, __FILE__, __LINE__);                     \
            return e_ == cudaErrorMemoryAllocation ? BD_ENOMEM : BD_ECUDA;           \
        }                                                                            \
    } while (0)

#define BD_LAUNCH_CHECK() BD_CUDA(cudaGetLastError())

#define BD_TRY(x)                                                                    \
    do {                                                                             \
        int s_ = (x);                                                                \
        if (s_ != BD_OK) return s_;                                                  \
    } while (0)

// ------------------------------------------------------------------ device buffers
// Owning, move-only device allocation.  Every allocation of the library goes
// through here so that the destructors of the handles release everything.
template <class T>
struct DBuf {
    T *p = nullptr;
    size_t n = 0;
    DBuf() = default;
    DBuf(const DBuf &) = delete;
    DBuf &operator=(const DBuf &) = delete;
    DBuf(DBuf &&o) noexcept : p(o.p), n(o.n) { o.p = nullptr; o.n = 0; }
    DBuf &operator=(DBuf &&o) noexcept {
        if (this != &o) { release(); p = o.p; n = o.n; o.p = nullptr; o.n = 0; }
        return *this;
    }
    ~DBuf() { release(); }
    int alloc(size_t count) {
        release();
        if (count == 0) count = 1;
        cudaError_t e = cudaMalloc((void **)&p, count * sizeof(T));
        if (e != cudaSuccess) {
            p = nullptr;
            record_cuda_error(e, "cudaMalloc", __FILE__, __LINE__);
            return BD_ENOMEM;
        }
        n = count;
        return BD_OK;
    }
    void release() {
        if (p) cudaFree(p);
        p = nullptr;
        n = 0;
    }
    size_t bytes() const { return n * sizeof(T); }
};

// 2x2-block CSR: block row i holds blocks (i, ci[t]) for t in [rp[i], rp[i+1]),
// columns ascending; the block values are v[4t..4t+3] = [a00 a01 a10 a11].
struct BSR {
    int nbr = 0, nbc = 0;  // block rows / block columns
    long long nb = 0;      // blocks
    DBuf<int> rp, ci;
    DBuf<double> v;
};

// scalar CSR with int32 indices (node graphs)
struct CSR {
    int nr = 0, nc = 0;
    long long nnz = 0;
    DBuf<int> rp, ci;
    DBuf<double> v;
};

// ------------------------------------------------------------------ utilities
constexpr int kSM = 152;  // GB300 streaming multiprocessors (grid sizing)

inline int grid_for(long long work, int block, int per_sm_cap = 8) {
    long long g = (work + block - 1) / block;
    long long cap = (long long)kSM * per_sm_cap * 4;
    if (g > cap) g = cap;
    if (g < 1) g = 1;
    return (int)g;
}

// out[0..n] = exclusive prefix sum of in[0..n) (out[n] = total); *total gets the
// total on the host (stream synchronised).  BD_ERANGE if the total exceeds 2^31-1.
int exclusive_scan(const int *in, int *out, int n, long long *total, cudaStream_t s);

// *slot = max(0, a[0..n)) on the device, stream-ordered (slot: one device int;
// the caller reads it back after its next synchronisation).
int device_max(const int *a, int n, int *slot, cudaStream_t s);

// Sort the keys of every segment [seg[i], seg[i+1]) ascending (keys unique
// within a segment), permuting `payload` alongside when it is not NULL.
// BD_ERANGE if a segment is longer than kMaxSortSeg.
constexpr int kMaxSortSeg = 8192;
int sort_segments(int *keys, int *payload, const int *seg, int nseg, int max_len,
                  cudaStream_t s);

// Correctly rounded dot product sum_i x[i]*y[i] (each product rounded, then an
// exact long accumulator and one rounding to nearest-even), written to *out on
// the device.  Order-independent, hence bit-reproducible.  `acc` must hold
// kExactLimbs+1 long longs of scratch.
constexpr int kExactLimbs = 68;
int exact_dot(const double *x, const double *y, int n, double *out, long long *acc,
              cudaStream_t s);

// Copy helpers between caller arrays (host or device) and device buffers.
int copy_in(void *dst_dev, const void *src, size_t bytes, int src_on_device, cudaStream_t s);
int copy_out(void *dst, const void *src_dev, size_t bytes, int dst_on_device, cudaStream_t s);

// Scalar CSR (2N x 2M, full 2x2 node blocks) <-> BSR conversion on the device.
int bsr_from_scalar_csr(int n, const int *rp, const int *ci, const double *v, BSR &out,
                        cudaStream_t s);
int bsr_to_scalar_csr_host(const BSR &a, int *rp, int *ci, double *v, cudaStream_t s);

}  // namespace bd

// ------------------------------------------------------------------ handles
struct bd_system {
    bd_mesh mesh{};
    bd_params params{};
    int N = 0;              // nodes
    bd::BSR A;              // block operator, 2x2 blocks per node pair
    bd::DBuf<double> M;     // lumped mass (N)
    bd::DBuf<double> Ki;    // node-pattern stiffness values (shared pattern with A)
    bd::DBuf<double> Ke;
};
