// amg_internal.cuh -- hierarchy layout shared by the setup and solve units.
#pragma once

#include "bd_common.cuh"

namespace bd {

constexpr int kMaxLevels = 16;
constexpr int kMaxCoarse = 4096;   // unknowns of the dense coarsest level
constexpr int kRedBlocks = 1216;   // blocks of the solve's reduction kernels (8 x SMs)

// A block-CSR operator of the V-cycle in sliced form: rows sorted by block
// count (descending, ties by row) within windows of kSliceWindow rows, slices
// of 32/K consecutive sorted rows, K lanes per row.  Group g of a slice holds
// entries gK .. gK+K-1 of each of its rows in 32 consecutive positions (lane
// i K + k: entry g K + k of the slice's row i), so every group is one
// coalesced load per warp and all lanes of a row-slice run the same trip
// count.  Positions past a row's end hold column 0 with zero values.
constexpr int kSliceWindow = 1024;
struct SlicedOp {
    int K = 0;                  // lanes per row (0: not built)
    int rows = 0;               // block rows
    int nsl = 0;                // slices
    long long groups = 0;       // 32-entry groups
    int warps = 0;              // warps of the launch (grid x 8)
    DBuf<int> order;            // rows padded to 32: row at each sorted position, -1 past the end
    DBuf<int> sptr;             // nsl + 1: first group of each slice
    DBuf<int> wsl;              // warps + 1: first slice of each warp (balanced by groups)
    DBuf<int> cnt;              // nsl: groups per slice (build scratch)
    DBuf<int> col;              // groups * 32 block columns
    DBuf<double> v;             // FP64: groups * 32 (a00, a01) pairs, then as many (a10, a11)
    DBuf<float> v32;            // FP32: groups * 32 float4 (a00, a01, a10, a11)
};

struct Level {
    int N = 0;                 // nodes (unknowns 2N)
    BSR A;                     // operator
    DBuf<double> invdiag;      // 1 / A(i,i), 2N
    DBuf<double> idc2, idt;    // FP64 sliced-ELL finest level: c2 / A(i,i) and 1 / (theta A(i,i))
    DBuf<double> B;            // near-null coefficients per field, 2N
    DBuf<unsigned char> mis;   // root flags (not on the coarsest)
    DBuf<int> agg;             // aggregate id per node
    int nagg = 0;
    double lam = 0.0;          // lambda_max(D^{-1} A) estimate
    BSR P, R;                  // prolongator / restriction (not on the coarsest)
    // solve workspace (double2 per node)
    DBuf<double> f, u, r, d, w;
    // FP32 V-cycle: value copies and workspace (float2 per node)
    DBuf<float> A32, P32, R32, invdiag32;
    DBuf<float> f32, u32, r32, d32, w32;
    // Chebyshev coefficients (host copies)
    double ch_inv_theta = 0, ch_c1 = 0, ch_c2 = 0;
    // lanes per block row of A, R and P in the V-cycle's precision: T > 0
    // block-CSR with T lanes (64..256: a thread block per row), -K the
    // sliced form sl[op] with K lanes per row
    int lanes[3] = {0, 0, 0};
    SlicedOp sl[3];
};

// Finest level in sliced-ELL form (32 rows per slice, slot-major), using the
// shared pattern of the Bidomain operator: per node pair only Ki and Ke are
// stored, since the block is [Ki, Ki; Ki, Ki+Ke] off the diagonal and the
// diagonal adds c M to the (v, v) entry.
struct FineSell {
    bool valid = false;
    int nslices = 0;
    long long slots = 0;        // padded slots (x 32 lanes)
    DBuf<int> sptr;             // nslices + 1, slot offset of each slice
    DBuf<int> col;              // slots * 32 column (FP64 kernels: an index costs no FP64 time)
    DBuf<unsigned char> code;   // slots * 32: neighbour q = p + off[code] (27-point stencil; FP32)
    int off[27] = {};           // node-index offset of each stencil position
    DBuf<double> kk;            // slots * 32 * 2: (Ki, Ke)
    DBuf<double> cm;            // c M_p per node
    DBuf<float> kk32, cm32;     // FP32 copies for the FP32 V-cycle
};

}  // namespace bd

struct amg_hierarchy {
    amg_options opts{};
    int nlev = 0;
    bool prec32 = false;        // V-cycle in FP32 inside an FP64 flexible CG
    bd::FineSell sell;
    bd::Level lev[bd::kMaxLevels];
    // coarsest level: dense inverse of A_c + s z z^T / z^T z, null vector z
    int nc = 0;
    bd::DBuf<double> cinv, zc;
    double zz = 0.0;
    // PCG workspace on the finest level
    bd::DBuf<double> x, r, z, p, q, fp, zold, fin;
    // whole-solve CUDA graph: pre-loop, a device-controlled WHILE node over one
    // PCG iteration, post-loop (built on first use, reused by every solve)
    cudaGraph_t graph = nullptr;
    cudaGraphExec_t graph_exec = nullptr;
    cudaStream_t cap_stream = nullptr, cap_stream2 = nullptr;
    bool graph_failed = false;
    long long graph_pre = 0, graph_body = 0, graph_post = 0;  // kernel nodes per section
    double *host_init = nullptr;  // pinned initial scalar block for a graph launch
    cudaEvent_t ev_solve[2] = {nullptr, nullptr};  // device time of a graph-form solve
    bd::DBuf<double> partial;   // kRedBlocks x 4 partial sums
    bd::DBuf<unsigned int> counter;  // arrival counter of the last-block reductions
    bd::DBuf<double> scal;      // device scalars of the PCG recurrences
    double *host_scal = nullptr;  // pinned mirror
    bd::DBuf<long long> exact_acc;
    // live timing of the finest-level operator applications
    int prof = 0;
    std::vector<cudaEvent_t> ev;      // pairs
    std::vector<double> ev_bytes, ev_flops, ev_ops;
    int ev_used = 0;
    amg_kernel_profile prof_sum{};
    // per-step breakdown (profiling level 2): label of each event pair and the
    // sums per label (level * 16 + role; level 15 holds the level-free steps)
    std::vector<int> ev_label;
    double trace_ms[256] = {};
    long long trace_n[256] = {};
    int batch_refs = 0;         // batches holding graphs of this hierarchy's kernels
    ~amg_hierarchy() {
        for (cudaEvent_t e : ev) cudaEventDestroy(e);
        if (graph_exec) cudaGraphExecDestroy(graph_exec);
        if (graph) cudaGraphDestroy(graph);
        if (cap_stream) cudaStreamDestroy(cap_stream);
        if (cap_stream2) cudaStreamDestroy(cap_stream2);
        if (host_init) cudaFreeHost(host_init);
        if (ev_solve[0]) cudaEventDestroy(ev_solve[0]);
        if (ev_solve[1]) cudaEventDestroy(ev_solve[1]);
    }
};

namespace bd {
// solve-phase entry points used by bd_step (amg_solve.cu)
int pcg_solve_device(amg_hierarchy *h, const double *f_dev, double *x_dev, int warm,
                     const solve_options *o, cudaStream_t s, solve_info *info);
int vcycle_device(amg_hierarchy *h, const double *r_dev, double *z_dev, cudaStream_t s);
int prepare_solve(amg_hierarchy *h, cudaStream_t s);
int pcg_solve_begin(amg_hierarchy *h, const double *f_dev, double *x_dev, int warm,
                    const solve_options *o, cudaStream_t s, solve_info *info, bool *pending);
int pcg_solve_end(amg_hierarchy *h, cudaStream_t s, solve_info *info);
int build_fine_sell(amg_hierarchy *h, const bd_system *sys, cudaStream_t s);
// Timed step of the solve phase (host-driven loop only).  `fine`: a
// finest-operator application, timed at profiling level 1 and summed into
// amg_kernel_profile; every labelled step is timed at level 2.
enum ProfRole {
    R_PRE = 0, R_RESID = 1, R_RESTRICT = 2, R_PROLONG = 3, R_POST1 = 4, R_POST2 = 5,
    R_COARSE = 15 * 16, R_VIN, R_VOUT, R_ZSTATS, R_PUPDATE, R_AP, R_XRUPDATE
};
int prof_begin(amg_hierarchy *h, cudaStream_t s, int label, bool fine);
void prof_end(amg_hierarchy *h, int slot, double bytes, double flops, cudaStream_t s, double ops = 0.0);
void prof_collect(amg_hierarchy *h);
}  // namespace bd
