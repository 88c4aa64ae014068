// bd_decoupled.cu -- the paper's own time-stepping scheme (Section 2.2,
// Eqs. 4-7 as printed): per step the gating update (Eq. 4), the elliptic
// system (Ai + Ae) u_e^n = -Ai v^n (Eq. 6) by AMG-PCG, then the parabolic
// system (c M + Ai) v^{n+1} = c M v^n - Ai u_e^n + M (I_app - chi I_ion)
// (Eq. 7, ionic sign as in the coupled step) by CG, Jacobi-preconditioned or
// unpreconditioned (the paper's GPU runs leave it unpreconditioned).
//
// The elliptic hierarchy is the block hierarchy of [I, 0; 0, Ai + Ae]
// (bd_elliptic_setup); its iterate is kept as (0, u_e) pairs, whose zero
// v-field the solve preserves.  The parabolic CG runs on the host loop with
// its inner products summed in a fixed order (per-block partials added on
// the host in block order), so it is reproducible run to run.
#include <cmath>
#include <new>

#include "amg_internal.cuh"

namespace {

constexpr int kParBlocks = 1216;  // fixed grid of the parabolic reductions
constexpr int kParVals = 3;       // partial sums per block

// sums of up to kParVals values over the block, in a fixed order, by thread 0
__device__ void block_partials(double a, double b, double c, double *partial)
{
    __shared__ double buf[kParVals][256];
    buf[0][threadIdx.x] = a;
    buf[1][threadIdx.x] = b;
    buf[2][threadIdx.x] = c;
    __syncthreads();
    const int w = threadIdx.x >> 5, l = threadIdx.x & 31;
    if (w < kParVals) {
        double t = buf[w][l];
        for (int i = l + 32; i < (int)blockDim.x; i += 32) t += buf[w][i];
        for (int o = 16; o; o >>= 1) t += __shfl_xor_sync(0xffffffffu, t, o);
        if (l == 0) partial[kParVals * blockIdx.x + w] = t;
    }
}

// Ai x on the node pattern, row p
__device__ __forceinline__ double ki_row(int p, const int *__restrict__ rp, const int *__restrict__ ci,
                                         const double *__restrict__ Ki, const double *__restrict__ x,
                                         int stride, int off)
{
    double a = 0.0;
    for (int t = rp[p]; t < rp[p + 1]; t++) a = fma(Ki[t], x[(size_t)stride * ci[t] + off], a);
    return a;
}

// elliptic right-hand side (0, -Ai v)
__global__ void k_ell_rhs(int N, const int *__restrict__ rp, const int *__restrict__ ci,
                          const double *__restrict__ Ki, const double *__restrict__ v, double2 *__restrict__ fe)
{
    for (int p = blockIdx.x * blockDim.x + threadIdx.x; p < N; p += gridDim.x * blockDim.x)
        fe[p] = make_double2(0.0, -ki_row(p, rp, ci, Ki, v, 1, 0));
}

// gating update (Eq. 4) and parabolic right-hand side (Eq. 7); u_e from the
// elliptic iterate (0, u_e)
__global__ void k_par_rhs(int N, const int *__restrict__ rp, const int *__restrict__ ci,
                          const double *__restrict__ Ki, const double *__restrict__ M,
                          const double *__restrict__ stim, int stim_on, double chi, double cm, double dt,
                          bd_rm_params rm, const double *__restrict__ v, double *__restrict__ w,
                          const double *__restrict__ xe, double *__restrict__ b)
{
    const double c = (chi * cm) / dt;
    for (int p = blockIdx.x * blockDim.x + threadIdx.x; p < N; p += gridDim.x * blockDim.x) {
        const double a = ki_row(p, rp, ci, Ki, xe, 2, 1);
        const double vk = v[p];
        const double wn = (w[p] + dt * rm.eta2 * vk / rm.vp) / (1.0 + dt * rm.eta2 * rm.eta3);
        const double iion = rm.G * vk * (1.0 - vk / rm.vth) * (1.0 - vk / rm.vp) + rm.eta1 * vk * wn;
        const double iapp = stim_on ? stim[p] : 0.0;
        b[p] = c * M[p] * vk - a + M[p] * (iapp - chi * iion);
        w[p] = wn;
    }
}

// inverse diagonal of c M + Ai (ones when unpreconditioned)
__global__ void k_par_dinv(int N, const int *__restrict__ rp, const int *__restrict__ ci,
                           const double *__restrict__ Ki, const double *__restrict__ M, double c, int jacobi,
                           double *__restrict__ dinv)
{
    for (int p = blockIdx.x * blockDim.x + threadIdx.x; p < N; p += gridDim.x * blockDim.x) {
        double d = c * M[p];
        for (int t = rp[p]; t < rp[p + 1]; t++)
            if (ci[t] == p) d = d + Ki[t];
        dinv[p] = jacobi ? 1.0 / d : 1.0;
    }
}

// r = b - (c M + Ai) v, z = D^{-1} r; partials r.r, r.z, b.b
__global__ void __launch_bounds__(256) k_par_resid(int N, const int *__restrict__ rp, const int *__restrict__ ci,
                                                   const double *__restrict__ Ki, const double *__restrict__ M, double c,
                                                   const double *__restrict__ v, const double *__restrict__ b,
                                                   const double *__restrict__ dinv, double *__restrict__ r,
                                                   double *__restrict__ z, double *__restrict__ partial)
{
    double rr = 0.0, rz = 0.0, bb = 0.0;
    for (int p = blockIdx.x * blockDim.x + threadIdx.x; p < N; p += gridDim.x * blockDim.x) {
        const double y = fma(c * M[p], v[p], ki_row(p, rp, ci, Ki, v, 1, 0));
        const double bp = b[p], rv = bp - y, zv = dinv[p] * rv;
        r[p] = rv;
        z[p] = zv;
        rr += rv * rv;
        rz += rv * zv;
        bb += bp * bp;
    }
    block_partials(rr, rz, bb, partial);
}

// q = (c M + Ai) p; partial p.q
__global__ void __launch_bounds__(256) k_par_apply(int N, const int *__restrict__ rp, const int *__restrict__ ci,
                                                   const double *__restrict__ Ki, const double *__restrict__ M, double c,
                                                   const double *__restrict__ pv, double *__restrict__ q,
                                                   double *__restrict__ partial)
{
    double pq = 0.0;
    for (int p = blockIdx.x * blockDim.x + threadIdx.x; p < N; p += gridDim.x * blockDim.x) {
        const double y = fma(c * M[p], pv[p], ki_row(p, rp, ci, Ki, pv, 1, 0));
        q[p] = y;
        pq += pv[p] * y;
    }
    block_partials(pq, 0.0, 0.0, partial);
}

// v += alpha p, r -= alpha q, z = D^{-1} r; partials r.r, r.z
__global__ void __launch_bounds__(256) k_par_update(int N, double alpha, const double *__restrict__ pv,
                                                    const double *__restrict__ q, const double *__restrict__ dinv,
                                                    double *__restrict__ v, double *__restrict__ r,
                                                    double *__restrict__ z, double *__restrict__ partial)
{
    double rr = 0.0, rz = 0.0;
    for (int p = blockIdx.x * blockDim.x + threadIdx.x; p < N; p += gridDim.x * blockDim.x) {
        v[p] = fma(alpha, pv[p], v[p]);
        const double rv = fma(-alpha, q[p], r[p]), zv = dinv[p] * rv;
        r[p] = rv;
        z[p] = zv;
        rr += rv * rv;
        rz += rv * zv;
    }
    block_partials(rr, rz, 0.0, partial);
}

__global__ void k_par_direction(int N, double beta, const double *__restrict__ z, double *__restrict__ pv, int first)
{
    for (int p = blockIdx.x * blockDim.x + threadIdx.x; p < N; p += gridDim.x * blockDim.x)
        pv[p] = first ? z[p] : fma(beta, pv[p], z[p]);
}

__global__ void k_split(int N, const double2 *__restrict__ xe, double *__restrict__ ue)
{
    for (int p = blockIdx.x * blockDim.x + threadIdx.x; p < N; p += gridDim.x * blockDim.x) ue[p] = xe[p].y;
}

__global__ void k_join(int N, const double *__restrict__ ue, double2 *__restrict__ xe)
{
    for (int p = blockIdx.x * blockDim.x + threadIdx.x; p < N; p += gridDim.x * blockDim.x)
        xe[p] = make_double2(0.0, ue[p]);
}

}  // namespace

struct bd_dsim {
    const bd_system *sys = nullptr;
    amg_hierarchy *h = nullptr;
    bd_rm_params rm{};
    int N = 0, jacobi = 1;
    long long step = 0;
    double stim_ms = 0.0;
    bd::DBuf<double> v, w, stim;   // N each
    bd::DBuf<double> xe, fe;       // elliptic iterate (0, u_e) and right-hand side, 2N
    bd::DBuf<double> b, r, z, p, q, dinv, partial;
    double *host_part = nullptr;   // pinned kParBlocks x kParVals
    cudaEvent_t ev[2] = {nullptr, nullptr};
    ~bd_dsim()
    {
        if (host_part) cudaFreeHost(host_part);
        if (ev[0]) cudaEventDestroy(ev[0]);
        if (ev[1]) cudaEventDestroy(ev[1]);
    }
};

using namespace bd;

namespace {

// block partials -> host, summed in block order
int read_sums(bd_dsim *S, cudaStream_t s, int nv, double *out)
{
    BD_CUDA(cudaMemcpyAsync(S->host_part, S->partial.p, sizeof(double) * kParVals * kParBlocks,
                            cudaMemcpyDeviceToHost, s));
    BD_CUDA(cudaStreamSynchronize(s));
    for (int k = 0; k < nv; k++) {
        double t = 0.0;
        for (int i = 0; i < kParBlocks; i++) t += S->host_part[kParVals * i + k];
        out[k] = t;
    }
    return BD_OK;
}

// (c M + Ai) v = b by (Jacobi-)CG from the current v; iterations and the
// recurrence / true residuals into info
int parabolic_cg(bd_dsim *S, const solve_options *o, cudaStream_t s, solve_info *info)
{
    const bd_system *sys = S->sys;
    const bd_params &P = sys->params;
    const int N = S->N;
    const double c = (P.chi * P.cm) / P.dt;
    const int *rp = sys->A.rp.p, *ci = sys->A.ci.p;
    const int G = kParBlocks;
    double sums[3];
    k_par_resid<<<G, 256, 0, s>>>(N, rp, ci, sys->Ki.p, sys->M.p, c, S->v.p, S->b.p, S->dinv.p, S->r.p, S->z.p,
                                  S->partial.p); note_launch();
    BD_LAUNCH_CHECK();
    BD_TRY(read_sums(S, s, 3, sums));
    const double nb = std::sqrt(sums[2]);
    double rr = std::sqrt(sums[0]), rz = sums[1];
    int it = 0, status = BD_OK;
    if (nb == 0.0) {
        BD_CUDA(cudaMemsetAsync(S->v.p, 0, S->v.bytes(), s));
        rr = 0.0;
    } else if (!(rr <= o->rtol * nb)) {
        status = BD_ENOTCONV;
        k_par_direction<<<grid_for(N, 256), 256, 0, s>>>(N, 0.0, S->z.p, S->p.p, 1); note_launch();
        while (it < o->max_it) {
            k_par_apply<<<G, 256, 0, s>>>(N, rp, ci, sys->Ki.p, sys->M.p, c, S->p.p, S->q.p, S->partial.p);
            note_launch();
            BD_LAUNCH_CHECK();
            BD_TRY(read_sums(S, s, 1, sums));
            const double pq = sums[0];
            if (!(pq > 0.0) || !std::isfinite(pq)) {
                status = BD_EBREAKDOWN;
                break;
            }
            const double alpha = rz / pq;
            k_par_update<<<G, 256, 0, s>>>(N, alpha, S->p.p, S->q.p, S->dinv.p, S->v.p, S->r.p, S->z.p,
                                           S->partial.p); note_launch();
            BD_LAUNCH_CHECK();
            BD_TRY(read_sums(S, s, 2, sums));
            it++;
            rr = std::sqrt(sums[0]);
            if (rr <= o->rtol * nb) {
                status = BD_OK;
                break;
            }
            const double beta = sums[1] / rz;
            rz = sums[1];
            k_par_direction<<<grid_for(N, 256), 256, 0, s>>>(N, beta, S->z.p, S->p.p, 0); note_launch();
        }
    }
    // true residual
    k_par_resid<<<G, 256, 0, s>>>(N, rp, ci, sys->Ki.p, sys->M.p, c, S->v.p, S->b.p, S->dinv.p, S->r.p, S->z.p,
                                  S->partial.p); note_launch();
    BD_LAUNCH_CHECK();
    BD_TRY(read_sums(S, s, 1, sums));
    if (info) {
        info->status = status;
        info->iters = it;
        info->rel_res = nb > 0.0 ? rr / nb : 0.0;
        info->true_rel_res = nb > 0.0 ? std::sqrt(sums[0]) / nb : 0.0;
    }
    return status;
}

}  // namespace

extern "C" int bd_dsim_create(const bd_system *sys, amg_hierarchy *h_elliptic, const bd_rm_params *rm,
                              const double *stim, int stim_on_device, double stim_ms, int jacobi, void *stream,
                              bd_dsim **out)
{
    if (!sys || !h_elliptic || !out) return BD_EINVAL;
    *out = nullptr;
    if (h_elliptic->lev[0].N != sys->N || h_elliptic->sell.valid) return BD_EINVAL;
    cudaStream_t s = (cudaStream_t)stream;
    bd_dsim *S = new (std::nothrow) bd_dsim();
    if (!S) return BD_ENOMEM;
    S->sys = sys;
    S->h = h_elliptic;
    if (rm) S->rm = *rm;
    else bd_rm_params_default(&S->rm);
    S->N = sys->N;
    S->jacobi = jacobi ? 1 : 0;
    S->stim_ms = stim ? stim_ms : 0.0;
    const size_t N = (size_t)sys->N;
    int st;
    if ((st = S->v.alloc(N)) || (st = S->w.alloc(N)) || (st = S->stim.alloc(N)) || (st = S->xe.alloc(2 * N)) ||
        (st = S->fe.alloc(2 * N)) || (st = S->b.alloc(N)) || (st = S->r.alloc(N)) || (st = S->z.alloc(N)) ||
        (st = S->p.alloc(N)) || (st = S->q.alloc(N)) || (st = S->dinv.alloc(N)) ||
        (st = S->partial.alloc((size_t)kParVals * kParBlocks))) {
        delete S;
        return st;
    }
    if (cudaMallocHost((void **)&S->host_part, sizeof(double) * kParVals * kParBlocks) != cudaSuccess ||
        cudaEventCreate(&S->ev[0]) != cudaSuccess || cudaEventCreate(&S->ev[1]) != cudaSuccess) {
        delete S;
        return BD_ECUDA;
    }
    const bd_params &P = sys->params;
    if (cudaMemsetAsync(S->v.p, 0, S->v.bytes(), s) || cudaMemsetAsync(S->w.p, 0, S->w.bytes(), s) ||
        cudaMemsetAsync(S->stim.p, 0, S->stim.bytes(), s) || cudaMemsetAsync(S->xe.p, 0, S->xe.bytes(), s) ||
        cudaMemsetAsync(S->partial.p, 0, S->partial.bytes(), s)) {
        delete S;
        return BD_ECUDA;
    }
    k_par_dinv<<<grid_for(sys->N, 256), 256, 0, s>>>(sys->N, sys->A.rp.p, sys->A.ci.p, sys->Ki.p, sys->M.p,
                                                     (P.chi * P.cm) / P.dt, S->jacobi, S->dinv.p); note_launch();
    if (cudaGetLastError() != cudaSuccess) {
        delete S;
        return BD_ECUDA;
    }
    if (stim && (st = copy_in(S->stim.p, stim, N * sizeof(double), stim_on_device, s))) {
        delete S;
        return st;
    }
    if (cudaStreamSynchronize(s) != cudaSuccess) {
        delete S;
        return BD_ECUDA;
    }
    *out = S;
    return BD_OK;
}

extern "C" int bd_dsim_set_state(bd_dsim *S, const double *v, const double *ue, const double *w, int on_device,
                                 void *stream)
{
    if (!S) return BD_EINVAL;
    cudaStream_t s = (cudaStream_t)stream;
    const size_t bytes = sizeof(double) * (size_t)S->N;
    if (v) BD_TRY(copy_in(S->v.p, v, bytes, on_device, s));
    if (w) BD_TRY(copy_in(S->w.p, w, bytes, on_device, s));
    if (ue) {
        DBuf<double> t;
        BD_TRY(t.alloc((size_t)S->N));
        BD_TRY(copy_in(t.p, ue, bytes, on_device, s));
        k_join<<<grid_for(S->N, 256), 256, 0, s>>>(S->N, t.p, (double2 *)S->xe.p); note_launch();
        BD_LAUNCH_CHECK();
        BD_CUDA(cudaStreamSynchronize(s));
    }
    BD_CUDA(cudaStreamSynchronize(s));
    return BD_OK;
}

extern "C" int bd_dsim_get_state(const bd_dsim *S, double *v, double *ue, double *w, int on_device, void *stream)
{
    if (!S) return BD_EINVAL;
    cudaStream_t s = (cudaStream_t)stream;
    const size_t bytes = sizeof(double) * (size_t)S->N;
    if (v) BD_TRY(copy_out(v, S->v.p, bytes, on_device, s));
    if (w) BD_TRY(copy_out(w, S->w.p, bytes, on_device, s));
    if (ue) {
        DBuf<double> t;
        BD_TRY(t.alloc((size_t)S->N));
        k_split<<<grid_for(S->N, 256), 256, 0, s>>>(S->N, (const double2 *)S->xe.p, t.p); note_launch();
        BD_LAUNCH_CHECK();
        BD_TRY(copy_out(ue, t.p, bytes, on_device, s));
        BD_CUDA(cudaStreamSynchronize(s));
    }
    BD_CUDA(cudaStreamSynchronize(s));
    return BD_OK;
}

extern "C" int bd_dsim_step(bd_dsim *S, int nsteps, const solve_options *opts, void *stream,
                            solve_info *elliptic, solve_info *parabolic)
{
    if (!S || nsteps < 0) return BD_EINVAL;
    solve_options o;
    solve_options_default(&o);
    if (opts) o = *opts;
    if (!(o.rtol > 0.0) || o.max_it < 0) return BD_EINVAL;
    cudaStream_t s = (cudaStream_t)stream;
    const bd_system *sys = S->sys;
    const bd_params &P = sys->params;
    solve_info ie{}, ip{};
    long long te = 0, tp = 0;
    int st = BD_OK;
    for (int k = 0; k < nsteps && st == BD_OK; k++) {
        const double t = (double)S->step * P.dt;
        // Eq. 6: (Ai + Ae) u_e^n = -Ai v^n, warm from the previous u_e
        k_ell_rhs<<<grid_for(S->N, 256), 256, 0, s>>>(S->N, sys->A.rp.p, sys->A.ci.p, sys->Ki.p, S->v.p,
                                                      (double2 *)S->fe.p); note_launch();
        BD_LAUNCH_CHECK();
        st = pcg_solve_device(S->h, S->fe.p, S->xe.p, 1, &o, s, &ie);
        te += ie.iters;
        if (st != BD_OK) break;
        // Eqs. 4 and 7, then the parabolic solve warm from v^n
        k_par_rhs<<<grid_for(S->N, 256), 256, 0, s>>>(S->N, sys->A.rp.p, sys->A.ci.p, sys->Ki.p, sys->M.p,
                                                      S->stim.p, t < S->stim_ms, P.chi, P.cm, P.dt, S->rm, S->v.p,
                                                      S->w.p, S->xe.p, S->b.p); note_launch();
        BD_LAUNCH_CHECK();
        BD_CUDA(cudaEventRecord(S->ev[0], s));
        st = parabolic_cg(S, &o, s, &ip);
        BD_CUDA(cudaEventRecord(S->ev[1], s));
        BD_CUDA(cudaEventSynchronize(S->ev[1]));
        float ms = 0.0f;
        cudaEventElapsedTime(&ms, S->ev[0], S->ev[1]);
        ip.solve_ms = ms;
        tp += ip.iters;
        S->step++;
    }
    ie.total_iters = te;
    ip.total_iters = tp;
    if (elliptic) *elliptic = ie;
    if (parabolic) *parabolic = ip;
    return st;
}

extern "C" void bd_dsim_destroy(bd_dsim *S) { delete S; }
