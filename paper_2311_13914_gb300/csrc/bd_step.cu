// bd_step.cu -- a12: semi-implicit time stepping of the coupled Bidomain
// system (Section 2.2, Eqs. 4-7 in coupled form) with the Rogers-McCulloch
// membrane model in place of the paper's TP06.
//
// One kernel per step fuses the implicit gating update, the explicit ionic
// current and the right-hand side [M (c v + I_app - chi I_ion); 0]; the solve
// then runs warm-started from the state, which is kept interleaved (v, u_e)
// so that it is the PCG iterate itself.
#include <new>

#include "amg_internal.cuh"

struct bd_sim {
    const bd_system *sys = nullptr;
    amg_hierarchy *h = nullptr;
    bd_rm_params rm{};
    int N = 0;
    long long step = 0;
    double stim_ms = 0.0;
    bd::DBuf<double> x;     // interleaved (v, u_e), 2N
    bd::DBuf<double> w;     // gating variable, N
    bd::DBuf<double> stim;  // applied current, N
    bd::DBuf<double> f;     // right-hand side, 2N
};

namespace bd {

__global__ void k_rm_rhs(int N, double2 *__restrict__ x, double *__restrict__ w,
                         const double *__restrict__ M, const double *__restrict__ stim, int stim_on,
                         double chi, double cm, double dt, bd_rm_params rm, double2 *__restrict__ f)
{
    const double c = (chi * cm) / dt;
    for (int k = blockIdx.x * blockDim.x + threadIdx.x; k < N; k += gridDim.x * blockDim.x) {
        double v = x[k].x;
        double wn = (w[k] + dt * rm.eta2 * v / rm.vp) / (1.0 + dt * rm.eta2 * rm.eta3);
        double iion = rm.G * v * (1.0 - v / rm.vth) * (1.0 - v / rm.vp) + rm.eta1 * v * wn;
        double iapp = stim_on ? stim[k] : 0.0;
        f[k] = make_double2(M[k] * (c * v + iapp - chi * iion), 0.0);
        w[k] = wn;
    }
}

__global__ void k_interleave(int N, const double *__restrict__ v, const double *__restrict__ ue,
                             double2 *__restrict__ x)
{
    for (int k = blockIdx.x * blockDim.x + threadIdx.x; k < N; k += gridDim.x * blockDim.x)
        x[k] = make_double2(v ? v[k] : 0.0, ue ? ue[k] : 0.0);
}

__global__ void k_deinterleave(int N, const double2 *__restrict__ x, double *__restrict__ v,
                               double *__restrict__ ue)
{
    for (int k = blockIdx.x * blockDim.x + threadIdx.x; k < N; k += gridDim.x * blockDim.x) {
        double2 a = x[k];
        if (v) v[k] = a.x;
        if (ue) ue[k] = a.y;
    }
}

// One time step split in two for callers that overlap several simulations:
// begin fuses the membrane update and right-hand side, then enqueues the
// warm-started solve; end waits for it and advances the step counter.
int sim_step_begin(bd_sim *sim, const solve_options *o, cudaStream_t s, solve_info *info,
                   bool *pending)
{
    const bd_params &P = sim->sys->params;
    const double t = (double)sim->step * P.dt;
    const int on = t < sim->stim_ms;
    k_rm_rhs<<<grid_for(sim->N, 256), 256, 0, s>>>(sim->N, (double2 *)sim->x.p, sim->w.p,
                                                   sim->sys->M.p, sim->stim.p, on, P.chi, P.cm,
                                                   P.dt, sim->rm, (double2 *)sim->f.p); ::bd::note_launch();
    BD_LAUNCH_CHECK();
    return pcg_solve_begin(sim->h, sim->f.p, sim->x.p, 1, o, s, info, pending);
}

int sim_step_end(bd_sim *sim, cudaStream_t s, solve_info *info, bool pending)
{
    int st = pending ? pcg_solve_end(sim->h, s, info) : info->status;
    sim->step++;
    return st;
}

}  // namespace bd

using namespace bd;

extern "C" int bd_sim_create(const bd_system *sys, amg_hierarchy *h, const bd_rm_params *rm,
                             const double *stim, int stim_on_device, double stim_ms, void *stream,
                             bd_sim **out)
{
    if (!sys || !h || !out) return BD_EINVAL;
    *out = nullptr;
    if (h->lev[0].N != sys->N) return BD_EINVAL;
    cudaStream_t s = (cudaStream_t)stream;
    bd_sim *sim = new (std::nothrow) bd_sim();
    if (!sim) return BD_ENOMEM;
    sim->sys = sys;
    sim->h = h;
    if (rm) sim->rm = *rm;
    else bd_rm_params_default(&sim->rm);
    sim->N = sys->N;
    sim->stim_ms = stim ? stim_ms : 0.0;
    size_t N = (size_t)sys->N;
    int st;
    if ((st = sim->x.alloc(2 * N)) || (st = sim->w.alloc(N)) || (st = sim->stim.alloc(N)) ||
        (st = sim->f.alloc(2 * N))) {
        delete sim;
        return st;
    }
    if (cudaMemsetAsync(sim->x.p, 0, sim->x.bytes(), s) || cudaMemsetAsync(sim->w.p, 0, sim->w.bytes(), s) ||
        cudaMemsetAsync(sim->stim.p, 0, sim->stim.bytes(), s)) {
        delete sim;
        return BD_ECUDA;
    }
    if (stim && (st = copy_in(sim->stim.p, stim, N * sizeof(double), stim_on_device, s))) {
        delete sim;
        return st;
    }
    if (cudaStreamSynchronize(s) != cudaSuccess) {
        delete sim;
        return BD_ECUDA;
    }
    *out = sim;
    return BD_OK;
}

extern "C" int bd_sim_set_state(bd_sim *sim, const double *v, const double *ue, const double *w,
                                int on_device, void *stream)
{
    if (!sim) return BD_EINVAL;
    cudaStream_t s = (cudaStream_t)stream;
    size_t N = (size_t)sim->N;
    DBuf<double> tv, tu;
    const double *pv = v, *pu = ue;
    if (!on_device) {
        if (v) {
            BD_TRY(tv.alloc(N));
            BD_TRY(copy_in(tv.p, v, N * sizeof(double), 0, s));
            pv = tv.p;
        }
        if (ue) {
            BD_TRY(tu.alloc(N));
            BD_TRY(copy_in(tu.p, ue, N * sizeof(double), 0, s));
            pu = tu.p;
        }
    }
    if (v || ue) {
        // keep the component that is not given
        DBuf<double> keepv, keepu;
        if (!v || !ue) {
            BD_TRY(keepv.alloc(N));
            BD_TRY(keepu.alloc(N));
            k_deinterleave<<<grid_for(sim->N, 256), 256, 0, s>>>(sim->N, (const double2 *)sim->x.p,
                                                                 keepv.p, keepu.p); ::bd::note_launch();
            BD_LAUNCH_CHECK();
            if (!v) pv = keepv.p;
            if (!ue) pu = keepu.p;
        }
        k_interleave<<<grid_for(sim->N, 256), 256, 0, s>>>(sim->N, pv, pu, (double2 *)sim->x.p); ::bd::note_launch();
        BD_LAUNCH_CHECK();
        BD_CUDA(cudaStreamSynchronize(s));
    }
    if (w) BD_TRY(copy_in(sim->w.p, w, N * sizeof(double), on_device, s));
    BD_CUDA(cudaStreamSynchronize(s));
    return BD_OK;
}

extern "C" int bd_sim_get_state(const bd_sim *sim, double *v, double *ue, double *w, int on_device,
                                void *stream)
{
    if (!sim) return BD_EINVAL;
    cudaStream_t s = (cudaStream_t)stream;
    size_t N = (size_t)sim->N;
    if (on_device) {
        if (v || ue) {
            k_deinterleave<<<grid_for(sim->N, 256), 256, 0, s>>>(sim->N, (const double2 *)sim->x.p, v, ue); ::bd::note_launch();
            BD_LAUNCH_CHECK();
        }
        if (w) BD_TRY(copy_out(w, sim->w.p, N * sizeof(double), 1, s));
        BD_CUDA(cudaStreamSynchronize(s));
        return BD_OK;
    }
    DBuf<double> tv, tu;
    if (v || ue) {
        BD_TRY(tv.alloc(N));
        BD_TRY(tu.alloc(N));
        k_deinterleave<<<grid_for(sim->N, 256), 256, 0, s>>>(sim->N, (const double2 *)sim->x.p, tv.p, tu.p); ::bd::note_launch();
        BD_LAUNCH_CHECK();
        if (v) BD_TRY(copy_out(v, tv.p, N * sizeof(double), 0, s));
        if (ue) BD_TRY(copy_out(ue, tu.p, N * sizeof(double), 0, s));
    }
    if (w) BD_TRY(copy_out(w, sim->w.p, N * sizeof(double), 0, s));
    BD_CUDA(cudaStreamSynchronize(s));
    return BD_OK;
}

extern "C" int bd_step(bd_sim *sim, int nsteps, const solve_options *opts, void *stream,
                       solve_info *last)
{
    if (!sim || nsteps < 0) return BD_EINVAL;
    solve_options o;
    solve_options_default(&o);
    if (opts) o = *opts;
    if (!(o.rtol > 0.0) || o.max_it < 0) return BD_EINVAL;
    cudaStream_t s = (cudaStream_t)stream;
    const bd_params &P = sim->sys->params;
    long long total = 0;
    solve_info info{};
    int st = BD_OK;
    (void)P;
    for (int k = 0; k < nsteps; k++) {
        bool pending = false;
        st = sim_step_begin(sim, &o, s, &info, &pending);
        if (st == BD_OK || !pending) st = sim_step_end(sim, s, &info, pending);
        total += info.iters;
        if (st != BD_OK) break;
    }
    info.total_iters = total;
    if (last) *last = info;
    return st;
}

extern "C" void bd_sim_destroy(bd_sim *sim) { delete sim; }
