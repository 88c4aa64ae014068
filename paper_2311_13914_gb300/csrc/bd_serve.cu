// bd_serve.cu -- continuous-batching serving loop for Bidomain simulations.
//
// Requests are whole simulations (a slab, its fibre field and stimulus, a
// number of time steps).  The scheduler admits queued requests in arrival
// order while their device-memory footprint fits the budget, keeps each
// admitted request's operator, hierarchy and state resident until its last
// step, and on every tick advances all admitted simulations by one time step:
// the steps are enqueued on one stream per request (each a whole-solve CUDA
// graph), so solves of different sizes overlap on the GPU; a request whose
// step has finished gets its next step enqueued at once, so small
// simulations advance while large ones are still solving.  Finished requests
// release their memory, which lets the next queued requests in.  Results do not depend on what else is running: every
// request owns its buffers and the kernels are deterministic.
#include <algorithm>
#include <chrono>
#include <deque>
#include <map>
#include <new>
#include <thread>
#include <vector>

#include "amg_internal.cuh"

namespace bd {
int sim_step_begin(bd_sim *sim, const solve_options *o, cudaStream_t s, solve_info *info, bool *pending);
int sim_step_end(bd_sim *sim, cudaStream_t s, solve_info *info, bool pending);
}  // namespace bd

namespace {

struct Request {
    long long id = 0;
    bd_mesh mesh{};
    bd_params params{};
    std::vector<double> fib, stim;
    double stim_ms = 0.0;
    int nsteps = 0;
    int state = 0;  // 0 queued, 1 active, 2 done, < 0 failed with that status
    int steps_done = 0;
    long long iters = 0;
    double t_submit = 0.0, t_admit = -1.0, t_done = -1.0;
    long long footprint = 0;
    bd_system *sys = nullptr;
    amg_hierarchy *h = nullptr;
    bd_sim *sim = nullptr;
    cudaStream_t stream = nullptr;
    bool pending = false;   // a graph-form step is enqueued
    bool inflight = false;  // a step has been started and not yet completed
    solve_info info{};
    std::vector<double> v, ue, w;

    long long nodes() const { return (mesh.nx + 1LL) * (mesh.ny + 1LL) * (mesh.nz + 1LL); }
};

}  // namespace

struct bd_server {
    bd_server_options o{};
    std::chrono::steady_clock::time_point t0;
    std::map<long long, Request> reqs;
    std::deque<long long> queue;
    std::vector<long long> active;
    long long next_id = 1;
    long long resident = 0;
    double bytes_per_node = 3000.0;  // footprint estimate, refined by measurement
    long long solves = 0;

    double now_ms() const
    {
        return std::chrono::duration<double, std::milli>(std::chrono::steady_clock::now() - t0).count();
    }
};

static void release(Request &r)
{
    if (r.sim) bd_sim_destroy(r.sim);
    if (r.h) amg_destroy(r.h);
    if (r.sys) bd_system_destroy(r.sys);
    if (r.stream) cudaStreamDestroy(r.stream);
    r.sim = nullptr;
    r.h = nullptr;
    r.sys = nullptr;
    r.stream = nullptr;
}

static void fail(bd_server *S, Request &r, int status)
{
    release(r);
    S->resident -= r.footprint;
    r.footprint = 0;
    r.state = status < 0 ? status : BD_ECUDA;
    r.t_done = S->now_ms();
}

// Build the request's operator, hierarchy and simulation on its own stream.
static int admit(bd_server *S, Request &r)
{
    r.t_admit = S->now_ms();
    if (cudaStreamCreateWithFlags(&r.stream, cudaStreamNonBlocking) != cudaSuccess) return BD_ECUDA;
    size_t free0 = 0, free1 = 0, total = 0;
    cudaMemGetInfo(&free0, &total);
    int st = bd_assemble(&r.mesh, &r.params, r.fib.data(), 0, r.stream, &r.sys);
    if (st) return st;
    amg_options ao;
    amg_options_default(&ao);
    ao.precision = S->o.precision;
    if ((st = amg_setup(r.sys, &ao, r.stream, &r.h))) return st;
    bd_rm_params rm;
    bd_rm_params_default(&rm);
    if ((st = bd_sim_create(r.sys, r.h, &rm, r.stim.data(), 0, r.stim_ms, r.stream, &r.sim))) return st;
    cudaMemGetInfo(&free1, &total);
    r.footprint = free0 > free1 ? (long long)(free0 - free1) : 0;
    if (r.footprint > 0)
        S->bytes_per_node = 0.5 * S->bytes_per_node + 0.5 * (double)r.footprint / (double)r.nodes();
    S->resident += r.footprint;
    r.state = 1;
    return BD_OK;
}

static void retire(bd_server *S, Request &r)
{
    const size_t N = (size_t)r.nodes();
    r.v.resize(N);
    r.ue.resize(N);
    r.w.resize(N);
    int st = bd_sim_get_state(r.sim, r.v.data(), r.ue.data(), r.w.data(), 0, r.stream);
    release(r);
    S->resident -= r.footprint;
    r.footprint = 0;
    r.state = st == BD_OK ? 2 : st;
    r.t_done = S->now_ms();
}

extern "C" void bd_server_options_default(bd_server_options *o)
{
    if (!o) return;
    o->hbm_budget = 0;
    o->max_active = 16;
    o->precision = 0;
    o->rtol = 1e-8;
    o->max_it = 500;
}

extern "C" int bd_server_create(const bd_server_options *opts, bd_server **out)
{
    if (!out) return BD_EINVAL;
    *out = nullptr;
    bd_server *S = new (std::nothrow) bd_server();
    if (!S) return BD_ENOMEM;
    bd_server_options_default(&S->o);
    if (opts) S->o = *opts;
    if (S->o.max_active < 1 || S->o.hbm_budget < 0 || (S->o.precision != 0 && S->o.precision != 1) ||
        !(S->o.rtol > 0.0) || S->o.max_it < 1) {
        delete S;
        return BD_EINVAL;
    }
    if (S->o.hbm_budget == 0) {
        size_t fr = 0, tot = 0;
        if (cudaMemGetInfo(&fr, &tot) != cudaSuccess) {
            delete S;
            return BD_ECUDA;
        }
        S->o.hbm_budget = (long long)(0.8 * (double)fr);
    }
    S->t0 = std::chrono::steady_clock::now();
    *out = S;
    return BD_OK;
}

extern "C" int bd_server_submit(bd_server *S, const bd_mesh *mesh, const bd_params *params,
                                const double *fib, const double *stim, double stim_ms, int nsteps,
                                long long *id)
{
    if (!S || !mesh || !params || !fib || !id || nsteps < 1) return BD_EINVAL;
    if (mesh->nx < 1 || mesh->ny < 1 || mesh->nz < 1) return BD_EINVAL;
    Request r;
    r.id = S->next_id++;
    r.mesh = *mesh;
    r.params = *params;
    r.fib.assign(fib, fib + (size_t)mesh->nz * 6);
    const size_t N = (size_t)r.nodes();
    if (stim) r.stim.assign(stim, stim + N);
    else r.stim.assign(N, 0.0);
    r.stim_ms = stim ? stim_ms : 0.0;
    r.nsteps = nsteps;
    r.t_submit = S->now_ms();
    *id = r.id;
    S->queue.push_back(r.id);
    S->reqs.emplace(r.id, std::move(r));
    return BD_OK;
}

extern "C" int bd_server_tick(bd_server *S, int *n_active, int *n_queued)
{
    if (!S) return BD_EINVAL;
    // 1. admission in arrival order while the footprint fits
    while (!S->queue.empty() && (int)S->active.size() < S->o.max_active) {
        Request &r = S->reqs[S->queue.front()];
        const long long est = (long long)(S->bytes_per_node * (double)r.nodes());
        if (est > S->o.hbm_budget) {  // can never fit
            S->queue.pop_front();
            fail(S, r, BD_ENOMEM);
            continue;
        }
        if (S->resident + est > S->o.hbm_budget && !S->active.empty()) break;
        S->queue.pop_front();
        int st = admit(S, r);
        if (st != BD_OK) {
            fail(S, r, st);
            continue;
        }
        S->active.push_back(r.id);
    }
    // 2. start a step of every admitted simulation that is idle, each on its stream
    solve_options so;
    solve_options_default(&so);
    so.rtol = S->o.rtol;
    so.max_it = S->o.max_it;
    auto start = [&](Request &r) {
        r.info = solve_info{};
        int st = bd::sim_step_begin(r.sim, &so, r.stream, &r.info, &r.pending);
        if (st != BD_OK && r.pending) r.pending = false, r.info.status = st;
        r.inflight = true;
    };
    // completes a started step; returns true when the request left the active set
    auto complete = [&](Request &r) -> bool {
        int st = bd::sim_step_end(r.sim, r.stream, &r.info, r.pending);
        r.inflight = false;
        r.pending = false;
        r.iters += r.info.iters;
        r.steps_done++;
        S->solves++;
        if (st != BD_OK) {
            fail(S, r, st);
            return true;
        }
        if (r.steps_done >= r.nsteps) {
            retire(S, r);
            return true;
        }
        start(r);  // next step right away
        return false;
    };
    for (long long id : S->active) {
        Request &r = S->reqs[id];
        if (!r.inflight) start(r);
    }
    // 3. wait until at least one started step has completed; complete all that have
    if (!S->active.empty()) {
        std::vector<long long> still;
        bool any = false;
        for (long long spins = 0;; spins++) {
            still.clear();
            for (long long id : S->active) {
                Request &r = S->reqs[id];
                const bool ready = !r.pending || cudaStreamQuery(r.stream) != cudaErrorNotReady;
                if (r.inflight && ready) {
                    any = true;
                    if (complete(r)) continue;
                }
                still.push_back(id);
            }
            S->active.swap(still);
            if (any || S->active.empty()) break;
            if (spins < 2000) {
                std::this_thread::yield();
            } else {  // long steps: block on the first in-flight stream instead of spinning
                cudaStreamSynchronize(S->reqs[S->active.front()].stream);
            }
        }
    }
    if (n_active) *n_active = (int)S->active.size();
    if (n_queued) *n_queued = (int)S->queue.size();
    return BD_OK;
}

extern "C" int bd_server_drain(bd_server *S)
{
    if (!S) return BD_EINVAL;
    int a = 0, q = 0;
    do {
        BD_TRY(bd_server_tick(S, &a, &q));
    } while (a > 0 || q > 0);
    return BD_OK;
}

extern "C" int bd_server_request(const bd_server *S, long long id, bd_request_info *out)
{
    if (!S || !out) return BD_EINVAL;
    auto it = S->reqs.find(id);
    if (it == S->reqs.end()) return BD_EINVAL;
    const Request &r = it->second;
    out->state = r.state;
    out->steps_done = r.steps_done;
    out->total_iters = r.iters;
    out->submit_ms = r.t_submit;
    out->admit_ms = r.t_admit;
    out->done_ms = r.t_done;
    out->footprint = r.footprint;
    out->n_nodes = (int)r.nodes();
    return BD_OK;
}

extern "C" int bd_server_result(const bd_server *S, long long id, double *v, double *ue, double *w)
{
    if (!S) return BD_EINVAL;
    auto it = S->reqs.find(id);
    if (it == S->reqs.end()) return BD_EINVAL;
    const Request &r = it->second;
    if (r.state != 2) return BD_ESTATE;
    const size_t N = r.v.size();
    if (v) std::copy(r.v.begin(), r.v.end(), v);
    if (ue) std::copy(r.ue.begin(), r.ue.end(), ue);
    if (w) std::copy(r.w.begin(), r.w.begin() + N, w);
    return BD_OK;
}

extern "C" int bd_server_stats(const bd_server *S, long long *solves, long long *resident_bytes,
                               long long *budget_bytes)
{
    if (!S) return BD_EINVAL;
    if (solves) *solves = S->solves;
    if (resident_bytes) *resident_bytes = S->resident;
    if (budget_bytes) *budget_bytes = S->o.hbm_budget;
    return BD_OK;
}

extern "C" void bd_server_destroy(bd_server *S)
{
    if (!S) return;
    for (auto &kv : S->reqs) release(kv.second);
    delete S;
}
