/*
 * bidomain.h -- C ABI of the GB300 (sm_103a) smoothed-aggregation AMG-PCG
 * solver for the coupled Bidomain system of arXiv 2311.13914.
 *
 * The operation: every semi-implicit time step of the parabolic-elliptic
 * Bidomain model (Section 2, Eq. 1; block form Eq. 3; time scheme Eqs. 4-7)
 * yields one symmetric positive semi-definite system A x = f (Section 4,
 * Eq. 9) with the interleaved 2x2-block operator
 *     A = [c M + Ki, Ki; Ki, Ki + Ke],   c = chi*Cm/dt,
 * whose null space is (v, u_e) = (0, 1).  It is solved by conjugate gradients
 * preconditioned with one algebraic-multigrid V-cycle (Algorithm 2) over a
 * smoothed-aggregation hierarchy (Algorithm 1; modified MIS, cluster rule and
 * P_ij = |C_j|^{-1/2} of Section 4; GAMG options of Appendix A).
 *
 * Conventions shared by every call
 *  - Return value: BD_OK (0) or a negative BD_E* code; bd_strerror() names it.
 *    No call aborts, traps or exits; inputs are validated before any launch.
 *  - Handles (bd_system, amg_hierarchy, bd_sim) are opaque, owned by the
 *    library, released with the matching *_destroy (NULL is accepted).
 *  - Caller arrays stay owned by the caller and are never retained after a
 *    call returns.  Arguments named *_on_device select device pointers
 *    (valid in the current CUDA context, ordered on `stream`) or host
 *    pointers (pageable or pinned; the call copies them and synchronises).
 *  - `stream` is a cudaStream_t passed as void* (NULL = legacy default
 *    stream).  Calls that return host-visible results synchronise `stream`.
 *  - Node numbering of an nx*ny*nz-element slab: k = i + (nx+1)(j + (ny+1) l).
 *    Unknowns are interleaved: x[2k] = v_k (mV), x[2k+1] = u_e,k (mV).
 *  - Units: length cm, time ms, conductivity mS/cm, capacitance uF/cm^2,
 *    current density uA/cm^2 (membrane) or uA/cm^3 (volumetric).
 *  - Scalar CSR exchange format: int32 row_ptr[n+1], int32 col[nnz] (sorted
 *    ascending within a row), double val[nnz].
 */
#ifndef BIDOMAIN_H
#define BIDOMAIN_H

#ifdef __cplusplus
extern "C" {
#endif

#define BD_OK 0
#define BD_EINVAL (-1)        /* invalid argument (NULL, size, layout, option)   */
#define BD_ENOMEM (-2)        /* device or host allocation failed                */
#define BD_ENOTCONV (-3)      /* PCG hit max_it before rtol                      */
#define BD_EBREAKDOWN (-4)    /* PCG breakdown: p^T A p <= 0, NaN or Inf         */
#define BD_ETIMEOUT (-5)      /* a bounded device-side loop gave up              */
#define BD_ECUDA (-6)         /* a CUDA runtime call failed                      */
#define BD_EINCONSISTENT (-7) /* strict mode: f not orthogonal to the null space */
#define BD_ERANGE (-8)        /* a size exceeds a documented maximum             */
#define BD_ESTATE (-9)        /* handle used in the wrong state                  */

typedef struct bd_system bd_system;
typedef struct amg_hierarchy amg_hierarchy;
typedef struct bd_sim bd_sim;

/* Slab [0,lx]x[0,ly]x[0,lz] (cm) meshed by nx*ny*nz uniform Q1 hexahedra. */
typedef struct {
    int nx, ny, nz;
    double lx, ly, lz;
} bd_mesh;

/* chi (1/cm), Cm (uF/cm^2), dt (ms); conductivities (mS/cm) along (l) and
 * across (t) the fibre, intracellular (i) and extracellular (e); the normal
 * conductivity equals the transversal one (Eq. 2 with sigma_n = sigma_t). */
typedef struct {
    double chi, cm, dt;
    double sil, sit, sel, set;
} bd_params;

/* Options of the hierarchy (amg_options_default: the Appendix A values, except that
 * the graph is squared on every level, not on the first one only). */
typedef struct {
    double theta;          /* strength threshold, Section 4 (0.06)                  */
    int coarse_eq_limit;   /* stop coarsening at <= this many unknowns (100)        */
    int max_levels;        /* (10), at most 16                                      */
    int cheb_degree;       /* Chebyshev-Jacobi sweeps per smoothing (2)             */
    int esteig_steps;      /* CG steps of the lambda_max estimate (10), <= 64       */
    int square_levels;     /* levels whose MIS runs on the squared graph (16: all;
                              Appendix A squares the first level only, 1)           */
    double eig_lo, eig_hi; /* Chebyshev interval [eig_lo, eig_hi]*lambda (0.05,1.05) */
    unsigned long long seed; /* MIS priorities and Lanczos start vector (0)         */
    int precision;         /* 0: FP64 V-cycle; 1: FP32 V-cycle (values and vectors
                              of every level in FP32, coarsest solve in FP64) inside
                              an FP64 flexible CG (Polak-Ribiere beta) (0)          */
    int autotune;          /* 0: form of the V-cycle's block operators (see
                              amg_level_lanes) from a row-count and row-length
                              rule; 1: amg_setup times the candidate forms of
                              every operator of at least 20000 blocks on this
                              GPU (warm, median of three) and keeps the
                              fastest unless the rule's form is within 3 %.
                              Either way the choice is fixed per hierarchy, so its
                              solves are reproducible; the two choices differ in
                              the summation order of row sums (last bits) (0)       */
} amg_options;

typedef struct {
    double rtol;       /* stop when ||r||_2 <= rtol ||f||_2 (1e-8)                  */
    int max_it;        /* (500)                                                     */
    int warm_start;    /* 1: x holds the initial guess on entry                     */
    int strict;        /* 1: return BD_EINCONSISTENT if f has a null-space part     */
} solve_options;

typedef struct {
    int status;          /* BD_OK, BD_ENOTCONV or BD_EBREAKDOWN                     */
    int iters;           /* PCG iterations of this solve                            */
    double rel_res;      /* recurrence residual / ||f||                             */
    double true_rel_res; /* ||f - A x|| / ||f|| recomputed after the solve          */
    double solve_ms;     /* device time of the solve (CUDA events on `stream`)      */
    long long total_iters; /* bd_step: sum of iterations over the steps taken       */
} solve_info;

/* Rogers-McCulloch membrane model (the paper's TP06 is replaced):
 * I_ion = G v (1 - v/vth)(1 - v/vp) + eta1 v w,  dw/dt = eta2 (v/vp - eta3 w).
 * G, eta1 in mS/cm^2; vth, vp in mV; eta2 in 1/ms; eta3 dimensionless. */
typedef struct {
    double G, vth, vp, eta1, eta2, eta3;
} bd_rm_params;

const char *bd_strerror(int status);
/* Number of CUDA kernels this library has launched in the process so far. */
long long bd_launch_count(void);
/* Sparse matrix products the hierarchy setup has formed in the process so far,
 * by path: *hash_calls through the warp-per-row shared-memory hash (rows of at
 * most 4096 block products), *dense_calls through the block-per-row dense
 * accumulator (longer rows).  Both paths add every entry in ascending middle
 * index, so the path never changes a bit; the counts let a test show which
 * path a setup exercised.  Errors: BD_EINVAL (NULL). */
int bd_spgemm_path_counts(long long *hash_calls, long long *dense_calls);
void amg_options_default(amg_options *o);
void solve_options_default(solve_options *o);
void bd_rm_params_default(bd_rm_params *p);

/* ---- reproducible inner product --------------------------------------------
 * *out = the correctly rounded value of sum_i x[i]*y[i] (each product rounded
 * to double, the sum accumulated exactly in a fixed-point long accumulator,
 * then rounded once to nearest-even).  The result does not depend on the
 * launch configuration or the order of the additions; the hierarchy setup
 * uses the same operation for its eigen-estimate (Appendix A, CG steps).
 * x, y: n doubles, host or device; out: host.  The call allocates a small
 * device accumulator and synchronises `stream`.  Errors: BD_EINVAL (NULL,
 * n < 0), BD_ERANGE (n > 2^31 - 1, the accumulator's carry headroom). */
int bd_dot_exact(const double *x, const double *y, long long n, int on_device, double *out,
                 void *stream);

/* Same result as bd_dot_exact, computed without allocating anything.  The
 * paper has no counterpart: this entry point exists for callers that cannot
 * call cudaMalloc -- hosts whose device memory is owned by another allocator
 * (an application that reserves the GPU's memory for its own pool up front,
 * leaving none for the library to take), and latency-critical loops in which
 * an allocation would synchronise the device and stall the pipeline.
 * x, y: n doubles in device memory; out: one double in device memory, written
 * in stream order (the call does not synchronise).  Scratch: one 552-byte
 * accumulator in a static device array that every GPU loading the library
 * holds until exit; each call clears it on `stream` before use.  All calls
 * share that array, so calls whose work overlaps on the GPU (different
 * streams, or concurrent host threads) race and must be serialised by the
 * caller.  The first call on a device looks up the array's device address
 * (cudaGetSymbolAddress) and keeps it for the life of the process; make that
 * first call before any stream capture.  The kept address is not valid after
 * cudaDeviceReset on that device: do not call this entry point after such a
 * reset.  Errors: BD_EINVAL (NULL, n < 0), BD_ERANGE (n > 2^31 - 1, the
 * accumulator's carry headroom), BD_ECUDA. */
int bd_dot_exact_noalloc(const double *x, const double *y, long long n, double *out, void *stream);

/* ---- a0: Q1 assembly (Section 2.2; Eq. 2; Eq. 3) --------------------------
 * fib: fibre unit vector a_l at the two Gauss z-levels of every element layer,
 *   fib[(ez*2 + gz)*3 + d], d = x,y,z; gz = 0 at (ez + (1-1/sqrt3)/2)*lz/nz,
 *   gz = 1 at (ez + (1+1/sqrt3)/2)*lz/nz; nz*6 doubles, host or device.
 * Builds on the device: Ki, Ke (27-point), lumped mass M (N), and the block
 * operator A in 2x2-block CSR.  Values are bit-identical to the evaluation
 * order documented with the oracle (Gauss points ascending, elements
 * ascending, no fused multiply-add).  Errors: BD_EINVAL (sizes < 1, lengths
 * <= 0, NULL), BD_ERANGE (more than 2^31-1 blocks), BD_ENOMEM, BD_ECUDA. */
int bd_assemble(const bd_mesh *mesh, const bd_params *params, const double *fib,
                int fib_on_device, void *stream, bd_system **out);

/* Sizes of an assembled system: nodes N (unknowns 2N) and scalar nnz of A. */
int bd_system_info(const bd_system *sys, int *n_nodes, long long *nnz);

/* Copy A (scalar CSR, 2N rows, sizes from bd_system_info) and M (N) to HOST
 * arrays; any pointer may be NULL.  Synchronises `stream`. */
int bd_system_export(const bd_system *sys, int *row_ptr, int *col, double *val,
                     double *M, void *stream);

void bd_system_destroy(bd_system *sys);

/* ---- a1..a9: hierarchy setup (Algorithm 1) --------------------------------
 * Builds, entirely with device kernels: strength graph (Section 4), squared
 * graph on the first square_levels levels (Appendix A square_graph),
 * hash-priority MIS, aggregates, tentative prolongator, CG-Lanczos lambda_max
 * of D^{-1}A, smoothed prolongator P = (I - 4/(3 lambda) D^{-1}A) Pt,
 * R = P^T, Galerkin A_c = R (A P), and a dense factor of the coarsest level.
 * Aggregates and patterns are bit-identical to the oracle; hierarchy values
 * follow its evaluation order.  The hierarchy is reused by every solve.
 * Errors: BD_EINVAL, BD_ERANGE (a Galerkin row wider than 8192 blocks, or a
 * coarsest level above 4096 unknowns), BD_ENOMEM, BD_ECUDA. */
int amg_setup(const bd_system *sys, const amg_options *opts, void *stream, amg_hierarchy **out);

/* Same from a caller matrix: n = 2N unknowns (even), interleaved 2-unknown
 * nodes, scalar CSR whose pattern is made of full 2x2 node blocks, symmetric
 * positive semi-definite with null vector (0,1).  Arrays host or device. */
int amg_setup_from_csr(int n, const int *row_ptr, const int *col, const double *val,
                       int on_device, const amg_options *opts, void *stream,
                       amg_hierarchy **out);

/* Level sizes: unknowns n, scalar nnz of A_l, aggregates built on level l
 * (0 on the coarsest), lambda_max estimate (0 on the coarsest), and the scalar
 * nnz of P_l (0 on the coarsest). */
int amg_num_levels(const amg_hierarchy *h, int *nlevels);
int amg_level_info(const amg_hierarchy *h, int level, int *n, long long *nnz, int *n_agg,
                   double *lambda, long long *p_nnz);

/* Form in which the V-cycle applies A_l, R_l and P_l on level `level`
 * (lanes[0..2]):
 *   T = 1..32       block-CSR, T lanes per 2x2-block row (a butterfly sums them);
 *   T = 64..256     block-CSR, one thread block of T threads per row;
 *   T = -K (K = 1, 2, 4, 8)  sliced: rows sorted by block count (descending,
 *                   stable) within windows of 1024 rows, 32/K rows per warp,
 *                   K lanes per row, entries stored group-major so every load
 *                   of a warp is contiguous; it gives the same bits as T = K;
 *   0               not applied in block form (A on a sliced-ELL finest level,
 *                   everything on the coarsest level, solved densely).
 * The sliced form is never used for A on the finest level. */
int amg_level_lanes(const amg_hierarchy *h, int level, int lanes[3]);

/* Override the forms chosen by amg_setup (values as amg_level_lanes returns
 * them; 0 keeps an operator's current form).  Builds the sliced forms it
 * needs in the V-cycle's precision and drops the hierarchy's captured solve
 * graph (the next solve captures it anew).  No solve with h may be in flight
 * on any stream; synchronises `stream`.  Errors: BD_EINVAL (NULL, level out
 * of range, a value not listed above, a nonzero value for an operator the
 * level does not apply in block form, or a sliced form for A on the finest
 * level), BD_ESTATE (a batch of amg_batch_create holds h), BD_ENOMEM, BD_ECUDA. */
int amg_set_level_lanes(amg_hierarchy *h, int level, const int lanes[3], void *stream);

/* Copy level data to HOST arrays (sizes from amg_level_info; any pointer may
 * be NULL): A_l as scalar CSR, MIS flags and aggregate ids per node, P_l as
 * scalar CSR (n rows, 2*n_agg columns).  Synchronises `stream`. */
int amg_export_level(const amg_hierarchy *h, int level, int *a_row_ptr, int *a_col,
                     double *a_val, unsigned char *mis, int *agg, int *p_row_ptr,
                     int *p_col, double *p_val, void *stream);

/* ---- a10: one V-cycle z = B r (Algorithm 2) --------------------------------
 * r, z: n doubles (host or device).  z is not projected. */
int amg_vcycle(amg_hierarchy *h, const double *r, double *z, int on_device, void *stream);

/* ---- a11: projected PCG solve of A x = f ----------------------------------
 * Runs as one CUDA graph per solve (built on the first solve and reused): the
 * iteration loop is a WHILE node whose condition the last reduction kernel of
 * each iteration sets on the device (converged, breakdown, or max_it reached),
 * so the host synchronises once per solve.  A hierarchy serves one solve at a
 * time.  With profiling on or strict mode, a host-driven loop with the same
 * kernels in the same order runs instead (identical results).
 * f, x: n = 2N doubles, host or device.  f is projected orthogonal to (0,1)
 * (Euclidean mean of the u_e entries removed) unless opts->strict, in which
 * case a relative null-space part above 1e-8 returns BD_EINCONSISTENT.  On
 * return x has mean-zero u_e.  info may be NULL.  Returns info->status. */
int amg_solve(amg_hierarchy *h, const double *f, double *x, int on_device,
              const solve_options *opts, void *stream, solve_info *info);

void amg_destroy(amg_hierarchy *h);

/* ---- many independent solves in one launch ---------------------------------
 * The batched form of amg_solve for many small systems (each too small to fill
 * the GPU on its own): the whole solves of `count` hierarchies (each as in
 * amg_solve: projected PCG with the V-cycle of Algorithm 2) are captured as
 * the branches of ONE CUDA graph with no edges between them, so a single
 * graph launch runs all of them concurrently.  The paper has no counterpart.
 *
 * amg_batch_create: h[0..count-1] distinct hierarchies (each one's buffers
 *   serve one branch; BD_EINVAL on a repeat).  The batch does not own them;
 *   destroy the batch before any of them, and use none of them elsewhere while
 *   a batch solve runs.  While the batch exists amg_set_level_lanes refuses
 *   its hierarchies (BD_ESTATE).
 * amg_batch_solve: f[k], x[k]: DEVICE pointers to 2 n_k doubles each (f_k
 *   right-hand side; x_k initial guess if opts->warm_start, solution out),
 *   valid on `stream`.  One solve_options for all (strict mode is not
 *   supported: BD_EINVAL).  info: NULL or count entries (solve_ms is the
 *   whole batch's device time).  The graph is built on the first call and
 *   rebuilt when the f/x pointers change.  Synchronises `stream`.  Returns
 *   BD_OK or the first failing solve's status.  Results equal those of
 *   amg_solve with the same hierarchy and options bit for bit. */
typedef struct amg_batch amg_batch;
int amg_batch_create(amg_hierarchy *const *h, int count, amg_batch **out);
int amg_batch_solve(amg_batch *b, const double *const *f, double *const *x, const solve_options *opts,
                    void *stream, solve_info *info);
void amg_batch_destroy(amg_batch *b);

/* ---- f2, stacked: one launch per V-cycle step for many hierarchies ----------
 * The solves of `count` hierarchies advanced together (no counterpart in the
 * paper, which solves one system per time step; the batching form of the
 * many-slab workload).  Level l of the stack holds level l of every member
 * that has one, the members' operators placed block-diagonally, so every
 * V-cycle step of Algorithm 2 (Chebyshev(2)-Jacobi smoothing of Appendix A,
 * residual, restriction, the dense coarsest solves, prolongation) is ONE
 * kernel launch for all members; the projected PCG of Section 2.2 keeps its
 * scalars (null-space means, alpha, beta, the stopping test on ||r||_2) per
 * member, each reduced over that member's nodes in a fixed order.  A batch
 * solve is one CUDA graph whose WHILE loop runs until no member iterates;
 * members that stop (converged, breakdown, max_it) keep their iterate.  Each
 * member's result agrees with amg_solve of its hierarchy to rounding (the
 * stacked reductions sum in another order) and meets the same rtol.
 * amg_stack_create: h[0..count) distinct hierarchies of one V-cycle precision
 *   with Chebyshev degree 2; their operators are copied into the stack (the
 *   hierarchies must outlive it and keep their forms: amg_set_level_lanes
 *   refuses them with BD_ESTATE while the stack exists).  Synchronises
 *   `stream`.  Errors: BD_EINVAL, BD_ERANGE (more than 2^30 nodes on a level),
 *   BD_ENOMEM, BD_ECUDA.
 * amg_stack_solve: f[k], x[k]: DEVICE pointers to 2 n_k doubles (f_k the
 *   right-hand side; x_k the initial guess if opts->warm_start, the solution
 *   on return, with mean-zero u_e).  strict mode is not supported (BD_EINVAL).
 *   info: NULL or count entries (solve_ms: the whole batch's device time).
 *   The graph is built on the first call and rebuilt when the pointers change.
 *   Synchronises `stream`.  Returns BD_OK or the first failing member's status.
 * amg_stack_info: stack levels and kernel launches per PCG iteration (all
 *   members together; after the first solve). */
typedef struct amg_stack amg_stack;
int amg_stack_create(amg_hierarchy *const *h, int count, void *stream, amg_stack **out);
int amg_stack_solve(amg_stack *b, const double *const *f, double *const *x, const solve_options *opts,
                    void *stream, solve_info *info);
int amg_stack_info(const amg_stack *b, int *levels, long long *launches_per_iteration);
void amg_stack_destroy(amg_stack *b);

/* ---- live timing of the dominant kernel ------------------------------------
 * When enabled, every application of the finest-level operator (the fused
 * SpMV launches of the V-cycle, and of PCG when the V-cycle is FP64) is
 * bracketed by CUDA events on the launching stream; the durations, the
 * algorithmic bytes (matrix values and indices once, each vector stream once)
 * and the flops the kernels execute (an FMA counts 2; the sliced-ELL form of
 * the finest level needs 2 FMA per stored node pair with its gathered vector
 * in (v + u, u) form, 2 FMA and an add otherwise, where the 2x2-block operator
 * would take 8 flops per block) are summed; the last post-smoothing launch
 * with the PCG's z statistics counts its FP64 streams (r read, z written, and
 * z_old read in the flexible form) too.  Switching it on resets the sums, switching it off keeps them
 * for amg_profile_read; reading requires no pending work.  enable: 0 off,
 * 1 on, 2 on with the per-step breakdown below.  While it is on,
 * solves run the host-driven loop (one launch at a time) instead of the
 * whole-solve CUDA graph. */
typedef struct {
    long long launches;
    double total_ms;
    double bytes;
    double flops;
    int precision;     /* 0: the timed launches are FP64, 1: FP32 (V-cycle) */
    double fp64_ops;   /* FP64 pipe operations of those launches: a fused
                          multiply-add, an add or a multiply counts one (2 FMA
                          per stored node pair in the (v + u, u) form, and the
                          fused epilogue's operations per node) */
} amg_kernel_profile;
int amg_profile_enable(amg_hierarchy *h, int enable);
int amg_profile_read(const amg_hierarchy *h, amg_kernel_profile *out);

/* Per-step breakdown: with amg_profile_enable(h, 2) every step of the solve
 * phase (host-driven loop) is bracketed by CUDA events as well, and the
 * device time and count of each step kind are summed into ms[256] and
 * count[256], index 16 * level + role for the V-cycle steps of a level
 * (role 0 pre-smoother, 1 residual, 2 restriction, 3 prolongation, 4 and 5
 * the post-smoother's two steps) and 240 + k for the rest (k = 0 coarsest
 * solve, 1 V-cycle input, 2 V-cycle output, 3 preconditioned-residual
 * statistics, 4 search-direction update, 5 A p with p.Ap, 6 iterate and
 * residual update).  Steps fused into others have no entry of their own: on a
 * sliced-ELL finest level the statistics ride on the last post-smoothing step
 * (16 * 0 + 5), and in the PCG the V-cycle input is written by the residual
 * update (so k = 1, 2, 3 appear only for amg_vcycle or a finest level in
 * block-CSR form).  Steps shorter than the host's launch rate read high.
 * Switching profiling on from off resets these sums too. */
int amg_profile_breakdown(const amg_hierarchy *h, double *ms, long long *count);

/* ---- a12: time stepping (Eqs. 4-7 in coupled form) ------------------------
 * A simulation owns device state v, u_e, w (N each, zero at creation) and
 * borrows sys and h (which must outlive it).  stim: per-node applied current
 * (uA/cm^3, N doubles, host or device), applied while t < stim_ms.
 * Each step: w^{n+1} = (w + dt eta2 v/vp)/(1 + dt eta2 eta3);
 * f = [M (c v + I_app - chi I_ion(v, w^{n+1})); 0]; solve with warm start;
 * then t += dt.  bd_step runs nsteps steps; `last` receives the last solve
 * plus the total iteration count. */
int bd_sim_create(const bd_system *sys, amg_hierarchy *h, const bd_rm_params *rm,
                  const double *stim, int stim_on_device, double stim_ms, void *stream,
                  bd_sim **out);
int bd_sim_set_state(bd_sim *s, const double *v, const double *ue, const double *w,
                     int on_device, void *stream);
int bd_sim_get_state(const bd_sim *s, double *v, double *ue, double *w, int on_device,
                     void *stream);
int bd_step(bd_sim *s, int nsteps, const solve_options *opts, void *stream, solve_info *last);
void bd_sim_destroy(bd_sim *s);

/* ---- the paper's decoupled scheme (Section 2.2, Eqs. 4-7 as printed) ------
 * Per step: the gating update (Eq. 4); the elliptic system
 * (Ai + Ae) u_e^n = -Ai v^n (Eq. 6) by projected AMG-PCG, warm from the
 * previous u_e; the parabolic system (c M + Ai) v^{n+1} = c M v^n - Ai u_e^n
 * + M (I_app - chi I_ion(v^n, w^{n+1})) (Eq. 7, ionic sign as in bd_step) by
 * CG from v^n, Jacobi-preconditioned (jacobi = 1) or unpreconditioned (0, the
 * paper's GPU runs).  Both solves stop at ||r||_2 <= rtol ||f||_2.
 *
 * bd_elliptic_setup builds the hierarchy of the elliptic operator in the
 * block form the hierarchy code takes, [I, 0; 0, Ai + Ae] on the node pattern
 * (its u-field is smoothed aggregation on Ai + Ae with the strength of
 * amg_options; the identity v-field stays zero), with the same options and
 * determinism as amg_setup.  A decoupled simulation borrows sys and that
 * hierarchy (which must outlive it) and owns v, u_e, w (N each, zero at
 * creation).  bd_dsim_step runs nsteps steps; `elliptic` and `parabolic`
 * (either may be NULL) receive the last step's solves and the total
 * iteration counts; solve_ms of `parabolic` is its device time.  Returns the
 * first failing solve's status (BD_EINVAL for a hierarchy that was not built
 * by bd_elliptic_setup). */
typedef struct bd_dsim bd_dsim;
int bd_elliptic_setup(const bd_system *sys, const amg_options *opts, void *stream,
                      amg_hierarchy **out);
int bd_dsim_create(const bd_system *sys, amg_hierarchy *h_elliptic, const bd_rm_params *rm,
                   const double *stim, int stim_on_device, double stim_ms, int jacobi,
                   void *stream, bd_dsim **out);
int bd_dsim_set_state(bd_dsim *s, const double *v, const double *ue, const double *w,
                      int on_device, void *stream);
int bd_dsim_get_state(const bd_dsim *s, double *v, double *ue, double *w, int on_device,
                      void *stream);
int bd_dsim_step(bd_dsim *s, int nsteps, const solve_options *opts, void *stream,
                 solve_info *elliptic, solve_info *parabolic);
void bd_dsim_destroy(bd_dsim *s);

/* ---- serving: continuous batching of simulations ---------------------------
 * A request is a whole simulation (slab, fibre table, stimulus, number of time
 * steps, as for bd_assemble / bd_sim_create; host arrays, copied at submit).
 * Each tick of the scheduler (1) admits queued requests in arrival order while
 * the estimated device-memory footprint of the resident requests stays within
 * hbm_budget (estimate from the measured bytes per node of earlier requests;
 * a request that alone exceeds the budget fails with BD_ENOMEM), builds their
 * operator and hierarchy, which stay resident until the request finishes;
 * (2) starts a time step of every idle admitted simulation, each on its own
 * stream, so solves of different sizes overlap on the GPU; (3) waits until at
 * least one started step has finished, starts the next step of each request
 * whose step finished (small simulations advance while large ones solve) and
 * retires finished requests, whose memory admits the next ones.  A
 * request's result does not depend on the other requests in flight (every
 * request owns its buffers; the kernels are deterministic).  Times are host
 * milliseconds since bd_server_create.  Not thread-safe: one host thread
 * drives a server. */
typedef struct bd_server bd_server;
typedef struct {
    long long hbm_budget; /* bytes the resident requests may hold (0: 80 % of free memory) */
    int max_active;       /* simulations advanced per tick (16)                     */
    int precision;        /* V-cycle precision of every request (0: FP64, 1: FP32)  */
    double rtol;          /* (1e-8)                                                 */
    int max_it;           /* (500)                                                  */
} bd_server_options;
typedef struct {
    int state;            /* 0 queued, 1 active, 2 done, < 0 failed with that status */
    int steps_done;
    long long total_iters;
    double submit_ms, admit_ms, done_ms;
    long long footprint;  /* measured device bytes while resident (0 when not)       */
    int n_nodes;
} bd_request_info;
void bd_server_options_default(bd_server_options *o);
int bd_server_create(const bd_server_options *opts, bd_server **out);
int bd_server_submit(bd_server *s, const bd_mesh *mesh, const bd_params *params, const double *fib,
                     const double *stim, double stim_ms, int nsteps, long long *id);
int bd_server_tick(bd_server *s, int *n_active, int *n_queued);
int bd_server_drain(bd_server *s); /* tick until nothing is queued or active */
int bd_server_request(const bd_server *s, long long id, bd_request_info *out);
/* final (v, u_e, w) of a finished request into host arrays of n_nodes doubles */
int bd_server_result(const bd_server *s, long long id, double *v, double *ue, double *w);
int bd_server_stats(const bd_server *s, long long *solves, long long *resident_bytes,
                    long long *budget_bytes);
void bd_server_destroy(bd_server *s);

#ifdef __cplusplus
}
#endif
#endif /* BIDOMAIN_H */
