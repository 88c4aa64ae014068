/*
 * bd_oracle.h -- plain, slow, FP64 CPU oracle for the smoothed-aggregation
 * AMG-preconditioned CG solve of the coupled Bidomain block system.
 *
 * TEST INFRASTRUCTURE ONLY.  Nothing in the product library includes, links or
 * calls this file; only the test-suite, the smoke check and the CPU-baseline
 * leg of the benchmark load it.  It shares no code with the CUDA path.
 *
 * Every function follows a passage of the paper (arXiv 2311.13914, "A comparison
 * of Algebraic Multigrid Bidomain solvers on hybrid CPU-GPU architectures"),
 * cited as section / equation / algorithm.  Where the paper is silent the
 * reading used is stated in the function's comment.
 *
 * Conventions.  Nodes of an nx*ny*nz-element box are numbered
 * k = i + (nx+1)*(j + (ny+1)*l).  The coupled unknown vector is interleaved:
 * x[2k] = v_k (transmembrane), x[2k+1] = u_e,k (extracellular).
 * All matrices are scalar CSR with sorted column indices, owned by the oracle
 * and released with oc_csr_free.  Return value 0 = ok, negative = error.
 */
#ifndef BD_ORACLE_H
#define BD_ORACLE_H
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef struct {
    int nrows, ncols;
    int64_t nnz;
    int64_t *rp;   /* nrows+1 */
    int *ci;       /* nnz */
    double *v;     /* nnz */
} oc_csr;

void oc_csr_free(oc_csr *a);

/* Threads of the solve phase (OpenMP build): only loops with independent
 * iterations run in parallel and every reduction stays serial, so results are
 * bitwise independent of the thread count.  oc_set_threads returns nonzero if
 * the count cannot be set (n < 1, or n > 1 in a build without OpenMP). */
int oc_set_threads(int n);
int oc_get_threads(void);

/* Correctly rounded sum of the rounded products x[i]*y[i] (exact long
 * accumulator, then one rounding to nearest-even). */
double oc_dot_exact(int64_t n, const double *x, const double *y);
/* Correctly rounded sum of x[0..n). */
double oc_sum_exact(int64_t n, const double *x);

/* ---- a0: Q1 assembly (Section 2.2, Eq. 2, Eq. 3) ---------------------------
 * fib: fibre unit vector a_l at the two Gauss z-levels of every element layer,
 *      fib[((ez*2)+gz)*3 + d], gz=0 at z0+hz*(1-1/sqrt3)/2, gz=1 at z0+hz*(1+1/sqrt3)/2.
 * Outputs: Ki, Ke (N x N scalar, 27-point), M (lumped mass, N), A (2N x 2N
 * interleaved block [cM+Ki, Ki; Ki, Ki+Ke], c = chi*Cm/dt). Any output may be NULL. */
int oc_assemble(int nx, int ny, int nz, double lx, double ly, double lz,
                const double *fib, double sil, double sit, double sel, double set,
                double chi, double cm, double dt,
                oc_csr *Ki, oc_csr *Ke, double *M, oc_csr *A);

/* ---- generic sparse helpers ---------------------------------------------- */
int oc_spmv(const oc_csr *A, const double *x, double *y);          /* y = A x  */
int oc_transpose(const oc_csr *A, oc_csr *T);                      /* T = A^T  */
int oc_spgemm(const oc_csr *A, const oc_csr *B, oc_csr *C);        /* C = A B  */

/* ---- a1: strength graph (Section 4, modified MIS, first phase) ------------
 * Node graph of the 2x2-block matrix A (2N x 2N).  S holds, for every node p,
 * the strong neighbours q != p (ascending) with S.v = w_pq. */
int oc_strength(const oc_csr *A, double theta, oc_csr *S);
/* Appendix A square_graph: S2 = (I+W)^2 without diagonal. */
int oc_square_graph(const oc_csr *S, oc_csr *S2);

/* ---- a2: MIS (Section 4): lexicographically-first MIS in priority order ---- */
uint64_t oc_mix64(uint64_t z);
uint64_t oc_level_key(uint64_t seed, int level, int stream);
int oc_mis(const oc_csr *S, uint64_t key, unsigned char *in_set);

/* ---- a3: aggregation (Section 4, cluster rule) ----------------------------- */
int oc_aggregate(const oc_csr *S, const unsigned char *in_set, int *agg, int *n_agg);

/* ---- a4: tentative prolongator (Section 4, P_ij = |C_j|^{-1/2}) ------------
 * B: per-field near-null coefficients on this level (2N), Bc: next level (2*n_agg). */
int oc_ptent(int N, const int *agg, int n_agg, const double *B, oc_csr *Pt, double *Bc);

/* ---- a5: lambda_max of D^{-1}A by 10-step CG-Lanczos (Appendix A) ---------- */
int oc_lambda_max(const oc_csr *A, int steps, uint64_t key, double *lam, int *steps_done);
double oc_tridiag_max_eig(int m, const double *diag, const double *off);

/* ---- a6: smoothed prolongator P = (I - omega D^{-1} A) Pt (Appendix A) ----- */
int oc_smooth_p(const oc_csr *A, const oc_csr *Pt, double omega, oc_csr *P);

/* ---- hierarchy: Algorithm 1 with a1..a9 ----------------------------------- */
typedef struct {
    double theta;          /* strength threshold (0.06) */
    int coarse_eq_limit;   /* stop at <= this many unknowns (100) */
    int max_levels;        /* (10) */
    int cheb_degree;       /* (2) */
    int esteig_steps;      /* (10) */
    double eig_lo, eig_hi; /* Chebyshev interval factors (0.05, 1.05) */
    uint64_t seed;
    int square_levels;     /* levels whose MIS runs on the squared graph */
} oc_amg_opts;

typedef struct oc_hier oc_hier;
int oc_setup(const oc_csr *A, const oc_amg_opts *o, oc_hier **out);
void oc_hier_free(oc_hier *h);
int oc_hier_nlevels(const oc_hier *h);
/* Level accessors (pointers stay owned by h). */
const oc_csr *oc_hier_A(const oc_hier *h, int l);
const oc_csr *oc_hier_P(const oc_hier *h, int l);   /* NULL on the coarsest */
const oc_csr *oc_hier_Pt(const oc_hier *h, int l);
const int *oc_hier_agg(const oc_hier *h, int l);
const unsigned char *oc_hier_mis(const oc_hier *h, int l);
int oc_hier_nagg(const oc_hier *h, int l);
double oc_hier_lambda(const oc_hier *h, int l);
const double *oc_hier_null(const oc_hier *h, int l); /* z-hat on level l (2N_l) */

/* ---- a10: smoother and V-cycle (Algorithm 2, Appendix A) ------------------- */
/* degree-k Chebyshev-Jacobi on D^{-1}A over [lo, hi]; x updated in place. */
int oc_chebyshev(const oc_csr *A, const double *f, double *x, int x_is_zero,
                 int degree, double lo, double hi);
int oc_coarse_solve(const oc_hier *h, const double *r, double *x);
int oc_vcycle(const oc_hier *h, const double *r, double *z);

/* ---- a11: projected PCG (Section 2.2 closing paragraph, Eq. 9) ------------- */
int oc_pcg(const oc_hier *h, const double *f, double *x, int warm, double rtol,
           int max_it, int *iters, double *rel_res, double *true_rel_res);

/* ---- a12: one semi-implicit step with the Rogers-McCulloch membrane ------- */
typedef struct {
    double G, vth, vp, eta1, eta2, eta3;
} oc_rm_params;
/* state: v, ue, w per node (N).  Iapp: volumetric applied current per node
 * for this step.  Builds rhs, solves with warm start, updates state. */
int oc_bd_step(const oc_hier *h, const double *M, int N, double chi, double cm,
               double dt, const oc_rm_params *rm, const double *Iapp,
               double *v, double *ue, double *w, double rtol, int max_it,
               int *iters);

/* ---- f4: the paper's decoupled scheme (Section 2.2, Eqs. 4-7 as printed) --
 * Elliptic operator Ai + Ae (symmetric positive semi-definite, null vector 1)
 * in the 2x2-block form the hierarchy code takes: block (p,q) =
 * [delta_pq, 0; 0, Ki_pq + Ke_pq] on the pattern of Ki (explicit zeros kept),
 * so the u-field of the block hierarchy is smoothed aggregation on Ai + Ae and
 * the v-field an identity that stays zero when its right-hand side is. */
int oc_elliptic_block(const oc_csr *Ki, const oc_csr *Ke, oc_csr *out);

/* Parabolic system (c M + Ai) v = b (Eq. 7, symmetric positive definite) by
 * CG, Jacobi-preconditioned when jacobi != 0, unpreconditioned otherwise (the
 * paper's GPU runs), from v (warm start), to ||r||_2 <= rtol ||b||_2. */
int oc_parabolic_cg(const oc_csr *Ki, const double *M, double c, const double *b, double *v,
                    double rtol, int max_it, int jacobi, int *iters, double *rel_res);

/* One decoupled step: w^{n+1} (Eq. 4); elliptic (Ai+Ae) u_e^n = -Ai v^n
 * (Eq. 6) by oc_pcg on the hierarchy he of oc_elliptic_block, warm from ue;
 * parabolic (c M + Ai) v^{n+1} = c M v^n - Ai u_e^n + M (I_app - chi I_ion)
 * (Eq. 7, ionic sign as in oc_bd_step) warm from v^n. */
int oc_bd_step_decoupled(const oc_hier *he, const oc_csr *Ki, const double *M, int N, double chi,
                         double cm, double dt, const oc_rm_params *rm, const double *Iapp,
                         double *v, double *ue, double *w, double rtol, int max_it, int jacobi,
                         int *it_ell, int *it_par);

#ifdef __cplusplus
}
#endif
#endif
