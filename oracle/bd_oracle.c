/*
 * bd_oracle.c -- plain FP64 CPU oracle (TEST INFRASTRUCTURE ONLY; see
 * bd_oracle.h).  Compiled with -O2 -ffp-contract=off so that every a*b+c is a
 * rounded multiply followed by a rounded add, in the order written.
 *
 * Paper: arXiv 2311.13914.  Citations name the paper's section, equation or
 * algorithm.  The readings taken where the paper is silent are stated inline.
 */
#include "bd_oracle.h"

#include <math.h>
#include <stdlib.h>
#include <string.h>
#ifdef _OPENMP
#include <omp.h>
#endif

#define OC_EINVAL (-1)
#define OC_ENOMEM (-2)
#define OC_EBREAK (-3)
#define OC_ENOTCONV (-4)

/* Threads of the solve phase.  Only loops whose iterations are independent
 * (SpMV rows, element-wise vector updates, per-node time-step updates) run in
 * parallel; every reduction (dot products, means) stays a serial loop in
 * index order, so the results are bitwise the same for any thread count.
 * Built without OpenMP the oracle is serial and reports one thread. */
int oc_set_threads(int n)
{
#ifdef _OPENMP
    if (n < 1) return OC_EINVAL;
    omp_set_num_threads(n);
    return 0;
#else
    return n == 1 ? 0 : OC_EINVAL;
#endif
}

int oc_get_threads(void)
{
#ifdef _OPENMP
    return omp_get_max_threads();
#else
    return 1;
#endif
}

void oc_csr_free(oc_csr *a)
{
    if (!a) return;
    free(a->rp);
    free(a->ci);
    free(a->v);
    memset(a, 0, sizeof(*a));
}

static int csr_alloc(oc_csr *a, int nrows, int ncols, int64_t nnz)
{
    a->nrows = nrows;
    a->ncols = ncols;
    a->nnz = nnz;
    a->rp = (int64_t *)calloc((size_t)nrows + 1, sizeof(int64_t));
    a->ci = (int *)malloc(sizeof(int) * (size_t)(nnz > 0 ? nnz : 1));
    a->v = (double *)malloc(sizeof(double) * (size_t)(nnz > 0 ? nnz : 1));
    if (!a->rp || !a->ci || !a->v) {
        oc_csr_free(a);
        return OC_ENOMEM;
    }
    return 0;
}

/* position of column j in row i, or -1 (binary search; columns are sorted) */
static int64_t csr_find(const oc_csr *a, int i, int j)
{
    int64_t lo = a->rp[i], hi = a->rp[i + 1] - 1;
    while (lo <= hi) {
        int64_t mid = lo + (hi - lo) / 2;
        if (a->ci[mid] == j) return mid;
        if (a->ci[mid] < j) lo = mid + 1;
        else hi = mid - 1;
    }
    return -1;
}

/* ======================================================================
 * Correctly rounded summation.  Each addend is split exactly into 32-bit
 * digits of a fixed-point number whose unit is 2^-1074 (the smallest
 * subnormal), so the running total is exact; one final rounding to nearest,
 * ties to even, gives the correctly rounded sum.  (Long-accumulator method of
 * Collange, Defour, Graillat and Iakymchuk, 2015.)
 * ====================================================================== */
#define OC_LIMBS 68
typedef struct {
    int64_t l[OC_LIMBS];
    int64_t adds;
    int special;
    double special_sum;
} oc_acc;

static void acc_normalize(oc_acc *a)
{
    for (int i = 0; i < OC_LIMBS - 1; i++) {
        int64_t lo = a->l[i] & (int64_t)0xffffffff;
        int64_t carry = (a->l[i] - lo) / (int64_t)4294967296LL;
        a->l[i] = lo;
        a->l[i + 1] += carry;
    }
    a->adds = 0;
}

static void acc_add(oc_acc *a, double x)
{
    uint64_t b;
    memcpy(&b, &x, 8);
    int neg = (int)(b >> 63);
    int E = (int)((b >> 52) & 0x7ff);
    uint64_t m = b & 0xFFFFFFFFFFFFFULL;
    if (E == 0x7ff) {
        a->special = 1;
        a->special_sum += x;
        return;
    }
    int off;
    if (E == 0) {
        off = 0;
    } else {
        m |= (1ULL << 52);
        off = E - 1;
    }
    if (m == 0) return;
    int li = off / 32, sh = off % 32;
    uint64_t t0 = (m & 0xffffffffULL) << sh; /* < 2^63 */
    uint64_t t1 = (m >> 32) << sh;           /* < 2^52 */
    uint64_t d0 = t0 & 0xffffffffULL;
    uint64_t u1 = (t0 >> 32) + (t1 & 0xffffffffULL);
    uint64_t d1 = u1 & 0xffffffffULL;
    uint64_t d2 = (u1 >> 32) + (t1 >> 32);
    if (neg) {
        a->l[li] -= (int64_t)d0;
        a->l[li + 1] -= (int64_t)d1;
        a->l[li + 2] -= (int64_t)d2;
    } else {
        a->l[li] += (int64_t)d0;
        a->l[li + 1] += (int64_t)d1;
        a->l[li + 2] += (int64_t)d2;
    }
    if (++a->adds >= (1 << 24)) acc_normalize(a);
}

static int acc_bit(const oc_acc *a, int pos)
{
    return (int)((a->l[pos / 32] >> (pos % 32)) & 1);
}

static double acc_round(oc_acc *a)
{
    if (a->special) return a->special_sum;
    acc_normalize(a);
    double sign = 1.0;
    if (a->l[OC_LIMBS - 1] < 0) {
        for (int i = 0; i < OC_LIMBS; i++) a->l[i] = -a->l[i];
        acc_normalize(a);
        sign = -1.0;
    }
    int top = -1;
    for (int i = OC_LIMBS - 1; i >= 0; i--)
        if (a->l[i] != 0) {
            top = i;
            break;
        }
    if (top < 0) return 0.0;
    if (a->l[top] >= ((int64_t)1 << 32)) return sign * INFINITY;
    int H = 32 * top;
    for (int b = 31; b >= 0; b--)
        if ((a->l[top] >> b) & 1) {
            H += b;
            break;
        }
    uint64_t mant = 0;
    if (H < 53) {
        for (int p = H; p >= 0; p--) mant = (mant << 1) | (uint64_t)acc_bit(a, p);
        return sign * ldexp((double)mant, -1074);
    }
    for (int p = H; p >= H - 52; p--) mant = (mant << 1) | (uint64_t)acc_bit(a, p);
    int rbit = acc_bit(a, H - 53);
    int sticky = 0;
    for (int p = H - 54; p >= 0 && !sticky; p--) sticky |= acc_bit(a, p);
    if (rbit && (sticky || (mant & 1))) {
        mant += 1;
        if (mant == (1ULL << 53)) {
            mant >>= 1;
            H += 1;
        }
    }
    return sign * ldexp((double)mant, H - 52 - 1074);
}

double oc_sum_exact(int64_t n, const double *x)
{
    oc_acc a;
    memset(&a, 0, sizeof(a));
    for (int64_t i = 0; i < n; i++) acc_add(&a, x[i]);
    return acc_round(&a);
}

double oc_dot_exact(int64_t n, const double *x, const double *y)
{
    oc_acc a;
    memset(&a, 0, sizeof(a));
    for (int64_t i = 0; i < n; i++) {
        double p = x[i] * y[i];
        acc_add(&a, p);
    }
    return acc_round(&a);
}

/* ======================================================================
 * a0.  Q1 hexahedral assembly (Section 2.2; conductivity tensor Eq. 2; block
 * operator of Eq. 3).
 *
 * Readings: the box [0,lx]x[0,ly]x[0,lz] is meshed by uniform trilinear
 * hexahedra; D = sigma_t I + (sigma_l - sigma_t) a_l a_l^T (sigma_n = sigma_t,
 * Eq. 2 with the third term dropped) is sampled at the 2x2x2 Gauss points;
 * the lumped mass of a node is the sum of |e|/8 over the elements around it
 * (row-sum lumping of the Q1 mass matrix on boxes).
 *
 * Evaluation order (fixed so that any implementation following it produces
 * the same bits): Gauss points q = gx + 2 gy + 4 gz in ascending q, each
 * element entry accumulated as K = K + w*c starting from 0.0, element entries
 * added into the global entry in ascending element index.
 * ====================================================================== */
static void q1_element(double hx, double hy, double hz, const double *fib_layer,
                       double sl, double st, double K[8][8])
{
    const double r = 1.0 / sqrt(3.0);
    const double g[2] = {(1.0 - r) * 0.5, (1.0 + r) * 0.5};
    const double ih[3] = {1.0 / hx, 1.0 / hy, 1.0 / hz};
    const double wq = ((hx * hy) * hz) * 0.125;
    const double dl = sl - st;
    for (int a = 0; a < 8; a++)
        for (int b = 0; b < 8; b++) K[a][b] = 0.0;
    for (int q = 0; q < 8; q++) {
        int gq[3] = {q & 1, (q >> 1) & 1, (q >> 2) & 1};
        double xi[3] = {g[gq[0]], g[gq[1]], g[gq[2]]};
        const double *al = fib_layer + 3 * gq[2];
        double D[3][3];
        for (int i = 0; i < 3; i++)
            for (int j = 0; j < 3; j++) {
                D[i][j] = dl * (al[i] * al[j]);
                if (i == j) D[i][j] = D[i][j] + st;
            }
        double G[8][3];
        for (int a = 0; a < 8; a++) {
            int ad[3] = {a & 1, (a >> 1) & 1, (a >> 2) & 1};
            double n[3], s[3];
            for (int d = 0; d < 3; d++) {
                n[d] = ad[d] ? xi[d] : 1.0 - xi[d];
                s[d] = ad[d] ? ih[d] : -ih[d];
            }
            G[a][0] = s[0] * (n[1] * n[2]);
            G[a][1] = s[1] * (n[0] * n[2]);
            G[a][2] = s[2] * (n[0] * n[1]);
        }
        for (int a = 0; a < 8; a++)
            for (int b = a; b < 8; b++) {
                double t0 = (D[0][0] * G[b][0] + D[0][1] * G[b][1]) + D[0][2] * G[b][2];
                double t1 = (D[1][0] * G[b][0] + D[1][1] * G[b][1]) + D[1][2] * G[b][2];
                double t2 = (D[2][0] * G[b][0] + D[2][1] * G[b][1]) + D[2][2] * G[b][2];
                double c = (G[a][0] * t0 + G[a][1] * t1) + G[a][2] * t2;
                K[a][b] = K[a][b] + wq * c;
            }
    }
    for (int a = 0; a < 8; a++)
        for (int b = 0; b < a; b++) K[a][b] = K[b][a];
}

/* 27-point node pattern (neighbours in ascending node index) */
static int pattern27(int nx, int ny, int nz, oc_csr *P)
{
    int NX = nx + 1, NY = ny + 1, NZ = nz + 1;
    int N = NX * NY * NZ;
    int64_t nnz = 0;
    for (int l = 0; l < NZ; l++)
        for (int j = 0; j < NY; j++)
            for (int i = 0; i < NX; i++) {
                int cx = 1 + (i > 0) + (i < NX - 1), cy = 1 + (j > 0) + (j < NY - 1),
                    cz = 1 + (l > 0) + (l < NZ - 1);
                nnz += cx * cy * cz;
            }
    if (csr_alloc(P, N, N, nnz)) return OC_ENOMEM;
    int64_t pos = 0;
    for (int l = 0; l < NZ; l++)
        for (int j = 0; j < NY; j++)
            for (int i = 0; i < NX; i++) {
                int k = i + NX * (j + NY * l);
                P->rp[k] = pos;
                for (int dz = -1; dz <= 1; dz++)
                    for (int dy = -1; dy <= 1; dy++)
                        for (int dx = -1; dx <= 1; dx++) {
                            int ii = i + dx, jj = j + dy, ll = l + dz;
                            if (ii < 0 || ii >= NX || jj < 0 || jj >= NY || ll < 0 || ll >= NZ)
                                continue;
                            P->ci[pos] = ii + NX * (jj + NY * ll);
                            P->v[pos] = 0.0;
                            pos++;
                        }
            }
    P->rp[N] = pos;
    return 0;
}

int oc_assemble(int nx, int ny, int nz, double lx, double ly, double lz,
                const double *fib, double sil, double sit, double sel, double set,
                double chi, double cm, double dt,
                oc_csr *Ki_out, oc_csr *Ke_out, double *M_out, oc_csr *A_out)
{
    if (nx < 1 || ny < 1 || nz < 1 || !(lx > 0) || !(ly > 0) || !(lz > 0) || !fib)
        return OC_EINVAL;
    int NX = nx + 1, NY = ny + 1;
    oc_csr Ki, Ke;
    memset(&Ki, 0, sizeof(Ki));
    memset(&Ke, 0, sizeof(Ke));
    if (pattern27(nx, ny, nz, &Ki) || pattern27(nx, ny, nz, &Ke)) {
        oc_csr_free(&Ki);
        oc_csr_free(&Ke);
        return OC_ENOMEM;
    }
    int N = Ki.nrows;
    double *M = (double *)calloc((size_t)N, sizeof(double));
    if (!M) {
        oc_csr_free(&Ki);
        oc_csr_free(&Ke);
        return OC_ENOMEM;
    }
    double hx = lx / nx, hy = ly / ny, hz = lz / nz;
    double vol8 = ((hx * hy) * hz) * 0.125;
    double Kie[8][8], Kee[8][8];
    for (int ez = 0; ez < nz; ez++)
        for (int ey = 0; ey < ny; ey++)
            for (int ex = 0; ex < nx; ex++) {
                const double *fl = fib + (size_t)ez * 6;
                q1_element(hx, hy, hz, fl, sil, sit, Kie);
                q1_element(hx, hy, hz, fl, sel, set, Kee);
                int node[8];
                for (int a = 0; a < 8; a++)
                    node[a] = (ex + (a & 1)) + NX * ((ey + ((a >> 1) & 1)) + NY * (ez + ((a >> 2) & 1)));
                for (int a = 0; a < 8; a++) {
                    M[node[a]] = M[node[a]] + vol8;
                    for (int b = 0; b < 8; b++) {
                        int64_t p = csr_find(&Ki, node[a], node[b]);
                        Ki.v[p] = Ki.v[p] + Kie[a][b];
                        Ke.v[p] = Ke.v[p] + Kee[a][b];
                    }
                }
            }
    if (A_out) {
        /* Eq. 3 with backward Euler on the diffusion: the coupled operator
         * [c M + Ki, Ki; Ki, Ki + Ke], c = chi*Cm/dt, unknowns interleaved. */
        double c = (chi * cm) / dt;
        oc_csr *A = A_out;
        if (csr_alloc(A, 2 * N, 2 * N, 4 * Ki.nnz)) {
            free(M);
            oc_csr_free(&Ki);
            oc_csr_free(&Ke);
            return OC_ENOMEM;
        }
        int64_t pos = 0;
        for (int p = 0; p < N; p++)
            for (int f = 0; f < 2; f++) {
                A->rp[2 * p + f] = pos;
                for (int64_t t = Ki.rp[p]; t < Ki.rp[p + 1]; t++) {
                    int q = Ki.ci[t];
                    double ki = Ki.v[t], ke = Ke.v[t];
                    double vv = ki, vu = ki, uv = ki, uu = ki + ke;
                    if (q == p) vv = c * M[p] + ki;
                    A->ci[pos] = 2 * q;
                    A->v[pos++] = (f == 0) ? vv : uv;
                    A->ci[pos] = 2 * q + 1;
                    A->v[pos++] = (f == 0) ? vu : uu;
                }
            }
        A->rp[2 * N] = pos;
    }
    if (M_out) memcpy(M_out, M, sizeof(double) * (size_t)N);
    free(M);
    if (Ki_out) *Ki_out = Ki;
    else oc_csr_free(&Ki);
    if (Ke_out) *Ke_out = Ke;
    else oc_csr_free(&Ke);
    return 0;
}

/* ======================================================================
 * Generic sparse helpers
 * ====================================================================== */
int oc_spmv(const oc_csr *A, const double *x, double *y)
{
#pragma omp parallel for schedule(static) if (A->nrows > 4096)
    for (int i = 0; i < A->nrows; i++) {
        double s = 0.0;
        for (int64_t t = A->rp[i]; t < A->rp[i + 1]; t++) s = s + A->v[t] * x[A->ci[t]];
        y[i] = s;
    }
    return 0;
}

/* stable transpose: the entries of each output row keep ascending order */
int oc_transpose(const oc_csr *A, oc_csr *T)
{
    if (csr_alloc(T, A->ncols, A->nrows, A->nnz)) return OC_ENOMEM;
    for (int64_t t = 0; t < A->nnz; t++) T->rp[A->ci[t] + 1]++;
    for (int j = 0; j < A->ncols; j++) T->rp[j + 1] += T->rp[j];
    int64_t *next = (int64_t *)malloc(sizeof(int64_t) * (size_t)(A->ncols + 1));
    if (!next) {
        oc_csr_free(T);
        return OC_ENOMEM;
    }
    memcpy(next, T->rp, sizeof(int64_t) * (size_t)(A->ncols + 1));
    for (int i = 0; i < A->nrows; i++)
        for (int64_t t = A->rp[i]; t < A->rp[i + 1]; t++) {
            int64_t p = next[A->ci[t]]++;
            T->ci[p] = i;
            T->v[p] = A->v[t];
        }
    free(next);
    return 0;
}

/* C = A B, row by row (Gustavson).  Every entry C(i,j) is accumulated as
 * acc = acc + A(i,k)*B(k,j) over the middle index k in ascending order,
 * starting from 0.0; the pattern of C is every (i,j) reached, even if the
 * value is zero.  Columns of each row are emitted in ascending order. */
int oc_spgemm(const oc_csr *A, const oc_csr *B, oc_csr *C)
{
    if (A->ncols != B->nrows) return OC_EINVAL;
    int n = A->nrows, m = B->ncols;
    int *mark = (int *)malloc(sizeof(int) * (size_t)(m > 0 ? m : 1));
    double *acc = (double *)calloc((size_t)(m > 0 ? m : 1), sizeof(double));
    int *cols = (int *)malloc(sizeof(int) * (size_t)(m > 0 ? m : 1));
    int64_t *rp = (int64_t *)calloc((size_t)n + 1, sizeof(int64_t));
    if (!mark || !acc || !cols || !rp) {
        free(mark); free(acc); free(cols); free(rp);
        return OC_ENOMEM;
    }
    for (int j = 0; j < m; j++) mark[j] = -1;
    /* symbolic */
    for (int i = 0; i < n; i++) {
        int cnt = 0;
        for (int64_t t = A->rp[i]; t < A->rp[i + 1]; t++) {
            int k = A->ci[t];
            for (int64_t s = B->rp[k]; s < B->rp[k + 1]; s++) {
                int j = B->ci[s];
                if (mark[j] != i) {
                    mark[j] = i;
                    cnt++;
                }
            }
        }
        rp[i + 1] = rp[i] + cnt;
    }
    if (csr_alloc(C, n, m, rp[n])) {
        free(mark); free(acc); free(cols); free(rp);
        return OC_ENOMEM;
    }
    memcpy(C->rp, rp, sizeof(int64_t) * ((size_t)n + 1));
    for (int j = 0; j < m; j++) mark[j] = -1;
    for (int i = 0; i < n; i++) {
        int cnt = 0;
        for (int64_t t = A->rp[i]; t < A->rp[i + 1]; t++) {
            int k = A->ci[t];
            double a = A->v[t];
            for (int64_t s = B->rp[k]; s < B->rp[k + 1]; s++) {
                int j = B->ci[s];
                if (mark[j] != i) {
                    mark[j] = i;
                    acc[j] = 0.0;
                    cols[cnt++] = j;
                }
                acc[j] = acc[j] + a * B->v[s];
            }
        }
        /* insertion sort of the (short) column list */
        for (int x = 1; x < cnt; x++) {
            int key = cols[x], y = x - 1;
            while (y >= 0 && cols[y] > key) {
                cols[y + 1] = cols[y];
                y--;
            }
            cols[y + 1] = key;
        }
        for (int x = 0; x < cnt; x++) {
            C->ci[C->rp[i] + x] = cols[x];
            C->v[C->rp[i] + x] = acc[cols[x]];
        }
    }
    free(mark); free(acc); free(cols); free(rp);
    return 0;
}

/* ======================================================================
 * a1.  Strength graph (Section 4: w_ij = a_ij / sqrt(a_ii a_jj); edges with
 * weight below the threshold are cut).
 *
 * Readings: for the coupled system the graph is over nodes and uses the
 * elliptic (u_e,u_e) entry of every 2x2 node block -- on the fine level that
 * entry is exactly the paper's elliptic matrix A_i + A_e, for which the
 * threshold 0.06 was tuned (Section 6.1).  Magnitudes are used (stiffness
 * off-diagonals are mostly negative), and the numerator is the mean of the
 * two transposed magnitudes so that the graph is symmetric even when a
 * Galerkin operator is symmetric only up to rounding.  "Cut if less than the
 * threshold" keeps w >= theta.
 * ====================================================================== */
int oc_strength(const oc_csr *A, double theta, oc_csr *S)
{
    if (A->nrows != A->ncols || (A->nrows & 1)) return OC_EINVAL;
    int N = A->nrows / 2;
    double *du = (double *)malloc(sizeof(double) * (size_t)(N > 0 ? N : 1));
    if (!du) return OC_ENOMEM;
    for (int p = 0; p < N; p++) {
        int64_t t = csr_find(A, 2 * p + 1, 2 * p + 1);
        du[p] = t >= 0 ? A->v[t] : 0.0;
    }
    /* two passes: count, then fill */
    for (int pass = 0; pass < 2; pass++) {
        int64_t pos = 0;
        for (int p = 0; p < N; p++) {
            if (pass == 1) S->rp[p] = pos;
            int r = 2 * p + 1;
            for (int64_t t = A->rp[r]; t < A->rp[r + 1]; t++) {
                int c = A->ci[t];
                if (!(c & 1)) continue;
                int q = c / 2;
                if (q == p) continue;
                int64_t tt = csr_find(A, 2 * q + 1, 2 * p + 1);
                double apq = fabs(A->v[t]);
                double aqp = tt >= 0 ? fabs(A->v[tt]) : 0.0;
                double num = 0.5 * (apq + aqp);
                double den = sqrt(du[p] * du[q]);
                if (!(den > 0.0)) continue;
                double w = num / den;
                if (w >= theta) {
                    if (pass == 1) {
                        S->ci[pos] = q;
                        S->v[pos] = w;
                    }
                    pos++;
                }
            }
        }
        if (pass == 0) {
            if (csr_alloc(S, N, N, pos)) {
                free(du);
                return OC_ENOMEM;
            }
        } else {
            S->rp[N] = pos;
        }
    }
    free(du);
    return 0;
}

/* Squared strength graph (Appendix A, square_graph 1: the MIS of the first
 * level runs on the square of the filtered graph, i.e. aggressive
 * coarsening).  Reading: with W the filtered weights (symmetric, zero
 * diagonal) and Wh = I + W, the squared graph is Wh*Wh without its diagonal;
 * its entries (sums over the middle node in ascending order) are the weights
 * the cluster rule compares.  Direct strong neighbours therefore carry
 * 2 w_pq plus their two-step paths and outrank nodes two steps away. */
int oc_square_graph(const oc_csr *S, oc_csr *S2)
{
    int N = S->nrows;
    oc_csr Wh, Q;
    memset(&Wh, 0, sizeof(Wh));
    memset(&Q, 0, sizeof(Q));
    if (csr_alloc(&Wh, N, N, S->nnz + N)) return OC_ENOMEM;
    int64_t pos = 0;
    for (int p = 0; p < N; p++) {
        Wh.rp[p] = pos;
        int diag_done = 0;
        for (int64_t t = S->rp[p]; t < S->rp[p + 1]; t++) {
            if (!diag_done && S->ci[t] > p) {
                Wh.ci[pos] = p;
                Wh.v[pos++] = 1.0;
                diag_done = 1;
            }
            Wh.ci[pos] = S->ci[t];
            Wh.v[pos++] = S->v[t];
        }
        if (!diag_done) {
            Wh.ci[pos] = p;
            Wh.v[pos++] = 1.0;
        }
    }
    Wh.rp[N] = pos;
    int rc = oc_spgemm(&Wh, &Wh, &Q);
    oc_csr_free(&Wh);
    if (rc) return rc;
    if (csr_alloc(S2, N, N, Q.nnz - N)) {
        oc_csr_free(&Q);
        return OC_ENOMEM;
    }
    pos = 0;
    for (int p = 0; p < N; p++) {
        S2->rp[p] = pos;
        for (int64_t t = Q.rp[p]; t < Q.rp[p + 1]; t++) {
            if (Q.ci[t] == p) continue;
            S2->ci[pos] = Q.ci[t];
            S2->v[pos++] = Q.v[t];
        }
    }
    S2->rp[N] = pos;
    S2->nnz = pos;
    oc_csr_free(&Q);
    return 0;
}

/* ======================================================================
 * a2.  Maximal independent set (Section 4: "a greedy MIS or the parallel
 * implementation (Luby)").  Reading: node k has priority (h(k), -k) with
 * h(k) = SplitMix64 finalizer of (k XOR key); the set is the one the
 * sequential greedy algorithm builds when it visits nodes in decreasing
 * priority (the lexicographically-first MIS of that order).  Luby's rounds
 * with the same fixed priorities return exactly this set.
 * ====================================================================== */
uint64_t oc_mix64(uint64_t z)
{
    z = (z ^ (z >> 30)) * 0xbf58476d1ce4e5b9ULL;
    z = (z ^ (z >> 27)) * 0x94d049bb133111ebULL;
    return z ^ (z >> 31);
}

uint64_t oc_level_key(uint64_t seed, int level, int stream)
{
    return oc_mix64(seed + 0x9E3779B97F4A7C15ULL * (uint64_t)(2 * level + stream + 1));
}

typedef struct {
    uint64_t h;
    int k;
} prio_t;

static int prio_cmp(const void *a, const void *b)
{
    const prio_t *x = (const prio_t *)a, *y = (const prio_t *)b;
    if (x->h != y->h) return x->h > y->h ? -1 : 1; /* larger hash first */
    return x->k < y->k ? -1 : (x->k > y->k); /* then smaller index */
}

int oc_mis(const oc_csr *S, uint64_t key, unsigned char *in_set)
{
    int N = S->nrows;
    prio_t *order = (prio_t *)malloc(sizeof(prio_t) * (size_t)(N > 0 ? N : 1));
    if (!order) return OC_ENOMEM;
    for (int k = 0; k < N; k++) {
        order[k].h = oc_mix64((uint64_t)k ^ key);
        order[k].k = k;
        in_set[k] = 0;
    }
    qsort(order, (size_t)N, sizeof(prio_t), prio_cmp);
    for (int t = 0; t < N; t++) {
        int k = order[t].k, ok = 1;
        for (int64_t s = S->rp[k]; s < S->rp[k + 1]; s++)
            if (in_set[S->ci[s]]) {
                ok = 0;
                break;
            }
        in_set[k] = (unsigned char)ok;
    }
    free(order);
    return 0;
}

/* ======================================================================
 * a3.  Aggregation (Section 4: i not in S joins C_j, j in S, with the largest
 * w_ij).  Reading: ties go to the smaller root index; roots are numbered in
 * ascending node index.  Every i outside S has a strong neighbour in S
 * because S is maximal, so the rule assigns every node.
 * ====================================================================== */
int oc_aggregate(const oc_csr *S, const unsigned char *in_set, int *agg, int *n_agg)
{
    int N = S->nrows, na = 0;
    for (int k = 0; k < N; k++) agg[k] = in_set[k] ? na++ : -1;
    for (int k = 0; k < N; k++) {
        if (in_set[k]) continue;
        int best = -1;
        double bw = -1.0;
        for (int64_t s = S->rp[k]; s < S->rp[k + 1]; s++) {
            int q = S->ci[s];
            if (in_set[q] && S->v[s] > bw) {
                bw = S->v[s];
                best = q;
            }
        }
        if (best < 0) return OC_EINVAL; /* not maximal: cannot happen for a MIS */
        agg[k] = agg[best];
    }
    *n_agg = na;
    return 0;
}

/* ======================================================================
 * a4.  Tentative prolongator (Section 4: P_ij = |C_j|^{-1/2} if i in C_j).
 * Reading: for the 2-unknown system the near-null space is one vector per
 * field, so every aggregate gives one coarse unknown per field:
 * Pt(2k+f, 2J+f) = B(2k+f) / ||B restricted to field f of C_J||, and the
 * coarse near-null coefficients are Bc(2J+f) = that norm.  On the finest
 * level B = 1 and this is exactly |C_J|^{-1/2}; on coarser levels it keeps
 * the constant vector in the range of the prolongators.  Sums run over the
 * members of C_J in ascending node index.
 * ====================================================================== */
int oc_ptent(int N, const int *agg, int n_agg, const double *B, oc_csr *Pt, double *Bc)
{
    for (int J = 0; J < 2 * n_agg; J++) Bc[J] = 0.0;
    for (int k = 0; k < N; k++)
        for (int f = 0; f < 2; f++) {
            double b = B[2 * k + f];
            Bc[2 * agg[k] + f] = Bc[2 * agg[k] + f] + b * b;
        }
    for (int J = 0; J < 2 * n_agg; J++) Bc[J] = sqrt(Bc[J]);
    if (csr_alloc(Pt, 2 * N, 2 * n_agg, 2 * (int64_t)N)) return OC_ENOMEM;
    for (int k = 0; k < N; k++)
        for (int f = 0; f < 2; f++) {
            int i = 2 * k + f;
            Pt->rp[i] = i;
            Pt->ci[i] = 2 * agg[k] + f;
            Pt->v[i] = B[i] / Bc[2 * agg[k] + f];
        }
    Pt->rp[2 * N] = 2 * (int64_t)N;
    return 0;
}

/* ======================================================================
 * a5.  Largest eigenvalue of D^{-1}A (Appendix A: Chebyshev bounds from a
 * 10-step CG eigenvalue estimate with the Jacobi preconditioner).
 * CG on A x = b, x0 = 0, preconditioned by D = diag(A); the Lanczos
 * tridiagonal built from the CG coefficients (T_00 = 1/alpha_0,
 * T_jj = 1/alpha_j + beta_{j-1}/alpha_{j-1}, T_j,j+1 = sqrt(beta_j)/alpha_j)
 * has the Ritz values of D^{-1}A; the largest is found by Sturm-sequence
 * bisection to the last bit.  Reading: b_i uniform in [-1,1) from a
 * counter-based hash of (key, i); dot products are correctly rounded.
 * ====================================================================== */
static int sturm_count_below(int m, const double *d, const double *e, double x)
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

double oc_tridiag_max_eig(int m, const double *d, const double *e)
{
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
    return hi;
}

int oc_lambda_max(const oc_csr *A, int steps, uint64_t key, double *lam, int *steps_done)
{
    int n = A->nrows;
    if (steps < 1 || steps > 64 || n < 1) return OC_EINVAL;
    double *D = (double *)malloc(sizeof(double) * (size_t)n);
    double *r = (double *)malloc(sizeof(double) * (size_t)n);
    double *z = (double *)malloc(sizeof(double) * (size_t)n);
    double *p = (double *)malloc(sizeof(double) * (size_t)n);
    double *q = (double *)malloc(sizeof(double) * (size_t)n);
    double *al = (double *)malloc(sizeof(double) * (size_t)steps);
    double *be = (double *)malloc(sizeof(double) * (size_t)steps);
    if (!D || !r || !z || !p || !q || !al || !be) {
        free(D); free(r); free(z); free(p); free(q); free(al); free(be);
        return OC_ENOMEM;
    }
    for (int i = 0; i < n; i++) {
        int64_t t = csr_find(A, i, i);
        D[i] = t >= 0 ? A->v[t] : 0.0;
        uint64_t h = oc_mix64(key ^ (uint64_t)i);
        double u = (double)(h >> 11) * (1.0 / 9007199254740992.0);
        r[i] = 2.0 * u - 1.0;
        z[i] = r[i] / D[i];
        p[i] = z[i];
    }
    double rz = oc_dot_exact(n, r, z);
    int m = 0;
    for (int j = 0; j < steps; j++) {
        oc_spmv(A, p, q);
        double pq = oc_dot_exact(n, p, q);
        if (!(pq > 0.0) || !(rz > 0.0)) break;
        double alpha = rz / pq;
        for (int i = 0; i < n; i++) {
            r[i] = r[i] - alpha * q[i];
            z[i] = r[i] / D[i];
        }
        double rz1 = oc_dot_exact(n, r, z);
        double beta = rz1 / rz;
        al[j] = alpha;
        be[j] = beta;
        m = j + 1;
        if (!(rz1 > 0.0)) break;
        for (int i = 0; i < n; i++) p[i] = z[i] + beta * p[i];
        rz = rz1;
    }
    int ret = 0;
    if (m == 0) {
        ret = OC_EBREAK;
    } else {
        double d[64], e[64];
        for (int j = 0; j < m; j++) {
            d[j] = 1.0 / al[j];
            if (j > 0) d[j] = d[j] + be[j - 1] / al[j - 1];
            if (j < m - 1) e[j] = sqrt(be[j]) / al[j];
        }
        *lam = oc_tridiag_max_eig(m, d, e);
    }
    if (steps_done) *steps_done = m;
    free(D); free(r); free(z); free(p); free(q); free(al); free(be);
    return ret;
}

/* ======================================================================
 * a6.  Smoothed prolongator (Appendix A, one smoothing step of the
 * aggregates' prolongator): P = Pt - omega D^{-1} (A Pt).  Reading:
 * omega = 4/(3 lambda), D = diag(A) (point Jacobi), no dropping; entry by
 * entry P(i,j) = Pt(i,j) - s_i * (A Pt)(i,j) with s_i = omega / A(i,i).
 * ====================================================================== */
int oc_smooth_p(const oc_csr *A, const oc_csr *Pt, double omega, oc_csr *P)
{
    oc_csr AP;
    memset(&AP, 0, sizeof(AP));
    int rc = oc_spgemm(A, Pt, &AP);
    if (rc) return rc;
    for (int i = 0; i < AP.nrows; i++) {
        int64_t td = csr_find(A, i, i);
        double s = omega / A->v[td];
        for (int64_t t = AP.rp[i]; t < AP.rp[i + 1]; t++) {
            int64_t tp = csr_find(Pt, i, AP.ci[t]);
            double pt = tp >= 0 ? Pt->v[tp] : 0.0;
            AP.v[t] = pt - s * AP.v[t];
        }
    }
    *P = AP;
    return 0;
}

/* ======================================================================
 * Hierarchy: Algorithm 1 ("AMG setup phase"), with the GAMG options of
 * Appendix A (agg_nsmooths 1, coarse_eq_limit 100, Chebyshev(2)-Jacobi with
 * bounds [0.05, 1.05] x the 10-step CG estimate).  Reading for the coarsest
 * level (the paper only says "direct solver", Algorithm 2): a dense Cholesky
 * factor of A_c + s zz^T/(z^T z), s = max diag(A_c), where z is the
 * null vector (0,1) carried through the levels; right-hand sides are
 * projected orthogonal to z first, so the result is the minimum-norm
 * solution orthogonal to z.
 * ====================================================================== */
#define OC_MAXLEV 32
struct oc_hier {
    int nlev;
    oc_csr A[OC_MAXLEV], P[OC_MAXLEV], R[OC_MAXLEV], Pt[OC_MAXLEV];
    int *agg[OC_MAXLEV];
    unsigned char *mis[OC_MAXLEV];
    int nagg[OC_MAXLEV];
    double lam[OC_MAXLEV];
    double *diag[OC_MAXLEV];
    double *B[OC_MAXLEV];    /* near-null coefficients per field */
    double *zhat[OC_MAXLEV]; /* null vector: B on the u-field, 0 on v */
    int cheb_degree;
    double eig_lo, eig_hi;
    int nc;
    double *L;  /* dense Cholesky factor, nc x nc, row-major lower */
};

void oc_hier_free(oc_hier *h)
{
    if (!h) return;
    for (int l = 0; l < OC_MAXLEV; l++) {
        oc_csr_free(&h->A[l]);
        oc_csr_free(&h->P[l]);
        oc_csr_free(&h->R[l]);
        oc_csr_free(&h->Pt[l]);
        free(h->agg[l]);
        free(h->mis[l]);
        free(h->diag[l]);
        free(h->B[l]);
        free(h->zhat[l]);
    }
    free(h->L);
    free(h);
}

static int csr_copy(const oc_csr *a, oc_csr *b)
{
    if (csr_alloc(b, a->nrows, a->ncols, a->nnz)) return OC_ENOMEM;
    memcpy(b->rp, a->rp, sizeof(int64_t) * ((size_t)a->nrows + 1));
    memcpy(b->ci, a->ci, sizeof(int) * (size_t)a->nnz);
    memcpy(b->v, a->v, sizeof(double) * (size_t)a->nnz);
    return 0;
}

static int dense_cholesky(int n, double *a)
{
    for (int j = 0; j < n; j++) {
        double s = a[(size_t)j * n + j];
        for (int k = 0; k < j; k++) s = s - a[(size_t)j * n + k] * a[(size_t)j * n + k];
        if (!(s > 0.0)) return OC_EBREAK;
        double d = sqrt(s);
        a[(size_t)j * n + j] = d;
        for (int i = j + 1; i < n; i++) {
            double t = a[(size_t)i * n + j];
            for (int k = 0; k < j; k++) t = t - a[(size_t)i * n + k] * a[(size_t)j * n + k];
            a[(size_t)i * n + j] = t / d;
        }
        for (int i = 0; i < j; i++) a[(size_t)i * n + j] = 0.0;
    }
    return 0;
}

int oc_setup(const oc_csr *A0, const oc_amg_opts *o, oc_hier **out)
{
    if (!A0 || !o || A0->nrows != A0->ncols || (A0->nrows & 1) || A0->nrows < 2) return OC_EINVAL;
    oc_hier *h = (oc_hier *)calloc(1, sizeof(oc_hier));
    if (!h) return OC_ENOMEM;
    h->cheb_degree = o->cheb_degree;
    h->eig_lo = o->eig_lo;
    h->eig_hi = o->eig_hi;
    int rc = csr_copy(A0, &h->A[0]);
    if (rc) goto fail;
    int n0 = A0->nrows;
    h->B[0] = (double *)malloc(sizeof(double) * (size_t)n0);
    if (!h->B[0]) { rc = OC_ENOMEM; goto fail; }
    for (int i = 0; i < n0; i++) h->B[0][i] = 1.0;
    int maxlev = o->max_levels < OC_MAXLEV ? o->max_levels : OC_MAXLEV;
    int l = 0;
    for (;;) {
        oc_csr *A = &h->A[l];
        int n = A->nrows, N = n / 2;
        h->diag[l] = (double *)malloc(sizeof(double) * (size_t)n);
        h->zhat[l] = (double *)malloc(sizeof(double) * (size_t)n);
        if (!h->diag[l] || !h->zhat[l]) { rc = OC_ENOMEM; goto fail; }
        for (int i = 0; i < n; i++) {
            int64_t t = csr_find(A, i, i);
            h->diag[l][i] = t >= 0 ? A->v[t] : 0.0;
            h->zhat[l][i] = (i & 1) ? h->B[l][i] : 0.0;
        }
        if (n <= o->coarse_eq_limit || l == maxlev - 1) break;
        oc_csr S;
        memset(&S, 0, sizeof(S));
        if ((rc = oc_strength(A, o->theta, &S))) goto fail;
        if (l < o->square_levels) {
            oc_csr S2;
            memset(&S2, 0, sizeof(S2));
            rc = oc_square_graph(&S, &S2);
            oc_csr_free(&S);
            if (rc) goto fail;
            S = S2;
        }
        h->mis[l] = (unsigned char *)malloc((size_t)N);
        h->agg[l] = (int *)malloc(sizeof(int) * (size_t)N);
        if (!h->mis[l] || !h->agg[l]) { oc_csr_free(&S); rc = OC_ENOMEM; goto fail; }
        rc = oc_mis(&S, oc_level_key(o->seed, l, 0), h->mis[l]);
        if (!rc) rc = oc_aggregate(&S, h->mis[l], h->agg[l], &h->nagg[l]);
        oc_csr_free(&S);
        if (rc) goto fail;
        if (2 * h->nagg[l] >= n) { /* no coarsening: this level is the coarsest */
            free(h->mis[l]); h->mis[l] = NULL;
            free(h->agg[l]); h->agg[l] = NULL;
            h->nagg[l] = 0;
            break;
        }
        int steps_done = 0;
        if ((rc = oc_lambda_max(A, o->esteig_steps, oc_level_key(o->seed, l, 1), &h->lam[l], &steps_done)))
            goto fail;
        h->B[l + 1] = (double *)malloc(sizeof(double) * (size_t)(2 * h->nagg[l]));
        if (!h->B[l + 1]) { rc = OC_ENOMEM; goto fail; }
        if ((rc = oc_ptent(N, h->agg[l], h->nagg[l], h->B[l], &h->Pt[l], h->B[l + 1]))) goto fail;
        double omega = 4.0 / (3.0 * h->lam[l]);
        if ((rc = oc_smooth_p(A, &h->Pt[l], omega, &h->P[l]))) goto fail;
        if ((rc = oc_transpose(&h->P[l], &h->R[l]))) goto fail;
        oc_csr AP;
        memset(&AP, 0, sizeof(AP));
        if ((rc = oc_spgemm(A, &h->P[l], &AP))) goto fail;
        rc = oc_spgemm(&h->R[l], &AP, &h->A[l + 1]);
        oc_csr_free(&AP);
        if (rc) goto fail;
        l++;
    }
    h->nlev = l + 1;
    {
        const oc_csr *Ac = &h->A[l];
        int nc = Ac->nrows;
        if (nc > 20000) { rc = OC_ENOMEM; goto fail; }
        h->nc = nc;
        h->L = (double *)calloc((size_t)nc * nc, sizeof(double));
        if (!h->L) { rc = OC_ENOMEM; goto fail; }
        double smax = 0.0, zz = 0.0;
        const double *z = h->zhat[l];
        for (int i = 0; i < nc; i++) {
            for (int64_t t = Ac->rp[i]; t < Ac->rp[i + 1]; t++) h->L[(size_t)i * nc + Ac->ci[t]] = Ac->v[t];
            if (h->diag[l][i] > smax) smax = h->diag[l][i];
            zz = zz + z[i] * z[i];
        }
        for (int i = 0; i < nc; i++)
            for (int j = 0; j < nc; j++)
                h->L[(size_t)i * nc + j] = h->L[(size_t)i * nc + j] + (smax * z[i]) * z[j] / zz;
        if ((rc = dense_cholesky(nc, h->L))) goto fail;
    }
    *out = h;
    return 0;
fail:
    oc_hier_free(h);
    return rc;
}

int oc_hier_nlevels(const oc_hier *h) { return h->nlev; }
const oc_csr *oc_hier_A(const oc_hier *h, int l) { return &h->A[l]; }
const oc_csr *oc_hier_P(const oc_hier *h, int l) { return l < h->nlev - 1 ? &h->P[l] : NULL; }
const oc_csr *oc_hier_Pt(const oc_hier *h, int l) { return l < h->nlev - 1 ? &h->Pt[l] : NULL; }
const int *oc_hier_agg(const oc_hier *h, int l) { return h->agg[l]; }
const unsigned char *oc_hier_mis(const oc_hier *h, int l) { return h->mis[l]; }
int oc_hier_nagg(const oc_hier *h, int l) { return h->nagg[l]; }
double oc_hier_lambda(const oc_hier *h, int l) { return h->lam[l]; }
const double *oc_hier_null(const oc_hier *h, int l) { return h->zhat[l]; }

/* ======================================================================
 * a10.  Smoother (Section 4, Richardson form, specialised by Appendix A to
 * two Chebyshev iterations on the Jacobi-preconditioned operator over
 * [lo, hi]).  Three-term Chebyshev iteration (Saad, Iterative Methods for
 * Sparse Linear Systems, 2nd ed., Algorithm 12.1), preconditioned by D:
 *   theta = (hi+lo)/2, delta = (hi-lo)/2, sigma = theta/delta, rho0 = 1/sigma
 *   r0 = f - A x0, d0 = D^{-1} r0 / theta
 *   x_{k+1} = x_k + d_k, r_{k+1} = r_k - A d_k,
 *   rho_{k+1} = 1/(2 sigma - rho_k),
 *   d_{k+1} = rho_{k+1} rho_k d_k + (2 rho_{k+1}/delta) D^{-1} r_{k+1}.
 * ====================================================================== */
int oc_chebyshev(const oc_csr *A, const double *f, double *x, int x_is_zero,
                 int degree, double lo, double hi)
{
    int n = A->nrows;
    double *r = (double *)malloc(sizeof(double) * (size_t)n);
    double *d = (double *)malloc(sizeof(double) * (size_t)n);
    double *q = (double *)malloc(sizeof(double) * (size_t)n);
    double *D = (double *)malloc(sizeof(double) * (size_t)n);
    if (!r || !d || !q || !D) {
        free(r); free(d); free(q); free(D);
        return OC_ENOMEM;
    }
#pragma omp parallel for schedule(static) if (n > 4096)
    for (int i = 0; i < n; i++) {
        int64_t t = csr_find(A, i, i);
        D[i] = A->v[t];
    }
    double theta = 0.5 * (hi + lo), delta = 0.5 * (hi - lo);
    double sigma = theta / delta, rho = 1.0 / sigma;
    if (x_is_zero) {
#pragma omp parallel for schedule(static) if (n > 4096)
        for (int i = 0; i < n; i++) {
            x[i] = 0.0;
            r[i] = f[i];
        }
    } else {
        oc_spmv(A, x, q);
#pragma omp parallel for schedule(static) if (n > 4096)
        for (int i = 0; i < n; i++) r[i] = f[i] - q[i];
    }
#pragma omp parallel for schedule(static) if (n > 4096)
    for (int i = 0; i < n; i++) d[i] = r[i] / D[i] / theta;
    for (int k = 1; k <= degree; k++) {
#pragma omp parallel for schedule(static) if (n > 4096)
        for (int i = 0; i < n; i++) x[i] = x[i] + d[i];
        if (k == degree) break;
        oc_spmv(A, d, q);
        double rho1 = 1.0 / (2.0 * sigma - rho);
#pragma omp parallel for schedule(static) if (n > 4096)
        for (int i = 0; i < n; i++) {
            r[i] = r[i] - q[i];
            d[i] = rho1 * rho * d[i] + (2.0 * rho1 / delta) * (r[i] / D[i]);
        }
        rho = rho1;
    }
    free(r); free(d); free(q); free(D);
    return 0;
}

int oc_coarse_solve(const oc_hier *h, const double *r, double *x)
{
    int nc = h->nc, l = h->nlev - 1;
    const double *z = h->zhat[l];
    const double *L = h->L;
    double zz = 0.0, zr = 0.0;
    for (int i = 0; i < nc; i++) {
        zz = zz + z[i] * z[i];
        zr = zr + z[i] * r[i];
    }
    double a = zz > 0.0 ? zr / zz : 0.0;
    for (int i = 0; i < nc; i++) x[i] = r[i] - a * z[i];
    for (int i = 0; i < nc; i++) { /* L y = b */
        double s = x[i];
        for (int k = 0; k < i; k++) s = s - L[(size_t)i * nc + k] * x[k];
        x[i] = s / L[(size_t)i * nc + i];
    }
    for (int i = nc - 1; i >= 0; i--) { /* L^T x = y */
        double s = x[i];
        for (int k = i + 1; k < nc; k++) s = s - L[(size_t)k * nc + i] * x[k];
        x[i] = s / L[(size_t)i * nc + i];
    }
    return 0;
}

/* Algorithm 2 (MGV), mu1 = mu2 = one degree-2 Chebyshev sweep, u^k = 0 on entry. */
static int vcycle_level(const oc_hier *h, int l, const double *f, double *u)
{
    if (l == h->nlev - 1) return oc_coarse_solve(h, f, u);
    const oc_csr *A = &h->A[l];
    int n = A->nrows, nc = h->A[l + 1].nrows;
    double lo = h->eig_lo * h->lam[l], hi = h->eig_hi * h->lam[l];
    double *r = (double *)malloc(sizeof(double) * (size_t)n);
    double *rc = (double *)malloc(sizeof(double) * (size_t)nc);
    double *ec = (double *)malloc(sizeof(double) * (size_t)nc);
    double *e = (double *)malloc(sizeof(double) * (size_t)n);
    if (!r || !rc || !ec || !e) {
        free(r); free(rc); free(ec); free(e);
        return OC_ENOMEM;
    }
    oc_chebyshev(A, f, u, 1, h->cheb_degree, lo, hi);         /* pre-smoothing */
    oc_spmv(A, u, r);
#pragma omp parallel for schedule(static) if (n > 4096)
    for (int i = 0; i < n; i++) r[i] = f[i] - r[i];            /* r = f - A u */
    oc_spmv(&h->R[l], r, rc);                                  /* r_c = R r  */
    int rc_ = vcycle_level(h, l + 1, rc, ec);                  /* recursion  */
    oc_spmv(&h->P[l], ec, e);                                  /* e = P e_c  */
#pragma omp parallel for schedule(static) if (n > 4096)
    for (int i = 0; i < n; i++) u[i] = u[i] + e[i];            /* correction */
    oc_chebyshev(A, f, u, 0, h->cheb_degree, lo, hi);          /* post-smoothing */
    free(r); free(rc); free(ec); free(e);
    return rc_;
}

int oc_vcycle(const oc_hier *h, const double *r, double *z)
{
    return vcycle_level(h, 0, r, z);
}

/* ======================================================================
 * a11.  Projected PCG (Section 2.2: PCG for the symmetric positive
 * semi-definite system; Algorithm 2 as preconditioner).  Readings: the
 * right-hand side and every preconditioned residual are projected
 * orthogonal to the null vector (0,1) (Euclidean mean of u_e removed); the
 * stopping test is the recurrence residual ||r||_2 <= rtol ||f||_2; the
 * returned x has mean-zero u_e.
 * ====================================================================== */
static void project_u(int n, double *x)
{
    int N = n / 2;
    double s = 0.0;
    for (int k = 0; k < N; k++) s = s + x[2 * k + 1];
    double m = s / N;
    for (int k = 0; k < N; k++) x[2 * k + 1] = x[2 * k + 1] - m;
}

static double dot(int n, const double *a, const double *b)
{
    double s = 0.0;
    for (int i = 0; i < n; i++) s = s + a[i] * b[i];
    return s;
}

int oc_pcg(const oc_hier *h, const double *f_in, double *x, int warm, double rtol,
           int max_it, int *iters, double *rel_res, double *true_rel_res)
{
    const oc_csr *A = &h->A[0];
    int n = A->nrows;
    double *f = (double *)malloc(sizeof(double) * (size_t)n);
    double *r = (double *)malloc(sizeof(double) * (size_t)n);
    double *z = (double *)malloc(sizeof(double) * (size_t)n);
    double *p = (double *)malloc(sizeof(double) * (size_t)n);
    double *q = (double *)malloc(sizeof(double) * (size_t)n);
    if (!f || !r || !z || !p || !q) {
        free(f); free(r); free(z); free(p); free(q);
        return OC_ENOMEM;
    }
    memcpy(f, f_in, sizeof(double) * (size_t)n);
    project_u(n, f);
    if (!warm)
        for (int i = 0; i < n; i++) x[i] = 0.0;
    double nf = sqrt(dot(n, f, f));
    int it = 0, ret = 0;
    double rr = 0.0;
    if (nf == 0.0) {
        for (int i = 0; i < n; i++) x[i] = 0.0;
    } else {
        oc_spmv(A, x, q);
#pragma omp parallel for schedule(static) if (n > 4096)
        for (int i = 0; i < n; i++) r[i] = f[i] - q[i];
        rr = sqrt(dot(n, r, r));
        if (rr > rtol * nf) {
            oc_vcycle(h, r, z);
            project_u(n, z);
            memcpy(p, z, sizeof(double) * (size_t)n);
            double rz = dot(n, r, z);
            ret = OC_ENOTCONV;
            while (it < max_it) {
                oc_spmv(A, p, q);
                double pq = dot(n, p, q);
                if (!(pq > 0.0)) {
                    ret = OC_EBREAK;
                    break;
                }
                double alpha = rz / pq;
#pragma omp parallel for schedule(static) if (n > 4096)
                for (int i = 0; i < n; i++) {
                    x[i] = x[i] + alpha * p[i];
                    r[i] = r[i] - alpha * q[i];
                }
                it++;
                rr = sqrt(dot(n, r, r));
                if (rr <= rtol * nf) {
                    ret = 0;
                    break;
                }
                oc_vcycle(h, r, z);
                project_u(n, z);
                double rz1 = dot(n, r, z);
                double beta = rz1 / rz;
#pragma omp parallel for schedule(static) if (n > 4096)
                for (int i = 0; i < n; i++) p[i] = z[i] + beta * p[i];
                rz = rz1;
            }
        }
    }
    project_u(n, x);
    if (iters) *iters = it;
    if (rel_res) *rel_res = nf > 0.0 ? rr / nf : 0.0;
    if (true_rel_res) {
        oc_spmv(A, x, q);
        for (int i = 0; i < n; i++) q[i] = f[i] - q[i];
        *true_rel_res = nf > 0.0 ? sqrt(dot(n, q, q)) / nf : 0.0;
    }
    free(f); free(r); free(z); free(p); free(q);
    return ret;
}

/* ======================================================================
 * a12.  One semi-implicit time step (Section 2.2, Eqs. 4-7 in coupled form).
 * The gating variable is updated implicitly (Eq. 4, sign read as
 * w^{n+1} - dt R(v^n, w^{n+1}) = w^n), the ionic current is explicit, the
 * diffusion implicit: [cM+Ki, Ki; Ki, Ki+Ke][v;u_e]^{n+1} =
 * [M (c v^n + I_app - chi I_ion(v^n, w^{n+1})); 0], c = chi Cm/dt.
 * Membrane model (not in the paper, which uses TP06): Rogers-McCulloch,
 *   I_ion = G v (1 - v/vth)(1 - v/vp) + eta1 v w,  dw/dt = eta2 (v/vp - eta3 w).
 * ====================================================================== */
int oc_bd_step(const oc_hier *h, const double *M, int N, double chi, double cm,
               double dt, const oc_rm_params *rm, const double *Iapp,
               double *v, double *ue, double *w, double rtol, int max_it, int *iters)
{
    int n = 2 * N;
    if (N < 1 || h->A[0].nrows != n) return OC_EINVAL;
    double *f = (double *)malloc(sizeof(double) * (size_t)n);
    double *x = (double *)malloc(sizeof(double) * (size_t)n);
    if (!f || !x) {
        free(f); free(x);
        return OC_ENOMEM;
    }
    double c = (chi * cm) / dt;
#pragma omp parallel for schedule(static) if (N > 4096)
    for (int k = 0; k < N; k++) {
        double vk = v[k];
        double wn = (w[k] + dt * rm->eta2 * vk / rm->vp) / (1.0 + dt * rm->eta2 * rm->eta3);
        double iion = rm->G * vk * (1.0 - vk / rm->vth) * (1.0 - vk / rm->vp) + rm->eta1 * vk * wn;
        f[2 * k] = M[k] * (c * vk + Iapp[k] - chi * iion);
        f[2 * k + 1] = 0.0;
        w[k] = wn;
        x[2 * k] = vk;
        x[2 * k + 1] = ue[k];
    }
    int it = 0;
    double rr, tr;
    int rc = oc_pcg(h, f, x, 1, rtol, max_it, &it, &rr, &tr);
    for (int k = 0; k < N; k++) {
        v[k] = x[2 * k];
        ue[k] = x[2 * k + 1];
    }
    if (iters) *iters = it;
    free(f); free(x);
    return rc;
}

/* ======================================================================
 * f4.  The decoupled scheme the paper runs (Section 2.2, Eqs. 4-7 as
 * printed): per step the elliptic system with matrix Ai + Ae, then the
 * parabolic system with matrix c M + Ai, each by its own CG.
 * ====================================================================== */
int oc_elliptic_block(const oc_csr *Ki, const oc_csr *Ke, oc_csr *out)
{
    int N = Ki->nrows;
    if (Ke->nrows != N || Ke->nnz != Ki->nnz) return OC_EINVAL;
    for (int p = 0; p <= N; p++)
        if (Ki->rp[p] != Ke->rp[p]) return OC_EINVAL;
    for (int64_t t = 0; t < Ki->nnz; t++)
        if (Ki->ci[t] != Ke->ci[t]) return OC_EINVAL;
    out->nrows = out->ncols = 2 * N;
    out->nnz = 4 * Ki->nnz;
    out->rp = (int64_t *)malloc(sizeof(int64_t) * (size_t)(2 * N + 1));
    out->ci = (int *)malloc(sizeof(int) * (size_t)out->nnz);
    out->v = (double *)malloc(sizeof(double) * (size_t)out->nnz);
    if (!out->rp || !out->ci || !out->v) {
        oc_csr_free(out);
        return OC_ENOMEM;
    }
    int64_t o = 0;
    for (int p = 0; p < N; p++) {
        for (int f = 0; f < 2; f++) {            /* row 2p + f */
            out->rp[2 * p + f] = o;
            for (int64_t t = Ki->rp[p]; t < Ki->rp[p + 1]; t++) {
                int q = Ki->ci[t];
                double kk = Ki->v[t] + Ke->v[t];
                out->ci[o] = 2 * q;                 /* (f, v) entry */
                out->v[o] = (f == 0 && q == p) ? 1.0 : 0.0;
                o++;
                out->ci[o] = 2 * q + 1;             /* (f, u) entry */
                out->v[o] = f == 1 ? kk : 0.0;
                o++;
            }
        }
    }
    out->rp[2 * N] = o;
    return 0;
}

/* y = (c M + Ai) x on the node pattern of Ki */
static void parabolic_apply(const oc_csr *Ki, const double *M, double c, const double *x, double *y)
{
    for (int p = 0; p < Ki->nrows; p++) {
        double a = 0.0;
        for (int64_t t = Ki->rp[p]; t < Ki->rp[p + 1]; t++) a = a + Ki->v[t] * x[Ki->ci[t]];
        y[p] = c * M[p] * x[p] + a;
    }
}

int oc_parabolic_cg(const oc_csr *Ki, const double *M, double c, const double *b, double *v,
                    double rtol, int max_it, int jacobi, int *iters, double *rel_res)
{
    int N = Ki->nrows;
    double *r = (double *)malloc(sizeof(double) * (size_t)N);
    double *z = (double *)malloc(sizeof(double) * (size_t)N);
    double *p = (double *)malloc(sizeof(double) * (size_t)N);
    double *q = (double *)malloc(sizeof(double) * (size_t)N);
    double *dinv = (double *)malloc(sizeof(double) * (size_t)N);
    if (!r || !z || !p || !q || !dinv) {
        free(r); free(z); free(p); free(q); free(dinv);
        return OC_ENOMEM;
    }
    /* Jacobi: inverse of the diagonal of c M + Ai */
    for (int i = 0; i < N; i++) {
        double d = c * M[i];
        for (int64_t t = Ki->rp[i]; t < Ki->rp[i + 1]; t++)
            if (Ki->ci[t] == i) d = d + Ki->v[t];
        dinv[i] = jacobi ? 1.0 / d : 1.0;
    }
    double nb = sqrt(dot(N, b, b));
    parabolic_apply(Ki, M, c, v, q);
    for (int i = 0; i < N; i++) r[i] = b[i] - q[i];
    double rr = sqrt(dot(N, r, r));
    int it = 0, ret = 0;
    if (nb == 0.0) {
        for (int i = 0; i < N; i++) v[i] = 0.0;
        rr = 0.0;
    } else if (rr > rtol * nb) {
        for (int i = 0; i < N; i++) z[i] = dinv[i] * r[i];
        memcpy(p, z, sizeof(double) * (size_t)N);
        double rz = dot(N, r, z);
        ret = OC_ENOTCONV;
        while (it < max_it) {
            parabolic_apply(Ki, M, c, p, q);
            double pq = dot(N, p, q);
            if (!(pq > 0.0)) {
                ret = OC_EBREAK;
                break;
            }
            double alpha = rz / pq;
            for (int i = 0; i < N; i++) {
                v[i] = v[i] + alpha * p[i];
                r[i] = r[i] - alpha * q[i];
            }
            it++;
            rr = sqrt(dot(N, r, r));
            if (rr <= rtol * nb) {
                ret = 0;
                break;
            }
            for (int i = 0; i < N; i++) z[i] = dinv[i] * r[i];
            double rz1 = dot(N, r, z);
            double beta = rz1 / rz;
            for (int i = 0; i < N; i++) p[i] = z[i] + beta * p[i];
            rz = rz1;
        }
    }
    if (iters) *iters = it;
    if (rel_res) *rel_res = nb > 0.0 ? rr / nb : 0.0;
    free(r); free(z); free(p); free(q); free(dinv);
    return ret;
}

int oc_bd_step_decoupled(const oc_hier *he, const oc_csr *Ki, const double *M, int N, double chi,
                         double cm, double dt, const oc_rm_params *rm, const double *Iapp,
                         double *v, double *ue, double *w, double rtol, int max_it, int jacobi,
                         int *it_ell, int *it_par)
{
    int n = 2 * N;
    if (N < 1 || Ki->nrows != N || he->A[0].nrows != n) return OC_EINVAL;
    double *f = (double *)malloc(sizeof(double) * (size_t)n);
    double *x = (double *)malloc(sizeof(double) * (size_t)n);
    double *kv = (double *)malloc(sizeof(double) * (size_t)N);
    double *b = (double *)malloc(sizeof(double) * (size_t)N);
    if (!f || !x || !kv || !b) {
        free(f); free(x); free(kv); free(b);
        return OC_ENOMEM;
    }
    double c = (chi * cm) / dt;
    /* Eq. 6: (Ai + Ae) u_e^n = -Ai v^n, in the block form (0, u_e) */
    oc_spmv(Ki, v, kv);
    for (int k = 0; k < N; k++) {
        f[2 * k] = 0.0;
        f[2 * k + 1] = -kv[k];
        x[2 * k] = 0.0;
        x[2 * k + 1] = ue[k];
    }
    int ie = 0, ip = 0;
    double rr, tr;
    int rc = oc_pcg(he, f, x, 1, rtol, max_it, &ie, &rr, &tr);
    for (int k = 0; k < N; k++) ue[k] = x[2 * k + 1];
    if (rc == 0) {
        /* Eq. 4 and Eq. 7 */
        oc_spmv(Ki, ue, kv);
        for (int k = 0; k < N; k++) {
            double vk = v[k];
            double wn = (w[k] + dt * rm->eta2 * vk / rm->vp) / (1.0 + dt * rm->eta2 * rm->eta3);
            double iion = rm->G * vk * (1.0 - vk / rm->vth) * (1.0 - vk / rm->vp) + rm->eta1 * vk * wn;
            b[k] = c * M[k] * vk - kv[k] + M[k] * (Iapp[k] - chi * iion);
            w[k] = wn;
        }
        rc = oc_parabolic_cg(Ki, M, c, b, v, rtol, max_it, jacobi, &ip, &rr);
    }
    if (it_ell) *it_ell = ie;
    if (it_par) *it_par = ip;
    free(f); free(x); free(kv); free(b);
    return rc;
}
