// bd_assemble.cu -- a0: Q1 hexahedral assembly of the coupled Bidomain block
// operator on the device (Section 2.2; conductivity tensor Eq. 2; block
// operator Eq. 3 with backward Euler on the diffusion).
//
// Compiled with -fmad=false: every value is formed by the same sequence of
// rounded multiplies and adds as the documented evaluation order (Gauss points
// ascending, element entries accumulated from 0.0, element contributions added
// in ascending element index), so the operator is bit-reproducible and
// bit-symmetric.
#include "bd_common.cuh"

namespace bd {

// Element matrices depend only on the element layer (the fibre field varies
// with z alone): Kel[(ez*2 + m)*64 + a*8 + b], m = 0 intracellular, 1 extra.
__global__ void k_element_matrices(int nz, double lx, double ly, double lz, int nx, int ny,
                                   const double *__restrict__ fib, double sil, double sit,
                                   double sel, double set, double *__restrict__ Kel)
{
    int id = blockIdx.x * blockDim.x + threadIdx.x;
    int total = nz * 2 * 64;
    if (id >= total) return;
    int ab = id & 63, m = (id >> 6) & 1, ez = id >> 7;
    int a = ab >> 3, b = ab & 7;
    if (b < a) {  // mirrored entry: computed by the (b, a) thread below
        int t = a;
        a = b;
        b = t;
    }
    double hx = lx / nx, hy = ly / ny, hz = lz / nz;
    double r = 1.0 / sqrt(3.0);
    double g[2] = {(1.0 - r) * 0.5, (1.0 + r) * 0.5};
    double ih[3] = {1.0 / hx, 1.0 / hy, 1.0 / hz};
    double wq = ((hx * hy) * hz) * 0.125;
    double sl = m ? sel : sil, st = m ? set : sit;
    double dl = sl - st;
    double K = 0.0;
    for (int q = 0; q < 8; q++) {
        int gq0 = q & 1, gq1 = (q >> 1) & 1, gq2 = (q >> 2) & 1;
        double xi[3] = {g[gq0], g[gq1], g[gq2]};
        const double *al = fib + ((size_t)ez * 2 + gq2) * 3;
        double D[3][3];
        for (int i = 0; i < 3; i++)
            for (int j = 0; j < 3; j++) {
                D[i][j] = dl * (al[i] * al[j]);
                if (i == j) D[i][j] = D[i][j] + st;
            }
        double Ga[3], Gb[3];
        {
            int ad[3] = {a & 1, (a >> 1) & 1, (a >> 2) & 1};
            double n[3], s[3];
            for (int d = 0; d < 3; d++) {
                n[d] = ad[d] ? xi[d] : 1.0 - xi[d];
                s[d] = ad[d] ? ih[d] : -ih[d];
            }
            Ga[0] = s[0] * (n[1] * n[2]);
            Ga[1] = s[1] * (n[0] * n[2]);
            Ga[2] = s[2] * (n[0] * n[1]);
        }
        {
            int bd_[3] = {b & 1, (b >> 1) & 1, (b >> 2) & 1};
            double n[3], s[3];
            for (int d = 0; d < 3; d++) {
                n[d] = bd_[d] ? xi[d] : 1.0 - xi[d];
                s[d] = bd_[d] ? ih[d] : -ih[d];
            }
            Gb[0] = s[0] * (n[1] * n[2]);
            Gb[1] = s[1] * (n[0] * n[2]);
            Gb[2] = s[2] * (n[0] * n[1]);
        }
        double t0 = (D[0][0] * Gb[0] + D[0][1] * Gb[1]) + D[0][2] * Gb[2];
        double t1 = (D[1][0] * Gb[0] + D[1][1] * Gb[1]) + D[1][2] * Gb[2];
        double t2 = (D[2][0] * Gb[0] + D[2][1] * Gb[1]) + D[2][2] * Gb[2];
        double c = (Ga[0] * t0 + Ga[1] * t1) + Ga[2] * t2;
        K = K + wq * c;
    }
    Kel[id] = K;
}

__device__ __forceinline__ int clampi(int v, int lo, int hi) { return v < lo ? lo : (v > hi ? hi : v); }

__global__ void k_row_counts(int nx, int ny, int nz, int *cnt)
{
    int NX = nx + 1, NY = ny + 1, NZ = nz + 1;
    long long N = (long long)NX * NY * NZ;
    long long p = blockIdx.x * (long long)blockDim.x + threadIdx.x;
    if (p >= N) return;
    int i = (int)(p % NX), j = (int)((p / NX) % NY), l = (int)(p / ((long long)NX * NY));
    int cx = 1 + (i > 0) + (i < NX - 1), cy = 1 + (j > 0) + (j < NY - 1), cz = 1 + (l > 0) + (l < NZ - 1);
    cnt[p] = cx * cy * cz;
}

// One thread per node row: every neighbour q in ascending node index, the
// element contributions of the elements shared by p and q in ascending
// element index.
__global__ void k_assemble_rows(int nx, int ny, int nz, double lx, double ly, double lz,
                                double chi, double cm, double dt, const double *__restrict__ Kel,
                                const int *__restrict__ rp, int *__restrict__ ci,
                                double *__restrict__ v, double *__restrict__ Ki_out,
                                double *__restrict__ Ke_out, double *__restrict__ M)
{
    int NX = nx + 1, NY = ny + 1, NZ = nz + 1;
    long long N = (long long)NX * NY * NZ;
    long long p = blockIdx.x * (long long)blockDim.x + threadIdx.x;
    if (p >= N) return;
    int pi = (int)(p % NX), pj = (int)((p / NX) % NY), pl = (int)(p / ((long long)NX * NY));
    double hx = lx / nx, hy = ly / ny, hz = lz / nz;
    double vol8 = ((hx * hy) * hz) * 0.125;
    // lumped mass: |e|/8 from every element around p, ascending element index
    double Mp = 0.0;
    for (int ez = clampi(pl - 1, 0, nz - 1); ez <= clampi(pl, 0, nz - 1); ez++)
        for (int ey = clampi(pj - 1, 0, ny - 1); ey <= clampi(pj, 0, ny - 1); ey++)
            for (int ex = clampi(pi - 1, 0, nx - 1); ex <= clampi(pi, 0, nx - 1); ex++) Mp = Mp + vol8;
    M[p] = Mp;
    double c = (chi * cm) / dt;
    int pos = rp[p];
    for (int dz = -1; dz <= 1; dz++)
        for (int dy = -1; dy <= 1; dy++)
            for (int dx = -1; dx <= 1; dx++) {
                int qi = pi + dx, qj = pj + dy, ql = pl + dz;
                if (qi < 0 || qi >= NX || qj < 0 || qj >= NY || ql < 0 || ql >= NZ) continue;
                double ki = 0.0, ke = 0.0;
                int exlo = (pi > qi ? pi : qi) - 1, exhi = (pi < qi ? pi : qi);
                int eylo = (pj > qj ? pj : qj) - 1, eyhi = (pj < qj ? pj : qj);
                int ezlo = (pl > ql ? pl : ql) - 1, ezhi = (pl < ql ? pl : ql);
                exlo = exlo < 0 ? 0 : exlo;
                eylo = eylo < 0 ? 0 : eylo;
                ezlo = ezlo < 0 ? 0 : ezlo;
                exhi = exhi > nx - 1 ? nx - 1 : exhi;
                eyhi = eyhi > ny - 1 ? ny - 1 : eyhi;
                ezhi = ezhi > nz - 1 ? nz - 1 : ezhi;
                for (int ez = ezlo; ez <= ezhi; ez++)
                    for (int ey = eylo; ey <= eyhi; ey++)
                        for (int ex = exlo; ex <= exhi; ex++) {
                            int a = (pi - ex) + 2 * (pj - ey) + 4 * (pl - ez);
                            int b = (qi - ex) + 2 * (qj - ey) + 4 * (ql - ez);
                            ki = ki + Kel[((size_t)ez * 2 + 0) * 64 + a * 8 + b];
                            ke = ke + Kel[((size_t)ez * 2 + 1) * 64 + a * 8 + b];
                        }
                long long q = qi + (long long)NX * (qj + (long long)NY * ql);
                double vv = (q == p) ? c * Mp + ki : ki;
                ci[pos] = (int)q;
                v[4 * (size_t)pos + 0] = vv;
                v[4 * (size_t)pos + 1] = ki;
                v[4 * (size_t)pos + 2] = ki;
                v[4 * (size_t)pos + 3] = ki + ke;
                Ki_out[pos] = ki;
                Ke_out[pos] = ke;
                pos++;
            }
}

}  // namespace bd

using namespace bd;

extern "C" int bd_assemble(const bd_mesh *mesh, const bd_params *params, const double *fib,
                           int fib_on_device, void *stream, bd_system **out)
{
    if (!mesh || !params || !fib || !out) return BD_EINVAL;
    *out = nullptr;
    if (mesh->nx < 1 || mesh->ny < 1 || mesh->nz < 1 || !(mesh->lx > 0) || !(mesh->ly > 0) ||
        !(mesh->lz > 0) || !(params->dt > 0) || !(params->chi > 0) || !(params->cm > 0))
        return BD_EINVAL;
    long long NX = mesh->nx + 1LL, NY = mesh->ny + 1LL, NZ = mesh->nz + 1LL;
    long long N = NX * NY * NZ;
    long long nb = (3 * NX - 2) * (3 * NY - 2) * (3 * NZ - 2);
    if (N > (1LL << 30) || nb > 2147483647LL) return BD_ERANGE;
    cudaStream_t s = (cudaStream_t)stream;
    bd_system *sys = new (std::nothrow) bd_system();
    if (!sys) return BD_ENOMEM;
    auto fail = [&](int st) {
        delete sys;
        return st;
    };
    sys->mesh = *mesh;
    sys->params = *params;
    sys->N = (int)N;
    DBuf<double> dfib, Kel;
    DBuf<int> cnt;
    int st;
    if ((st = dfib.alloc((size_t)mesh->nz * 6))) return fail(st);
    if ((st = copy_in(dfib.p, fib, (size_t)mesh->nz * 6 * sizeof(double), fib_on_device, s))) return fail(st);
    if ((st = Kel.alloc((size_t)mesh->nz * 128))) return fail(st);
    if ((st = cnt.alloc((size_t)N + 1))) return fail(st);
    BSR &A = sys->A;
    A.nbr = A.nbc = (int)N;
    if ((st = A.rp.alloc((size_t)N + 1))) return fail(st);
    int total = mesh->nz * 128;
    k_element_matrices<<<(total + 127) / 128, 128, 0, s>>>(mesh->nz, mesh->lx, mesh->ly, mesh->lz,
                                                          mesh->nx, mesh->ny, dfib.p, params->sil,
                                                          params->sit, params->sel, params->set, Kel.p); ::bd::note_launch();
    if (cudaGetLastError() != cudaSuccess) return fail(BD_ECUDA);
    int grid = (int)((N + 255) / 256);
    k_row_counts<<<grid, 256, 0, s>>>(mesh->nx, mesh->ny, mesh->nz, cnt.p); ::bd::note_launch();
    if (cudaGetLastError() != cudaSuccess) return fail(BD_ECUDA);
    long long tot = 0;
    if ((st = exclusive_scan(cnt.p, A.rp.p, (int)N, &tot, s))) return fail(st);
    if (tot != nb) return fail(BD_ECUDA);
    A.nb = tot;
    if ((st = A.ci.alloc((size_t)tot)) || (st = A.v.alloc(4 * (size_t)tot)) ||
        (st = sys->Ki.alloc((size_t)tot)) || (st = sys->Ke.alloc((size_t)tot)) ||
        (st = sys->M.alloc((size_t)N)))
        return fail(st);
    k_assemble_rows<<<grid, 256, 0, s>>>(mesh->nx, mesh->ny, mesh->nz, mesh->lx, mesh->ly, mesh->lz,
                                         params->chi, params->cm, params->dt, Kel.p, A.rp.p, A.ci.p,
                                         A.v.p, sys->Ki.p, sys->Ke.p, sys->M.p); ::bd::note_launch();
    if (cudaGetLastError() != cudaSuccess) return fail(BD_ECUDA);
    if (cudaStreamSynchronize(s) != cudaSuccess) return fail(BD_ECUDA);
    *out = sys;
    return BD_OK;
}

extern "C" int bd_system_info(const bd_system *sys, int *n_nodes, long long *nnz)
{
    if (!sys) return BD_EINVAL;
    if (n_nodes) *n_nodes = sys->N;
    if (nnz) *nnz = 4 * sys->A.nb;
    return BD_OK;
}

extern "C" int bd_system_export(const bd_system *sys, int *row_ptr, int *col, double *val,
                                double *M, void *stream)
{
    if (!sys) return BD_EINVAL;
    cudaStream_t s = (cudaStream_t)stream;
    if (row_ptr || col || val) BD_TRY(bsr_to_scalar_csr_host(sys->A, row_ptr, col, val, s));
    if (M) {
        BD_CUDA(cudaMemcpyAsync(M, sys->M.p, sizeof(double) * sys->N, cudaMemcpyDeviceToHost, s));
        BD_CUDA(cudaStreamSynchronize(s));
    }
    return BD_OK;
}

extern "C" void bd_system_destroy(bd_system *sys) { delete sys; }
