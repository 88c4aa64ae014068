"""Pins of the oracle's Q1 assembly and block operator (a0) against closed forms.

Section 2.2 (Q1 stiffness a_pj = int D grad phi_j . grad phi_p, lumped mass),
Eq. 2 (conductivity tensor), Eq. 3 (block operator).  None of these checks
re-types the oracle's formula: they use tensor-product identities, exact
integrals of linear functions, a manufactured solution and dense spectra.
"""
import json
import math
import os

import numpy as np
import pytest
import scipy.sparse as sp
import scipy.sparse.linalg as spla

from paper_2311_13914_gb300 import workloads as W

GOLD = os.path.join(os.path.dirname(__file__), "golden")


def _const_fib(mesh, a):
    a = np.asarray(a, float)
    return np.tile(a, (mesh["nz"], 2, 1))


def _params(sl, st, sel=None, se_t=None):
    p = dict(W.DEFAULT_PARAMS)
    p.update(sil=sl, sit=st, sel=sl if sel is None else sel, set=st if se_t is None else se_t)
    return p


def _k1d(n, h):
    main = np.full(n + 1, 2.0)
    main[0] = main[-1] = 1.0
    return sp.diags([-np.ones(n), main, -np.ones(n)], [-1, 0, 1]) / h


def _m1d(n, h):
    main = np.full(n + 1, 2.0 / 3.0)
    main[0] = main[-1] = 1.0 / 3.0
    return sp.diags([np.full(n, 1 / 6.0), main, np.full(n, 1 / 6.0)], [-1, 0, 1]) * h


def _c1d(n):
    # int N_i' N_j over the line: derivative on the left factor
    # element: [[-1/2, -1/2], [1/2, 1/2]] (rows test fn derivative, cols trial fn value)
    rows, cols, vals = [], [], []
    for e in range(n):
        loc = np.array([[-0.5, -0.5], [0.5, 0.5]])
        for a in range(2):
            for b in range(2):
                rows.append(e + a)
                cols.append(e + b)
                vals.append(loc[a, b])
    return sp.csr_matrix((vals, (rows, cols)), shape=(n + 1, n + 1))


def _kron3(mz, my, mx):
    return sp.kron(mz, sp.kron(my, mx)).tocsr()


def _tensor_stiffness(mesh, D):
    """K = sum_{d,d'} D[d,d'] int d_d phi_p d_d' phi_q, as tensor products of 1D
    integrals (exact for Q1 on boxes with constant D)."""
    nx, ny, nz = mesh["nx"], mesh["ny"], mesh["nz"]
    h = [mesh["lx"] / nx, mesh["ly"] / ny, mesh["lz"] / nz]
    n = [nx, ny, nz]
    Kd = [_k1d(n[d], h[d]) for d in range(3)]
    Md = [_m1d(n[d], h[d]) for d in range(3)]
    Cd = [_c1d(n[d]) for d in range(3)]  # int N_p' N_q
    K = None
    for d in range(3):
        for e in range(3):
            f = []
            for ax in range(3):
                if ax == d and ax == e:
                    f.append(Kd[ax])
                elif ax == d:
                    f.append(Cd[ax])  # derivative on test function p along d
                elif ax == e:
                    f.append(Cd[ax].T)  # derivative on trial function q along e
                else:
                    f.append(Md[ax])
            term = D[d, e] * _kron3(f[2], f[1], f[0])
            K = term if K is None else K + term
    return K.tocsr()


def test_isotropic_interior_stencil_matches_closed_form(oracle_lib):
    gold = json.load(open(os.path.join(GOLD, "q1_isotropic_stencil.json")))
    m = W.mesh(4, 4, 4)
    h = m["lx"] / m["nx"]
    sig = 2.5
    out = oracle_lib.assemble(m, _params(sig, sig), _const_fib(m, [1, 0, 0]))
    Ki = out["Ki"].toarray()
    NX = m["nx"] + 1
    p = 2 + NX * (2 + NX * 2)  # centre node
    for dz in (-1, 0, 1):
        for dy in (-1, 0, 1):
            for dx in (-1, 0, 1):
                q = p + dx + NX * (dy + NX * dz)
                k = abs(dx) + abs(dy) + abs(dz)
                want = gold[["center", "face", "edge", "corner"][k]] * sig * h
                assert Ki[p, q] == pytest.approx(want, rel=1e-13, abs=1e-15 * sig * h)


@pytest.mark.parametrize("angle", [0.0, 37.0, 90.0])
def test_constant_anisotropy_matches_tensor_product(oracle_lib, angle):
    m = W.mesh(3, 4, 2, 0.3, 0.5, 0.2)
    sl, st = 3.0, 0.31525
    th = math.radians(angle)
    a = np.array([math.cos(th), math.sin(th), 0.0])
    out = oracle_lib.assemble(m, _params(sl, st), _const_fib(m, a))
    D = st * np.eye(3) + (sl - st) * np.outer(a, a)
    Kref = _tensor_stiffness(m, D).toarray()
    Ki = out["Ki"].toarray()
    assert np.allclose(Ki, Kref, rtol=1e-12, atol=1e-14 * np.abs(Kref).max())


def test_general_constant_tensor_off_diagonal_terms(oracle_lib):
    # fibre with a z component exercises every off-diagonal D entry (a transposed
    # operand in the element formula would break symmetry of D[d,e] here)
    m = W.mesh(2, 3, 2, 0.2, 0.3, 0.25)
    a = np.array([0.48, -0.6, 0.64])
    out = oracle_lib.assemble(m, _params(2.0, 0.5), _const_fib(m, a))
    D = 0.5 * np.eye(3) + 1.5 * np.outer(a, a)
    Kref = _tensor_stiffness(m, D).toarray()
    assert np.allclose(out["Ki"].toarray(), Kref, rtol=1e-12, atol=1e-14 * np.abs(Kref).max())


def _gauss_layer_stiffness(mesh, sl, st, theta_of_z):
    """Stiffness of a slab whose conductivity varies with z only, by 2x2x2
    Gauss quadrature (Section 2.2): x and y integrated exactly by the 1D
    tensor factors, z sampled at numpy's two Gauss-Legendre points of every
    element layer, where D(z) = st I + (sl - st) a a^T with
    a = (cos theta(z), sin theta(z), 0) (Eq. 2) is evaluated directly."""
    nx, ny, nz = mesh["nx"], mesh["ny"], mesh["nz"]
    hx, hy, hz = mesh["lx"] / nx, mesh["ly"] / ny, mesh["lz"] / nz
    fx = dict(K=_k1d(nx, hx), M=_m1d(nx, hx), C=_c1d(nx))
    fy = dict(K=_k1d(ny, hy), M=_m1d(ny, hy), C=_c1d(ny))
    xi, wq = np.polynomial.legendre.leggauss(2)
    K = sp.csr_matrix(((nx + 1) * (ny + 1) * (nz + 1),) * 2)
    for ez in range(nz):
        for g in range(2):
            t = (1.0 + xi[g]) / 2.0                  # position inside the layer
            z = (ez + t) * hz
            th = theta_of_z(z)
            a = np.array([math.cos(th), math.sin(th), 0.0])
            D = st * np.eye(3) + (sl - st) * np.outer(a, a)
            N = np.array([1.0 - t, t])                # z basis values
            dN = np.array([-1.0, 1.0]) / hz           # z basis derivatives
            jw = wq[g] * hz / 2.0

            def zf(u, v):
                m = np.zeros((nz + 1, nz + 1))
                m[ez:ez + 2, ez:ez + 2] = jw * np.outer(u, v)
                return sp.csr_matrix(m)
            fz = dict(K=zf(dN, dN), M=zf(N, N), C=zf(dN, N))
            for d in range(3):
                for e in range(3):
                    if D[d, e] == 0.0:
                        continue
                    f = []
                    for ax, fac in enumerate((fx, fy, fz)):
                        if ax == d and ax == e:
                            f.append(fac["K"])
                        elif ax == d:
                            f.append(fac["C"])
                        elif ax == e:
                            f.append(fac["C"].T)
                        else:
                            f.append(fac["M"])
                    K = K + D[d, e] * _kron3(f[2], f[1], f[0])
    return K.toarray()


@pytest.mark.parametrize("rot,off", [(120.0, 5.0), (-75.0, 20.0)])
def test_z_varying_fibre_matches_gauss_quadrature(oracle_lib, rot, off):
    """The fibre table's Gauss z-levels (Section 2.2 quadrature, D sampled at
    the Gauss points) against an independent quadrature that evaluates
    theta(z) = off + rot (z/lz - 1/2) itself: a swapped or shifted z-level, or
    a table read at the wrong layer, changes the layer's stiffness."""
    m = W.mesh(2, 3, 3, 0.2, 0.25, 0.3)
    p = dict(W.DEFAULT_PARAMS)
    out = oracle_lib.assemble(m, p, W.fibre_table(m, rot, off))

    def theta(z):
        return math.radians(off) + math.radians(rot) * (z / m["lz"] - 0.5)
    for K, (sl, st) in ((out["Ki"], (p["sil"], p["sit"])), (out["Ke"], (p["sel"], p["set"]))):
        Kref = _gauss_layer_stiffness(m, sl, st, theta)
        assert np.allclose(K.toarray(), Kref, rtol=1e-12, atol=1e-13 * np.abs(Kref).max())


def test_row_sums_symmetry_mass(oracle_lib):
    m = W.SLAB_SMALL
    out = oracle_lib.assemble(m, W.DEFAULT_PARAMS, W.fibre_table(m))
    for K in (out["Ki"], out["Ke"]):
        d = K.diagonal()
        rs = np.asarray(K.sum(axis=1)).ravel()
        assert np.all(np.abs(rs) <= 1e-13 * d)
        D = (K - K.T).tocoo()
        assert np.all(D.data == 0.0)  # bitwise symmetric
    assert out["M"].sum() == pytest.approx(m["lx"] * m["ly"] * m["lz"], rel=1e-13)
    A = out["A"]
    assert np.all((A - A.T).tocoo().data == 0.0)


def test_patch_test_and_energy_of_linear_functions(oracle_lib):
    m = W.mesh(5, 4, 3, 0.5, 0.4, 0.3)
    a = np.array([0.6, 0.8, 0.0])
    sl, st = 3.0, 0.5
    out = oracle_lib.assemble(m, _params(sl, st), _const_fib(m, a))
    K = out["Ki"]
    NX, NY, NZ = m["nx"] + 1, m["ny"] + 1, m["nz"] + 1
    z, y, x = np.meshgrid(np.linspace(0, m["lz"], NZ), np.linspace(0, m["ly"], NY),
                          np.linspace(0, m["lx"], NX), indexing="ij")
    g = np.array([0.7, -1.3, 2.1])
    u = (g[0] * x + g[1] * y + g[2] * z).ravel()
    Ku = K @ u
    interior = ((x > 0) & (x < m["lx"] - 1e-12) & (y > 0) & (y < m["ly"] - 1e-12)
                & (z > 0) & (z < m["lz"] - 1e-12)).ravel()
    assert np.abs(Ku[interior]).max() <= 1e-12 * np.abs(Ku).max()
    D = st * np.eye(3) + (sl - st) * np.outer(a, a)
    vol = m["lx"] * m["ly"] * m["lz"]
    assert u @ Ku == pytest.approx(vol * g @ D @ g, rel=1e-12)


def test_manufactured_neumann_poisson_second_order(oracle_lib):
    """-sigma Lap u = f with u = cos(pi x/lx)cos(pi y/ly)cos(pi z/lz), zero Neumann
    data; the nodal error of the Q1 / lumped-mass solution falls as h^2."""
    errs = []
    for n in (6, 12):
        m = W.mesh(n, n, n, 1.0, 1.0, 1.0)
        sig = 1.3
        out = oracle_lib.assemble(m, _params(sig, sig), _const_fib(m, [1, 0, 0]))
        K, M = out["Ki"], out["M"]
        NX = n + 1
        c = np.linspace(0, 1, NX)
        z, y, x = np.meshgrid(c, c, c, indexing="ij")
        ue = (np.cos(np.pi * x) * np.cos(np.pi * y) * np.cos(np.pi * z)).ravel()
        f = sig * 3 * np.pi ** 2 * ue
        b = M * f
        b -= b.mean()
        # pin one node, solve, then remove the mean
        Kp = K.tolil()
        Kp[0, :] = 0
        Kp[0, 0] = 1.0
        bp = b.copy()
        bp[0] = 0.0
        uh = spla.spsolve(Kp.tocsc(), bp)
        uh -= uh.mean()
        err = np.abs(uh - (ue - ue.mean())).max()
        errs.append(err)
    rate = math.log2(errs[0] / errs[1])
    assert 1.8 < rate < 2.3, errs


def test_block_operator_null_space_and_energy(oracle_lib):
    p = dict(W.DEFAULT_PARAMS)
    for m in (W.mesh(2, 2, 1), W.mesh(3, 3, 2)):
        out = oracle_lib.assemble(m, p, W.fibre_table(m, 90.0, 10.0))
        A, Ki, Ke, M = out["A"], out["Ki"], out["Ke"], out["M"]
        N = M.size
        z = np.zeros(2 * N)
        z[1::2] = 1.0
        assert np.abs(A @ z).max() <= 1e-13 * np.abs(A.diagonal()).max()
        rng = np.random.default_rng(0)
        x = rng.standard_normal(2 * N)
        v, u = x[0::2], x[1::2]
        c = p["chi"] * p["cm"] / p["dt"]
        energy = c * v @ (M * v) + (v + u) @ (Ki @ (v + u)) + u @ (Ke @ u)
        assert x @ (A @ x) == pytest.approx(energy, rel=1e-12)
        ev = np.linalg.eigvalsh(A.toarray())
        tol = 1e-10 * ev.max()
        assert np.sum(np.abs(ev) <= tol) == 1  # exactly one-dimensional null space
        assert ev.min() >= -tol
