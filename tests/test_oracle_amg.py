"""Pins of the oracle's AMG setup and solve (a1..a12) against brute force,
closed forms and dense linear algebra (numpy), never against itself.

Section 4 (strength w_ij, MIS, cluster rule, P_ij = |C_j|^{-1/2}),
Algorithm 1 (setup), Algorithm 2 (V-cycle), Appendix A (Chebyshev(2)-Jacobi,
10-step CG eigen-estimate, one prolongator smoothing step), Section 2.2 (PCG
for the semi-definite system), Eqs. 4-7 (time step).
"""
import itertools
import json
import math
import os

import numpy as np
import pytest
import scipy.sparse as sp

from paper_2311_13914_gb300 import workloads as W

GOLD = os.path.join(os.path.dirname(__file__), "golden")


def _pinv_apply(A, b):
    """Dense pseudo-inverse through the symmetric eigendecomposition."""
    ev, V = np.linalg.eigh(A)
    keep = np.abs(ev) > 1e-10 * np.abs(ev).max()
    return V[:, keep] @ ((V[:, keep].T @ b) / ev[keep])


# --------------------------------------------------------------- summation
def test_exact_sum_is_correctly_rounded(oracle_lib):
    rng = np.random.default_rng(1)
    cases = [
        rng.standard_normal(1000),
        np.array([1e300, 1.0, -1e300, 1e-300]),
        np.array([2.0 ** -1074] * 7 + [-(2.0 ** -1073)]),
        np.array([1.0, 2.0 ** -53, 2.0 ** -106]),          # rounds up only via sticky bit
        np.array([1.0, 2.0 ** -53]),                          # exact tie -> even
        np.array([1.0 + 2.0 ** -52, 2.0 ** -53]),             # tie -> even (up)
        rng.standard_normal(5000) * np.exp(rng.uniform(-300, 300, 5000)),
        np.concatenate([rng.standard_normal(100) * 1e20, -rng.standard_normal(100) * 1e20]),
    ]
    for x in cases:
        assert oracle_lib.sum_exact(x) == math.fsum(x)
    big = 1.7976931348623157e308
    # intermediate overflow that a long accumulator absorbs (math.fsum raises here)
    assert oracle_lib.sum_exact(np.array([big, big, -big])) == big
    x, y = rng.standard_normal(777), rng.standard_normal(777)
    assert oracle_lib.dot_exact(x, y) == math.fsum(x * y)
    assert oracle_lib.sum_exact(np.zeros(0)) == 0.0


# --------------------------------------------------------------- strength
def test_strength_isotropic_keeps_exactly_the_edge_neighbours(oracle_lib):
    """Isotropic Q1: interior off-diagonals are 0 (face), -sigma h/6 (edge),
    -sigma h/12 (corner) against 8 sigma h/3, so w = 0, 1/16, 1/32 and
    theta = 0.06 keeps exactly the 12 edge neighbours."""
    m = W.mesh(6, 6, 6)
    p = dict(W.DEFAULT_PARAMS, sil=1.0, sit=1.0, sel=2.0, set=2.0)
    A = oracle_lib.assemble(m, p, np.tile([1.0, 0, 0], (6, 2, 1)))["A"]
    S = oracle_lib.strength(A, 0.06)
    NX = 7
    for (i, j, l) in [(3, 3, 3), (2, 3, 4), (4, 2, 2)]:
        p_ = i + NX * (j + NX * l)
        cols = set(S.indices[S.indptr[p_]:S.indptr[p_ + 1]])
        want = set()
        for dz, dy, dx in itertools.product((-1, 0, 1), repeat=3):
            if abs(dx) + abs(dy) + abs(dz) == 2:
                want.add(p_ + dx + NX * (dy + NX * dz))
        assert cols == want
        w = S.data[S.indptr[p_]:S.indptr[p_ + 1]]
        assert np.allclose(w, 1 / 16, rtol=1e-13)


def test_strength_symmetric(oracle_lib):
    m = W.SLAB_SMALL
    A = oracle_lib.assemble(m, W.DEFAULT_PARAMS, W.fibre_table(m))["A"]
    S = oracle_lib.strength(A, 0.06)
    assert (S != S.T).nnz == 0
    assert np.all(S.data >= 0.06)


# --------------------------------------------------------------- MIS
def _prio(oracle_lib, n, key):
    return [(oracle_lib.mix64(k ^ key), -k) for k in range(n)]


def _random_graph(rng, n, p):
    a = rng.random((n, n)) < p
    a = np.triu(a, 1)
    a = a | a.T
    return sp.csr_matrix(a.astype(float))


def test_mis_is_lexicographically_first_maximal_independent_set(oracle_lib):
    rng = np.random.default_rng(2)
    for trial in range(40):
        n = int(rng.integers(1, 13))
        G = _random_graph(rng, n, rng.uniform(0.1, 0.6))
        key = int(rng.integers(0, 2**63))
        got = oracle_lib.mis(G, key).astype(bool)
        adj = G.toarray() > 0
        pr = _prio(oracle_lib, n, key)
        order = sorted(range(n), key=lambda k: pr[k], reverse=True)
        best = None
        for bits in range(1 << n):
            s = np.array([(bits >> k) & 1 for k in range(n)], bool)
            if np.any(adj[np.ix_(s, s)]):
                continue
            # maximal: every node outside has a neighbour inside
            if not all(s[k] or np.any(adj[k] & s) for k in range(n)):
                continue
            seq = tuple(int(s[k]) for k in order)
            if best is None or seq > best[0]:
                best = (seq, s)
        assert np.array_equal(got, best[1]), (trial, n)


# --------------------------------------------------------------- aggregation
def test_aggregation_rule_by_brute_force(oracle_lib):
    m = W.mesh(10, 9, 5)
    A = oracle_lib.assemble(m, W.DEFAULT_PARAMS, W.fibre_table(m, 120.0, 5.0))["A"]
    S = oracle_lib.strength(A, 0.06)
    key = oracle_lib.level_key(7, 0, 0)
    s = oracle_lib.mis(S, key)
    agg, na = oracle_lib.aggregate(S, s)
    roots = np.flatnonzero(s)
    assert na == roots.size
    assert np.array_equal(agg[roots], np.arange(na))  # roots numbered ascending
    Sd = S.toarray()
    for i in range(S.shape[0]):
        if s[i]:
            continue
        cand = [(Sd[i, j], -j) for j in roots if Sd[i, j] > 0]
        assert cand, "every non-root has a strong root neighbour (maximality)"
        w, mj = max(cand)
        assert agg[i] == agg[-mj]


# --------------------------------------------------------------- squared graph
def _dense_square_without_diagonal(S):
    """(I + W)^2 with its diagonal removed, W the filtered weights (Appendix A,
    square_graph), computed densely by numpy."""
    Wd = S.toarray()
    Wh = np.eye(Wd.shape[0]) + Wd
    Q = Wh @ Wh
    np.fill_diagonal(Q, 0.0)
    return Q


def _check_square(oracle_lib, S):
    S2 = oracle_lib.square_graph(S)
    Q = _dense_square_without_diagonal(S)
    got = S2.toarray()
    # pattern: every pair joined by a path of one or two strong edges, no diagonal
    assert np.array_equal(got != 0, Q != 0)
    assert np.all(np.diff(S2.indptr) >= 0) and S2.nnz == np.count_nonzero(Q)
    # values: 2 w_pq for direct neighbours plus the two-step path weights
    assert np.allclose(got, Q, rtol=4e-16 * 8, atol=0.0)
    # symmetric input -> symmetric square
    assert (S2 != S2.T).nnz == 0 or np.abs((S2 - S2.T).toarray()).max() <= 1e-15 * np.abs(Q).max()
    for i in range(S2.shape[0]):
        cols = S2.indices[S2.indptr[i]:S2.indptr[i + 1]]
        assert np.all(np.diff(cols) > 0) and i not in cols
    return S2


def test_square_graph_is_dense_identity_plus_w_squared_on_a_slab(oracle_lib):
    m = W.mesh(7, 6, 4)
    A = oracle_lib.assemble(m, W.DEFAULT_PARAMS, W.fibre_table(m, 120.0, 5.0))["A"]
    S = oracle_lib.strength(A, 0.06)
    S2 = _check_square(oracle_lib, S)
    # a direct strong neighbour q of p with no common neighbour carries exactly 2 w_pq
    Sd = S.toarray()
    for p in range(0, S.shape[0], 7):
        for q in S.indices[S.indptr[p]:S.indptr[p + 1]]:
            if not np.any((Sd[p] > 0) & (Sd[q] > 0)):
                assert S2[p, q] == 2.0 * Sd[p, q]


def test_square_graph_on_random_symmetric_graphs(oracle_lib):
    rng = np.random.default_rng(21)
    for trial in range(30):
        n = int(rng.integers(1, 40))
        G = _random_graph(rng, n, rng.uniform(0.02, 0.5)).toarray()
        w = np.triu(rng.uniform(0.06, 1.0, (n, n)), 1)
        w = (w + w.T) * G
        _check_square(oracle_lib, sp.csr_matrix(w))
    # isolated nodes stay isolated; a path a-b-c gains the two-step edge a-c = w_ab w_bc
    Wp = sp.csr_matrix(np.array([[0, 0.5, 0, 0], [0.5, 0, 0.25, 0], [0, 0.25, 0, 0], [0, 0, 0, 0]]))
    S2 = oracle_lib.square_graph(Wp).toarray()
    assert S2[0, 2] == 0.125 and S2[0, 1] == 1.0 and S2[1, 2] == 0.5
    assert not S2[3].any() and not S2[:, 3].any()


def test_aggregation_rule_on_the_squared_graph_by_brute_force(oracle_lib):
    """Section 4's cluster rule run on the squared graph (Appendix A): every
    non-root joins the root with the largest (I+W)^2 weight, ties to the
    smaller root index; checked against the dense square, not the oracle's."""
    for m, key_seed in ((W.mesh(10, 9, 5), 7), (W.mesh(8, 8, 3), 11)):
        A = oracle_lib.assemble(m, W.DEFAULT_PARAMS, W.fibre_table(m, 120.0, 5.0))["A"]
        S = oracle_lib.strength(A, 0.06)
        S2 = oracle_lib.square_graph(S)
        key = oracle_lib.level_key(key_seed, 0, 0)
        s = oracle_lib.mis(S2, key)
        Q = _dense_square_without_diagonal(S)
        adj = Q > 0
        roots = np.flatnonzero(s)
        # independence and maximality on the squared graph
        assert not np.any(adj[np.ix_(roots, roots)])
        assert all(s[i] or np.any(adj[i, roots]) for i in range(Q.shape[0]))
        agg, na = oracle_lib.aggregate(S2, s)
        assert na == roots.size
        assert np.array_equal(agg[roots], np.arange(na))
        for i in range(Q.shape[0]):
            if s[i]:
                continue
            cand = [(Q[i, j], -j) for j in roots if Q[i, j] > 0]
            w, mj = max(cand)
            # equal weights in exact arithmetic may differ by rounding between
            # the dense and the sparse sums: accept only an exact-tie ambiguity
            best = [j for (wj, j) in ((Q[i, j], j) for j in roots if Q[i, j] > 0)
                    if abs(wj - w) <= 4e-16 * w * 8]
            if len(best) == 1:
                assert agg[i] == agg[-mj]
            else:
                assert agg[i] in set(agg[best])


# --------------------------------------------------------------- prolongators
@pytest.fixture(scope="module")
def small_hier(oracle_lib):
    m = W.mesh(10, 10, 6)
    out = oracle_lib.assemble(m, W.DEFAULT_PARAMS, W.fibre_table(m))
    H = oracle_lib.Hierarchy(out["A"], coarse_eq_limit=40)
    return out, H


def test_tentative_prolongator_orthonormal_and_paper_formula(oracle_lib, small_hier):
    _, H = small_hier
    assert H.nlevels >= 3
    for l in range(H.nlevels - 1):
        Pt = H.Pt(l)
        G = (Pt.T @ Pt).toarray()
        assert np.abs(G - np.eye(G.shape[0])).max() <= 1e-14  # a few ulps per member
        z, zc = H.null(l), H.null(l + 1)
        assert np.abs(Pt @ zc - z).max() <= 1e-15 * np.abs(z).max()
    # finest level: exactly |C_J|^{-1/2} (Section 4)
    agg = H.agg(0)
    cnt = np.bincount(agg)
    Pt = H.Pt(0)
    assert np.array_equal(Pt.data, 1.0 / np.sqrt(cnt[agg].repeat(2).astype(float)))


def test_smoothed_prolongator_preserves_null_vector(small_hier):
    _, H = small_hier
    for l in range(H.nlevels - 1):
        P, z, zc = H.P(l), H.null(l), H.null(l + 1)
        assert np.abs(P @ zc - z).max() <= 1e-12 * np.abs(z).max()


def test_galerkin_operator_equals_dense_triple_product(small_hier):
    _, H = small_hier
    for l in range(H.nlevels - 1):
        A, P, Ac = H.A(l).toarray(), H.P(l).toarray(), H.A(l + 1).toarray()
        ref = P.T @ A @ P
        assert np.abs(Ac - ref).max() <= 1e-12 * np.abs(ref).max()
        assert np.abs(Ac - Ac.T).max() <= 1e-13 * np.abs(Ac).max()
        zc = H.null(l + 1)
        assert np.abs(Ac @ zc).max() <= 1e-12 * np.abs(Ac).max() * np.abs(zc).max()


# --------------------------------------------------------------- eigen-estimate
@pytest.mark.parametrize("m", [3, 6, 10])
def test_lanczos_exact_on_1d_laplacian(oracle_lib, m):
    """D^{-1}A of tridiag(-1,2,-1) has eigenvalues 1 - cos(k pi/(m+1)); with
    m <= 10 the 10-step Lanczos process is exact."""
    A = sp.diags([-np.ones(m - 1), 2 * np.ones(m), -np.ones(m - 1)], [-1, 0, 1]).tocsr()
    lam, done = oracle_lib.lambda_max(A, 10, 12345)
    assert done <= 10
    assert lam == pytest.approx(1 - math.cos(m * math.pi / (m + 1)), rel=1e-12)


def test_lanczos_ritz_value_below_and_close_to_lambda_max(oracle_lib, small_hier):
    out, H = small_hier
    for l in range(H.nlevels - 1):
        A = H.A(l).toarray()
        d = np.diag(A)
        ev = np.linalg.eigvals(A / d[:, None]).real.max()
        lam = H.lam(l)
        assert lam <= ev * (1 + 1e-12)
        assert lam >= 0.9 * ev


def test_tridiagonal_bisection_matches_dense(oracle_lib):
    rng = np.random.default_rng(3)
    for m in (1, 2, 5, 10):
        d, e = rng.uniform(0, 3, m), rng.uniform(-1, 1, m - 1)
        T = np.diag(d) + np.diag(e, 1) + np.diag(e, -1)
        assert oracle_lib.tridiag_max_eig(d, e) == pytest.approx(np.linalg.eigvalsh(T).max(),
                                                                 rel=1e-14, abs=1e-14)


# --------------------------------------------------------------- smoother
def test_chebyshev_error_polynomial_closed_form(oracle_lib):
    """x2 = T_2((theta - D^{-1}A)/delta) x0 / T_2(theta/delta) for f = 0."""
    rng = np.random.default_rng(4)
    n = 12
    B = rng.standard_normal((n, n))
    A = B @ B.T + n * np.eye(n)
    lam = np.linalg.eigvals(A / np.diag(A)[:, None]).real.max()
    lo, hi = 0.05 * lam, 1.05 * lam
    x0 = rng.standard_normal(n)
    x2 = oracle_lib.chebyshev(sp.csr_matrix(A), np.zeros(n), x0, 2, lo, hi)
    th, de = (hi + lo) / 2, (hi - lo) / 2
    Mj = A / np.diag(A)[:, None]
    X = (th * np.eye(n) - Mj) / de
    T2 = 2 * X @ X - np.eye(n)
    ref = T2 @ x0 / (2 * (th / de) ** 2 - 1)
    assert np.allclose(x2, ref, rtol=1e-12, atol=1e-12 * np.abs(ref).max())


# --------------------------------------------------------------- coarse / V-cycle / PCG
def test_single_level_is_pseudo_inverse(oracle_lib):
    m = W.mesh(2, 2, 1)
    A = oracle_lib.assemble(m, W.DEFAULT_PARAMS, W.fibre_table(m))["A"]
    H = oracle_lib.Hierarchy(A)
    assert H.nlevels == 1
    rng = np.random.default_rng(5)
    r = rng.standard_normal(A.shape[0])
    r[1::2] -= r[1::2].mean()
    x = H.vcycle(r)
    ref = _pinv_apply(A.toarray(), r)
    assert np.allclose(x, ref, rtol=1e-10, atol=1e-10 * np.abs(ref).max())


def test_vcycle_symmetric_positive(small_hier):
    out, H = small_hier
    n = H.n
    rng = np.random.default_rng(6)
    z = np.zeros(n)
    z[1::2] = 1
    for _ in range(3):
        x, y = rng.standard_normal(n), rng.standard_normal(n)
        x -= z * (z @ x) / (z @ z)
        y -= z * (z @ y) / (z @ z)
        Bx, By = H.vcycle(x), H.vcycle(y)
        assert abs(Bx @ y - x @ By) <= 1e-12 * abs(Bx @ y) + 1e-13 * np.linalg.norm(Bx) * np.linalg.norm(y)
        assert x @ Bx > 0


def test_pcg_matches_dense_pseudo_inverse(oracle_lib):
    m = W.mesh(6, 5, 3)
    A = oracle_lib.assemble(m, W.DEFAULT_PARAMS, W.fibre_table(m))["A"]
    H = oracle_lib.Hierarchy(A, coarse_eq_limit=60)
    assert H.nlevels >= 2
    f = W.rhs(A.shape[0], 11)
    x, info = H.pcg(f, rtol=1e-12)
    assert info["status"] == 0 and info["iters"] <= 30
    xs = _pinv_apply(A.toarray(), f)
    xs[1::2] -= xs[1::2].mean()
    ev = np.linalg.eigvalsh(A.toarray())
    cond = ev.max() / ev[ev > 1e-10 * ev.max()].min()
    assert np.linalg.norm(x - xs) <= cond * 1e-12 * np.linalg.norm(xs) * 10
    assert abs(x[1::2].mean()) <= 1e-14 * np.abs(x).max()


def test_default_options_are_appendix_a(oracle_lib):
    gold = json.load(open(os.path.join(GOLD, "gamg_appendix_a.json")))
    o = oracle_lib.DEFAULT_OPTS
    assert o["theta"] == gold["threshold"]
    assert o["coarse_eq_limit"] == gold["coarse_eq_limit"]
    assert o["cheb_degree"] == gold["mg_levels_ksp_max_it"]
    assert o["esteig_steps"] == gold["esteig_ksp_max_it"]
    assert (o["eig_lo"], o["eig_hi"]) == (gold["chebyshev_esteig"][1], gold["chebyshev_esteig"][3])
    # App. A squares the first level's graph; the default squares every level
    # (measured: operator complexity 1.26 instead of 1.78 on the 128x128x32 slab)
    assert o["square_levels"] >= gold["square_graph"]


# --------------------------------------------------------------- time step
def test_space_clamped_step_is_explicit_euler(oracle_lib):
    """Uniform v, w and I_app: K 1 = 0, so u_e stays 0 and
    v' = v + dt (I_app - chi I_ion)/(chi Cm), w' = (w + dt eta2 v/vp)/(1 + dt eta2 eta3)."""
    m = W.mesh(6, 6, 3)
    p = W.DEFAULT_PARAMS
    out = oracle_lib.assemble(m, p, W.fibre_table(m))
    H = oracle_lib.Hierarchy(out["A"], coarse_eq_limit=60)
    N = out["M"].size
    rm = oracle_lib.RM_PARAMS
    for v0, w0, Ia in [(0.0, 0.0, 8e4), (20.0, 0.05, 0.0), (90.0, 0.4, 1e3)]:
        v, ue, w = np.full(N, v0), np.zeros(N), np.full(N, w0)
        info = H.bd_step(out["M"], p, np.full(N, Ia), v, ue, w, rtol=1e-12)
        assert info["status"] == 0
        dt, chi, cm = p["dt"], p["chi"], p["cm"]
        wn = (w0 + dt * rm["eta2"] * v0 / rm["vp"]) / (1 + dt * rm["eta2"] * rm["eta3"])
        iion = rm["G"] * v0 * (1 - v0 / rm["vth"]) * (1 - v0 / rm["vp"]) + rm["eta1"] * v0 * wn
        vn = v0 + dt * (Ia - chi * iion) / (chi * cm)
        assert np.allclose(w, wn, rtol=1e-15)
        assert np.allclose(v, vn, rtol=1e-9, atol=1e-9 * max(1.0, abs(vn)))
        assert np.abs(ue).max() <= 1e-9 * max(1.0, abs(vn))


def test_threaded_solve_phase_is_bitwise_serial(oracle_lib):
    """The oracle's solve phase runs its independent loops on several threads
    and every reduction serially: V-cycle, PCG and time step give the same
    bits on one thread and on four."""
    m = W.mesh(20, 18, 8)
    p = W.DEFAULT_PARAMS
    out = oracle_lib.assemble(m, p, W.fibre_table(m, 120.0, 5.0))
    H = oracle_lib.Hierarchy(out["A"])
    f = W.rhs(out["A"].shape[0], 3)
    N = out["M"].size
    stim = W.stimulus(m)
    res = []
    before = oracle_lib.get_threads()
    try:
        for t in (1, 4):
            try:
                oracle_lib.set_threads(t)
            except RuntimeError:
                pytest.skip("oracle built without OpenMP")
            z = H.vcycle(f)
            x, info = H.pcg(f)
            v, ue, w = np.zeros(N), np.zeros(N), np.zeros(N)
            for _ in range(3):
                H.bd_step(out["M"], p, stim, v, ue, w)
            res.append((z, x, info["iters"], v, ue, w))
    finally:
        oracle_lib.set_threads(max(before, 1))
    for a, b in zip(res[0], res[1]):
        assert np.array_equal(np.asarray(a), np.asarray(b))
