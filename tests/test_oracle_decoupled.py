"""Pins of the oracle's decoupled scheme (Section 2.2, Eqs. 4-7 as printed):
the elliptic block operator's structure and null space, the elliptic AMG-PCG
and the parabolic CG against dense direct solves, and the space-clamped step
against its closed form."""
import numpy as np
import pytest

from paper_2311_13914_gb300 import workloads as W


def _pinv_apply(A, b):
    ev, V = np.linalg.eigh(A)
    keep = np.abs(ev) > 1e-10 * np.abs(ev).max()
    return V[:, keep] @ ((V[:, keep].T @ b) / ev[keep])


@pytest.fixture(scope="module")
def tiny(oracle_lib):
    m = W.mesh(5, 4, 3, 0.5, 0.4, 0.3)
    out = oracle_lib.assemble(m, W.DEFAULT_PARAMS, W.fibre_table(m, 120.0, 10.0))
    return m, out


def test_elliptic_block_is_identity_plus_ai_ae(oracle_lib, tiny):
    _, out = tiny
    Ki, Ke = out["Ki"], out["Ke"]
    E = oracle_lib.elliptic_block(Ki, Ke)
    N = Ki.shape[0]
    assert E.shape == (2 * N, 2 * N) and E.nnz == 4 * Ki.nnz      # full 2x2 blocks
    D = E.toarray()
    assert np.array_equal(D[1::2, 1::2], (Ki + Ke).toarray())
    assert np.array_equal(D[0::2, 0::2], np.eye(N))
    assert not D[0::2, 1::2].any() and not D[1::2, 0::2].any()
    # null vector (0, 1): zero row sums of the stiffness blocks
    e = np.zeros(2 * N)
    e[1::2] = 1.0
    assert np.abs(D @ e).max() <= 1e-12 * np.abs(D).max()


def test_elliptic_pcg_matches_dense_pseudo_inverse(oracle_lib, tiny):
    _, out = tiny
    Ki, Ke = out["Ki"], out["Ke"]
    N = Ki.shape[0]
    H = oracle_lib.Hierarchy(oracle_lib.elliptic_block(Ki, Ke), coarse_eq_limit=40)
    assert H.nlevels >= 2
    v = np.random.default_rng(3).standard_normal(N)
    g = -(Ki @ v)
    f = np.zeros(2 * N)
    f[1::2] = g
    x, info = H.pcg(f, rtol=1e-12)
    assert info["status"] == 0
    ref = _pinv_apply((Ki + Ke).toarray(), g)
    assert np.abs(x[0::2]).max() == 0.0          # the v-field stays zero
    assert np.allclose(x[1::2], ref, rtol=1e-9, atol=1e-9 * np.abs(ref).max())


@pytest.mark.parametrize("jacobi", [True, False])
def test_parabolic_cg_matches_dense_solve(oracle_lib, tiny, jacobi):
    _, out = tiny
    Ki, M = out["Ki"], out["M"]
    p = W.DEFAULT_PARAMS
    c = p["chi"] * p["cm"] / p["dt"]
    rng = np.random.default_rng(4)
    b = rng.standard_normal(M.size)
    v0 = rng.standard_normal(M.size)
    v, info = oracle_lib.parabolic_cg(Ki, M, c, b, v0, rtol=1e-13, jacobi=jacobi)
    assert info["status"] == 0
    ref = np.linalg.solve(c * np.diag(M) + Ki.toarray(), b)
    assert np.allclose(v, ref, rtol=1e-11, atol=1e-11 * np.abs(ref).max())


def test_space_clamped_decoupled_step_is_explicit_euler(oracle_lib, tiny):
    """Uniform v, w and I_app: Ai 1 = 0 so the elliptic right-hand side is zero,
    u_e stays 0, and the parabolic solution is uniform with
    v' = v + dt (I_app - chi I_ion)/(chi Cm)."""
    _, out = tiny
    Ki, Ke, M = out["Ki"], out["Ke"], out["M"]
    p = W.DEFAULT_PARAMS
    H = oracle_lib.Hierarchy(oracle_lib.elliptic_block(Ki, Ke), coarse_eq_limit=40)
    N = M.size
    rm = oracle_lib.RM_PARAMS
    for v0, w0, Ia in [(0.0, 0.0, 8e4), (20.0, 0.05, 0.0), (90.0, 0.4, 1e3)]:
        v, ue, w = np.full(N, v0), np.zeros(N), np.full(N, w0)
        info = H.bd_step_decoupled(Ki, M, p, np.full(N, Ia), v, ue, w, rtol=1e-12)
        assert info["status"] == 0
        dt, chi, cm = p["dt"], p["chi"], p["cm"]
        wn = (w0 + dt * rm["eta2"] * v0 / rm["vp"]) / (1 + dt * rm["eta2"] * rm["eta3"])
        iion = rm["G"] * v0 * (1 - v0 / rm["vth"]) * (1 - v0 / rm["vp"]) + rm["eta1"] * v0 * wn
        vn = v0 + dt * (Ia - chi * iion) / (chi * cm)
        assert np.allclose(w, wn, rtol=1e-15)
        assert np.allclose(v, vn, rtol=1e-9, atol=1e-9 * max(1.0, abs(vn)))
        assert np.abs(ue).max() <= 1e-9 * max(1.0, abs(vn))


def test_decoupled_step_matches_dense_solves(oracle_lib, tiny):
    """A step from a non-uniform state: the elliptic solution against the dense
    pseudo-inverse (mean-zero u_e), the parabolic one against a dense solve."""
    _, out = tiny
    Ki, Ke, M = out["Ki"], out["Ke"], out["M"]
    p = W.DEFAULT_PARAMS
    H = oracle_lib.Hierarchy(oracle_lib.elliptic_block(Ki, Ke), coarse_eq_limit=40)
    N = M.size
    rng = np.random.default_rng(5)
    v = 40.0 * rng.random(N)
    w = 0.3 * rng.random(N)
    ue = np.zeros(N)
    Ia = np.where(rng.random(N) < 0.2, 8e4, 0.0)
    v0, w0 = v.copy(), w.copy()
    info = H.bd_step_decoupled(Ki, M, p, Ia, v, ue, w, rtol=1e-13)
    assert info["status"] == 0 and info["iters_elliptic"] > 0 and info["iters_parabolic"] > 0
    Kd, Ked = Ki.toarray(), Ke.toarray()
    ue_ref = _pinv_apply(Kd + Ked, -Kd @ v0)
    assert np.allclose(ue, ue_ref, rtol=1e-9, atol=1e-9 * np.abs(ue_ref).max())
    rm = oracle_lib.RM_PARAMS
    dt, chi, cm = p["dt"], p["chi"], p["cm"]
    c = chi * cm / dt
    iion = rm["G"] * v0 * (1 - v0 / rm["vth"]) * (1 - v0 / rm["vp"]) + rm["eta1"] * v0 * w
    b = c * M * v0 - Kd @ ue_ref + M * (Ia - chi * iion)
    v_ref = np.linalg.solve(c * np.diag(M) + Kd, b)
    assert np.allclose(v, v_ref, rtol=1e-9, atol=1e-9 * np.abs(v_ref).max())
