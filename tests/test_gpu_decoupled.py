"""The paper's decoupled scheme on the GPU (bd_elliptic_setup, bd_dsim_*)
against the oracle: the elliptic hierarchy bit for bit (the determinism
contract carries over), per-step iteration counts of both solves, and the
time-stepped state (Section 2.2, Eqs. 4-7 as printed)."""
import numpy as np
import pytest
import scipy.sparse as sp

from paper_2311_13914_gb300 import workloads as W

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def B():
    import torch

    if not torch.cuda.is_available():
        pytest.skip("needs a CUDA GPU")
    from paper_2311_13914_gb300 import _build, binding

    _build.build()
    return binding


def _same(a, b):
    a = sp.csr_matrix(a)
    b = sp.csr_matrix(b)
    a.sort_indices()
    b.sort_indices()
    assert a.shape == b.shape
    assert np.array_equal(a.indptr, b.indptr)
    assert np.array_equal(a.indices, b.indices)
    assert np.array_equal(a.data.view(np.uint64), b.data.view(np.uint64))


@pytest.mark.parametrize("m", [W.SLAB_SMALL, W.mesh(9, 7, 5, 0.9, 0.7, 0.5)])
def test_elliptic_hierarchy_bit_exact(B, oracle_lib, m):
    fib = W.fibre_table(m, 120.0, 3.0)
    sysh = B.bd_assemble(m, W.DEFAULT_PARAMS, fib)
    opts = {} if m is W.SLAB_SMALL else dict(coarse_eq_limit=60)
    h = B.bd_elliptic_setup(sysh, B.amg_options_default(**opts))
    o = oracle_lib.assemble(m, W.DEFAULT_PARAMS, fib)
    H = oracle_lib.Hierarchy(oracle_lib.elliptic_block(o["Ki"], o["Ke"]), **opts)
    nl = B.amg_num_levels(h)
    assert nl == H.nlevels and nl >= 2
    for l in range(nl):
        e = B.amg_export_level(h, l)
        n = e["n"]
        _same(sp.csr_matrix((e["A"][2], e["A"][1], e["A"][0]), shape=(n, n)), H.A(l))
        if l < nl - 1:
            assert np.array_equal(e["agg"], H.agg(l))
            assert e["lam"] == H.lam(l)
            _same(sp.csr_matrix((e["P"][2], e["P"][1], e["P"][0]), shape=(n, 2 * e["n_agg"])), H.P(l))


@pytest.mark.parametrize("jacobi", [True, False])
def test_decoupled_time_stepping_matches_oracle(B, oracle_lib, jacobi):
    m = W.mesh(16, 16, 8, 0.6, 0.6, 0.3)
    p = W.DEFAULT_PARAMS
    fib = W.fibre_table(m, 120.0, 10.0)
    stim = W.stimulus(m)
    sysh = B.bd_assemble(m, p, fib)
    h = B.bd_elliptic_setup(sysh)
    sim = B.bd_dsim_create(sysh, h, stim=stim, stim_ms=1.0, jacobi=jacobi)
    o = oracle_lib.assemble(m, p, fib)
    H = oracle_lib.Hierarchy(oracle_lib.elliptic_block(o["Ki"], o["Ke"]))
    N = W.n_nodes(m)
    v, ue, w = np.zeros(N), np.zeros(N), np.zeros(N)
    for k in range(30):
        Iapp = stim if k * p["dt"] < 1.0 else np.zeros(N)
        info = H.bd_step_decoupled(o["Ki"], o["M"], p, Iapp, v, ue, w, jacobi=jacobi)
        assert info["status"] == 0
        ie, ip = B.bd_dsim_step(sim, 1)
        assert ie["status"] == 0 and ip["status"] == 0
        assert abs(ie["iters"] - info["iters_elliptic"]) <= 1
        assert abs(ip["iters"] - info["iters_parabolic"]) <= 1
        assert ip["true_rel_res"] <= 1.01e-8
    gv, gu, gw = B.bd_dsim_get_state(sim, N)
    assert v.max() > 13.0  # the stimulus excited the corner
    for a, b in ((gv, v), (gu, ue), (gw, w)):
        assert np.linalg.norm(a - b) <= 1e-6 * np.linalg.norm(b)


def test_decoupled_needs_the_elliptic_hierarchy(B):
    m = W.mesh(6, 5, 4)
    sysh = B.bd_assemble(m, W.DEFAULT_PARAMS, W.fibre_table(m))
    h = B.amg_setup(sysh)  # the coupled operator's hierarchy
    with pytest.raises(B.BidomainError) as ei:
        B.bd_dsim_create(sysh, h)
    assert ei.value.status == B.BD_EINVAL
