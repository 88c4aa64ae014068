"""Parity at the benchmark's own size and options (CUDA path through the C ABI
against the FP64 oracle).

* The 128x128x32 slab (1,098,306 unknowns) with the time-stepping benchmark's
  hierarchy options (every level's graph squared, coarsest level up to 2000
  unknowns): every level's pattern, MIS flags, aggregates, eigen-estimate,
  prolongator and Galerkin values bit for bit (Algorithm 1, Section 4), one
  V-cycle to 1e-10 (Algorithm 2).
* A slab small enough for a quick oracle setup whose level-1 Galerkin rows
  exceed 4096 block products, so the setup's block-per-row dense SpGEMM runs
  (checked through bd_spgemm_path_counts): bit for bit as well.
* 100 time steps of the benchmark's workload (Section 2.2, Eqs. 4-7, coupled
  form) against the oracle's stored run: v, u_e and w within 1e-6 relative,
  iterations per step within 1.
"""
import json
import os

import numpy as np
import pytest
import scipy.sparse as sp

from paper_2311_13914_gb300 import workloads as W

pytestmark = pytest.mark.gpu

GOLD = os.path.join(os.path.dirname(__file__), "golden")
STEP_COARSE_EQ_LIMIT = 2000   # the time-stepping benchmark's coarsest-level limit


@pytest.fixture(scope="module")
def B():
    import torch

    if not torch.cuda.is_available():
        pytest.skip("needs a CUDA GPU")
    from paper_2311_13914_gb300 import _build, binding

    _build.build()
    return binding


def _same(a: sp.csr_matrix, b: sp.csr_matrix):
    a.sort_indices()
    b.sort_indices()
    assert a.shape == b.shape
    assert np.array_equal(a.indptr, b.indptr)
    assert np.array_equal(a.indices, b.indices)
    assert np.array_equal(a.data.view(np.uint64), b.data.view(np.uint64))


def _compare_hierarchy(B, oracle_lib, m, fib, limit, vcycle=True):
    dense0 = B.bd_spgemm_path_counts()
    sysh = B.bd_assemble(m, W.DEFAULT_PARAMS, fib)
    h = B.amg_setup(sysh, B.amg_options_default(coarse_eq_limit=limit))
    dense1 = B.bd_spgemm_path_counts()
    o = oracle_lib.assemble(m, W.DEFAULT_PARAMS, fib)
    H = oracle_lib.Hierarchy(o["A"], coarse_eq_limit=limit)
    nl = B.amg_num_levels(h)
    assert nl == H.nlevels
    for l in range(nl):
        e = B.amg_export_level(h, l)
        n = e["n"]
        _same(sp.csr_matrix((e["A"][2], e["A"][1], e["A"][0]), shape=(n, n)), H.A(l))
        if l < nl - 1:
            assert np.array_equal(e["mis"].astype(bool), H.mis(l).astype(bool))
            assert np.array_equal(e["agg"], H.agg(l))
            assert e["n_agg"] == H.nagg(l)
            assert e["lam"] == H.lam(l)
            P = e["P"]
            _same(sp.csr_matrix((P[2], P[1], P[0]), shape=(n, 2 * e["n_agg"])), H.P(l))
    if vcycle:
        rng = np.random.default_rng(23)
        r = rng.standard_normal(o["A"].shape[0])
        r[1::2] -= r[1::2].mean()
        zo = H.vcycle(r)
        assert np.linalg.norm(B.amg_vcycle(h, r) - zo) <= 1e-10 * np.linalg.norm(zo)
    return (dense1[0] - dense0[0], dense1[1] - dense0[1])


def test_dense_spgemm_path_hierarchy_bit_exact(B, oracle_lib):
    """48x48x12, coarsest level up to 2000 unknowns: the level-1 Galerkin
    product R (A P) has rows of 11,154 block products, above the hash path's
    4096, so the block-per-row dense accumulator forms them."""
    m = W.mesh(48, 48, 12)
    fib = W.fibre_table(m, 120.0, W.fibre_offset_from_seed(1))
    hash_calls, dense_calls = _compare_hierarchy(B, oracle_lib, m, fib, STEP_COARSE_EQ_LIMIT)
    assert dense_calls >= 1 and hash_calls >= 1


def test_paper_slab_hierarchy_bit_exact_with_bench_options(B, oracle_lib):
    m = W.SLAB_PAPER
    fib = W.fibre_table(m, 120.0, W.fibre_offset_from_seed(1))
    hash_calls, dense_calls = _compare_hierarchy(B, oracle_lib, m, fib, STEP_COARSE_EQ_LIMIT)
    assert dense_calls >= 1 and hash_calls >= 1


def test_paper_slab_100_steps_match_stored_oracle(B):
    """The benchmark's workload stepped 100 times on the GPU against the
    oracle's run stored by tests/golden/make_paper_slab_steps.py."""
    gold = json.load(open(os.path.join(GOLD, "paper_slab_steps_oracle.json")))
    m = W.SLAB_PAPER
    assert gold["mesh"] == m
    p = W.DEFAULT_PARAMS
    fib = W.fibre_table(m, gold["fibre_rotation_deg"], W.fibre_offset_from_seed(1))
    assert W.fibre_offset_from_seed(1) == gold["fibre_offset_deg"]
    stim = W.stimulus(m)
    sysh = B.bd_assemble(m, p, fib)
    h = B.amg_setup(sysh, B.amg_options_default(coarse_eq_limit=gold["coarse_eq_limit"]))
    assert [B.amg_level_info(h, l)["n"] for l in range(B.amg_num_levels(h))] == gold["levels"]
    sim = B.bd_sim_create(sysh, h, stim=stim, stim_ms=1.0)
    N = W.n_nodes(m)
    iters = []
    for _ in range(gold["steps"]):
        info = B.bd_step(sim, 1)
        iters.append(info["total_iters"])
    assert max(abs(a - b) for a, b in zip(iters, gold["iters"])) <= 1
    v, ue, w = B.bd_sim_get_state(sim, N)
    idx = np.asarray(gold["sample_index"])
    R = np.random.Generator(np.random.PCG64(gold["proj_seed"])).standard_normal((gold["n_proj"], N))
    for name, a in (("v", v), ("ue", ue), ("w", w)):
        g = gold["fields"][name]
        ref = g["norm2"]
        assert abs(np.linalg.norm(a) - ref) <= 1e-6 * ref, name
        assert np.abs(a[idx] - np.asarray(g["sample"])).max() <= 1e-6 * g["max_abs"], name
        # <a - a_oracle, rho> for a Gaussian rho is N(0, |a - a_oracle|^2): a 6-sigma
        # margin on the relative error bound 1e-6 |a_oracle|
        d = R @ a - np.asarray(g["proj"])
        assert np.abs(d).max() <= 6e-6 * ref, (name, d / ref)
    assert np.abs(v).max() > 13.0  # the stimulus excited the corner
