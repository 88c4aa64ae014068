"""Form choice by timing inside V-cycles (paper_2311_13914_gb300.forms): every
chosen form is one of the candidates and is what the hierarchy reports, the
timed table covers every coarse operator, the forms it started from are
restored by time_forms, and a solve with the tuned forms still meets the
oracle (Algorithm 2 V-cycle inside the projected PCG)."""
import numpy as np
import pytest

from paper_2311_13914_gb300 import workloads as W

pytestmark = pytest.mark.gpu

CANDS = (2, 8, 32, -1, -4)


@pytest.fixture(scope="module")
def B():
    import torch

    if not torch.cuda.is_available():
        pytest.skip("needs a CUDA GPU")
    from paper_2311_13914_gb300 import _build, binding

    _build.build()
    return binding


@pytest.mark.parametrize("precision", [0, 1])
def test_tune_forms_in_vcycle(B, oracle_lib, precision):
    from paper_2311_13914_gb300 import forms

    m = W.SLAB_SMALL
    fib = W.fibre_table(m, 120.0, 10.0)
    sysh = B.bd_assemble(m, W.DEFAULT_PARAMS, fib)
    h = B.amg_setup(sysh, B.amg_options_default(precision=precision))
    nl = B.amg_num_levels(h)
    n = 2 * W.n_nodes(m)
    r = W.rhs(n, 21)
    before = [B.amg_level_lanes(h, l) for l in range(nl)]
    times = forms.time_forms(h, r, CANDS, reps=2)
    assert [B.amg_level_lanes(h, l) for l in range(nl)] == before
    ops = {(l, op) for l in range(nl - 1) for op in (0, 1, 2) if not (l == 0 and op == 0)}
    assert set(times) == ops
    for row in times.values():
        assert set(row) == set(CANDS) and all(t > 0.0 for t in row.values())
    out = forms.tune_forms(h, r, CANDS, reps=2)
    for (l, op), form in out["forms"].items():
        assert B.amg_level_lanes(h, l)[op] == form
        assert form in CANDS or form == before[l][op]
    o = oracle_lib.assemble(m, W.DEFAULT_PARAMS, fib)
    H = oracle_lib.Hierarchy(o["A"])
    f = W.rhs(n, 22)
    xg, ig = B.amg_solve(h, f)
    assert ig["status"] == 0 and ig["true_rel_res"] <= 1e-8 * 1.01
    ref, _ = H.pcg(f, rtol=1e-13, max_it=1000)
    assert np.linalg.norm(xg - ref) <= 1e-7 * np.linalg.norm(ref)
