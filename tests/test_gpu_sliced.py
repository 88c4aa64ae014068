"""Sliced form of the V-cycle's block operators (rows sorted by block count
within windows of 1024, 32/K rows per warp, K lanes per row): it sums every
row in the order block-CSR with K lanes uses, so V-cycles and solves agree bit
for bit between the two forms; with every operator sliced the V-cycle and
the solve meet the oracle (Algorithm 2; Section 2.3 for the PCG); the rule
takes the sliced form where it should; amg_set_level_lanes rejects what it
must."""
import numpy as np
import pytest

from paper_2311_13914_gb300 import workloads as W

pytestmark = pytest.mark.gpu

# 41 x 37 x 13 = 19,721 nodes: the finest P has 20 windows of 1024 rows, the
# last one ragged
MESH = W.mesh(40, 36, 12, 1.0, 0.9, 0.3)
SMALL = W.SLAB_SMALL


@pytest.fixture(scope="module")
def B():
    import torch

    if not torch.cuda.is_available():
        pytest.skip("needs a CUDA GPU")
    from paper_2311_13914_gb300 import _build, binding

    _build.build()
    return binding


def _hier(B, m, **opts):
    fib = W.fibre_table(m, 120.0, 10.0)
    sysh = B.bd_assemble(m, W.DEFAULT_PARAMS, fib)
    return fib, sysh, B.amg_setup(sysh, B.amg_options_default(**opts))


def _set_all(B, h, T):
    """Every block operator of h in form T (T > 0 block CSR, -K sliced)."""
    nl = B.amg_num_levels(h)
    for l in range(nl - 1):
        B.amg_set_level_lanes(h, l, (0 if l == 0 else T, T, T))
        got = B.amg_level_lanes(h, l)
        assert got[1:] == (T, T) and (l == 0 or got[0] == T)


@pytest.mark.parametrize("precision", [0, 1])
@pytest.mark.parametrize("m", [SMALL, MESH])
def test_sliced_equals_block_csr_bit_for_bit(B, precision, m):
    _, sysh, h = _hier(B, m, precision=precision)
    n = 2 * W.n_nodes(m)
    f = W.rhs(n, seed=11)
    rng = np.random.default_rng(12)
    r = rng.standard_normal(n)
    for K in (1, 2, 4, 8):
        _set_all(B, h, K)
        zc = B.amg_vcycle(h, r)
        xc, ic = B.amg_solve(h, f)
        _set_all(B, h, -K)
        zs = B.amg_vcycle(h, r)
        xs, is_ = B.amg_solve(h, f)
        assert np.array_equal(zc, zs), f"K={K}"
        assert ic["iters"] == is_["iters"] and ic["status"] == is_["status"] == 0
        assert np.array_equal(xc, xs), f"K={K}"


@pytest.mark.parametrize("precision", [0, 1])
def test_sliced_forms_meet_oracle(B, oracle_lib, precision):
    fib, sysh, h = _hier(B, MESH, precision=precision)
    _set_all(B, h, -2)
    o = oracle_lib.assemble(MESH, W.DEFAULT_PARAMS, fib)
    H = oracle_lib.Hierarchy(o["A"])
    f = W.rhs(o["A"].shape[0], seed=13)
    if precision == 0:
        zo = H.vcycle(f)
        assert np.linalg.norm(B.amg_vcycle(h, f) - zo) <= 1e-10 * np.linalg.norm(zo)
    xg, ig = B.amg_solve(h, f)
    xo, io = H.pcg(f, rtol=1e-8)
    assert ig["status"] == 0 and ig["true_rel_res"] <= 1e-8 * 1.01
    assert abs(ig["iters"] - io["iters"]) <= (1 if precision == 0 else 3)
    ref, _ = H.pcg(f, rtol=1e-13, max_it=1000)
    assert np.linalg.norm(xg - ref) <= 1e-7 * np.linalg.norm(ref)


@pytest.mark.parametrize("precision", [0, 1])
def test_rule_takes_sliced_form_for_many_short_rows(B, precision):
    """65 x 65 x 17 = 71,825 nodes: the finest prolongator's rows (about 7
    blocks each) take the sliced form with one lane per row in FP64 and
    block-CSR in FP32; the solve converges either way."""
    m = W.mesh(64, 64, 16)
    _, sysh, h = _hier(B, m, precision=precision)
    lanes = B.amg_level_lanes(h, 0)
    assert lanes[2] == (-1 if precision == 0 else 2)
    x, info = B.amg_solve(h, W.rhs(2 * W.n_nodes(m), seed=15))
    assert info["status"] == 0 and info["true_rel_res"] <= 1e-8 * 1.01


def test_graph_recaptured_after_override(B):
    """A solve after an override runs the new forms (the captured graph is
    dropped): the graph form equals the host loop with the same forms."""
    _, sysh, h = _hier(B, MESH)
    f = W.rhs(2 * W.n_nodes(MESH), seed=14)
    B.amg_solve(h, f)  # captures the graph with the rule's forms
    _set_all(B, h, 4)
    xg, ig = B.amg_solve(h, f)
    B.amg_profile_enable(h, 1)  # host-driven loop, same kernels
    xl, il = B.amg_solve(h, f)
    B.amg_profile_enable(h, 0)
    assert ig["iters"] == il["iters"] and np.array_equal(xg, xl)
    _set_all(B, h, -2)
    xg2, _ = B.amg_solve(h, f)
    _set_all(B, h, 2)
    xc2, _ = B.amg_solve(h, f)
    assert np.array_equal(xg2, xc2)


def test_set_level_lanes_rejects(B):
    _, sysh, h = _hier(B, SMALL)
    nl = B.amg_num_levels(h)
    bad = [
        (0, (-1, 0, 0)),          # the finest A is sliced ELL already
        (0, (0, 3, 0)),           # not a power of two
        (0, (0, 512, 0)),
        (0, (0, -16, 0)),         # sliced K up to 8
        (nl - 1, (0, 1, 0)),      # nothing is applied in block form on the coarsest
        (nl, (0, 0, 0)),          # level out of range
        (-1, (0, 0, 0)),
    ]
    for level, lanes in bad:
        with pytest.raises(B.BidomainError) as ei:
            B.amg_set_level_lanes(h, level, lanes)
        assert ei.value.status == B.BD_EINVAL, (level, lanes)
    before = B.amg_level_lanes(h, 1)
    B.amg_set_level_lanes(h, 1, (0, 0, 0))  # all kept
    assert B.amg_level_lanes(h, 1) == before
    batch = B.amg_batch_create([h])
    with pytest.raises(B.BidomainError) as ei:
        B.amg_set_level_lanes(h, 1, (-1, -1, -1))
    assert ei.value.status == B.BD_ESTATE
    batch.close()
    B.amg_set_level_lanes(h, 1, (-1, -1, -1))
    assert B.amg_level_lanes(h, 1) == (-1, -1, -1)
