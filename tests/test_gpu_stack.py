"""Stacked batch (amg_stack_*): the hierarchies of many uneven slabs solved
together, one kernel launch per V-cycle step and level for all of them.

Each member's solve is the projected PCG of Section 2.2 with its own
hierarchy's V-cycle (Algorithm 2, Appendix A smoother), so it must agree with
amg_solve of that hierarchy to rounding (the stacked reductions add in another
order) and with the FP64 oracle to 1e-7, on the 64-slab workload (nx, ny in
16..64, nz in 8..16, seed 2).  Edge cases: a single-level member (its finest
level is its coarsest), a zero right-hand side, warm start from the solution,
max_it reached, mixed precisions, forms locked while stacked.
"""
import numpy as np
import pytest

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


def _setup(B, slabs, precision=0):
    import torch

    out = []
    for m, p, fib in slabs:
        sysh = B.bd_assemble(m, p, fib)
        h = B.amg_setup(sysh, B.amg_options_default(precision=precision))
        out.append((sysh, h, 2 * W.n_nodes(m)))
    torch.cuda.synchronize()
    return out


def _rhs(hs):
    import torch

    return [torch.tensor(W.rhs(n, 100 + k), device="cuda") for k, (_, _, n) in enumerate(hs)]


@pytest.mark.parametrize("precision", [0, 1])
def test_stack_of_64_slabs_matches_one_solve_per_hierarchy(B, precision):
    import torch

    slabs = W.batch_slabs(64, seed=2)
    hs = _setup(B, slabs, precision)
    fs = _rhs(hs)
    st = B.amg_stack_create([h for _, h, _ in hs])
    xs = [torch.zeros_like(f) for f in fs]
    infos = B.amg_stack_solve(st, fs, xs)
    info = B.amg_stack_info(st)
    nl = max(B.amg_num_levels(h) for _, h, _ in hs)
    assert info["levels"] == nl
    # one launch per V-cycle step and level for all 64 members, plus the
    # coarsest solves and five PCG kernels
    assert info["launches_per_iteration"] <= 7 * (nl - 1) + 1 + 6
    for (sysh, h, n), f, x, inf in zip(hs, fs, xs, infos):
        xr, ir = B.amg_solve(h, f.cpu().numpy())
        xg = x.cpu().numpy()
        assert inf["status"] == 0 and inf["true_rel_res"] <= 1.01e-8
        assert abs(inf["iters"] - ir["iters"]) <= 1
        assert np.linalg.norm(xg - xr) <= 1e-7 * np.linalg.norm(xr)
        assert abs(xg[1::2].mean()) <= 1e-12 * np.abs(xg).max()
    # a second solve through the same graph gives the same bits
    xs2 = [torch.zeros_like(f) for f in fs]
    infos2 = B.amg_stack_solve(st, fs, xs2)
    B.amg_stack_solve(st, fs, xs)
    for a, b, i1, i2 in zip(xs, xs2, infos, infos2):
        assert torch.equal(a, b) and i1["iters"] == i2["iters"]
    st.close()


def test_stack_members_match_the_oracle(B, oracle_lib):
    import torch

    slabs = W.batch_slabs(64, seed=2)
    sizes = [W.n_nodes(m) for m, _, _ in slabs]
    pick = sorted(range(64), key=lambda k: sizes[k])
    pick = pick[:4] + pick[-1:]          # the four smallest and the largest
    sub = [slabs[k] for k in pick]
    hs = _setup(B, sub)
    fs = _rhs(hs)
    st = B.amg_stack_create([h for _, h, _ in hs])
    xs = [torch.zeros_like(f) for f in fs]
    infos = B.amg_stack_solve(st, fs, xs)
    for (m, p, fib), f, x, inf in zip(sub, fs, xs, infos):
        o = oracle_lib.assemble(m, p, fib)
        H = oracle_lib.Hierarchy(o["A"])
        xo, io = H.pcg(f.cpu().numpy(), rtol=1e-8)
        assert abs(inf["iters"] - io["iters"]) <= 1
        assert np.linalg.norm(x.cpu().numpy() - xo) <= 1e-7 * np.linalg.norm(xo)
    st.close()


def test_stack_edge_cases(B):
    import torch

    slabs = W.batch_slabs(3, seed=5)
    m1 = W.mesh(1, 1, 1)                  # single level: its finest level is its coarsest
    slabs.append((m1, W.DEFAULT_PARAMS, W.fibre_table(m1)))
    hs = _setup(B, slabs)
    assert B.amg_num_levels(hs[-1][1]) == 1
    fs = _rhs(hs)
    fs[1].zero_()                          # zero right-hand side: zero solution, no iteration
    st = B.amg_stack_create([h for _, h, _ in hs])
    xs = [torch.zeros_like(f) for f in fs]
    infos = B.amg_stack_solve(st, fs, xs)
    assert infos[1]["iters"] == 0 and torch.count_nonzero(xs[1]) == 0
    for k in (0, 2, 3):
        xr, ir = B.amg_solve(hs[k][1], fs[k].cpu().numpy())
        assert infos[k]["status"] == 0
        assert np.linalg.norm(xs[k].cpu().numpy() - xr) <= 1e-7 * np.linalg.norm(xr)
    # warm start from the solutions (tightly converged): no iteration needed at rtol 1e-8
    tight = B.solve_options_default(rtol=1e-11)
    B.amg_stack_solve(st, fs, xs, opts=tight)
    warm = B.solve_options_default(warm_start=1, rtol=1e-8)
    infos = B.amg_stack_solve(st, fs, xs, opts=warm)
    assert all(i["iters"] == 0 and i["status"] == 0 for i in infos)
    # max_it reached: BD_ENOTCONV for the members still iterating
    for x in xs:
        x.zero_()
    infos = B.amg_stack_solve(st, fs, xs, opts=B.solve_options_default(max_it=1, rtol=1e-14),
                              raise_on_error=False)
    assert infos[0]["status"] == B.BD_ENOTCONV and infos[0]["iters"] == 1
    assert infos[1]["status"] == 0 and infos[1]["iters"] == 0
    # the members' forms are locked while the stack exists
    with pytest.raises(B.BidomainError) as ei:
        B.amg_set_level_lanes(hs[0][1], 0, [0, 4, 0])
    assert ei.value.status == B.BD_ESTATE
    st.close()
    B.amg_set_level_lanes(hs[0][1], 0, [0, 4, 0])
    # one V-cycle precision per stack
    h32 = B.amg_setup(hs[0][0], B.amg_options_default(precision=1))
    with pytest.raises(B.BidomainError) as ei:
        B.amg_stack_create([hs[2][1], h32])
    assert ei.value.status == B.BD_EINVAL
