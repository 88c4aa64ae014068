"""CUDA path (through the C ABI) against the FP64 oracle, element by element.

Bit-exact: assembled operator and lumped mass, every level's sparsity
pattern, MIS flags, aggregate ids, prolongator values, Galerkin values and
eigen-estimates (the determinism contract).  Floating-point solve phase: one
V-cycle to 1e-10 relative, PCG solutions to a relative error of 1e-7 at rtol
1e-8 after null-space projection, the time-stepped state to 1e-6.
"""
import numpy as np
import pytest
import scipy.sparse as sp

from paper_2311_13914_gb300 import workloads as W

pytestmark = pytest.mark.gpu

MESHES = [
    W.SLAB_SMALL,                         # 24x24x12, the small slab (4 levels)
    W.mesh(1, 1, 1),                      # degenerate: 8 nodes, single dense level
    W.mesh(7, 5, 3, 0.7, 0.5, 0.3),      # ragged, non-cubic elements
    W.mesh(33, 17, 9, 1.0, 0.5, 0.27),   # several tiles with ragged tails
]


@pytest.fixture(scope="module")
def B():
    import torch

    if not torch.cuda.is_available():
        pytest.skip("needs a CUDA GPU")
    from paper_2311_13914_gb300 import _build, binding

    _build.build()
    return binding


def _csr(rp, ci, v, n, m=None):
    return sp.csr_matrix((v, ci, rp), shape=(n, m if m is not None else n))


def _same(a: sp.csr_matrix, b: sp.csr_matrix):
    a.sort_indices()
    b.sort_indices()
    assert a.shape == b.shape
    assert np.array_equal(a.indptr, b.indptr)
    assert np.array_equal(a.indices, b.indices)
    assert np.array_equal(a.data.view(np.uint64), b.data.view(np.uint64))


def test_reproducible_dot_bit_exact(B, oracle_lib):
    """The device long-accumulator dot equals the oracle's correctly rounded
    dot bit for bit, on cancelling, wide-range, subnormal, sparse, constant
    and ragged inputs."""
    import torch

    rng = np.random.default_rng(12)
    cases = [
        (rng.standard_normal(1), rng.standard_normal(1)),
        (rng.standard_normal(1000003), rng.standard_normal(1000003)),
        (rng.standard_normal(4097) * np.exp(rng.uniform(-300, 300, 4097)), rng.standard_normal(4097)),
        (np.array([1e300, 1.0, -1e300, 3e-310]), np.array([1.0, 1e-16, 1.0, 1.0])),
        (np.array([1.0, 2.0 ** -53]), np.array([1.0, 1.0])),
        (np.zeros(0), np.zeros(0)),
        # half the products zero (lanes a warp's shared-limb sum skips), and a
        # long run of equal negative products (warp sums at full width)
        (rng.standard_normal(100003) * (rng.random(100003) < 0.5), rng.standard_normal(100003)),
        (np.full(65571, -3.0), np.full(65571, 7.0 + 2.0 ** -40)),
    ]
    for x, y in cases:
        want = oracle_lib.dot_exact(x, y)
        got = B.bd_dot_exact(x, y)
        assert np.float64(got).view(np.uint64) == np.float64(want).view(np.uint64)
        if x.size:
            gd = B.bd_dot_exact(torch.tensor(x, device="cuda"), torch.tensor(y, device="cuda"))
            assert gd == got


@pytest.mark.parametrize("mi", range(len(MESHES)))
def test_assembly_bit_exact(B, oracle_lib, mi):
    m = MESHES[mi]
    fib = W.fibre_table(m, 120.0, 7.0)
    sysh = B.bd_assemble(m, W.DEFAULT_PARAMS, fib)
    rp, ci, v, M = B.bd_system_export(sysh)
    o = oracle_lib.assemble(m, W.DEFAULT_PARAMS, fib)
    _same(_csr(rp, ci, v, rp.size - 1), o["A"])
    assert np.array_equal(M.view(np.uint64), o["M"].view(np.uint64))


def _gpu_hier(B, m, fib, **opts):
    sysh = B.bd_assemble(m, W.DEFAULT_PARAMS, fib)
    h = B.amg_setup(sysh, B.amg_options_default(**opts))
    return sysh, h


@pytest.mark.parametrize("mi", [0, 2, 3])
def test_hierarchy_bit_exact(B, oracle_lib, mi):
    m = MESHES[mi]
    fib = W.fibre_table(m, 120.0, 3.0)
    opts = dict(coarse_eq_limit=60) if mi == 2 else {}
    sysh, h = _gpu_hier(B, m, fib, **opts)
    o = oracle_lib.assemble(m, W.DEFAULT_PARAMS, fib)
    H = oracle_lib.Hierarchy(o["A"], **opts)
    nl = B.amg_num_levels(h)
    assert nl == H.nlevels
    for l in range(nl):
        e = B.amg_export_level(h, l)
        n = e["n"]
        _same(_csr(*e["A"], n), H.A(l))
        if l < nl - 1:
            assert np.array_equal(e["mis"].astype(bool), H.mis(l).astype(bool))
            assert np.array_equal(e["agg"], H.agg(l))
            assert e["n_agg"] == H.nagg(l)
            assert e["lam"] == H.lam(l)  # bitwise: correctly rounded dots, IEEE ops
            _same(_csr(*e["P"], n, 2 * e["n_agg"]), H.P(l))


def test_setup_from_csr_matches_assembled_path(B, oracle_lib):
    m = MESHES[0]
    fib = W.fibre_table(m)
    o = oracle_lib.assemble(m, W.DEFAULT_PARAMS, fib)
    A = o["A"]
    h = B.amg_setup_from_csr(A.shape[0], A.indptr.astype(np.int32), A.indices.astype(np.int32),
                             A.data)
    H = oracle_lib.Hierarchy(A)
    assert B.amg_num_levels(h) == H.nlevels
    for l in range(H.nlevels):
        e = B.amg_export_level(h, l)
        _same(_csr(*e["A"], e["n"]), H.A(l))
    # the block-CSR finest level (from_csr) and the sliced-ELL finest level
    # (assembled system) solve to the same answer
    sysh, h2 = _gpu_hier(B, m, fib)
    f = W.rhs(A.shape[0], 8)
    x1, i1 = B.amg_solve(h, f)
    x2, i2 = B.amg_solve(h2, f)
    xo, io = H.pcg(f)
    assert np.linalg.norm(x1 - xo) <= 1e-7 * np.linalg.norm(xo)
    assert np.linalg.norm(x2 - xo) <= 1e-7 * np.linalg.norm(xo)


def test_setup_rejects_bad_csr(B):
    # odd size and a pattern that is not made of full 2x2 blocks
    with pytest.raises(B.BidomainError) as ei:
        B.amg_setup_from_csr(3, np.array([0, 1, 2, 3], np.int32), np.array([0, 1, 2], np.int32),
                             np.ones(3))
    assert ei.value.status == B.BD_EINVAL
    rp = np.array([0, 1, 2], np.int32)
    with pytest.raises(B.BidomainError) as ei:
        B.amg_setup_from_csr(2, rp, np.array([0, 1], np.int32), np.ones(2))
    assert ei.value.status == B.BD_EINVAL


@pytest.mark.parametrize("mi", [0, 1, 3])
def test_vcycle_matches_oracle(B, oracle_lib, mi):
    m = MESHES[mi]
    fib = W.fibre_table(m)
    sysh, h = _gpu_hier(B, m, fib)
    o = oracle_lib.assemble(m, W.DEFAULT_PARAMS, fib)
    H = oracle_lib.Hierarchy(o["A"])
    rng = np.random.default_rng(5)
    for _ in range(2):
        r = rng.standard_normal(o["A"].shape[0])
        r[1::2] -= r[1::2].mean()
        zg = B.amg_vcycle(h, r)
        zo = H.vcycle(r)
        assert np.linalg.norm(zg - zo) <= 1e-10 * np.linalg.norm(zo)


def _ref_solution(H, f):
    x, info = H.pcg(f, rtol=1e-13, max_it=1000)
    return x


@pytest.mark.parametrize("mi", [0, 1, 2, 3])
def test_pcg_matches_oracle(B, oracle_lib, mi):
    m = MESHES[mi]
    fib = W.fibre_table(m)
    sysh, h = _gpu_hier(B, m, fib)
    o = oracle_lib.assemble(m, W.DEFAULT_PARAMS, fib)
    H = oracle_lib.Hierarchy(o["A"])
    f = W.rhs(o["A"].shape[0], seed=mi)
    xg, ig = B.amg_solve(h, f)
    xo, io = H.pcg(f, rtol=1e-8)
    assert ig["status"] == 0 and io["status"] == 0
    assert abs(ig["iters"] - io["iters"]) <= 1
    assert ig["true_rel_res"] <= 1e-8 * 1.01
    xs = _ref_solution(H, f)
    gap_go = np.linalg.norm(xg - xo) / np.linalg.norm(xo)
    assert gap_go <= 1e-7, (gap_go, np.linalg.norm(xg - xs) / np.linalg.norm(xs))
    assert abs(xg[1::2].mean()) <= 1e-12 * np.abs(xg).max()


def test_solve_edge_cases(B, oracle_lib):
    import torch

    m = MESHES[2]
    fib = W.fibre_table(m)
    sysh, h = _gpu_hier(B, m, fib)
    n = 2 * W.n_nodes(m)
    # zero right-hand side: zero solution, no iteration
    x, info = B.amg_solve(h, np.zeros(n))
    assert info["iters"] == 0 and np.all(x == 0.0)
    # a pure null-space right-hand side projects to zero
    f = np.zeros(n)
    f[1::2] = 3.0
    x, info = B.amg_solve(h, f)
    assert info["iters"] == 0 and np.abs(x).max() == 0.0
    # strict mode rejects an inconsistent right-hand side
    g = W.rhs(n, 3)
    g[1::2] += 0.5
    with pytest.raises(B.BidomainError) as ei:
        B.amg_solve(h, g, opts=B.solve_options_default(strict=1))
    assert ei.value.status == B.BD_EINCONSISTENT
    # warm start from the solution: converged before the first iteration
    f = W.rhs(n, 4)
    x, info = B.amg_solve(h, f, opts=B.solve_options_default(rtol=1e-10))
    x2, info2 = B.amg_solve(h, f, x=x.copy(), opts=B.solve_options_default(warm_start=1, rtol=1e-8))
    assert info2["iters"] == 0
    # max_it reached -> BD_ENOTCONV reported, not raised when asked
    x3, info3 = B.amg_solve(h, f, opts=B.solve_options_default(max_it=1, rtol=1e-14),
                            raise_on_error=False)
    assert info3["status"] == B.BD_ENOTCONV and info3["iters"] == 1
    # device tensors give the same answer as host arrays (same options, same kernels)
    xh, ih = B.amg_solve(h, f)
    fd = torch.tensor(f, device="cuda")
    xd = torch.zeros_like(fd)
    B.amg_solve(h, fd, xd, stream=torch.cuda.current_stream())
    torch.cuda.synchronize()
    assert np.array_equal(xd.cpu().numpy(), xh)


@pytest.mark.parametrize("precision", [0, 1])
def test_graph_solve_equals_host_loop_solve(B, precision):
    """The whole-solve CUDA graph (device-side WHILE loop) and the host-driven
    loop run the same kernels in the same order with deterministic reductions:
    identical iterates, iteration counts and statuses."""
    m = MESHES[3]
    sysh = B.bd_assemble(m, W.DEFAULT_PARAMS, W.fibre_table(m))
    h = B.amg_setup(sysh, B.amg_options_default(precision=precision))
    n = 2 * W.n_nodes(m)
    for seed, opts in ((1, {}), (2, dict(max_it=3, rtol=1e-14)), (3, dict(rtol=1e-3))):
        f = W.rhs(n, seed)
        o = B.solve_options_default(**opts)
        xg, ig = B.amg_solve(h, f, opts=o, raise_on_error=False)       # graph form
        B.amg_profile_enable(h, True)                                   # timed launches: host loop
        xl, il = B.amg_solve(h, f, opts=o, raise_on_error=False)
        B.amg_profile_enable(h, False)
        assert ig["iters"] == il["iters"] and ig["status"] == il["status"]
        assert np.array_equal(xg, xl)
        assert ig["true_rel_res"] == il["true_rel_res"]


@pytest.mark.parametrize("precision", [0, 1])
def test_autotuned_lanes_solve(B, oracle_lib, precision):
    """amg_options.autotune times the operator forms on the GPU: every chosen
    form is a valid kernel shape, the V-cycle stays within the V-cycle bound
    of the oracle (FP64), the solve still meets the oracle's solution, and the
    graph and loop forms agree bit for bit with the tuned choice."""
    m = MESHES[3]
    fib = W.fibre_table(m)
    sysh = B.bd_assemble(m, W.DEFAULT_PARAMS, fib)
    h = B.amg_setup(sysh, B.amg_options_default(precision=precision, autotune=1))
    nl = B.amg_num_levels(h)
    for l in range(nl):
        lanes = B.amg_level_lanes(h, l)
        if l == nl - 1:
            assert lanes == (0, 0, 0)
            continue
        forms = (1, 2, 4, 8, 16, 32, 64, 128, 256, -1, -2, -4, -8)  # -K: sliced
        assert lanes[0] == 0 if l == 0 else lanes[0] in forms
        assert lanes[1] in forms
        assert lanes[2] in forms
    o = oracle_lib.assemble(m, W.DEFAULT_PARAMS, fib)
    H = oracle_lib.Hierarchy(o["A"])
    f = W.rhs(o["A"].shape[0], seed=7)
    if precision == 0:
        r = f.copy()
        assert np.linalg.norm(B.amg_vcycle(h, r) - H.vcycle(r)) <= 1e-10 * np.linalg.norm(H.vcycle(r))
    xg, ig = B.amg_solve(h, f)
    xo, io = H.pcg(f, rtol=1e-8)
    assert ig["status"] == 0 and ig["true_rel_res"] <= 1e-8 * 1.01
    assert abs(ig["iters"] - io["iters"]) <= (1 if precision == 0 else 3)
    assert np.linalg.norm(xg - xo) <= 1e-7 * np.linalg.norm(xo)
    B.amg_profile_enable(h, True)
    xl, il = B.amg_solve(h, f)
    B.amg_profile_enable(h, False)
    assert il["iters"] == ig["iters"] and np.array_equal(xl, xg)


@pytest.mark.parametrize("m,limit", [(W.SLAB_SMALL, 2000), (W.mesh(32, 32, 10), 4000)])
def test_large_coarsest_level_matches_oracle(B, oracle_lib, m, limit):
    """Coarsest levels above 256 unknowns are inverted by multi-block
    Gauss-Jordan (and above 1024 solved by a multi-block mat-vec): the V-cycle
    and the PCG solution still meet the oracle's dense Cholesky solve."""
    fib = W.fibre_table(m)
    sysh, h = _gpu_hier(B, m, fib, coarse_eq_limit=limit)
    o = oracle_lib.assemble(m, W.DEFAULT_PARAMS, fib)
    H = oracle_lib.Hierarchy(o["A"], coarse_eq_limit=limit)
    nl = B.amg_num_levels(h)
    sizes = [B.amg_level_info(h, l)["n"] for l in range(nl)]
    assert sizes == [H.A(l).shape[0] for l in range(H.nlevels)] and sizes[-1] > 256
    rng = np.random.default_rng(8)
    r = rng.standard_normal(o["A"].shape[0])
    r[1::2] -= r[1::2].mean()
    zo = H.vcycle(r)
    assert np.linalg.norm(B.amg_vcycle(h, r) - zo) <= 1e-10 * np.linalg.norm(zo)
    f = W.rhs(o["A"].shape[0], seed=9)
    xg, ig = B.amg_solve(h, f)
    xo, io = H.pcg(f, rtol=1e-8)
    assert ig["status"] == 0 and abs(ig["iters"] - io["iters"]) <= 1
    assert np.linalg.norm(xg - xo) <= 1e-7 * np.linalg.norm(xo)


@pytest.mark.parametrize("precision", [0, 1])
def test_profile_breakdown_covers_the_solve(B, precision):
    """Profiling level 2 times every solve-phase step: all V-cycle steps of
    every level appear once per iteration, the PCG steps once per iteration
    (the fused ones not at all), and level 1 keeps its finest-operator sums."""
    m = MESHES[0]
    sysh = B.bd_assemble(m, W.DEFAULT_PARAMS, W.fibre_table(m))
    h = B.amg_setup(sysh, B.amg_options_default(precision=precision))
    nl = B.amg_num_levels(h)
    f = W.rhs(2 * W.n_nodes(m), 1)
    B.amg_profile_enable(h, 2)
    _, info = B.amg_solve(h, f)
    B.amg_profile_enable(h, 0)
    it = info["iters"]
    bd = B.amg_profile_breakdown(h)
    for l in range(nl - 1):
        for role in B.PROFILE_ROLES:
            assert bd[f"L{l}_{role}"][1] == it
    for step in ("coarse", "p_update", "A_p", "x_r_update"):
        assert bd[step][1] == it
    # the V-cycle's input rides on the residual update; the z statistics ride on
    # the last finest-level smoothing kernel in FP64 and on the conversion of
    # the FP32 V-cycle's output to z in FP32
    for step in ("vcycle_in", "vcycle_out"):
        assert step not in bd
    if precision:
        assert bd["z_stats"][1] == it
    else:
        assert "z_stats" not in bd
    assert all(ms > 0.0 for ms, _ in bd.values())
    prof = B.amg_profile_read(h)
    assert prof["launches"] == it * (4 if precision else 5)


def test_time_stepping_matches_oracle(B, oracle_lib):
    m = W.mesh(16, 16, 8, 0.6, 0.6, 0.3)
    p = W.DEFAULT_PARAMS
    fib = W.fibre_table(m, 120.0, 10.0)
    stim = W.stimulus(m)
    sysh, h = _gpu_hier(B, m, fib)
    sim = B.bd_sim_create(sysh, h, stim=stim, stim_ms=1.0)
    o = oracle_lib.assemble(m, p, fib)
    H = oracle_lib.Hierarchy(o["A"])
    N = W.n_nodes(m)
    v, ue, w = np.zeros(N), np.zeros(N), np.zeros(N)
    nsteps = 30
    for k in range(nsteps):
        Iapp = stim if k * p["dt"] < 1.0 else np.zeros(N)
        info = H.bd_step(o["M"], p, Iapp, v, ue, w)
        assert info["status"] == 0
    ginfo = B.bd_step(sim, nsteps)
    gv, gu, gw = B.bd_sim_get_state(sim, N)
    assert v.max() > 13.0  # the stimulus excited the corner
    for a, b in ((gv, v), (gu, ue), (gw, w)):
        assert np.linalg.norm(a - b) <= 1e-6 * np.linalg.norm(b)
    assert ginfo["total_iters"] > 0


@pytest.mark.parametrize("mi", [0, 1, 3])
def test_fp32_vcycle_flexible_pcg_matches_fp64_oracle(B, oracle_lib, mi):
    """FP32 V-cycle inside the FP64 flexible CG: the outer loop still drives the
    FP64 residual to rtol 1e-8, so the solution meets the same 1e-7 bound
    against the FP64 oracle; the iteration count may grow slightly."""
    m = MESHES[mi]
    fib = W.fibre_table(m)
    sysh = B.bd_assemble(m, W.DEFAULT_PARAMS, fib)
    h32 = B.amg_setup(sysh, B.amg_options_default(precision=1))
    h64 = B.amg_setup(sysh)
    o = oracle_lib.assemble(m, W.DEFAULT_PARAMS, fib)
    H = oracle_lib.Hierarchy(o["A"])
    f = W.rhs(o["A"].shape[0], seed=10 + mi)
    x32, i32 = B.amg_solve(h32, f)
    x64, i64 = B.amg_solve(h64, f)
    xo, io = H.pcg(f, rtol=1e-8)
    assert i32["status"] == 0 and i32["true_rel_res"] <= 1.01e-8
    assert np.linalg.norm(x32 - xo) <= 1e-7 * np.linalg.norm(xo)
    assert i32["iters"] <= i64["iters"] + 3
    # one FP32 V-cycle agrees with the FP64 one to FP32 accuracy
    r = W.rhs(o["A"].shape[0], seed=20 + mi)
    z32, z64 = B.amg_vcycle(h32, r), B.amg_vcycle(h64, r)
    assert np.linalg.norm(z32 - z64) <= 1e-4 * np.linalg.norm(z64)


def test_fp32_time_stepping_matches_oracle(B, oracle_lib):
    m = W.mesh(16, 16, 8, 0.6, 0.6, 0.3)
    p = W.DEFAULT_PARAMS
    fib = W.fibre_table(m, 120.0, 10.0)
    stim = W.stimulus(m)
    sysh = B.bd_assemble(m, p, fib)
    h = B.amg_setup(sysh, B.amg_options_default(precision=1))
    sim = B.bd_sim_create(sysh, h, stim=stim, stim_ms=1.0)
    o = oracle_lib.assemble(m, p, fib)
    H = oracle_lib.Hierarchy(o["A"])
    N = W.n_nodes(m)
    v, ue, w = np.zeros(N), np.zeros(N), np.zeros(N)
    for k in range(25):
        H.bd_step(o["M"], p, stim if k * p["dt"] < 1.0 else np.zeros(N), v, ue, w)
    B.bd_step(sim, 25)
    gv, gu, gw = B.bd_sim_get_state(sim, N)
    for a, b in ((gv, v), (gu, ue), (gw, w)):
        assert np.linalg.norm(a - b) <= 1e-6 * np.linalg.norm(b)


def test_full_size_slab_properties(B):
    """128x128x32 slab (1.1M unknowns): bit-symmetric operator, zero row sums
    of the stiffness part, total mass, converged solve with projected u_e."""
    m = W.SLAB_PAPER
    fib = W.fibre_table(m, 120.0, W.fibre_offset_from_seed(1))
    sysh = B.bd_assemble(m, W.DEFAULT_PARAMS, fib)
    rp, ci, v, M = B.bd_system_export(sysh)
    n = rp.size - 1
    A = _csr(rp, ci, v, n)
    assert (A != A.T).nnz == 0
    assert M.sum() == pytest.approx(m["lx"] * m["ly"] * m["lz"], rel=1e-12)
    z = np.zeros(n)
    z[1::2] = 1.0
    assert np.abs(A @ z).max() <= 1e-13 * np.abs(A.diagonal()).max()
    h = B.amg_setup(sysh)
    f = W.rhs(n, 1)
    x, info = B.amg_solve(h, f)
    assert info["status"] == 0 and info["true_rel_res"] <= 1.01e-8
    r = f - A @ x
    assert np.linalg.norm(r) <= 1.01e-8 * np.linalg.norm(f)
    assert abs(x[1::2].mean()) <= 1e-12 * np.abs(x).max()
    # the V-cycle is symmetric at full size
    rng = np.random.default_rng(9)
    a, b = rng.standard_normal(n), rng.standard_normal(n)
    a[1::2] -= a[1::2].mean()
    b[1::2] -= b[1::2].mean()
    Ba, Bb = B.amg_vcycle(h, a), B.amg_vcycle(h, b)
    assert abs(Ba @ b - a @ Bb) <= 1e-10 * abs(Ba @ b)
