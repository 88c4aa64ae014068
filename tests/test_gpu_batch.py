"""Batched form: many independent solves captured as the branches of one CUDA
graph (amg_batch_*) give the same iterates, bit for bit, as one amg_solve per
hierarchy, cold and warm-started; a member of the batch meets the oracle."""
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


@pytest.mark.parametrize("precision", [0, 1])
def test_batch_equals_one_solve_per_hierarchy(B, precision):
    import torch

    slabs = W.batch_slabs(6, seed=2)
    hs = _setup(B, slabs, precision)
    fs = [torch.tensor(W.rhs(n, k), device="cuda") for k, (_, _, n) in enumerate(hs)]
    ref = []
    for (sysh, h, n), f in zip(hs, fs):
        x = torch.zeros(n, dtype=torch.float64, device="cuda")
        _, info = B.amg_solve(h, f, x)
        ref.append((x.clone(), info))
    b = B.amg_batch_create([h for _, h, _ in hs])
    xs = [torch.full((n,), 7.0, dtype=torch.float64, device="cuda") for _, _, n in hs]
    for _ in range(2):  # second call reuses the graph
        infos = B.amg_batch_solve(b, fs, xs)
        for (xr, ir), x, i in zip(ref, xs, infos):
            assert i["status"] == 0 and i["iters"] == ir["iters"]
            assert i["true_rel_res"] == ir["true_rel_res"]
            assert torch.equal(x, xr)
    # warm start from a perturbed solution, against the single-solve warm start
    o = B.solve_options_default(warm_start=1)
    x0 = [xr + 1e-3 * torch.tensor(W.rhs(xr.numel(), 50 + k), device="cuda")
          for k, (xr, _) in enumerate(ref)]
    xw = [x.clone() for x in x0]
    infos = B.amg_batch_solve(b, fs, xw, opts=o)
    for (sysh, h, n), f, x00, x, i in zip(hs, fs, x0, xw, infos):
        xs1 = x00.clone()
        _, i1 = B.amg_solve(h, f, xs1, opts=o)
        assert i["iters"] == i1["iters"] and torch.equal(x, xs1)
    b.close()


def test_batch_member_matches_oracle(B, oracle_lib):
    import torch

    slabs = [s for s in W.batch_slabs(64, seed=2) if 2 * W.n_nodes(s[0]) < 20000][:2]
    hs = _setup(B, slabs)
    fs = [torch.tensor(W.rhs(n, 3), device="cuda") for _, _, n in hs]
    xs = [torch.zeros(n, dtype=torch.float64, device="cuda") for _, _, n in hs]
    b = B.amg_batch_create([h for _, h, _ in hs])
    infos = B.amg_batch_solve(b, fs, xs)
    for (m, p, fib), f, x, i in zip(slabs, fs, xs, infos):
        o = oracle_lib.assemble(m, p, fib)
        H = oracle_lib.Hierarchy(o["A"])
        xo, io = H.pcg(f.cpu().numpy(), rtol=1e-8)
        assert i["status"] == 0 and abs(i["iters"] - io["iters"]) <= 1
        assert np.linalg.norm(x.cpu().numpy() - xo) <= 1e-7 * np.linalg.norm(xo)
    b.close()


def test_batch_rejects_bad_arguments(B):
    import torch

    hs = _setup(B, W.batch_slabs(1, seed=4))
    h = hs[0][1]
    with pytest.raises(B.BidomainError) as ei:
        B.amg_batch_create([h, h])
    assert ei.value.status == B.BD_EINVAL
    b = B.amg_batch_create([h])
    n = hs[0][2]
    f = torch.tensor(W.rhs(n, 1), device="cuda")
    x = torch.zeros(n, dtype=torch.float64, device="cuda")
    with pytest.raises(B.BidomainError) as ei:
        B.amg_batch_solve(b, [f], [x], opts=B.solve_options_default(strict=1))
    assert ei.value.status == B.BD_EINVAL
    b.close()
