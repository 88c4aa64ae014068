"""Serving loop (continuous batching of Bidomain simulations), through the C ABI.

A request's result must not depend on what else is in flight: each request
owns its buffers and every kernel is deterministic, so the final state of a
simulation is compared bit for bit alone and in a mix of other sizes.
Admission keeps the measured resident footprint within the budget.
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


def _request(nx, ny, nz, rot=120.0):
    m = W.mesh(nx, ny, nz)
    return m, W.fibre_table(m, rot, 3.0), W.stimulus(m, corner=0.12)


def _submit(B, srv, req, nsteps):
    m, fib, stim = req
    return B.bd_server_submit(srv, m, W.DEFAULT_PARAMS, fib, stim, 1.0, nsteps)


@pytest.mark.parametrize("precision", [0, 1])
def test_result_alone_equals_result_in_the_mix(B, precision):
    x = _request(20, 18, 6)
    srv = B.bd_server_create(B.bd_server_options_default(precision=precision))
    ix = _submit(B, srv, x, 12)
    B.bd_server_drain(srv)
    alone = B.bd_server_result(srv, ix)
    assert B.bd_server_request(srv, ix)["state"] == 2

    srv2 = B.bd_server_create(B.bd_server_options_default(precision=precision, max_active=3))
    ids = [_submit(B, srv2, _request(24, 16, 6, 90.0), 20),
           _submit(B, srv2, _request(12, 12, 4, 60.0), 8),
           _submit(B, srv2, x, 12),
           _submit(B, srv2, _request(28, 28, 8, 150.0), 10),
           _submit(B, srv2, _request(16, 16, 8), 15)]
    peak = 0
    while True:
        a, q = B.bd_server_tick(srv2)
        peak = max(peak, a)
        if a == 0 and q == 0:
            break
    assert peak <= 3
    for i in ids:
        assert B.bd_server_request(srv2, i)["state"] == 2
    mixed = B.bd_server_result(srv2, ids[2])
    for a_, b_ in zip(alone, mixed):
        assert np.array_equal(a_, b_)
    info = B.bd_server_request(srv2, ids[2])
    assert info["steps_done"] == 12 and info["total_iters"] > 0
    assert info["done_ms"] >= info["admit_ms"] >= info["submit_ms"]


def test_admission_keeps_resident_footprint_within_budget(B):
    req = _request(40, 40, 10)
    probe = B.bd_server_create()
    i = _submit(B, probe, req, 2)
    B.bd_server_tick(probe)
    fp = B.bd_server_request(probe, i)["footprint"]
    B.bd_server_drain(probe)
    assert fp > 0
    budget = int(2.5 * fp)
    srv = B.bd_server_create(B.bd_server_options_default(hbm_budget=budget, max_active=16))
    ids = [_submit(B, srv, req, 3) for _ in range(5)]
    while True:
        a, q = B.bd_server_tick(srv)
        st = B.bd_server_stats(srv)
        assert st["resident_bytes"] <= budget
        assert a <= 2
        if a == 0 and q == 0:
            break
    assert all(B.bd_server_request(srv, i)["state"] == 2 for i in ids)


def test_request_larger_than_the_budget_fails_cleanly(B):
    srv = B.bd_server_create(B.bd_server_options_default(hbm_budget=1 << 20))
    i = _submit(B, srv, _request(24, 24, 12), 3)
    ok = _submit(B, srv, _request(2, 2, 1), 2)
    B.bd_server_drain(srv)
    assert B.bd_server_request(srv, i)["state"] == B.BD_ENOMEM
    with pytest.raises(B.BidomainError):
        B.bd_server_result(srv, i)


def test_served_simulation_matches_oracle(B, oracle_lib):
    m, fib, stim = _request(16, 16, 8)
    p = W.DEFAULT_PARAMS
    srv = B.bd_server_create()
    i = B.bd_server_submit(srv, m, p, fib, stim, 1.0, 25)
    B.bd_server_drain(srv)
    gv, gu, gw = B.bd_server_result(srv, i)
    o = oracle_lib.assemble(m, p, fib)
    H = oracle_lib.Hierarchy(o["A"])
    N = W.n_nodes(m)
    v, ue, w = np.zeros(N), np.zeros(N), np.zeros(N)
    for k in range(25):
        H.bd_step(o["M"], p, stim if k * p["dt"] < 1.0 else np.zeros(N), v, ue, w)
    for a_, b_ in ((gv, v), (gu, ue), (gw, w)):
        assert np.linalg.norm(a_ - b_) <= 1e-6 * np.linalg.norm(b_)
