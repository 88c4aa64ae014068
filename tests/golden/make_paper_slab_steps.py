"""Write paper_slab_steps_oracle.json: the oracle's 100 time steps of the
128x128x32 slab.

The paper-size slab (1,098,306 unknowns) time-stepped from rest with the
corner stimulus is the benchmark's workload (Section 2.2, Eqs. 4-7 in the
coupled form: Rogers-McCulloch update, then one AMG-PCG solve of the block
system per step, warm-started from the previous step).  The oracle takes
about ten minutes for the 100 steps, so it runs once, here, and the GPU test
compares against what this script stores: per-step iteration counts, the
norms of v, u_e and w, their values at seeded sample indices, and their
projections on seeded random vectors (which see every entry).

Inputs (same recipe as the benchmark): Q1 slab 1 x 1 x 0.5 cm, fibres
rotating 120 degrees through the thickness with the offset drawn from seed 1,
v = u_e = w = 0 at t = 0, stimulus 8e4 uA/cm^3 on the 0.1 cm corner cube while
t < 1 ms, dt = 0.05 ms, rtol 1e-8, hierarchy options as the oracle's defaults
except a coarsest level of up to 2000 unknowns (the benchmark's setting).

Run from the repository root:  python tests/golden/make_paper_slab_steps.py
Only oracle/ and the seeded input generators are called.
"""
import json
import os
import sys
import time

import numpy as np

ROOT = os.path.dirname(os.path.dirname(os.path.dirname(os.path.abspath(__file__))))
sys.path.insert(0, ROOT)

import oracle  # noqa: E402
from paper_2311_13914_gb300 import workloads as W  # noqa: E402

N_STEPS = 100
COARSE_EQ_LIMIT = 2000
N_SAMPLES = 1024
N_PROJ = 4


def projections(n):
    """Seeded unit-variance random directions (PCG64 seed 17)."""
    return np.random.Generator(np.random.PCG64(17)).standard_normal((N_PROJ, n))


def main():
    mesh = W.SLAB_PAPER
    p = W.DEFAULT_PARAMS
    off = W.fibre_offset_from_seed(1)
    fib = W.fibre_table(mesh, 120.0, off)
    stim = W.stimulus(mesh)
    t0 = time.time()
    sysd = oracle.assemble(mesh, p, fib)
    H = oracle.Hierarchy(sysd["A"], coarse_eq_limit=COARSE_EQ_LIMIT)
    t1 = time.time()
    N = W.n_nodes(mesh)
    v, ue, w = np.zeros(N), np.zeros(N), np.zeros(N)
    iters = []
    for k in range(N_STEPS):
        Iapp = stim if k * p["dt"] < 1.0 else np.zeros(N)
        info = H.bd_step(sysd["M"], p, Iapp, v, ue, w)
        assert info["status"] == 0, info
        iters.append(int(info["iters"]))
        print(k, info["iters"], flush=True)
    t2 = time.time()
    idx = np.sort(np.random.Generator(np.random.PCG64(13)).choice(N, N_SAMPLES, replace=False))
    # the stimulated corner and its neighbourhood, where the state varies most
    corner = np.flatnonzero(stim)[:64]
    idx = np.union1d(idx, corner)
    R = projections(N)
    fields = {}
    for name, a in (("v", v), ("ue", ue), ("w", w)):
        fields[name] = {"norm2": float(np.linalg.norm(a)), "max_abs": float(np.abs(a).max()),
                        "sample": a[idx].tolist(), "proj": (R @ a).tolist()}
    out = {
        "what": "oracle time stepping of the 128x128x32 Q1 Bidomain slab (coupled block system)",
        "mesh": mesh, "fibre_rotation_deg": 120.0, "fibre_offset_deg": off,
        "steps": N_STEPS, "dt": p["dt"], "stimulus": "8e4 uA/cm^3 on [0,0.1]^3 cm for t < 1 ms",
        "rtol": 1e-8, "coarse_eq_limit": COARSE_EQ_LIMIT,
        "levels": [int(H.A(l).shape[0]) for l in range(H.nlevels)],
        "iters": iters, "sample_index": idx.tolist(), "proj_seed": 17, "n_proj": N_PROJ,
        "fields": fields,
        "seconds": {"assemble_setup": t1 - t0, "steps": t2 - t1},
    }
    dst = os.path.join(os.path.dirname(os.path.abspath(__file__)), "paper_slab_steps_oracle.json")
    with open(dst, "w") as fh:
        json.dump(out, fh, indent=0)
    print(dst, sum(iters), out["seconds"])


if __name__ == "__main__":
    main()
