"""Write large_slab_oracle.json: the oracle's solve of the 256x256x64 slab.

The full-size slab (8,586,370 unknowns) is the size at which the FP32 V-cycle
form is compared with the FP64 form (Section 4's V-cycle inside PCG; the
flexible CG for the FP32 V-cycle).  The oracle takes minutes there, so it runs
once, here, and the GPU test compares against what this script stores:
iteration count, residuals, norms and the solution at seeded sample indices.

Inputs (same recipe as the GPU test): Q1 slab 1 x 1 x 0.5 cm, fibres rotating
120 degrees through the thickness with the offset drawn from seed 1, right-hand
side N(0,1) from PCG64 seed 0 with the u_e mean removed, rtol 1e-8 on the
recurrence residual, oracle defaults for the hierarchy.

Run from the repository root:  python tests/golden/make_large_slab_oracle.py
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

N_SAMPLES = 512


def main():
    mesh = W.SLAB_LARGE
    off = W.fibre_offset_from_seed(1)
    fib = W.fibre_table(mesh, 120.0, off)
    t0 = time.time()
    sysd = oracle.assemble(mesh, W.DEFAULT_PARAMS, fib)
    A = sysd["A"]
    t1 = time.time()
    H = oracle.Hierarchy(A)
    t2 = time.time()
    n = A.shape[0]
    f = W.rhs(n, 0)
    x, info = H.pcg(f, rtol=1e-8)
    t3 = time.time()
    idx = np.sort(np.random.Generator(np.random.PCG64(11)).choice(n, N_SAMPLES, replace=False))
    out = {
        "what": "oracle AMG-PCG solve of the 256x256x64 Q1 Bidomain slab (coupled block system)",
        "mesh": mesh, "fibre_rotation_deg": 120.0, "fibre_offset_deg": off,
        "rhs": "PCG64 seed 0 standard_normal, u_e mean removed", "rtol": 1e-8,
        "levels": [int(H.A(l).shape[0]) for l in range(H.nlevels)],
        "status": info["status"], "iters": info["iters"], "rel_res": info["rel_res"],
        "true_rel_res": info["true_rel_res"],
        "norm2_x": float(np.linalg.norm(x)), "max_abs_x": float(np.abs(x).max()),
        "sample_index": idx.tolist(), "sample_x": x[idx].tolist(),
        "seconds": {"assemble": t1 - t0, "setup": t2 - t1, "solve": t3 - t2},
    }
    dst = os.path.join(os.path.dirname(os.path.abspath(__file__)), "large_slab_oracle.json")
    with open(dst, "w") as fh:
        json.dump(out, fh, indent=1)
    print(dst, out["iters"], out["seconds"])


if __name__ == "__main__":
    main()
