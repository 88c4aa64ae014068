"""Choose the V-cycle's operator forms by timing them inside V-cycles.

The library picks the form of every coarse operator (block-CSR lanes per row
or the sliced block form, see amg_level_lanes) from a rule, or with
amg_options.autotune from single-launch timings at setup.  Single launches do
not rank every operator the way the V-cycle (Algorithm 2) runs it, so this
module times each candidate form where it matters: inside whole V-cycles,
through the library's per-step breakdown (amg_profile_enable level 2), one
operator at a time, the others left as they are.  It only sequences calls of
the C ABI; every timed step runs in the library's kernels.
"""
from __future__ import annotations

from . import binding as B

#: breakdown roles of each operator: A (four smoothing/residual steps), R, P
ROLES = {0: ("pre", "residual", "post1", "post2"), 1: ("restrict",), 2: ("prolong",)}
#: block-CSR lane counts and sliced forms (-K) tried by default
CANDIDATES = (1, 2, 4, 8, 16, 32, 64, 128, -1, -2, -4, -8)


def _operators(h):
    nl = B.amg_num_levels(h)
    for level in range(nl - 1):
        for op in (0, 1, 2):
            if op == 0 and level == 0:
                continue  # the finest A: sliced ELL, or block-CSR fused with the PCG
            yield level, op


def _valid(level: int, op: int, form: int) -> bool:
    if form > 0:
        return form <= 256 and form & (form - 1) == 0
    return -form in (1, 2, 4, 8) and not (op == 0 and level == 0)


def time_forms(h, r, candidates=CANDIDATES, reps: int = 5, warm: int = 2, stream=None) -> dict:
    """Microseconds per V-cycle of every candidate form of every coarse
    operator: {(level, op): {form: us}} (op 0 = A, 1 = R, 2 = P).  r: the
    V-cycle input (numpy array or CUDA tensor, 2N values).  Every operator is
    left in the form it had on entry."""
    # a CUDA tensor input needs a device output of the same shape
    z = r.new_empty(r.shape) if getattr(r, "is_cuda", False) else None
    table = {}
    for level, op in _operators(h):
        start = B.amg_level_lanes(h, level)[op]
        row = {}
        try:
            for form in candidates:
                if not _valid(level, op, form):
                    continue
                lanes = [0, 0, 0]
                lanes[op] = form
                B.amg_set_level_lanes(h, level, lanes, stream=stream)
                for _ in range(warm):
                    B.amg_vcycle(h, r, z, stream=stream)
                B.amg_profile_enable(h, 2)
                try:
                    for _ in range(reps):
                        B.amg_vcycle(h, r, z, stream=stream)
                    bd = B.amg_profile_breakdown(h)
                finally:
                    B.amg_profile_enable(h, 0)
                row[form] = sum(1000.0 * bd[f"L{level}_{role}"][0] / bd[f"L{level}_{role}"][1]
                                for role in ROLES[op])
        finally:
            # the operator goes back to its starting form even when a candidate
            # failed (e.g. BD_ENOMEM while building a sliced form)
            lanes = [0, 0, 0]
            lanes[op] = start
            B.amg_set_level_lanes(h, level, lanes, stream=stream)
        table[(level, op)] = row
    return table


def tune_forms(h, r, candidates=CANDIDATES, reps: int = 5, keep_within: float = 0.03,
               stream=None) -> dict:
    """Time the candidates (time_forms) and set every operator to its fastest
    form, keeping the current one when it is within keep_within of the best
    (near-ties then resolve the same way on every run).  Returns the table and
    the forms chosen: {"times": ..., "forms": {(level, op): form}}.  The
    choice, like the library's, is fixed for the hierarchy afterwards, so its
    solves stay reproducible."""
    times = time_forms(h, r, candidates, reps=reps, stream=stream)
    chosen = {}
    for (level, op), row in times.items():
        current = B.amg_level_lanes(h, level)[op]
        best = min(row, key=row.get)
        keep = current in row and row[current] <= (1.0 + keep_within) * row[best]
        form = current if keep else best
        lanes = [0, 0, 0]
        lanes[op] = form
        B.amg_set_level_lanes(h, level, lanes, stream=stream)
        chosen[(level, op)] = form
    return {"times": times, "forms": chosen}
