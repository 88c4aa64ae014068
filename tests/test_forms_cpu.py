"""Host logic of the in-V-cycle form tuner (paper_2311_13914_gb300.forms)
against a stand-in for the library: which operators and forms it visits, that
time_forms restores the forms it found, and how tune_forms picks (fastest, the
current form on a near-tie)."""
import pytest

from paper_2311_13914_gb300 import forms


class FakeLib:
    """Three levels; the breakdown reports a time per step that depends on the
    form of the operator the step applies."""

    def __init__(self, cost):
        self.nl = 3
        self.lanes = {0: [0, 4, 1], 1: [4, 32, 4], 2: [0, 0, 0]}
        self.cost = cost          # (level, op, form) -> us per launch
        self.prof = 0
        self.sums = {}
        self.sets = []

    def amg_num_levels(self, h):
        return self.nl

    def amg_level_lanes(self, h, level):
        return tuple(self.lanes[level])

    def amg_set_level_lanes(self, h, level, lanes, stream=None):
        for op, t in enumerate(lanes):
            if t:
                assert not (level == 0 and op == 0)
                assert forms._valid(level, op, t)
                self.lanes[level][op] = t
        self.sets.append((level, tuple(lanes)))

    def amg_vcycle(self, h, r, z=None, stream=None):
        if self.prof < 2:
            return
        for level in range(self.nl - 1):
            for op, roles in forms.ROLES.items():
                if level == 0 and op == 0:
                    roles = ("pre", "residual", "post1", "post2")  # the finest A: not tuned
                for role in roles:
                    us = self.cost(level, op, self.lanes[level][op])
                    ms, n = self.sums.get(f"L{level}_{role}", (0.0, 0))
                    self.sums[f"L{level}_{role}"] = (ms + us / 1000.0, n + 1)

    def amg_profile_enable(self, h, enable):
        if enable and not self.prof:
            self.sums = {}
        self.prof = enable

    def amg_profile_breakdown(self, h):
        return dict(self.sums)


@pytest.fixture
def fake(monkeypatch):
    def make(cost):
        lib = FakeLib(cost)
        monkeypatch.setattr(forms, "B", lib)
        return lib
    return make


def test_time_forms_visits_coarse_operators_and_restores(fake):
    lib = fake(lambda level, op, form: 10.0 + abs(form))
    start = {l: list(v) for l, v in lib.lanes.items()}
    t = forms.time_forms(None, None, candidates=(1, 4, 16, -1, -16), reps=3, warm=1)
    assert set(t) == {(0, 1), (0, 2), (1, 0), (1, 1), (1, 2)}
    for (level, op), row in t.items():
        assert set(row) == {1, 4, 16, -1}            # -16 is not a sliced form
        n = len(forms.ROLES[op])
        for form, us in row.items():
            assert us == pytest.approx(n * (10.0 + abs(form)))
    assert lib.lanes == start


def test_tune_forms_takes_the_fastest_and_keeps_near_ties(fake):
    # level 1's A: the current form 4 is 2 % slower than sliced 4 (kept);
    # level 0's P: sliced 1 is 20 % faster than the current form 1 (taken)
    def cost(level, op, form):
        if (level, op) == (1, 0):
            return {4: 10.2, -4: 10.0}.get(form, 30.0)
        if (level, op) == (0, 2):
            return {1: 12.0, -1: 10.0}.get(form, 30.0)
        return 20.0 - (form == 32) * 5.0
    lib = fake(cost)
    out = forms.tune_forms(None, None, candidates=(1, 4, 32, -1, -4), reps=2)
    assert out["forms"][(1, 0)] == 4
    assert out["forms"][(0, 2)] == -1
    assert out["forms"][(0, 1)] == 32 and out["forms"][(1, 1)] == 32
    for (level, op), form in out["forms"].items():
        assert lib.lanes[level][op] == form
    assert lib.lanes[0][0] == 0                      # the finest A untouched


def test_time_forms_restores_the_starting_form_when_a_candidate_fails(fake):
    lib = fake(lambda level, op, form: 10.0)
    start = {l: list(v) for l, v in lib.lanes.items()}
    real_set = lib.amg_set_level_lanes

    def failing_set(h, level, lanes, stream=None):
        if level == 1 and lanes[0] == -2:
            # the library's own fallback after a failed sliced build
            lib.lanes[1][0] = 4
            raise RuntimeError("amg_set_level_lanes: out of memory")
        real_set(h, level, lanes, stream)
    lib.amg_set_level_lanes = failing_set
    with pytest.raises(RuntimeError):
        forms.time_forms(None, None, candidates=(1, 8, -2), reps=1, warm=0)
    assert lib.lanes == start
    assert lib.sets[-1] == (1, (start[1][0], 0, 0))
