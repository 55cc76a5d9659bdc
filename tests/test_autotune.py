"""The launch autotuner: picks the fastest candidate by the library's stage
timings and leaves the handle in that form (CPU, with a stand-in solver), and
on the GPU leaves results unchanged (every launch form is bitwise equal)."""
import numpy as np
import pytest

from paper_2501_06717_gb300 import autotune as A
from paper_2501_06717_gb300 import workloads as W


class _FakeSolver:
    """Stage time per launch form from a table; records the calls."""

    def __init__(self, cost):
        self.cost = cost
        self.form = None
        self.calls = []

    def set_launch(self, persistent=0, blocks_per_cta=1, ctas_per_sm=0, use_graph=0):
        self.form = (persistent, blocks_per_cta, ctas_per_sm)
        self.calls.append(("set_launch", persistent, blocks_per_cta, ctas_per_sm, use_graph))

    def step(self, n, cfl):
        self.calls.append(("step", n))
        self.last_n = n

    def timings(self):
        from paper_2501_06717_gb300 import bats as B
        t = [0.0, 0.0, 0.0]
        t[B.BATS_PHASE_STAGE] = self.cost[self.form] * self.last_n
        return t


def test_autotune_picks_the_fastest_form_and_enables_the_graph():
    cost = {c: 10.0 + i for i, c in enumerate(A.DEFAULT_CANDIDATES)}
    cost[(1, 4, 0)] = 3.0
    s = _FakeSolver(cost)
    best, table = A.autotune(s, 0.8, steps=3)
    assert best == (1, 4, 0, None)      # no staging knob on this handle
    assert dict(table)[(1, 4, 0, None)] == pytest.approx(3.0)
    assert s.calls[-1] == ("set_launch", 1, 4, 0, 1)
    # every candidate timed with eager launches (per-stage events) after one warm step
    tuned = [c for c in s.calls if c[0] == "set_launch"][:-1]
    assert [c[1:4] for c in tuned] == A.DEFAULT_CANDIDATES and all(c[4] == 0 for c in tuned)


class _FakeMixedSolver(_FakeSolver):
    """A mixed-form handle: stage time per (launch form, staging layout)."""

    def __init__(self, cost):
        super().__init__(cost)
        from paper_2501_06717_gb300 import bats as B
        self.precision = B.BATS_MIXED
        self.st = None

    def set_staging(self, tma):
        self.st = tma
        self.calls.append(("set_staging", tma))

    def timings(self):
        from paper_2501_06717_gb300 import bats as B
        t = [0.0, 0.0, 0.0]
        t[B.BATS_PHASE_STAGE] = self.cost[self.form + (self.st,)] * self.last_n
        return t


@pytest.mark.parametrize("winner", [(0, 2, 0, 0), (1, 8, 0, 1)])
def test_autotune_sweeps_the_staging_layouts_of_a_mixed_handle(winner):
    cost = {tuple(c) + (st,): 10.0 + i + 0.5 * st for st in A.STAGING_LAYOUTS
            for i, c in enumerate(A.DEFAULT_CANDIDATES)}
    cost[winner] = 1.0
    s = _FakeMixedSolver(cost)
    best, table = A.autotune(s, 0.8, steps=2)
    assert best == winner
    assert len(table) == len(A.DEFAULT_CANDIDATES) * len(A.STAGING_LAYOUTS)
    assert {k[3] for k, _ in table} == set(A.STAGING_LAYOUTS)
    # the handle is left in the winner's staging layout and launch form, graph on
    assert s.st == winner[3]
    assert s.calls[-1] == ("set_launch",) + winner[:3] + (1,)


@pytest.mark.gpu
def test_autotuned_handle_gives_the_same_result():
    from paper_2501_06717_gb300 import bats as B
    q = W.blast()
    outs = []
    for tune in (False, True):
        with B.Solver(q, precision=B.BATS_MIXED) as s:
            s.set_state(0, q.U0)
            if tune:
                best, table = A.autotune(s, 0.8, steps=1)
                assert best[:3] in A.DEFAULT_CANDIDATES and best[3] in A.STAGING_LAYOUTS
                assert len(table) == len(A.DEFAULT_CANDIDATES) * len(A.STAGING_LAYOUTS)
                s.set_state(0, q.U0)
            s.step(3, 0.8)
            outs.append(s.get_state(0))
    assert np.array_equal(outs[0], outs[1])
