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
    assert best == (1, 4, 0)
    assert dict(table)[(1, 4, 0)] == pytest.approx(3.0)
    assert s.calls[-1] == ("set_launch", 1, 4, 0, 1)
    # every candidate timed with eager launches (per-stage events) after one warm step
    tuned = [c for c in s.calls if c[0] == "set_launch"][:-1]
    assert [c[1:4] for c in tuned] == A.DEFAULT_CANDIDATES and all(c[4] == 0 for c in tuned)


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
                assert best in A.DEFAULT_CANDIDATES and len(table) == len(A.DEFAULT_CANDIDATES)
                s.set_state(0, q.U0)
            s.step(3, 0.8)
            outs.append(s.get_state(0))
    assert np.array_equal(outs[0], outs[1])
