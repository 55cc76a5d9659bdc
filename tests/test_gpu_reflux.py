"""Refluxing (conservative flux correction at resolution changes) on the GPU
against the oracle, and exact conservation on a periodic AMR grid."""
import copy

import numpy as np
import pytest

from oracle import oracle as O
from paper_2501_06717_gb300 import workloads as W

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def B():
    from paper_2501_06717_gb300 import bats
    bats.lib()
    return bats


def _with(q, **kw):
    q2 = copy.copy(q)
    for k, v in kw.items():
        setattr(q2, k, v)
    return q2


def _scaled(g, o):
    g = np.asarray(g).reshape(8, -1)
    o = np.asarray(o).reshape(8, -1)
    s = np.abs(o).max(1)
    s[1:4] = s[1:4].max()
    s[4:7] = s[4:7].max()
    s = np.where(s > 0, s, 1.0)
    return np.abs(g - o).max(1) / s


def _amr(seed, periodic=True, powell=0, limiter=W.LIM_MC):
    lv = W.random_amr_tree(seed, root=(3, 3, 3), periodic=periodic, frac=0.3)
    bc = (W.BC_PERIODIC,) * 6 if periodic else (W.BC_OUTFLOW, W.BC_INFLOW, W.BC_OUTFLOW, W.BC_OUTFLOW,
                                                  W.BC_INFLOW, W.BC_OUTFLOW)
    q = W.Problem("amr", (-1, -1, -1), (1, 1, 1), (3, 3, 3), lv, bc, limiter=limiter, powell=powell)
    q.inflow = np.array([1.1, 0.2, -0.1, 0.05, 0.3, 0.1, -0.2, 0.8])
    X = W.cell_centres(q.lo, q.hi, q.root, q.leaves)
    tp = 2 * np.pi
    q = W.with_state(q, [1 + 0.3 * np.sin(tp * X[0] / 2) * np.cos(tp * X[1] / 2), 0.3 * np.cos(tp * X[2] / 2),
                         0.2 * np.sin(tp * X[0] / 2), -0.1 + 0 * X[0], 0.4 * np.sin(tp * X[1] / 2),
                         0.3 + 0.1 * np.cos(tp * X[2] / 2), 0.2 * np.cos(tp * X[0] / 2),
                         1 + 0.2 * np.cos(tp * (X[0] + X[2]) / 2)])
    q.inflow = np.array([1.1, 0.2, -0.1, 0.05, 0.3, 0.1, -0.2, 0.8])
    return q


CASES = {
    "amr_periodic_midpoint": lambda: _with(_amr(3), reflux=1),
    "amr_inflow_powell_ssp": lambda: _with(_amr(4, periodic=False, powell=1), reflux=1, rk=W.RK_SSP2),
    "magnetosphere": lambda: _with(W.magnetosphere(), reflux=1),
    "amr_local_dt_first_order": lambda: _with(_amr(5), reflux=1, local_dt=1, rk=W.RK_EULER, limiter=W.LIM_NONE),
}


@pytest.mark.parametrize("case", sorted(CASES))
def test_fp64_refluxing_matches_oracle(B, case):
    q = CASES[case]()
    n = 3 if case == "magnetosphere" else 8
    cfl = 0.8
    with B.Solver(q) as s:
        s.set_state(0, q.U0)
        s.step(n, cfl)
        Ug = s.get_state(0)
        tg = s.time(0)
    Uo, _, to = O.run(q, q.U0, n, cfl=cfl)
    err = _scaled(Ug, Uo)
    print(case, "FP64 scaled error per variable", err)
    assert err.max() <= 1e-12, err
    assert tg == pytest.approx(to, rel=1e-13)
    Un, _, _ = O.run(_with(q, reflux=0), q.U0, n, cfl=cfl)
    assert _scaled(Un, Uo).max() > 1e-9   # refluxing does change these runs


@pytest.mark.parametrize("case", ["amr_periodic_midpoint", "magnetosphere"])
def test_mixed_refluxing_one_step(B, case):
    q = CASES[case]()
    with B.Solver(q, precision=B.BATS_MIXED) as s:
        s.set_state(0, q.U0)
        s.step(1, 0.8)
        Ug = s.get_state(0)
    Uo, _, _ = O.run(q, q.U0, 1, cfl=0.8)
    err = _scaled(Ug, Uo)
    print(case, "mixed scaled error per variable", err)
    assert err.max() <= 1e-5, err


@pytest.mark.parametrize("prec", [0, 1])
def test_refluxing_conserves_on_the_gpu(B, prec):
    """Totals of the 8 conserved variables over 10 steps: FP64 to round-off;
    the mixed form's per-cell residual is an FP32 sum of FP32 face-flux
    differences, so there the totals drift at the FP32 rounding of dt R
    (bound 1e-10 relative, against 1e-7 and more without refluxing)."""
    q = CASES["amr_periodic_midpoint"]()
    lev = np.asarray(q.leaves)[:, 0]
    vol = (2.0 / 24.0) ** 3 / 8.0 ** lev

    def totals(U):
        return (np.asarray(U).reshape(8, q.nb, 512) * vol[None, :, None]).sum(axis=(1, 2))

    with B.Solver(q, precision=prec, persistent=1, use_graph=1) as s:
        s.set_state(0, q.U0)
        s.step(10, 0.8)
        U = s.get_state(0)
    t0 = totals(q.U0)
    assert np.abs(totals(U) - t0).max() <= (1e-13 if prec == 0 else 1e-10) * np.abs(t0).max()


def test_graph_replay_equals_eager_with_refluxing(B):
    q = CASES["amr_local_dt_first_order"]()
    outs = []
    for graph in (0, 1):
        with B.Solver(q, persistent=graph, use_graph=graph) as s:
            s.set_state(0, q.U0)
            s.step(3, 0.8)
            s.step(3, 0.8)
            outs.append(s.get_state(0))
    assert np.array_equal(outs[0], outs[1])


def test_refluxing_with_learned_is_rejected(B):
    q = _with(W.blast(), reflux=1, learned=1)
    with pytest.raises(B.BatsError):
        B.Solver(q)
