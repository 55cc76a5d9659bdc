"""Pins of the oracle's first-order one-stage scheme and local time stepping
(Section 5.2: the time-accurate session's first-order 1-stage scheme at CFL
0.85, and the steady-state session advanced with local time steps).  CPU only.
"""
import copy
import math

import numpy as np
import pytest

from oracle import oracle as O
from paper_2501_06717_gb300 import workloads as W


def _l1(a, b):
    return float(np.abs(np.asarray(a) - np.asarray(b)).mean())


def _with(q, **kw):
    q2 = copy.copy(q)
    for k, v in kw.items():
        setattr(q2, k, v)
    return q2


def test_first_order_sound_wave_converges_at_first_order():
    """No slopes (piecewise-constant faces) with the one-stage scheme: the L1
    error of a linear sound wave halves per refinement (order near 1), where
    the limited second-order scheme reaches 2."""
    errs = []
    for n in (32, 64, 128):
        q = _with(W.sound_wave(0, n, limiter=W.LIM_NONE), rk=W.RK_EULER)
        steps = int(round(0.5 / (0.2 / n)))
        U, _, t = O.run(q, q.U0, steps, dt=0.5 / steps)
        errs.append(_l1(U, W.sound_wave(0, n, t_shift=t).U0))
    orders = [math.log2(errs[i] / errs[i + 1]) for i in range(2)]
    assert errs[0] > errs[1] > errs[2]
    assert 0.8 <= orders[-1] <= 1.3, (errs, orders)


@pytest.mark.parametrize("rk", [W.RK_EULER, W.RK_MIDPOINT])
def test_first_order_rusanov_keeps_a_contact_within_its_bounds(rk):
    """A density step moving with a uniform flow (uniform p, B = 0): the
    first-order Rusanov scheme is monotone at CFL <= 1, so rho never leaves
    [rho_min, rho_max], and the step does spread (it is not frozen)."""
    n = 64
    q = W._line_problem("contact", 0, n, limiter=W.LIM_NONE)
    q.rk = rk
    X = W.cell_centres(q.lo, q.hi, q.root, q.leaves)
    rho = np.where((X[0] > 0.25) & (X[0] < 0.5), 2.0, 1.0)
    one = np.ones_like(rho)
    q = W.with_state(q, [rho, 0.7 * one, 0 * one, 0 * one, 0 * one, 0 * one, 0 * one, one])
    q.rk = rk
    U, _, _ = O.run(q, q.U0, 60, cfl=0.85)
    assert U[0].min() >= 1.0 - 1e-12 and U[0].max() <= 2.0 + 1e-12
    inner = (U[0] > 1.05) & (U[0] < 1.95)
    assert inner.sum() > 8 * 64


@pytest.mark.parametrize("limiter", [W.LIM_NONE, W.LIM_MINMOD])
def test_one_stage_step_is_one_stage_with_the_cfl_dt(limiter):
    q = _with(W.blast(), limiter=limiter, rk=W.RK_EULER)
    dt = 0.85 / O.cfl_smax(q, q.U0)
    U1, dtl, t = O.run(q, q.U0, 1, cfl=0.85)
    assert dtl == dt and t == dt
    assert np.array_equal(U1, O.stage(q, q.U0, q.U0, 0, dt))


def test_first_order_uniform_state_and_conservation():
    lv = W.random_amr_tree(5, root=(3, 3, 3), periodic=True, frac=0.3)
    q = W.Problem("u", (0, 0, 0), (1, 1, 1), (3, 3, 3), lv, (W.BC_PERIODIC,) * 6, limiter=W.LIM_NONE,
                  rk=W.RK_EULER)
    W.uniform_state(q, [1.3, 0.4, -0.2, 0.3, 0.7, -0.5, 0.25, 0.9])
    U, _, _ = O.run(q, q.U0, 3, cfl=0.85)
    assert np.array_equal(U, q.U0)
    # conservation on a uniform periodic grid with a non-trivial state
    qo = _with(W.orszag_tang(), limiter=W.LIM_NONE, rk=W.RK_EULER)
    U, _, _ = O.run(qo, qo.U0, 5, cfl=0.85)
    s0 = qo.U0.reshape(8, -1).sum(1)
    s1 = U.reshape(8, -1).sum(1)
    scale = np.abs(qo.U0).reshape(8, -1).sum(1) + 1e-300
    assert (np.abs(s1 - s0) / scale).max() < 1e-13


def test_local_dt_is_the_cfl_bound_of_each_cell():
    """dt_i = cfl / s_i: its smallest value is the global CFL dt, every dt_i
    times the cell's own speed bound gives cfl, and on an AMR grid with a
    uniform state the finer cells get exactly half the coarser cells' dt."""
    q = W.magnetosphere()
    dtc = O.local_dt(q, q.U0, 0.6)
    X = W.cell_centres(q.lo, q.hi, q.root, q.leaves)
    body = (X[0] ** 2 + X[1] ** 2 + X[2] ** 2 < q.body_r ** 2).reshape(q.nb, 512)
    assert np.all(dtc[body] == 0.0) and np.all(dtc[~body] > 0.0)
    assert dtc[~body].min() == pytest.approx(0.6 / O.cfl_smax(q, q.U0), rel=1e-15)
    lv = W.random_amr_tree(6, root=(3, 3, 3), periodic=True, frac=0.3)
    qu = W.Problem("u", (0, 0, 0), (1, 1, 1), (3, 3, 3), lv, (W.BC_PERIODIC,) * 6)
    W.uniform_state(qu, [1.3, 0.4, -0.2, 0.3, 0.7, -0.5, 0.25, 0.9])
    d = O.local_dt(qu, qu.U0, 0.8)
    lev = np.asarray(qu.leaves)[:, 0]
    for l in np.unique(lev):
        vals = d[lev == l]
        assert np.all(vals == vals.flat[0])
    top = d[lev == lev.min()].flat[0]
    for l in np.unique(lev):
        assert d[lev == l].flat[0] == pytest.approx(top / 2.0 ** (l - lev.min()), rel=1e-15)


def test_local_time_step_is_the_per_cell_update():
    """One local-time-step Euler step: every cell moves by its own dt_i times
    the residual of the step's initial state; the midpoint scheme's first
    stage uses dt_i / 2 the same way."""
    q = _with(W.blast(), local_dt=1, rk=W.RK_EULER, limiter=W.LIM_MINMOD)
    dtc = O.local_dt(q, q.U0, 0.6)
    R = O.residual(q, q.U0)
    U1, _, _ = O.run(q, q.U0, 1, cfl=0.6)
    dt_cell = dtc.reshape(1, q.nb, 8, 8, 8)
    expect = q.U0 + dt_cell * R
    assert np.abs(U1 - expect).max() <= 1e-14 * np.abs(q.U0).max()
    qm = _with(q, rk=W.RK_MIDPOINT)
    Us = O.stage(qm, q.U0, q.U0, 0, 0.5, dtc=dtc)
    assert np.abs(Us - (q.U0 + 0.5 * dt_cell * R)).max() <= 1e-14 * np.abs(q.U0).max()


def test_local_time_stepping_equals_global_when_all_speeds_agree():
    """A shear layer (u_y = +-0.3 in x) on a uniform grid: every cell has the
    same speed bound, so dt_i is the global dt and the first steps are
    bitwise equal (the residual is not zero: Rusanov diffuses the shear)."""
    q = W._line_problem("shear", 0, 32)
    X = W.cell_centres(q.lo, q.hi, q.root, q.leaves)
    one = np.ones_like(X[0])
    uy = np.where(np.sin(2 * np.pi * X[0]) > 0, 0.3, -0.3)
    q = W.with_state(q, [one, 0 * one, uy, 0 * one, 0.5 * one, 0 * one, 0 * one, one])
    for rk in (W.RK_MIDPOINT, W.RK_EULER):
        qr = _with(q, rk=rk)
        Ug, _, _ = O.run(qr, q.U0, 1, cfl=0.8)
        Ul, _, _ = O.run(_with(qr, local_dt=1), q.U0, 1, cfl=0.8)
        assert not np.array_equal(Ug, q.U0)
        assert np.array_equal(Ug, Ul)


def test_local_time_stepping_reaches_the_same_steady_state_sooner():
    """Inflow at -x, outflow at +x, one refined root block: a pressure and
    density bump is swept out and both runs settle to the uniform inflow
    state (which each preserves exactly); with local steps the coarse cells
    are not held to the fine cells' dt and after the same number of steps the
    local-step run is far closer to it."""
    def inside(b0, b1, p=(0.7, 0.3, 0.3)):
        return all(b0[a] <= p[a] < b1[a] for a in range(3))
    lv = W.refine_where(W.uniform_leaves((4, 2, 2)), inside, (0, 0, 0), (2, 1, 1), (4, 2, 2), 1)
    lv = W.as_leaf_array(W.balance(lv, (4, 2, 2), (False, True, True)))
    bc = (W.BC_INFLOW, W.BC_OUTFLOW, W.BC_PERIODIC, W.BC_PERIODIC, W.BC_PERIODIC, W.BC_PERIODIC)
    q = W.Problem("channel", (0, 0, 0), (2, 1, 1), (4, 2, 2), lv, bc, limiter=W.LIM_MINMOD)
    inflow = np.array([1.0, 1.5, 0.0, 0.0, 0.3, 0.2, 0.0, 1.0])
    X = W.cell_centres(q.lo, q.hi, q.root, q.leaves)
    bump = 0.2 * np.exp(-40 * ((X[0] - 1.2) ** 2 + (X[1] - 0.5) ** 2))
    q = W.with_state(q, [inflow[v] + (bump if v in (0, 7) else 0 * X[0]) for v in range(8)])
    q.inflow = inflow
    target = W.with_state(q, [inflow[v] + 0 * X[0] for v in range(8)]).U0
    Ut, _, _ = O.run(_with(q, local_dt=1), target, 5, cfl=0.6)
    assert np.array_equal(Ut, target)
    Ug, _, _ = O.run(q, q.U0, 1000, cfl=0.6)
    Ul, _, _ = O.run(_with(q, local_dt=1), q.U0, 1000, cfl=0.6)
    eg, el = _l1(Ug, target), _l1(Ul, target)
    e0 = _l1(q.U0, target)
    assert el < 0.05 * e0, (e0, eg, el)
    assert el < 0.25 * eg, (e0, eg, el)
