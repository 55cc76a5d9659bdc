"""Pins of the oracle's HLL flux option (two-state Harten-Lax-van Leer flux
with Davis wave-speed bounds), the stand-in for the Linde flux that the
paper's solver uses (Section 5; the paper does not print it).  Each pin is a
fact fixed by the mathematics of HLL, not a retyping of its formula."""
import math

import numpy as np
import pytest

from oracle import oracle as O
from paper_2501_06717_gb300 import workloads as W


def _face_problem(flux, gamma=5.0 / 3.0):
    q = W.uniform_state(W.Problem("face", (0, 0, 0), (1, 1, 1), (1, 1, 1), W.as_leaf_array([(0, 0, 0, 0)]),
                                  (W.BC_PERIODIC,) * 6, gamma=gamma), [1, 0, 0, 0, 0, 0, 0, 1])
    q.flux = flux
    return q


def _rot(direction, wn, wt1, wt2):
    """A vector with normal component wn along `direction` and the two
    tangential ones in cyclic order."""
    v = [0.0, 0.0, 0.0]
    v[direction] = wn
    v[(direction + 1) % 3] = wt1
    v[(direction + 2) % 3] = wt2
    return v


def _prim(rho, u, B, p):
    return np.array([rho, *u, *B, p], dtype=np.float64)


def _physical_flux(direction, Wf, gamma=5.0 / 3.0):
    # with identical face states the Rusanov flux is the physical flux exactly:
    # (F + F)/2 - cmax * 0 / 2 = F
    return O.numerical_flux(_face_problem(W.FLUX_RUSANOV, gamma), direction, Wf, Wf)


@pytest.mark.parametrize("direction", [0, 1, 2])
def test_supersonic_faces_take_the_upwind_physical_flux_exactly(direction):
    """When every wave moves right (S_L >= 0) HLL is F_L, when every wave
    moves left (S_R <= 0) it is F_R, bitwise."""
    hll = _face_problem(W.FLUX_HLL)
    WL = _prim(1.0, _rot(direction, 3.0, 0.2, -0.1), _rot(direction, 0.1, 0.2, 0.05), 0.2)
    WR = _prim(0.7, _rot(direction, 2.5, -0.3, 0.4), _rot(direction, 0.1, -0.2, 0.1), 0.15)
    assert np.array_equal(O.numerical_flux(hll, direction, WL, WR), _physical_flux(direction, WL))
    WLm = WL.copy()
    WRm = WR.copy()
    WLm[1 + direction] *= -1
    WRm[1 + direction] *= -1
    assert np.array_equal(O.numerical_flux(hll, direction, WLm, WRm), _physical_flux(direction, WRm))
    # and neither is the Rusanov flux, which adds dissipation regardless
    rus = O.numerical_flux(_face_problem(W.FLUX_RUSANOV), direction, WL, WR)
    assert np.abs(rus - _physical_flux(direction, WL)).max() > 0.1


@pytest.mark.parametrize("direction", [0, 1, 2])
def test_symmetric_wave_speeds_give_the_rusanov_flux(direction):
    """With S_L = -S_R (both states at rest along the normal with the same
    fast speed) HLL reduces to (F_L + F_R)/2 - S_R (U_R - U_L)/2, which is the
    Rusanov flux."""
    b = 0.5
    WL = _prim(1.2, _rot(direction, 0.0, 0.4, -0.3), _rot(direction, 0.3, 0.6 * b, 0.8 * b), 0.9)
    WR = _prim(1.2, _rot(direction, 0.0, -0.5, 0.2), _rot(direction, 0.3, 0.8 * b, -0.6 * b), 0.9)
    h = O.numerical_flux(_face_problem(W.FLUX_HLL), direction, WL, WR)
    r = O.numerical_flux(_face_problem(W.FLUX_RUSANOV), direction, WL, WR)
    assert np.abs(h - r).max() <= 1e-14 * np.abs(r).max()
    assert np.abs(h - _physical_flux(direction, WL)).max() > 1e-2  # a real jump


@pytest.mark.parametrize("seed", range(6))
def test_hll_flux_satisfies_the_jump_conditions_of_its_two_waves(seed):
    """HLL is the flux of a two-wave fan with one constant middle state
    U* = (S_R U_R - S_L U_L - (F_R - F_L)) / (S_R - S_L): the flux equals
    F_L + S_L (U* - U_L) and F_R + S_R (U* - U_R) (the Rankine-Hugoniot
    relations across the left and right waves)."""
    rng = np.random.default_rng(seed)
    gamma = 5.0 / 3.0
    d = int(rng.integers(0, 3))
    B0 = rng.uniform(-0.5, 0.5, 3)
    q = _face_problem(W.FLUX_HLL, gamma)
    WL = np.concatenate([[rng.uniform(0.5, 2)], rng.uniform(-0.5, 0.5, 3), rng.uniform(-1, 1, 3),
                         [rng.uniform(0.5, 2)]])
    WR = np.concatenate([[rng.uniform(0.5, 2)], rng.uniform(-0.5, 0.5, 3), rng.uniform(-1, 1, 3),
                         [rng.uniform(0.5, 2)]])
    F = O.numerical_flux(q, d, WL, WR, B0)
    # physical fluxes (identical-state Rusanov), states and wave-speed bounds
    r = _face_problem(W.FLUX_RUSANOV, gamma)
    FL = O.numerical_flux(r, d, WL, WL, B0)
    FR = O.numerical_flux(r, d, WR, WR, B0)
    UL = O.cons_from_prim(gamma, WL)
    UR = O.cons_from_prim(gamma, WR)
    cfL = O.fast_speed(gamma, WL, B0 + WL[4:7], d)
    cfR = O.fast_speed(gamma, WR, B0 + WR[4:7], d)
    SL = min(WL[1 + d] - cfL, WR[1 + d] - cfR)
    SR = max(WL[1 + d] + cfL, WR[1 + d] + cfR)
    assert SL < 0 < SR
    Us = (SR * UR - SL * UL - (FR - FL)) / (SR - SL)
    scale = np.abs(F).max() + np.abs(FL).max() + np.abs(FR).max()
    assert np.abs(F - (FL + SL * (Us - UL))).max() <= 1e-14 * scale
    assert np.abs(F - (FR + SR * (Us - UR))).max() <= 1e-14 * scale


@pytest.mark.parametrize("case", ["periodic_amr", "inflow_amr_b0"])
def test_uniform_state_preserved_bitwise_with_hll(case):
    periodic = case == "periodic_amr"
    lv = W.random_amr_tree(3, root=(3, 3, 3), periodic=periodic, frac=0.3)
    bc = (W.BC_PERIODIC,) * 6 if periodic else (W.BC_OUTFLOW,) * 6
    q = W.Problem(case, (-1, -1, -1), (1, 1, 1), (3, 3, 3), lv, bc, limiter=W.LIM_MC, powell=1,
                  flux=W.FLUX_HLL)
    Wu = [1.3, 0.4, -0.2, 0.3, 0.7, -0.5, 0.25, 0.9]
    if not periodic:
        q.bc = (W.BC_INFLOW, W.BC_OUTFLOW, W.BC_OUTFLOW, W.BC_INFLOW, W.BC_OUTFLOW, W.BC_OUTFLOW)
        q.inflow = np.array(Wu)
        q.b0 = W.B0_UNIFORM
        q.b0_param = np.array([0.3, -1.1, 0.6] + [0.0] * 9)
    W.uniform_state(q, Wu)
    U, dt, _ = O.run(q, q.U0, 2, cfl=0.8)
    assert dt > 0
    assert np.array_equal(U, q.U0)


def test_hll_conserves_every_total_on_a_periodic_grid():
    q = W.orszag_tang()
    q.flux = W.FLUX_HLL
    U, _, _ = O.run(q, q.U0, 5, cfl=0.8)
    s0 = q.U0.reshape(8, -1).sum(1)
    s1 = U.reshape(8, -1).sum(1)
    scale = np.abs(q.U0).reshape(8, -1).max(1) * q.U0[0].size
    assert np.all(np.abs(s1 - s0) <= 1e-14 * scale)
    q.flux = W.FLUX_RUSANOV
    Ur, _, _ = O.run(q, q.U0, 5, cfl=0.8)
    assert np.abs(U - Ur).max() > 1e-3  # the option changes the result


@pytest.mark.parametrize("n", [32, 64, 128])
def test_first_order_damping_of_a_carried_density_wave(n):
    """First order (piecewise-constant faces): a density wave carried by the
    flow u decays like exp(-nu k^2 t) with the numerical viscosity
    nu = D dx / 2, where D is the flux's dissipation coefficient for a wave
    moving at u: |u| + c_f for Rusanov, and for HLL
    ((S_R + S_L) u - 2 S_R S_L) / (S_R - S_L) = c_f (S = u -/+ c_f).  The L1
    error of rho is then A (1 - exp(-nu k^2 t)) 2/pi; both fluxes match it
    to 2 %, so HLL damps the wave (1 + |u|/c_f) times less at small nu."""
    gamma, u, A = 5.0 / 3.0, 1.0, 0.2
    a2, b2, bn2 = gamma, 0.14, 0.09  # rho = p = 1, B = (0.3, 0.2, 0.1) along x
    cf = math.sqrt(0.5 * (a2 + b2 + math.sqrt((a2 + b2) ** 2 - 4 * a2 * bn2)))
    k = 2 * math.pi
    errs = {}
    for flux, D in ((W.FLUX_RUSANOV, u + cf), (W.FLUX_HLL, cf)):
        q = W.entropy_wave(0, n, amplitude=A, speed=u, limiter=W.LIM_NONE)
        q.flux = flux
        steps = int(round(1.0 / (0.3 / n)))
        U, _, t = O.run(q, q.U0, steps, dt=1.0 / steps)
        ex = W.entropy_wave(0, n, amplitude=A, speed=u, t_shift=t).U0
        err = np.abs(U[0] - ex[0]).mean()
        pred = A * (1 - math.exp(-D * (1.0 / n) / 2 * k * k * t)) * 2 / math.pi
        assert abs(err / pred - 1) < 0.02, (flux, err, pred)
        errs[flux] = err
    assert errs[W.FLUX_HLL] < errs[W.FLUX_RUSANOV]


def test_second_order_hll_converges_on_a_carried_density_wave():
    errs = []
    for n in (32, 64, 128):
        q = W.entropy_wave(2, n, amplitude=0.05)
        q.flux = W.FLUX_HLL
        steps = int(round(1.0 / (0.3 / n)))
        U, _, t = O.run(q, q.U0, steps, dt=1.0 / steps)
        errs.append(np.abs(U - W.entropy_wave(2, n, amplitude=0.05, t_shift=t).U0).mean())
    orders = [math.log2(errs[i] / errs[i + 1]) for i in range(2)]
    assert orders[-1] >= 1.7, (errs, orders)


def test_brio_wu_with_hll_is_identical_along_each_axis():
    prof = []
    for axis in range(3):
        q = W.brio_wu(axis, ncells=64, nsteps=30)
        q.flux = W.FLUX_HLL
        U, _, _ = O.run(q, q.U0, q.nsteps, dt=1.1e-3)
        U6 = U.reshape(8, *q.root[::-1], 8, 8, 8)
        full = U6.transpose(0, 1, 4, 2, 5, 3, 6).reshape(8, q.root[2] * 8, q.root[1] * 8, q.root[0] * 8)
        line = [full[:, 0, 0, :], full[:, 0, :, 0], full[:, :, 0, 0]][axis]
        rot = [0, 1 + axis, 1 + (axis + 1) % 3, 1 + (axis + 2) % 3,
               4 + axis, 4 + (axis + 1) % 3, 4 + (axis + 2) % 3, 7]
        prof.append(line[rot])
    assert np.array_equal(prof[0], prof[1])
    assert np.array_equal(prof[0], prof[2])
    assert np.all(prof[0][0] > 0) and np.all(prof[0][7] > 0)


def test_hll_with_the_learned_correction_is_rejected():
    """The learned correction is clipped by the Rusanov dissipation, so it is
    defined on the Rusanov flux only; unknown flux kinds are rejected too."""
    q = W.orszag_tang()
    assert O.validate(q) == 0
    for flux in (W.FLUX_HLL, W.FLUX_LINDE):
        q.flux = flux
        assert O.validate(q) == 0
        q.learned = 1
        q.mlp = np.zeros(O.MLP_NPARAM)
        assert O.validate(q) != 0
        q.learned = 0
    for flux in (-1, 3):
        q.flux = flux
        assert O.validate(q) != 0
