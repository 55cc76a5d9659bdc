"""Pins of the oracle's Linde flux: the two-state HLL flux with its contact
(entropy) wave restored, the flux of the paper's fast-wave runs (Section
5.1).  The paper cites the flux without printing it; the reading (HLL minus
the contact part of its dissipation, weighted by c / (c + |u_n|)) is stated
in the oracle.  Each pin is a property that any contact-restoring two-state
HLL flux has, checked against the mathematics rather than a retyped formula:
exact upwinding, reduction to HLL when the restored part is off, the exact
flux of a stationary contact, a stationary contact that stays put on a grid,
a moving one smeared less than by HLL, and conservation."""
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
    v = [0.0, 0.0, 0.0]
    v[direction] = wn
    v[(direction + 1) % 3] = wt1
    v[(direction + 2) % 3] = wt2
    return v


def _prim(rho, u, B, p):
    return np.array([rho, *u, *B, p], dtype=np.float64)


def _physical_flux(direction, Wf):
    # identical face states: the Rusanov flux is the physical flux exactly
    return O.numerical_flux(_face_problem(W.FLUX_RUSANOV), direction, Wf, Wf)


@pytest.mark.parametrize("direction", [0, 1, 2])
def test_supersonic_faces_take_the_upwind_physical_flux_exactly(direction):
    """Every wave moving right: F = F_L; every wave moving left: F = F_R,
    bitwise (the restored part carries the factor S_L S_R = 0 there)."""
    linde = _face_problem(W.FLUX_LINDE)
    WL = _prim(1.0, _rot(direction, 3.0, 0.2, -0.1), _rot(direction, 0.1, 0.2, 0.05), 0.2)
    WR = _prim(0.7, _rot(direction, 2.5, -0.3, 0.4), _rot(direction, 0.1, -0.2, 0.1), 0.15)
    assert np.array_equal(O.numerical_flux(linde, direction, WL, WR), _physical_flux(direction, WL))
    WLm, WRm = WL.copy(), WR.copy()
    WLm[1 + direction] *= -1
    WRm[1 + direction] *= -1
    assert np.array_equal(O.numerical_flux(linde, direction, WLm, WRm), _physical_flux(direction, WRm))


@pytest.mark.parametrize("seed", range(8))
def test_with_the_contact_part_off_it_is_hll_bitwise(seed):
    rng = np.random.default_rng(seed)
    d = int(rng.integers(3))
    WL = _prim(rng.uniform(0.5, 2), rng.normal(0, 0.5, 3), rng.normal(0, 0.7, 3), rng.uniform(0.3, 2))
    WR = _prim(rng.uniform(0.5, 2), rng.normal(0, 0.5, 3), rng.normal(0, 0.7, 3), rng.uniform(0.3, 2))
    hll = O.numerical_flux(_face_problem(W.FLUX_HLL), d, WL, WR)
    off = O.numerical_flux(_face_problem(W.FLUX_LINDE), d, WL, WR, contact=0.0)
    assert np.array_equal(off, hll)
    # with a density jump at equal pressures the restored part is not zero
    WR[7] = WL[7]
    hll = O.numerical_flux(_face_problem(W.FLUX_HLL), d, WL, WR)
    on = O.numerical_flux(_face_problem(W.FLUX_LINDE), d, WL, WR)
    assert np.abs(on - hll).max() > 1e-6


@pytest.mark.parametrize("direction", [0, 1, 2])
def test_equal_states_give_the_physical_flux(direction):
    Wf = _prim(1.3, _rot(direction, 0.4, -0.2, 0.1), _rot(direction, 0.5, 0.3, -0.4), 0.8)
    F = O.numerical_flux(_face_problem(W.FLUX_LINDE), direction, Wf, Wf)
    P = _physical_flux(direction, Wf)
    assert np.abs(F - P).max() <= 1e-15 * np.abs(P).max()


@pytest.mark.parametrize("direction", [0, 1, 2])
def test_stationary_contact_gets_its_exact_flux(direction):
    """A density jump at rest (same pressure and field on both sides, normal
    field not zero): both physical fluxes are equal and no mass crosses the
    face; the Linde flux is that flux, HLL lets mass diffuse."""
    B = _rot(direction, 0.6, 0.4, -0.3)
    WL = _prim(1.0, [0, 0, 0], B, 0.7)
    WR = _prim(3.0, [0, 0, 0], B, 0.7)
    P = _physical_flux(direction, WL)
    assert np.allclose(P, _physical_flux(direction, WR), rtol=0, atol=1e-15)
    F = O.numerical_flux(_face_problem(W.FLUX_LINDE), direction, WL, WR)
    assert np.abs(F - P).max() <= 1e-14 * np.abs(P).max()
    assert abs(F[0]) <= 1e-15
    hll = O.numerical_flux(_face_problem(W.FLUX_HLL), direction, WL, WR)
    assert abs(hll[0]) > 0.1


def _contact_line(axis, speed, flux, ncells=32, limiter=W.LIM_MINMOD):
    """Two density jumps (rho 1 | 2.5 | 1) in a uniform flow u_n = speed at
    pressure 1 and field (0.5, 0.3, -0.2) (normal component 0.5), periodic."""
    prob = W._line_problem("contact", axis, ncells, limiter=limiter)
    prob.flux = flux
    X = W.cell_centres(prob.lo, prob.hi, prob.root, prob.leaves)
    s = X[axis]
    one = np.ones_like(s)
    rho = np.where((s > 0.25) & (s < 0.625), 2.5, 1.0)
    u = W._axis_vec(axis, speed * one, 0 * one, 0 * one)
    B = W._axis_vec(axis, 0.5 * one, 0.3 * one, -0.2 * one)
    return W.with_state(prob, [rho, u[0], u[1], u[2], B[0], B[1], B[2], one])


@pytest.mark.parametrize("axis", [0, 1, 2])
def test_stationary_contact_stays_put_on_a_grid(axis):
    """Second-order midpoint steps of the stationary two-contact state: with
    the Linde flux the density profile does not move (round-off), with HLL
    it smears at once."""
    q = _contact_line(axis, 0.0, W.FLUX_LINDE)
    U, _, _ = O.run(q, q.U0, 20, cfl=0.8)
    assert np.abs(U - q.U0).max() <= 1e-13
    h = _contact_line(axis, 0.0, W.FLUX_HLL)
    Uh, _, _ = O.run(h, h.U0, 20, cfl=0.8)
    assert np.abs(Uh[0] - h.U0[0]).max() > 1e-2


def test_moving_contact_is_smeared_less_than_by_hll():
    """The contact part is only partly restored in a moving flow
    (c / (c + |u_n|) < 1): the carried profile stays closer to the exact
    shifted one than with HLL, and both keep the pressure and velocity
    uniform (a contact carries no pressure or velocity jump)."""
    errs = {}
    for flux in (W.FLUX_HLL, W.FLUX_LINDE):
        q = _contact_line(0, 0.5, flux, ncells=64)
        U, _, t = O.run(q, q.U0, 128, dt=1.0 / 1024)
        Wp = np.moveaxis(O.prim_from_cons(q.gamma, np.moveaxis(U, 0, -1)), -1, 0)
        X = W.cell_centres(q.lo, q.hi, q.root, q.leaves)[0]
        s = np.mod(X - 0.5 * t, 1.0)
        exact = np.where((s > 0.25) & (s < 0.625), 2.5, 1.0)
        errs[flux] = np.abs(Wp[0] - exact).mean()
        assert np.abs(Wp[7] - 1.0).max() <= 1e-12
        assert np.abs(Wp[1] - 0.5).max() <= 1e-12
    assert errs[W.FLUX_LINDE] < 0.85 * errs[W.FLUX_HLL], errs


def test_conservation_on_a_periodic_amr_grid():
    """Without the Powell terms all 8 totals (cell-volume weighted) are
    conserved to round-off on a periodic block-adaptive grid (the coarse face
    at a resolution change takes the mean of the fine fluxes: refluxing)."""
    q = W.random_smooth_grid(27, seed=4)
    q.flux = W.FLUX_LINDE
    q.reflux = 1
    U, _, _ = O.run(q, q.U0, 4, cfl=0.8)
    vol = np.array([8.0 ** -lv for lv in q.leaves[:, 0]])[None, :, None, None, None]
    s0 = (q.U0 * vol).reshape(8, -1).sum(1)
    s1 = (U * vol).reshape(8, -1).sum(1)
    scale = (np.abs(q.U0) * vol).reshape(8, -1).sum(1)
    assert np.all(np.abs(s1 - s0) <= 1e-13 * scale), (s1 - s0) / scale
    assert np.abs(U - q.U0).max() > 1e-3


def test_convergence_of_a_smooth_density_wave():
    """A smooth density wave carried by the flow converges at second order
    with the Linde flux (MC limiter), as with the other fluxes."""
    errs = []
    for n in (32, 64, 128):
        q = W.entropy_wave(0, n, amplitude=0.2, speed=1.0)
        q.flux = W.FLUX_LINDE
        dt = 0.2 / n
        steps = int(round(0.25 / dt))
        U, _, t = O.run(q, q.U0, steps, dt=dt)
        ex = W.entropy_wave(0, n, amplitude=0.2, speed=1.0, t_shift=t)
        errs.append(np.abs(U[0] - ex.U0[0]).mean())
    order = math.log2(errs[1] / errs[2])
    assert order >= 1.8, errs


@pytest.mark.parametrize("direction", [0, 1, 2])
def test_sound_jumps_are_left_to_hll(direction):
    """Only the contact is restored: a small jump along a sound wave
    (rho' = rho e, u_n' = c e, p' = c^2 rho e, c^2 = gamma p / rho) has no
    contact part to first order, so the Linde flux differs from HLL by O(e^2)
    there, while for a density jump of the same size it differs by O(e)."""
    gamma = 5.0 / 3.0
    rho, p, e = 1.2, 0.9, 1e-4
    c = math.sqrt(gamma * p / rho)
    WL = _prim(rho, [0, 0, 0], [0, 0, 0], p)
    WS = _prim(rho * (1 + e), _rot(direction, c * e, 0, 0), [0, 0, 0], p + c * c * rho * e)
    WC = _prim(rho * (1 + e), [0, 0, 0], [0, 0, 0], p)
    lin, hll = _face_problem(W.FLUX_LINDE), _face_problem(W.FLUX_HLL)
    ds = np.abs(O.numerical_flux(lin, direction, WL, WS) - O.numerical_flux(hll, direction, WL, WS)).max()
    dc = np.abs(O.numerical_flux(lin, direction, WL, WC) - O.numerical_flux(hll, direction, WL, WC)).max()
    assert dc > 0.3 * c * rho * e
    assert ds < 10 * e * dc


def test_restored_density_jump_is_bounded_by_the_density_jump():
    """A strong pressure rise over a small density rise: the linear contact
    strength (rho_R - rho_L) - (p_R - p_L) / c^2 is large and of the other
    sign, so the restored part, limited to the density jump's sign and size,
    is zero and the flux is HLL; over a large density drop the restored mass
    flux is at most the HLL dissipation of that drop, |d rho| S_R |S_L| /
    (S_R - S_L) (a limit that keeps the magnetosphere stand-in physical)."""
    gamma = 5.0 / 3.0
    WL = _prim(1.0, [0.1, 0, 0], [0.2, 0.1, 0], 0.1)
    WR = _prim(1.05, [-0.1, 0, 0], [0.2, -0.1, 0], 10.0)
    hll = O.numerical_flux(_face_problem(W.FLUX_HLL), 0, WL, WR)
    lin = O.numerical_flux(_face_problem(W.FLUX_LINDE), 0, WL, WR)
    assert np.array_equal(lin, hll)
    WL = _prim(1.0, [0.1, 0, 0], [0.2, 0.1, 0], 10.0)
    WR = _prim(0.2, [-0.1, 0, 0], [0.2, -0.1, 0], 0.1)
    hll = O.numerical_flux(_face_problem(W.FLUX_HLL), 0, WL, WR)
    lin = O.numerical_flux(_face_problem(W.FLUX_LINDE), 0, WL, WR)
    cfl_ = O.fast_speed(gamma, WL, WL[4:7], 0)
    cfr_ = O.fast_speed(gamma, WR, WR[4:7], 0)
    sl = min(WL[1] - cfl_, WR[1] - cfr_)
    sr = max(WL[1] + cfl_, WR[1] + cfr_)
    bound = abs(WR[0] - WL[0]) * sr * abs(sl) / (sr - sl)
    assert 0 < abs(lin[0] - hll[0]) <= bound * (1 + 1e-12)
