"""Pins of the oracle's inner-body hold (Section 5.2: the inner boundary is a
sphere around the planet; cells whose centre lies strictly inside the radius
take the body state and are not advanced).

The grid here puts cell centres on the integers (dx = 1, lo = -8.5), so the
centre (0, 3, 4) lies exactly on a sphere of radius 5: "inside" (r < R) must
leave it a normal, updated cell.  Each test would fail on a plausible slip in
the oracle: `<=` for `<`, a body cell left in the CFL maximum, a body cell
updated instead of held, a held value that is not the body state, or a body
cell that leaks into cells outside its stencil.  CPU only.
"""
import numpy as np
import pytest

from oracle import oracle as O
from paper_2501_06717_gb300 import workloads as W

R_BODY = 5.0
# gamma = 2 makes p/(gamma - 1) exact, so the body state's conservative form
# is the same number however it is computed
GAMMA = 2.0
BODY_W = np.array([4.0, 0.0, 0.0, 0.0, 0.0, 0.0, 0.0, 0.3])


def _grid(state="random", seed=7):
    root = (2, 2, 2)
    lo, hi = (-8.5,) * 3, (7.5,) * 3
    leaves = W.as_leaf_array(W.morton_sort(W.uniform_leaves(root)))
    q = W.Problem("body_pin", lo, hi, root, leaves, (W.BC_OUTFLOW,) * 6, gamma=GAMMA, limiter=W.LIM_MINMOD,
                  body_r=R_BODY, body=BODY_W.copy(), cfl=0.8)
    x, y, z = W.cell_centres(lo, hi, root, leaves)
    if state == "body":
        Wf = [np.full(x.shape, BODY_W[v]) for v in range(8)]
    else:
        rng = np.random.default_rng(seed)
        sh = x.shape
        Wf = [rng.uniform(0.5, 2.0, sh), rng.uniform(-0.3, 0.3, sh), rng.uniform(-0.3, 0.3, sh),
              rng.uniform(-0.3, 0.3, sh), rng.uniform(-0.5, 0.5, sh), rng.uniform(-0.5, 0.5, sh),
              rng.uniform(-0.5, 0.5, sh), rng.uniform(0.5, 2.0, sh)]
    q = W.with_state(q, Wf)
    return q, (x, y, z)


def _masks(X):
    r2 = X[0] ** 2 + X[1] ** 2 + X[2] ** 2
    return r2 < R_BODY ** 2, r2 == R_BODY ** 2


def _ubody():
    return W.prim_to_cons(BODY_W.reshape(8, 1), GAMMA).reshape(8)


def test_grid_has_a_centre_exactly_on_the_sphere():
    q, X = _grid()
    body, on = _masks(X)
    assert int(on.sum()) > 0          # (0, 3, 4) and its permutations and reflections
    assert int(body.sum()) > 0
    assert not np.any(body & on)


def test_body_cells_hold_the_body_state_exactly():
    """After a stage, every cell strictly inside the sphere equals the body
    state bit for bit, whatever its input; every other cell is advanced."""
    q, X = _grid()
    body, on = _masks(X)
    U = q.U0.reshape(8, q.nb, 8, 8, 8)
    Uo = O.stage(q, U, U, 0, 0.05)
    Ub = _ubody()
    for v in range(8):
        held = Uo[v][body]
        assert np.all(held == held[0]), v
        assert held[0] == Ub[v], v
    # the input there was not the body state, so the hold did something
    assert np.all(np.abs(U[0][body] - Ub[0]) > 1e-3)
    # cells on the sphere (r == R) are not inside: updated, not held
    assert np.all(Uo[0][on] != U[0][on])
    assert np.all(np.abs(Uo[0][on] - Ub[0]) > 1e-3)
    outside = ~body
    changed = np.abs(Uo - U).max(axis=0)[outside] > 0.0
    assert changed.mean() > 0.99


def test_body_cells_hold_in_both_midpoint_stages():
    """A full midpoint step equals the two stages with the body held after
    each; the intermediate state already has the body state in the body."""
    q, X = _grid()
    body, _ = _masks(X)
    U = q.U0.reshape(8, q.nb, 8, 8, 8)
    dt = 0.05
    Us = O.stage(q, U, U, 0, 0.5 * dt)
    Ub = _ubody()
    for v in range(8):
        held = Us[v][body]
        assert np.all(held == held[0])
        assert held[0] == Ub[v]
    U1 = O.stage(q, Us, U, 0, dt)
    Ur, _, _ = O.run(q, U, 1, dt=dt)
    assert np.array_equal(U1, Ur)
    # a stage-2 that saw the unheld stage-1 body values would differ: the
    # body's stage-2 input differs from its stage-1 input
    assert not np.array_equal(Us[0][body], U[0][body])


def test_body_cells_do_not_enter_the_cfl_bound():
    """A body cell with an enormous speed leaves cfl_smax (and so dt)
    unchanged; the same speed in the cell on the sphere raises it."""
    q, X = _grid()
    body, on = _masks(X)
    U = q.U0.reshape(8, q.nb, 8, 8, 8).copy()
    s0 = O.cfl_smax(q, U)
    Ufast = U.copy()
    for c in (1, 2, 3):
        Ufast[c][body] = 1e6 * U[0][body]
    Ufast[7][body] = U[7][body] + 0.5 * 3 * 1e12 * U[0][body]
    assert O.cfl_smax(q, Ufast) == s0
    _, dt0, _ = O.run(q, U, 1, cfl=0.8)
    _, dt1, _ = O.run(q, Ufast, 1, cfl=0.8)
    assert dt1 == dt0
    Uon = U.copy()
    Uon[1][on] = 1e6 * U[0][on]
    Uon[7][on] = U[7][on] + 0.5 * 1e12 * U[0][on]
    assert O.cfl_smax(q, Uon) > 1e5 * s0


def test_uniform_body_state_stays_bitwise_uniform():
    """With the whole domain at the body state, holding the body changes
    nothing: the state stays bitwise uniform over several steps."""
    q, X = _grid(state="body")
    U = q.U0.reshape(8, q.nb, 8, 8, 8)
    Ur, _, _ = O.run(q, U, 4, cfl=0.8)
    for v in range(8):
        assert np.all(Ur[v] == U[v].flat[0]), v


def _stencil_reach(mask):
    """Cells within two cells along one axis of a cell in mask (the
    dimension-by-dimension stencil), on the 16^3 grid of the 2^3 blocks."""
    nb = mask.shape[0]
    # blocks 0..7 in Morton order of a 2x2x2 root: block b at (b & 1, b >> 1 & 1, b >> 2)
    full = np.zeros((16, 16, 16), dtype=bool)
    for b in range(nb):
        bi, bj, bk = b & 1, (b >> 1) & 1, b >> 2
        full[8 * bk:8 * bk + 8, 8 * bj:8 * bj + 8, 8 * bi:8 * bi + 8] = mask[b]
    reach = full.copy()
    for ax in range(3):
        for s in (-2, -1, 1, 2):
            sh = np.roll(full, s, axis=ax)
            if s > 0:
                sl = [slice(None)] * 3
                sl[ax] = slice(0, s)
                sh[tuple(sl)] = False
            else:
                sl = [slice(None)] * 3
                sl[ax] = slice(16 + s, 16)
                sh[tuple(sl)] = False
            reach |= sh
    out = np.zeros_like(mask)
    for b in range(nb):
        bi, bj, bk = b & 1, (b >> 1) & 1, b >> 2
        out[b] = reach[8 * bk:8 * bk + 8, 8 * bj:8 * bj + 8, 8 * bi:8 * bi + 8]
    return out


def test_block_order_is_the_one_the_reach_map_assumes():
    q, X = _grid()
    for b in range(q.nb):
        l, i, j, k = q.leaves[b]
        assert (i, j, k) == (b & 1, (b >> 1) & 1, b >> 2)


def test_deep_body_inputs_change_nothing_and_shallow_ones_do():
    """Inputs of body cells that no outside cell's stencil reaches have no
    effect on the stage result (they are replaced by the body state); inputs
    of body cells next to the surface enter the neighbouring fluxes."""
    q, X = _grid()
    body, _ = _masks(X)
    outside = ~body
    reach = _stencil_reach(outside)
    deep = body & ~reach
    shallow = body & reach
    assert deep.sum() > 0 and shallow.sum() > 0
    U = q.U0.reshape(8, q.nb, 8, 8, 8)
    dt = 0.05
    Uo = O.stage(q, U, U, 0, dt)
    rng = np.random.default_rng(3)
    Ud = U.copy()
    Ud[0][deep] = rng.uniform(5, 9, int(deep.sum()))
    Ud[7][deep] = rng.uniform(5, 9, int(deep.sum()))
    assert np.array_equal(O.stage(q, Ud, Ud, 0, dt), Uo)
    Us = U.copy()
    Us[0][shallow] *= 3.0
    Us[7][shallow] *= 3.0
    Uso = O.stage(q, Us, Us, 0, dt)
    diff = np.abs(Uso - Uo).max(axis=0)
    assert np.all(diff[body] == 0.0)
    assert diff[outside].max() > 0.0
    # and only inside the shallow cells' own stencil
    near = _stencil_reach(shallow)
    assert np.all(diff[outside & ~near] == 0.0)


def test_without_the_body_the_same_cells_are_advanced():
    """Body off (radius 0): the cells inside the sphere advance like all
    others, and the cells beyond the body's stencil give the same result as
    with the body on."""
    q, X = _grid()
    body, _ = _masks(X)
    U = q.U0.reshape(8, q.nb, 8, 8, 8)
    q0 = W.Problem(q.name, q.lo, q.hi, q.root, q.leaves, q.bc, gamma=q.gamma, limiter=q.limiter, body_r=0.0,
                   body=q.body, U0=q.U0)
    dt = 0.05
    Ub = O.stage(q, U, U, 0, dt)
    Un = O.stage(q0, U, U, 0, dt)
    far = ~_stencil_reach(body)
    assert np.array_equal(Ub[:, far], Un[:, far])
    assert np.all(np.abs(Un[0][body] - _ubody()[0]) > 1e-3)
