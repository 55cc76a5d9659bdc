"""Degenerate grids on the GPU against the oracle: one block that is its own
neighbour on every face (periodic), one block with outflow on every face, a
line of blocks with inflow and outflow ends, and the smallest refined grid (a
2 x 1 x 1 root grid with one root refined)."""
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


def _state(q, seed):
    X = W.cell_centres(q.lo, q.hi, q.root, q.leaves)
    rng = np.random.default_rng(seed)
    ph = rng.uniform(0, 2 * np.pi, 8)
    L = [q.hi[a] - q.lo[a] for a in range(3)]
    f = [np.sin(2 * np.pi * X[0] / L[0] + ph[v]) * np.cos(2 * np.pi * X[1] / L[1] + ph[v] / 2)
         + 0.5 * np.sin(2 * np.pi * X[2] / L[2] + ph[v] / 3) for v in range(8)]
    Wp = [1 + 0.2 * f[0], 0.3 * f[1], 0.3 * f[2], 0.3 * f[3], 0.4 + 0.2 * f[4], 0.2 * f[5], 0.3 * f[6], 1 + 0.2 * f[7]]
    return W.with_state(q, Wp)


def _problems():
    one = W.as_leaf_array([(0, 0, 0, 0)])
    periodic = W.Problem("one_periodic", (0, 0, 0), (1, 1, 1), (1, 1, 1), one, (W.BC_PERIODIC,) * 6,
                         limiter=W.LIM_MC, powell=1)
    outflow = W.Problem("one_outflow", (0, 0, 0), (1, 1, 1), (1, 1, 1), one, (W.BC_OUTFLOW,) * 6)
    line = W.Problem("line", (0, 0, 0), (1, 1, 4), (1, 1, 4), W.as_leaf_array(W.uniform_leaves((1, 1, 4))),
                     (W.BC_PERIODIC, W.BC_PERIODIC, W.BC_PERIODIC, W.BC_PERIODIC, W.BC_INFLOW, W.BC_OUTFLOW),
                     powell=1)
    line.inflow = np.array([1.2, 0.1, 0.0, 0.3, 0.4, 0.0, 0.2, 1.1])
    lv = W.uniform_leaves((2, 1, 1))
    lv = [x for x in lv if x != (0, 0, 0, 0)] + W._children((0, 0, 0, 0))
    lv = W.as_leaf_array(W.balance(lv, (2, 1, 1), (True, True, True)))
    amr = W.Problem("amr_small", (0, 0, 0), (2, 1, 1), (2, 1, 1), lv, (W.BC_PERIODIC,) * 6, limiter=W.LIM_MC)
    out = {}
    for i, q in enumerate((periodic, outflow, line, amr)):
        inflow = q.inflow
        q = _state(q, i)
        q.inflow = inflow
        out[q.name] = q
    return out


PROBS = _problems()


def _scaled(g, o):
    g = np.asarray(g).reshape(8, -1)
    o = np.asarray(o).reshape(8, -1)
    s = np.abs(o).max(1)
    s[1:4] = s[1:4].max()
    s[4:7] = s[4:7].max()
    s = np.where(s > 0, s, 1.0)
    return np.abs(g - o).max(1) / s


@pytest.mark.parametrize("name", sorted(PROBS))
@pytest.mark.parametrize("prec,steps,tol", [(0, 10, 1e-12), (1, 1, 1e-5)])
def test_degenerate_grids_match_oracle(B, name, prec, steps, tol):
    q = PROBS[name]
    for reflux in (0, 1):
        q.reflux = reflux
        with B.Solver(q, precision=prec) as s:
            s.set_state(0, q.U0)
            s.step(steps, 0.8)
            Ug = s.get_state(0)
        Uo, _, _ = O.run(q, q.U0, steps, cfl=0.8)
        err = _scaled(Ug, Uo)
        print(name, prec, reflux, err.max())
        assert err.max() <= tol, (name, reflux, err)
    q.reflux = 0
