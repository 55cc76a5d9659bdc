"""Longer runs against the oracle: the blast of 120 blocks for its full 100
steps and the magnetosphere stand-in for 20 steps, in both precisions.  The
FP64 path stays at round-off; the mixed form's error against the FP64 oracle
is reported per variable (scaled by each quantity's largest magnitude) and
bounded."""
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


def _scaled(g, o):
    g = np.asarray(g).reshape(8, -1)
    o = np.asarray(o).reshape(8, -1)
    s = np.abs(o).max(1)
    s[1:4] = s[1:4].max()
    s[4:7] = s[4:7].max()
    s = np.where(s > 0, s, 1.0)
    return np.abs(g - o).max(1) / s


@pytest.mark.parametrize("name,steps,fp64_tol,mixed_tol", [("blast", 100, 1e-12, 1e-5),
                                                           ("magnetosphere", 20, 1e-12, 1e-5)])
def test_long_runs(B, name, steps, fp64_tol, mixed_tol):
    q = W.blast() if name == "blast" else W.magnetosphere()
    Uo, _, to = O.run(q, q.U0, steps, cfl=0.8)
    for prec, tol in ((B.BATS_FP64, fp64_tol), (B.BATS_MIXED, mixed_tol)):
        with B.Solver(q, precision=prec, persistent=1, use_graph=1) as s:
            s.set_state(0, q.U0)
            s.step(steps, 0.8)
            Ug = s.get_state(0)
            tg = s.time(0)
        err = _scaled(Ug, Uo)
        Wg = O.prim_from_cons(q.gamma, np.moveaxis(Ug.reshape(8, -1), 0, -1))
        Wo = O.prim_from_cons(q.gamma, np.moveaxis(Uo.reshape(8, -1), 0, -1))
        ep = np.abs(Wg[:, 7] - Wo[:, 7]).max() / np.abs(Wo[:, 7]).max()
        print("%s %d steps, precision %d: scaled error per variable %s, pressure %.3e, time %.3e vs %.3e"
              % (name, steps, prec, np.array2string(err, precision=2), ep, tg, to))
        assert err.max() <= tol and ep <= tol, (err, ep)
