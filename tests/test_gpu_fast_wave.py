"""The paper's own test problem on the GPU: the Eq. 6 fast magnetosonic wave
on the Table 2 grid for one GPU at m = 3 (4^3 root blocks on [-32, 32]^3,
the -x-y-z octant refined once: 120 blocks of 8^3 cells), periodic, minmod,
with the Rusanov flux and with the HLL flux (Section 5.1 runs it with the
Linde flux, whose HLL base this is).  The FP64 path must match the oracle
to 1e-12 of each variable's scale after 10 steps at CFL 0.8 (a vector
component is scaled by its vector's largest magnitude); the mixed form to
1e-5 after one step."""
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


def _errs(g, o):
    g = np.asarray(g).reshape(8, -1)
    o = np.asarray(o).reshape(8, -1)
    s = np.abs(o).max(1)
    s[1:4] = s[1:4].max()
    s[4:7] = s[4:7].max()
    s = np.where(s > 0, s, 1.0)
    return np.abs(g - o).max(1) / s


def _problem(flux):
    q = W.fast_wave(m=3, nsteps=10)
    assert q.nb == 120
    q.flux = flux
    return q


@pytest.mark.parametrize("flux", [W.FLUX_RUSANOV, W.FLUX_HLL])
def test_fast_wave_fp64_ten_steps(B, flux):
    q = _problem(flux)
    with B.Solver(q) as s:
        s.set_state(0, q.U0)
        t = s.step(10, q.cfl)
        Ug = s.get_state(0)
    Uo, _, to = O.run(q, q.U0, 10, cfl=q.cfl)
    assert t == pytest.approx(to, rel=1e-12)
    err = _errs(Ug, Uo)
    print("fast wave flux", flux, "FP64 scaled error per variable", err)
    assert err.max() <= 1e-12, err
    # the wave moved: the state is not the initial one
    assert np.abs(Uo[0] - q.U0.reshape(Uo.shape)[0]).max() > 1e-4


@pytest.mark.parametrize("flux", [W.FLUX_RUSANOV, W.FLUX_HLL])
def test_fast_wave_mixed_one_step(B, flux):
    q = _problem(flux)
    with B.Solver(q, precision=B.BATS_MIXED) as s:
        s.set_state(0, q.U0)
        s.step(1, q.cfl)
        Ug = s.get_state(0)
    Uo, _, _ = O.run(q, q.U0, 1, cfl=q.cfl)
    err = _errs(Ug, Uo)
    print("fast wave flux", flux, "mixed scaled error per variable", err)
    assert err.max() <= 1e-5, err
