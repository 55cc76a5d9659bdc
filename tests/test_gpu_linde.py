"""The Linde flux option (HLL with the contact wave restored, the flux of the
paper's fast-wave runs) on the GPU through the C ABI against the FP64 oracle.

Tolerances are those of the Rusanov and HLL parity tests: FP64 path 1e-12 of
each variable's largest magnitude (a vector component: of its vector's) after
10 steps (and 1e-10 per cell with that scale as a floor at 1e-3), mixed form
1e-5 after one step.  The kernels add the restored part to the branch-free HLL
form, the oracle to the textbook three-branch HLL; they agree to rounding."""
import numpy as np
import pytest

from oracle import oracle as O
from paper_2501_06717_gb300 import workloads as W

from test_gpu_hll import _amr_problem, _errs
from test_oracle_linde import _contact_line

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def B():
    from paper_2501_06717_gb300 import bats
    bats.lib()
    return bats


def _case(name):
    if name == "orszag_tang":
        q = W.orszag_tang()
    elif name == "blast":
        q = W.blast()
    elif name == "amr_inflow_powell":
        q = _amr_problem(2, False)
    elif name == "magnetosphere":
        q = W.magnetosphere()
    elif name == "brio_wu_y":
        q = W.brio_wu(1, ncells=64)
    elif name == "fast_wave_m3":
        q = W.fast_wave(m=3)
    else:  # first order, a density wave carried through the periodic box
        q = W.entropy_wave(2, 64, limiter=W.LIM_NONE)
    q.flux = W.FLUX_LINDE
    return q


@pytest.mark.parametrize("case", ["orszag_tang", "blast", "amr_inflow_powell", "magnetosphere", "brio_wu_y",
                                  "fast_wave_m3", "entropy_first_order"])
def test_linde_fp64_ten_steps(B, case):
    q = _case(case)
    with B.Solver(q) as s:
        s.set_state(0, q.U0)
        t = s.step(10, q.cfl)
        Ug = s.get_state(0)
    Uo, _, to = O.run(q, q.U0, 10, cfl=q.cfl)
    assert t == pytest.approx(to, rel=1e-12)
    scaled, rel = _errs(Ug, Uo)
    print(case, "Linde FP64 scaled", scaled.max(), "cell-relative", rel.max())
    assert scaled.max() <= 1e-12, scaled
    assert rel.max() <= 1e-10, rel
    # the option reaches the kernel: the HLL run is a different result
    q.flux = W.FLUX_HLL
    Uh, _, _ = O.run(q, q.U0, 10, cfl=q.cfl)
    assert np.abs(Uh - Uo).max() > 1e3 * np.abs(Ug - Uo).max()


@pytest.mark.parametrize("case", ["orszag_tang", "blast", "amr_inflow_powell", "magnetosphere", "fast_wave_m3"])
def test_linde_mixed_one_step(B, case):
    q = _case(case)
    with B.Solver(q, precision=B.BATS_MIXED) as s:
        s.set_state(0, q.U0)
        s.step(1, q.cfl)
        Ug = s.get_state(0)
    Uo, _, _ = O.run(q, q.U0, 1, cfl=q.cfl)
    scaled, _ = _errs(Ug, Uo)
    print(case, "Linde mixed scaled per variable", scaled)
    assert scaled.max() <= 1e-5, scaled


@pytest.mark.parametrize("axis", [0, 1, 2])
def test_stationary_contact_stays_put(B, axis):
    """The stationary two-contact state of the oracle's pin: 20 steps leave it
    in place, to round-off in FP64 and to the FP32 rounding of the residuals
    in the mixed form, while HLL smears it."""
    q = _contact_line(axis, 0.0, W.FLUX_LINDE)
    for prec, tol in ((B.BATS_FP64, 1e-13), (B.BATS_MIXED, 1e-5)):
        with B.Solver(q, precision=prec) as s:
            s.set_state(0, q.U0)
            s.step(20, 0.8)
            assert np.abs(s.get_state(0) - q.U0).max() <= tol, prec
    h = _contact_line(axis, 0.0, W.FLUX_HLL)
    with B.Solver(h) as s:
        s.set_state(0, h.U0)
        s.step(20, 0.8)
        assert np.abs(s.get_state(0)[0] - h.U0[0]).max() > 1e-2


def test_linde_uniform_state_preserved_bitwise(B):
    lv = W.random_amr_tree(2, root=(3, 3, 3), periodic=False, frac=0.3)
    q = W.Problem("u", (-1, -1, -1), (1, 1, 1), (3, 3, 3), lv,
                  (W.BC_INFLOW, W.BC_OUTFLOW, W.BC_OUTFLOW, W.BC_INFLOW, W.BC_OUTFLOW, W.BC_OUTFLOW),
                  limiter=W.LIM_MC, powell=1, b0=W.B0_UNIFORM, b0_param=np.r_[0.3, -1.1, 0.6, np.zeros(9)],
                  flux=W.FLUX_LINDE)
    Wu = [1.3, 0.4, -0.2, 0.3, 0.7, -0.5, 0.25, 0.9]
    q.inflow = np.array(Wu)
    W.uniform_state(q, Wu)
    for prec in (B.BATS_FP64, B.BATS_MIXED):
        with B.Solver(q, precision=prec) as s:
            s.set_state(0, q.U0)
            s.step(3, 0.8)
            assert np.array_equal(s.get_state(0), q.U0), prec


@pytest.mark.parametrize("prec", [0, 1])
def test_linde_launch_forms_staging_and_batching_bitwise_equal(B, prec):
    probs = [_case("blast"), _case("amr_inflow_powell")]
    probs[0].powell = 1  # one handle's grids share the physics of the first
    ref = None
    for persistent, bpc, graph, staging in [(0, 1, 0, 1), (1, 4, 0, 1), (1, 2, 1, 1), (0, 4, 0, 0)]:
        with B.Solver(probs, precision=prec, persistent=persistent, blocks_per_cta=bpc, use_graph=graph) as s:
            if prec == B.BATS_MIXED:
                s.set_staging(staging)
            s.set_states()
            s.step(2, 0.8)
            s.step(2, 0.8)
            U = [s.get_state(g) for g in range(2)]
        if ref is None:
            ref = U
        else:
            for g in range(2):
                assert np.array_equal(U[g], ref[g]), (persistent, bpc, graph, staging, g)
    with B.Solver(probs[1], precision=prec) as s:
        s.set_state(0, probs[1].U0)
        s.step(4, 0.8)
        assert np.array_equal(s.get_state(0), ref[1])


@pytest.mark.parametrize("case", ["orszag_tang", "brio_wu_y"])
def test_linde_noalloc_entry_matches_the_handle(B, case):
    q = _case(case)
    with B.Solver(q) as s:
        s.set_state(0, q.U0)
        s.step(3, 0.8)
        Uh = s.get_state(0)
    U = q.U0.copy()
    B.bats_step_noalloc(q, B.physics_from(q), U, 3, cfl=0.8)
    assert np.array_equal(U, Uh)


def test_linde_refuses_the_learned_correction(B):
    q = _case("blast")
    with B.Solver(q) as s:
        with pytest.raises(B.BatsError) as e:
            s.set_mlp(np.zeros(O.MLP_NPARAM, np.float32))
        assert e.value.code == B.BATS_ERR_INVALID_ARG
