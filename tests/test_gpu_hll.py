"""The HLL flux option on the GPU (through the C ABI) against the FP64 oracle.

Tolerances are those of the Rusanov parity tests: FP64 path 1e-12 of each
variable's largest magnitude (a vector component: of its vector's) after 10
steps (and 1e-10 per cell with that scale as a floor at 1e-3), mixed form
1e-5 after one step.  The kernel writes
HLL as F_L - S_L/(S_R - S_L) ((F_R - F_L) - S_R (U_R - U_L)) with S_L, S_R
clamped at 0, the oracle as the textbook three-branch form; they agree to
rounding."""
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


def _errs(g, o, floor=1e-3):
    """Per variable max|g - o| / s_v and per cell |g - o| / max(|o|, floor s_v);
    s_v is the variable's largest magnitude, for a vector component that of
    the whole vector (a component that is zero in the solution carries only
    round-off on both sides)."""
    g = np.asarray(g).reshape(8, -1)
    o = np.asarray(o).reshape(8, -1)
    s = np.abs(o).max(1)
    s[1:4] = s[1:4].max()
    s[4:7] = s[4:7].max()
    s = np.where(s > 0, s, 1.0)
    d = np.abs(g - o)
    return d.max(1) / s, (d / np.maximum(np.abs(o), floor * s[:, None])).max(1)


def _amr_problem(seed, periodic):
    """A random 2:1 tree; the open version takes a partly supersonic flow in
    through a fixed-state face at -x (the inflow state is the flow's value
    there) and lets it out through zero-gradient faces."""
    lv = W.random_amr_tree(seed, root=(3, 3, 3), periodic=periodic, frac=0.3)
    bc = (W.BC_PERIODIC,) * 6 if periodic else (W.BC_INFLOW,) + (W.BC_OUTFLOW,) * 5
    q = W.Problem("amr%d" % seed, (-1, -1, -1), (1, 1, 1), (3, 3, 3), lv, bc, powell=1, limiter=W.LIM_MC)
    X = W.cell_centres(q.lo, q.hi, q.root, q.leaves)
    tp = 2 * np.pi
    Wp = [1 + 0.2 * np.sin(tp * X[1] / 2) * np.cos(tp * X[2] / 2), 0.6 + 0.3 * np.cos(tp * X[2] / 2),
          0.1 * np.sin(tp * X[0] / 2), -0.1 + 0 * X[0], 0.3 + 0 * X[0], 0.2 * np.sin(tp * X[0] / 2),
          0.2 * np.cos(tp * X[1] / 2), 0.3 + 0.1 * np.cos(tp * (X[1] + X[2]) / 2)]
    q.inflow = np.array([1.0, 0.9, 0.0, -0.1, 0.3, 0.0, 0.0, 0.3])
    return W.with_state(q, Wp)


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
    else:  # first order, a density wave carried through the periodic box
        q = W.entropy_wave(2, 64, limiter=W.LIM_NONE)
    q.flux = W.FLUX_HLL
    return q


@pytest.mark.parametrize("case", ["orszag_tang", "blast", "amr_inflow_powell", "magnetosphere", "brio_wu_y",
                                  "entropy_first_order"])
def test_hll_fp64_ten_steps(B, case):
    q = _case(case)
    with B.Solver(q) as s:
        s.set_state(0, q.U0)
        t = s.step(10, q.cfl)
        Ug = s.get_state(0)
    Uo, _, to = O.run(q, q.U0, 10, cfl=q.cfl)
    assert t == pytest.approx(to, rel=1e-12)
    scaled, rel = _errs(Ug, Uo)
    print(case, "HLL FP64 scaled", scaled.max(), "cell-relative", rel.max())
    assert scaled.max() <= 1e-12, scaled
    assert rel.max() <= 1e-10, rel
    # the option reaches the kernel: the Rusanov run is a different result
    q.flux = W.FLUX_RUSANOV
    Ur, _, _ = O.run(q, q.U0, 10, cfl=q.cfl)
    assert np.abs(Ur - Uo).max() > 1e3 * np.abs(Ug - Uo).max()


@pytest.mark.parametrize("case", ["orszag_tang", "blast", "amr_inflow_powell", "magnetosphere"])
def test_hll_mixed_one_step(B, case):
    q = _case(case)
    with B.Solver(q, precision=B.BATS_MIXED) as s:
        s.set_state(0, q.U0)
        s.step(1, q.cfl)
        Ug = s.get_state(0)
    Uo, _, _ = O.run(q, q.U0, 1, cfl=q.cfl)
    scaled, _ = _errs(Ug, Uo)
    print(case, "HLL mixed scaled per variable", scaled)
    assert scaled.max() <= 1e-5, scaled


def test_hll_uniform_state_preserved_bitwise(B):
    lv = W.random_amr_tree(2, root=(3, 3, 3), periodic=False, frac=0.3)
    q = W.Problem("u", (-1, -1, -1), (1, 1, 1), (3, 3, 3), lv,
                  (W.BC_INFLOW, W.BC_OUTFLOW, W.BC_OUTFLOW, W.BC_INFLOW, W.BC_OUTFLOW, W.BC_OUTFLOW),
                  limiter=W.LIM_MC, powell=1, b0=W.B0_UNIFORM, b0_param=np.r_[0.3, -1.1, 0.6, np.zeros(9)],
                  flux=W.FLUX_HLL)
    Wu = [1.3, 0.4, -0.2, 0.3, 0.7, -0.5, 0.25, 0.9]
    q.inflow = np.array(Wu)
    W.uniform_state(q, Wu)
    for prec in (B.BATS_FP64, B.BATS_MIXED):
        with B.Solver(q, precision=prec) as s:
            s.set_state(0, q.U0)
            s.step(3, 0.8)
            assert np.array_equal(s.get_state(0), q.U0), prec


@pytest.mark.parametrize("prec", [0, 1])
def test_hll_launch_forms_and_batching_bitwise_equal(B, prec):
    probs = [_case("blast"), _case("amr_inflow_powell")]
    probs[0].powell = 1  # one handle's grids share the physics of the first
    ref = None
    for persistent, bpc, graph in [(0, 1, 0), (1, 4, 0), (1, 2, 1)]:
        with B.Solver(probs, precision=prec, persistent=persistent, blocks_per_cta=bpc, use_graph=graph) as s:
            s.set_states()
            s.step(2, 0.8)
            s.step(2, 0.8)
            U = [s.get_state(g) for g in range(2)]
        if ref is None:
            ref = U
        else:
            for g in range(2):
                assert np.array_equal(U[g], ref[g]), (persistent, bpc, graph, g)
    with B.Solver(probs[1], precision=prec) as s:
        s.set_state(0, probs[1].U0)
        s.step(4, 0.8)
        assert np.array_equal(s.get_state(0), ref[1])


@pytest.mark.parametrize("case", ["orszag_tang", "brio_wu_y"])
def test_hll_noalloc_entry_matches_the_handle(B, case):
    q = _case(case)
    with B.Solver(q) as s:
        s.set_state(0, q.U0)
        s.step(3, 0.8)
        Uh = s.get_state(0)
    U = q.U0.copy()
    B.bats_step_noalloc(q, B.physics_from(q), U, 3, cfl=0.8)
    assert np.array_equal(U, Uh)


def test_hll_refuses_the_learned_correction_and_face_data(B):
    q = _case("blast")
    with B.Solver(q) as s:
        with pytest.raises(B.BatsError) as e:
            s.set_mlp(np.zeros(O.MLP_NPARAM, np.float32))
        assert e.value.code == B.BATS_ERR_INVALID_ARG
        with pytest.raises(B.BatsError) as e:
            s.face_data(0)
        assert e.value.code == B.BATS_ERR_INVALID_ARG
