"""Parity of the CUDA path (through the C ABI) with the FP64 CPU oracle.

Tolerances:
  * ghost fill: bitwise (copy, pairwise-summed restriction and the
    power-of-two-weighted prolongation are exact operations on both sides);
  * FP64 path: |gpu - oracle| <= 1e-12 * s_v per variable v after 10 steps,
    s_v = max |oracle_v| (the per-variable scale), plus the per-cell relative
    error with the scale as a floor at zero crossings (see _errs);
  * mixed form: 1e-5 * s_v after one step from the same FP64 state;
  * CFL time step: 1e-13 relative (a max of per-cell speeds).
"""
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
    """Per-variable scaled error max|g-o|/s_v and per-cell relative error
    max |g-o| / max(|o|, floor * s_v)."""
    g = np.asarray(g).reshape(8, -1)
    o = np.asarray(o).reshape(8, -1)
    s = np.abs(o).max(1)
    s = np.where(s > 0, s, 1.0)
    d = np.abs(g - o)
    scaled = d.max(1) / s
    rel = (d / np.maximum(np.abs(o), floor * s[:, None])).max(1)
    return scaled, rel


def _face_mask():
    m = np.zeros((12, 12, 12), bool)
    m[2:10, 2:10, :] = True
    m[2:10, :, 2:10] = True
    m[:, 2:10, 2:10] = True
    return m


def _amr_problem(seed, periodic):
    lv = W.random_amr_tree(seed, root=(3, 3, 3), periodic=periodic, frac=0.3)
    bc = (W.BC_PERIODIC,) * 6 if periodic else (W.BC_OUTFLOW, W.BC_INFLOW, W.BC_OUTFLOW, W.BC_OUTFLOW,
                                                  W.BC_INFLOW, W.BC_OUTFLOW)
    q = W.Problem("amr%d" % seed, (-1, -1, -1), (1, 1, 1), (3, 3, 3), lv, bc, powell=1, limiter=W.LIM_MC)
    q.inflow = np.array([1.1, 0.2, -0.1, 0.05, 0.3, 0.1, -0.2, 0.8])
    rng = np.random.default_rng(seed)
    X = W.cell_centres(q.lo, q.hi, q.root, q.leaves)
    tp = 2 * np.pi
    Wp = [1 + 0.3 * np.sin(tp * X[0] / 2) * np.cos(tp * X[1] / 2), 0.3 * np.cos(tp * X[2] / 2),
          0.2 * np.sin(tp * X[0] / 2), -0.1 + 0 * X[0], 0.4 * np.sin(tp * X[1] / 2), 0.3 + 0.1 * X[2],
          0.2 * np.cos(tp * X[0] / 2), 1 + 0.2 * np.cos(tp * (X[0] + X[2]) / 2)]
    q = W.with_state(q, Wp)
    q.U0 = q.U0 * (1 + 1e-3 * rng.standard_normal(q.U0.shape))
    return q


def test_integer_conversions_match_cuda(B):
    rng = np.random.default_rng(0)
    f = np.concatenate([rng.standard_normal(20000).astype(np.float32) * 10.0 ** rng.integers(-30, 30, 20000),
                        np.array([0.0, -0.0, 1.0, -1.0, 3.4e38, 1.2e-38], np.float32)]).astype(np.float32)
    d = np.concatenate([rng.standard_normal(20000) * 10.0 ** rng.integers(-35, 35, 20000),
                        np.array([0.0, -0.0, 1.0, -2.5, 3.0e38, 2e-38])])
    f2d, d2f = B.bats_debug_check_conversions(f, d)
    assert np.array_equal(f2d, f.astype(np.float64))
    ref = d.astype(np.float32)
    ok = np.abs(d) >= 1.1754943508222875e-38
    ulp = np.abs(d2f[ok].view(np.int32).astype(np.int64) - ref[ok].view(np.int32).astype(np.int64))
    assert ulp.max() <= 1
    assert np.all(d2f[~ok] == 0.0)


@pytest.mark.parametrize("case", ["amr_periodic", "amr_inflow", "magnetosphere"])
def test_ghost_fill_bitwise(B, case):
    if case == "magnetosphere":
        q = W.magnetosphere()
        rng = np.random.default_rng(3)
        q.U0 = q.U0 * (1 + 0.01 * rng.standard_normal(q.U0.shape))
    else:
        q = _amr_problem(1 if case == "amr_periodic" else 2, case == "amr_periodic")
    with B.Solver(q) as s:
        s.set_state(0, q.U0)
        Tg = s.fill_ghosts(0)
    To, deep = O.fill_ghosts(q, q.U0)
    assert deep == 0
    m = _face_mask()
    assert np.array_equal(Tg[:, :, m], To[:, :, m])


@pytest.mark.parametrize("staging", [1, 0])
@pytest.mark.parametrize("case", ["amr_periodic", "amr_inflow", "magnetosphere", "blast"])
def test_mixed_ghost_fill_matches_oracle(B, case, staging):
    """The mixed form fills ghosts from the FP32 primitives alone: at
    resolution changes the restriction and prolongation are the oracle's
    conservative ones written in primitive form.  Against the oracle's FP64
    fill turned into primitives, face slabs and interior, per variable scaled
    by its largest magnitude: FP32 rounding of a few operations, bound 4e-6.
    The view is the stage kernel's own staged tile (swizzled interior, face
    slabs by tensor copies or by thread gathers) read back through its
    layout, in both staging layouts."""
    if case == "amr_periodic":
        q = _amr_problem(3, True)
    elif case == "amr_inflow":
        q = _amr_problem(4, False)
    elif case == "magnetosphere":
        q = W.magnetosphere()
    else:
        q = W.blast()
        X = W.cell_centres(q.lo, q.hi, q.root, q.leaves)
        q = W.with_state(q, [1 + 0.5 * np.exp(-4 * (X[0] ** 2 + X[1] ** 2)), 0.3 * np.sin(3 * X[1]),
                             0.2 * np.cos(2 * X[2]), 0.1 * X[0], 0.5 + 0.2 * X[2], 0.3 * np.cos(X[0]),
                             -0.2 + 0 * X[0], 1 + 0.5 * np.exp(-3 * (X[1] ** 2 + X[2] ** 2))])
    with B.Solver(q, precision=B.BATS_MIXED) as s:
        s.set_staging(staging)
        assert s.staging() == staging
        s.set_state(0, q.U0)
        Tg = s.fill_ghosts_w(0)
    To, _ = O.fill_ghosts(q, q.U0)
    Wo = O.prim_from_cons(q.gamma, np.moveaxis(To.reshape(8, -1), 0, -1))
    Wo = np.moveaxis(Wo, -1, 0).reshape(To.shape)
    m = _face_mask()
    g = Tg[:, :, m].reshape(8, -1)
    o = Wo[:, :, m].reshape(8, -1)
    scale = np.abs(o).max(1)
    scale = np.where(scale > 0, scale, 1.0)
    err = np.abs(g - o).max(1) / scale
    print(case, "mixed ghost fill scaled error per variable", err)
    assert err.max() <= 4e-6, err


@pytest.mark.parametrize("case", ["orszag_tang", "blast", "amr_inflow_powell", "linear_b0", "magnetosphere"])
def test_residual_fp64(B, case):
    if case == "orszag_tang":
        q = W.orszag_tang()
    elif case == "blast":
        q = W.blast()
    elif case == "amr_inflow_powell":
        q = _amr_problem(2, False)
    elif case == "linear_b0":
        q = _amr_problem(4, True)
        G = np.array([[0.3, 0.1, 0.0], [0.8, -0.1, 0.2], [0.0, 0.4, 0.5]])
        q.b0, q.b0_param = W.B0_LINEAR, np.r_[0.2, 0.1, -0.4, G.reshape(-1)]
    else:
        q = W.magnetosphere()
    with B.Solver(q) as s:
        s.set_state(0, q.U0)
        Rg = s.residual(0)
    Ro = O.residual(q, q.U0)
    if q.body_r > 0:  # the debug view reports 0 for the fixed body cells
        X = W.cell_centres(q.lo, q.hi, q.root, q.leaves)
        Ro[:, (X[0] ** 2 + X[1] ** 2 + X[2] ** 2) < q.body_r ** 2] = 0.0
    scaled, _ = _errs(Rg, Ro)
    assert scaled.max() <= 1e-12, scaled


@pytest.mark.parametrize("case", ["orszag_tang", "blast", "amr_inflow_powell", "magnetosphere"])
def test_fp64_ten_steps(B, case):
    if case == "orszag_tang":
        q = W.orszag_tang()
    elif case == "blast":
        q = W.blast()
    elif case == "amr_inflow_powell":
        q = _amr_problem(2, False)
    else:
        q = W.magnetosphere()
    nsteps = 10
    with B.Solver(q) as s:
        s.set_state(0, q.U0)
        dt0 = s.dt(0, q.cfl)
        t = s.step(nsteps, q.cfl)
        Ug = s.get_state(0)
    smax0 = O.cfl_smax(q, q.U0)
    assert dt0 == pytest.approx(q.cfl / smax0, rel=1e-13)
    Uo, _, to = O.run(q, q.U0, nsteps, cfl=q.cfl)
    assert t == pytest.approx(to, rel=1e-12)
    scaled, rel = _errs(Ug, Uo)
    print(case, "scaled", scaled.max(), "cell-relative", rel.max())
    assert scaled.max() <= 1e-12, scaled
    assert rel.max() <= 1e-10, rel
    assert np.abs(Uo - q.U0).max() > 0


def test_fixed_dt_and_ssp_rk2(B):
    q = _amr_problem(5, True)
    q.rk = W.RK_SSP2
    with B.Solver(q) as s:
        s.set_state(0, q.U0)
        s.step_dt(5, 2e-3)
        Ug = s.get_state(0)
    Uo, _, _ = O.run(q, q.U0, 5, dt=2e-3)
    scaled, _ = _errs(Ug, Uo)
    assert scaled.max() <= 1e-12, scaled


@pytest.mark.parametrize("case", ["orszag_tang", "blast", "magnetosphere", "amr_inflow_powell"])
def test_mixed_one_step(B, case):
    if case == "orszag_tang":
        q = W.orszag_tang()
    elif case == "blast":
        q = W.blast()
    elif case == "amr_inflow_powell":
        q = _amr_problem(2, False)
    else:
        q = W.magnetosphere()
    with B.Solver(q, precision=B.BATS_MIXED) as s:
        s.set_state(0, q.U0)
        s.step(1, q.cfl)
        Ug = s.get_state(0)
    Uo, _, _ = O.run(q, q.U0, 1, cfl=q.cfl)
    scaled, rel = _errs(Ug, Uo)
    print(case, "mixed scaled per variable", scaled)
    assert scaled.max() <= 1e-5, scaled
    # primitive pressure from both states
    Wg = O.prim_from_cons(q.gamma, np.moveaxis(Ug.reshape(8, -1), 0, -1))
    Wo = O.prim_from_cons(q.gamma, np.moveaxis(Uo.reshape(8, -1), 0, -1))
    ep = np.abs(Wg[:, 7] - Wo[:, 7]).max() / np.abs(Wo[:, 7]).max()
    assert ep <= 1e-5, ep


def test_uniform_state_preserved_bitwise_gpu(B):
    lv = W.random_amr_tree(2, root=(3, 3, 3), periodic=False, frac=0.3)
    q = W.Problem("u", (-1, -1, -1), (1, 1, 1), (3, 3, 3), lv,
                  (W.BC_INFLOW, W.BC_OUTFLOW, W.BC_OUTFLOW, W.BC_INFLOW, W.BC_OUTFLOW, W.BC_OUTFLOW),
                  limiter=W.LIM_MC, powell=1, b0=W.B0_UNIFORM, b0_param=np.r_[0.3, -1.1, 0.6, np.zeros(9)])
    Wu = [1.3, 0.4, -0.2, 0.3, 0.7, -0.5, 0.25, 0.9]
    q.inflow = np.array(Wu)
    W.uniform_state(q, Wu)
    for prec in (B.BATS_FP64, B.BATS_MIXED):
        with B.Solver(q, precision=prec) as s:
            s.set_state(0, q.U0)
            s.step(3, 0.8)
            Ug = s.get_state(0)
        # the mixed form's ghost values at resolution changes are formed
        # from increments and variances, which vanish exactly here
        assert np.array_equal(Ug, q.U0), prec


def test_batched_grids_equal_single_runs_bitwise(B):
    probs = [_amr_problem(7, True), W.orszag_tang(), _amr_problem(8, False)]
    probs[1].limiter = W.LIM_MC
    probs[1].powell = 1
    for p in probs:
        p.limiter, p.powell = W.LIM_MC, 1
    with B.Solver(probs) as s:
        s.set_states()
        s.step(4, 0.8)
        batched = [s.get_state(g) for g in range(3)]
        times = [s.time(g) for g in range(3)]
    for g, p in enumerate(probs):
        with B.Solver(p) as s:
            s.set_state(0, p.U0)
            s.step(4, 0.8)
            assert np.array_equal(s.get_state(0), batched[g])
            assert s.time(0) == times[g]


@pytest.mark.parametrize("case", ["blast", "magnetosphere", "periodic_amr"])
def test_staging_layouts_bitwise_equal(B, case):
    """The mixed form's two staging layouts (same-level face slabs by tensor
    copies or gathered by the threads) give the same state bit for bit, on
    a grid with resolution changes and outflow faces, one with inflow faces,
    a dipole B0 and the inner body, and a periodic one, in every launch form
    the autotuner tries (persistent or not, one to eight blocks per CTA)."""
    if case == "blast":
        q = W.blast()
    elif case == "magnetosphere":
        q = W.magnetosphere()
    else:
        q = _amr_problem(3, True)
    ref = None
    for staging in (1, 0):
        for persistent, bpc in [(0, 1), (0, 4), (1, 2), (1, 8)]:
            with B.Solver(q, precision=B.BATS_MIXED, persistent=persistent, blocks_per_cta=bpc) as s:
                s.set_staging(staging)
                s.set_state(0, q.U0)
                s.step(3, 0.8)
                U = s.get_state(0)
            if ref is None:
                ref = U
            else:
                assert np.array_equal(U, ref), (staging, persistent, bpc)


def test_staging_layout_is_validated(B):
    q = W.orszag_tang()
    with B.Solver(q, precision=B.BATS_MIXED) as s:
        with pytest.raises(B.BatsError):
            s.set_staging(2)
        assert s.staging() == 1


@pytest.mark.parametrize("prec", [0, 1])
def test_launch_forms_bitwise_equal(B, prec):
    q = W.blast()
    ref = None
    for persistent, bpc, graph in [(0, 1, 0), (1, 1, 0), (1, 4, 0), (1, 2, 1), (0, 1, 1)]:
        with B.Solver(q, precision=prec, persistent=persistent, blocks_per_cta=bpc, use_graph=graph) as s:
            s.set_state(0, q.U0)
            s.step(3, 0.8)
            s.step(3, 0.8)   # graph replay on the second call
            U = s.get_state(0)
        if ref is None:
            ref = U
        else:
            assert np.array_equal(U, ref), (persistent, bpc, graph)


def test_run_to_run_bitwise(B):
    q = _amr_problem(9, True)
    outs = []
    for _ in range(2):
        with B.Solver(q, precision=B.BATS_MIXED) as s:
            s.set_state(0, q.U0)
            s.step(5, 0.8)
            outs.append(s.get_state(0))
    assert np.array_equal(outs[0], outs[1])


def test_checkpoint_resume_bitwise(B):
    """5 + 5 steps through get_state/set_state equal 10 steps (fixed dt)."""
    q = _amr_problem(10, True)
    with B.Solver(q) as s:
        s.set_state(0, q.U0)
        s.step_dt(10, 1e-3)
        U10 = s.get_state(0)
        s.set_state(0, q.U0)
        s.step_dt(5, 1e-3)
        mid = s.get_state(0)
    with B.Solver(q) as s:
        s.set_state(0, mid)
        s.step_dt(5, 1e-3)
        assert np.array_equal(s.get_state(0), U10)


def test_nonphysical_state_is_reported(B):
    q = W.orszag_tang()
    U = q.U0.copy()
    U[7, 3, 2, 2, 2] = -1.0  # negative energy -> negative pressure
    with B.Solver(q) as s:
        s.set_state(0, U)
        with pytest.raises(B.BatsError) as e:
            s.step(1, 0.8)
        assert e.value.code == B.BATS_ERR_NONPHYSICAL


def test_device_tensors_in_and_out(B):
    torch = pytest.importorskip("torch")
    q = W.orszag_tang()
    with B.Solver(q) as s:
        Ud = torch.from_numpy(q.U0.copy()).cuda()
        s.set_state(0, Ud)
        s.step(2, 0.8)
        out = torch.zeros_like(Ud)
        B.bats_get_state(s.h, 0, out)
        host = s.get_state(0)
    assert np.array_equal(out.cpu().numpy(), host)


def test_graph_replay_of_many_steps(B):
    """A 60-step graph, replayed twice, equals 120 eager steps (bitwise), and
    both eager runs and graph replays report per-stage event timings (the
    replay's from the graph's own event nodes)."""
    q = W.orszag_tang()
    with B.Solver(q, precision=B.BATS_MIXED) as s:
        s.set_state(0, q.U0)
        s.step(120, 0.8)
        ref = s.get_state(0)
        ms = s.timings()
        assert ms[B.BATS_PHASE_STAGE] > 0 and ms[B.BATS_PHASE_TOTAL] >= ms[B.BATS_PHASE_STAGE]
    with B.Solver(q, precision=B.BATS_MIXED, persistent=1, use_graph=1) as s:
        s.set_state(0, q.U0)
        s.step(60, 0.8)
        s.step(60, 0.8)
        assert np.array_equal(s.get_state(0), ref)
        assert s.launch_count() == 4 * 60
        g = s.timings()
        assert g[B.BATS_PHASE_STAGE] > 0 and g[B.BATS_PHASE_TOTAL] >= g[B.BATS_PHASE_STAGE]
        assert g[B.BATS_PHASE_DT] >= 0
        # the replay's stage time is that of its 60 steps (half the 120 eager ones, to a factor)
        assert 0.2 * ms[B.BATS_PHASE_STAGE] < g[B.BATS_PHASE_STAGE] < 1.5 * ms[B.BATS_PHASE_STAGE]


def test_batched_state_transfer_equals_per_grid_transfer(B):
    """bats_set_states / bats_get_states over the whole batch (host and
    device buffers) act like bats_set_state / bats_get_state on every grid."""
    import torch
    probs = [_amr_problem(9, True), W.orszag_tang(), _amr_problem(10, False)]
    flat = np.concatenate([np.ascontiguousarray(p.U0).reshape(-1) for p in probs])
    for prec in (B.BATS_FP64, B.BATS_MIXED):
        with B.Solver(probs, precision=prec) as s:
            s.set_states()
            s.step(2, 0.8)
            ref = [s.get_state(g) for g in range(3)]
        with B.Solver(probs, precision=prec) as s:
            B.bats_set_states(s.h, flat.copy())
            s.step(2, 0.8)
            out = B.bats_get_states(s.h, np.zeros_like(flat))
            dev = torch.zeros(flat.size, dtype=torch.float64, device="cuda")
            B.bats_get_states(s.h, dev)
            assert np.array_equal(dev.cpu().numpy(), out)
            pinned = torch.zeros(flat.size, dtype=torch.float64).pin_memory()
            B.bats_get_states(s.h, pinned)
            assert np.array_equal(pinned.numpy(), out)
            B.bats_set_states(s.h, dev)
            assert np.array_equal(np.concatenate([s.get_state(g).reshape(-1) for g in range(3)]), out)
            B.bats_set_states(s.h, pinned)
            assert np.array_equal(np.concatenate([s.get_state(g).reshape(-1) for g in range(3)]), out)
        off = 0
        for g, p in enumerate(probs):
            n = p.U0.size
            assert np.array_equal(out[off:off + n].reshape(p.U0.shape), ref[g]), (prec, g)
            off += n
