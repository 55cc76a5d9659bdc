"""bats_step_noalloc: stepping one grid without any device allocation.

For callers that cannot allocate device memory when they step (an external
memory manager owns the device, or the runtime forbids cudaMalloc after
start-up): the entry point keeps its scratch in a fixed array the library
reserves at load time.  Its results must match the allocating path
(bats_create + bats_step) on the same state, call after call, although every
call reuses the array left by the previous one.  Collected last so that a
failure here stops a -x run only after every other test has run.
"""
import numpy as np
import pytest

from paper_2501_06717_gb300 import workloads as W

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def B():
    from paper_2501_06717_gb300 import bats
    bats.lib()
    return bats


def _problem():
    lv = W.random_amr_tree(3, root=(2, 2, 2), periodic=False, max_level=1, frac=0.5)
    q = W.Problem("noalloc", (-1, -1, -1), (1, 1, 1), (2, 2, 2), lv,
                  (W.BC_OUTFLOW, W.BC_INFLOW, W.BC_OUTFLOW, W.BC_OUTFLOW, W.BC_OUTFLOW, W.BC_OUTFLOW),
                  limiter=W.LIM_MC, powell=1)
    q.inflow = np.array([1.1, -0.3, 0.0, 0.1, 0.2, 0.1, -0.1, 0.9])
    X = W.cell_centres(q.lo, q.hi, q.root, q.leaves)
    Wp = [1 + 0.2 * np.sin(np.pi * X[0]), 0.2 * np.cos(np.pi * X[1]), 0.1 + 0 * X[0], -0.1 * X[2],
          0.3 + 0.1 * X[1], 0.2 * np.sin(np.pi * X[2]), 0.1, 1 + 0.1 * np.cos(np.pi * (X[0] + X[1]))]
    return W.with_state(q, Wp)


def _scaled(a, b):
    s = np.abs(b).reshape(8, -1).max(1)
    return (np.abs(a - b).reshape(8, -1).max(1) / np.where(s > 0, s, 1)).max()


def test_noalloc_matches_allocating_path_on_consecutive_calls(B):
    q = _problem()
    assert 0 < q.nb <= B.BATS_NOALLOC_MAX_BLOCKS
    ph = B.physics_from(q)
    # allocating path: 3 + 3 steps
    with B.Solver(q) as s:
        s.set_state(0, q.U0)
        s.step(3, 0.8)
        ref1 = s.get_state(0)
        s.step(3, 0.8)
        ref2 = s.get_state(0)
    # no-alloc path, host buffer: two calls in a row, the second continuing the first
    U = q.U0.copy()
    t1 = B.bats_step_noalloc(q, ph, U, 3, cfl=0.8)
    assert t1 > 0 and _scaled(U, ref1) <= 1e-12
    B.bats_step_noalloc(q, ph, U, 3, cfl=0.8)
    assert _scaled(U, ref2) <= 1e-12
    # device buffer, fixed dt, twice from the same start: same answer both times
    torch = pytest.importorskip("torch")
    with B.Solver(q) as s:
        s.set_state(0, q.U0)
        s.step_dt(4, 2e-3)
        ref3 = s.get_state(0)
    for _ in range(2):
        Ud = torch.from_numpy(q.U0.copy()).cuda()
        B.bats_step_noalloc(q, ph, Ud, 4, dt=2e-3)
        assert _scaled(Ud.cpu().numpy(), ref3) <= 1e-12


def test_noalloc_rejects_grids_beyond_its_limit(B):
    root = (6, 6, 4)  # 144 blocks > 128
    lv = W.as_leaf_array(W.uniform_leaves(root))
    q = W.Problem("big", (0, 0, 0), (1, 1, 1), root, lv, (W.BC_PERIODIC,) * 6)
    W.uniform_state(q, [1, 0, 0, 0, 0, 0, 0, 1])
    with pytest.raises(B.BatsError) as e:
        B.bats_step_noalloc(q, B.physics_from(q), q.U0.copy(), 1, cfl=0.8)
    assert e.value.code == B.BATS_ERR_INVALID_ARG and "BATS_NOALLOC_MAX_BLOCKS" in str(e.value)


@pytest.mark.parametrize("option", ["reflux", "local_dt"])
def test_noalloc_refuses_options_it_cannot_honour(B, option):
    """Refluxing and local time steps change the physics and need buffers the
    entry point does not keep: they are refused with a message, not ignored."""
    q = _problem()
    setattr(q, option, 1)
    U = q.U0.copy()
    with pytest.raises(B.BatsError) as e:
        B.bats_step_noalloc(q, B.physics_from(q), U, 1, cfl=0.8)
    assert e.value.code == B.BATS_ERR_INVALID_ARG and option in str(e.value)
    assert np.array_equal(U, q.U0)  # the caller's state is untouched


@pytest.mark.parametrize("nsteps", [3, 4])
def test_noalloc_one_stage_scheme_matches_allocating_path(B, nsteps):
    """The one-stage first-order scheme (alternating buffers; an odd step
    count ends in the other buffer) gives the allocating path's result."""
    q = _problem()
    q.rk = W.RK_EULER
    q.limiter = W.LIM_NONE
    ph = B.physics_from(q)
    with B.Solver(q) as s:
        s.set_state(0, q.U0)
        s.step(nsteps, 0.8)
        ref = s.get_state(0)
    U = q.U0.copy()
    B.bats_step_noalloc(q, ph, U, nsteps, cfl=0.8)
    assert _scaled(U, ref) <= 1e-12


def test_noalloc_allocates_no_device_memory(B):
    """After a first call (which loads the kernels), further calls on host and
    device buffers leave the device's free memory unchanged."""
    torch = pytest.importorskip("torch")
    q = _problem()
    ph = B.physics_from(q)
    Uh = q.U0.copy()
    Ud = torch.from_numpy(q.U0.copy()).cuda()
    B.bats_step_noalloc(q, ph, Uh, 1, cfl=0.8)
    B.bats_step_noalloc(q, ph, Ud, 1, cfl=0.8)
    torch.cuda.synchronize()
    free0, _ = torch.cuda.mem_get_info()
    for _ in range(3):
        B.bats_step_noalloc(q, ph, Uh, 2, cfl=0.8)
        B.bats_step_noalloc(q, ph, Ud, 2, dt=1e-3)
    torch.cuda.synchronize()
    free1, _ = torch.cuda.mem_get_info()
    assert free1 == free0, (free0, free1)
