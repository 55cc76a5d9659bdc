"""Pins of the oracle's conservative flux correction at resolution changes
(refluxing): the flux through a coarse face that borders a refined region is
the mean of the 4 fine fluxes through it.  CPU only."""
import copy

import numpy as np
import pytest

from oracle import oracle as O
from paper_2501_06717_gb300 import workloads as W


def _with(q, **kw):
    q2 = copy.copy(q)
    for k, v in kw.items():
        setattr(q2, k, v)
    return q2


def _amr(seed, limiter=W.LIM_MC):
    lv = W.random_amr_tree(seed, root=(3, 3, 3), periodic=True, frac=0.3)
    q = W.Problem("amr", (-1, -1, -1), (1, 1, 1), (3, 3, 3), lv, (W.BC_PERIODIC,) * 6, limiter=limiter)
    X = W.cell_centres(q.lo, q.hi, q.root, q.leaves)
    tp = 2 * np.pi
    return W.with_state(q, [1 + 0.3 * np.sin(tp * X[0] / 2) * np.cos(tp * X[1] / 2), 0.3 * np.cos(tp * X[2] / 2),
                            0.2 * np.sin(tp * X[0] / 2), -0.1 + 0 * X[0], 0.4 * np.sin(tp * X[1] / 2),
                            0.3 + 0.1 * np.cos(tp * X[2] / 2), 0.2 * np.cos(tp * X[0] / 2),
                            1 + 0.2 * np.cos(tp * (X[0] + X[2]) / 2)])


def _totals(q, U):
    lev = np.asarray(q.leaves)[:, 0]
    vol = np.prod([(q.hi[a] - q.lo[a]) / (q.root[a] * 8) for a in range(3)]) / 8.0 ** lev
    return (np.asarray(U).reshape(8, q.nb, 512) * vol[None, :, None]).sum(axis=(1, 2))


@pytest.mark.parametrize("seed,limiter,rk", [(3, W.LIM_MC, W.RK_MIDPOINT), (4, W.LIM_MINMOD, W.RK_SSP2),
                                             (5, W.LIM_NONE, W.RK_EULER)])
def test_refluxing_conserves_every_variable_on_amr_grids(seed, limiter, rk):
    """Periodic block-adaptive grid, no sources: with refluxing the volume
    integrals of all 8 conserved variables stay constant to round-off (they
    do not without it: a coarse face and its 4 fine sub-faces carry different
    fluxes)."""
    q = _with(_amr(seed, limiter), rk=rk)
    t0 = _totals(q, q.U0)
    scale = np.abs(t0).max()
    U, _, _ = O.run(_with(q, reflux=1), q.U0, 5, cfl=0.8)
    assert np.abs(_totals(q, U) - t0).max() <= 1e-14 * scale
    U0, _, _ = O.run(q, q.U0, 5, cfl=0.8)
    assert np.abs(_totals(q, U0) - t0).max() > 1e-9 * scale


def test_refluxing_changes_only_coarse_cells_at_refined_faces():
    """One stage: the update differs from the uncorrected one only in the
    layer of coarse cells that touch a refined neighbour region."""
    q = _amr(6)
    dt = 0.8 / O.cfl_smax(q, q.U0)
    A = O.stage(q, q.U0, q.U0, 0, dt)
    B = O.stage(_with(q, reflux=1), q.U0, q.U0, 0, dt)
    diff = (np.abs(A - B).reshape(8, q.nb, 8, 8, 8).max(0) > 0)   # block, k, j, i
    L = np.asarray(q.leaves)
    pos = {tuple(x): i for i, x in enumerate(L.tolist())}
    allowed = np.zeros_like(diff)
    for b, (l, i, j, k) in enumerate(L.tolist()):
        for s in range(6):
            d, side = s // 2, s % 2
            p = [i, j, k]
            p[d] += 1 if side else -1
            n = q.root[d] << l
            p[d] %= n
            if (l, *p) in pos or (l >= 1 and (l - 1, p[0] >> 1, p[1] >> 1, p[2] >> 1) in pos):
                continue
            idx = [slice(None)] * 3
            idx[2 - d] = 7 if side else 0
            allowed[b][tuple(idx)] = True
    assert diff.any()
    assert not (diff & ~allowed).any()


def test_refluxing_is_void_on_uniform_grids_and_uniform_states():
    qo = W.orszag_tang()
    A, _, _ = O.run(qo, qo.U0, 3, cfl=0.8)
    B, _, _ = O.run(_with(qo, reflux=1), qo.U0, 3, cfl=0.8)
    assert np.array_equal(A, B)
    q = _amr(7)
    W.uniform_state(q, [1.3, 0.4, -0.2, 0.3, 0.7, -0.5, 0.25, 0.9])
    U, _, _ = O.run(_with(q, reflux=1), q.U0, 3, cfl=0.8)
    assert np.array_equal(U, q.U0)


def test_refluxing_with_the_learned_correction_is_rejected():
    q = _with(W.blast(), reflux=1, learned=1, mlp=np.zeros(O.MLP_NPARAM))
    with pytest.raises(Exception):
        O.run(q, q.U0, 1, cfl=0.8)
