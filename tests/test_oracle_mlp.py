"""Pins of the oracle's learned flux correction (MLP 40 -> 64 -> 64 -> 8).

Backprop against central finite differences, GELU identities, the exact
reduction to plain Rusanov with zero weights, and the invariance of the
normalised inputs (and the matching scaling of the correction) under the
similarity scaling of ideal MHD.  CPU only.
"""
import math

import numpy as np
import pytest

from oracle import oracle as O
from paper_2501_06717_gb300 import workloads as W

from learned_nets import double_dissipation_net, physical_per_block


def _params(seed, scale=0.3):
    rng = np.random.default_rng(seed)
    return rng.normal(0, scale, size=O.MLP_NPARAM)


def test_gelu_identities():
    """tanh-form GELU (Hendrycks & Gimpel): gelu(0) = 0, gelu(x) - gelu(-x) = x,
    gelu(1) = 0.84119199..., gelu(x) -> x for large x."""
    assert O.gelu(0.0) == 0.0
    assert O.gelu(1.0) == pytest.approx(0.8411919906082768, rel=1e-14)
    for x in (0.3, 1.7, -2.2, 5.0):
        assert O.gelu(x) - O.gelu(-x) == pytest.approx(x, rel=1e-14, abs=1e-15)
    assert O.gelu(12.0) == pytest.approx(12.0, rel=1e-15)


def test_backprop_matches_central_differences():
    rng = np.random.default_rng(4)
    P = _params(1)
    X = rng.normal(size=(37, O.MLP_IN))
    T = rng.normal(size=(37, O.MLP_OUT))
    loss, g = O.mlp_loss_grad(P, X, T)
    assert loss > 0
    idx = rng.choice(O.MLP_NPARAM, size=60, replace=False)
    # include every parameter group: W1, b1, W2, b2, W3, b3
    starts = np.cumsum([0, 64 * 40, 64, 64 * 64, 64, 8 * 64])
    idx = np.concatenate([idx, starts + 3])
    h = 1e-5  # central differences: truncation O(h^2) and round-off O(eps L / h) both below 1e-8 here
    for i in idx:
        Pp = P.copy()
        Pm = P.copy()
        Pp[i] += h
        Pm[i] -= h
        fd = (O.mlp_loss_grad(Pp, X, T)[0] - O.mlp_loss_grad(Pm, X, T)[0]) / (2 * h)
        assert abs(fd - g[i]) <= 1e-6 * abs(g[i]) + 2e-9, (i, fd, g[i])


def test_forward_matches_loss_definition():
    """mlp_forward and the loss use the same network: L = mean (y - t)^2."""
    rng = np.random.default_rng(2)
    P = _params(3)
    X = rng.normal(size=(5, O.MLP_IN))
    T = rng.normal(size=(5, O.MLP_OUT))
    ys = np.array([O.mlp_forward(P, x)[2] for x in X])
    loss, _ = O.mlp_loss_grad(P, X, T)
    assert loss == pytest.approx(np.mean((ys - T) ** 2), rel=1e-13)
    # zero weights: output is the last bias
    Z = np.zeros(O.MLP_NPARAM)
    Z[-8:] = np.arange(8)
    assert np.array_equal(O.mlp_forward(Z, X[0])[2], np.arange(8.0))


def test_zero_network_is_plain_rusanov_bitwise():
    q = W.blast(nsteps=2)
    U0, _, _ = O.run(q, q.U0, 2, cfl=0.8)
    ql = W.Problem(**{**q.__dict__, "learned": 1, "mlp": np.zeros(O.MLP_NPARAM)})
    U1, _, _ = O.run(ql, q.U0, 2, cfl=0.8)
    assert np.array_equal(U0, U1)


def _stencil(rng):
    Ws = np.zeros((4, 8))
    Ws[:, 0] = rng.uniform(0.5, 2, 4)
    Ws[:, 1:7] = rng.normal(0, 0.5, (4, 6))
    Ws[:, 7] = rng.uniform(0.5, 2, 4)
    WL = Ws[1] + rng.normal(0, 0.01, 8)
    WR = Ws[2] + rng.normal(0, 0.01, 8)
    return Ws, WL, WR


def _scale_prim(Wv, a, b):
    out = Wv.copy()
    out[..., 0] *= a
    out[..., 1:4] *= b
    out[..., 4:7] *= math.sqrt(a) * b
    out[..., 7] *= a * b * b
    return out


def test_features_are_similarity_invariant_and_rotate_with_the_face():
    rng = np.random.default_rng(7)
    Ws, WL, WR = _stencil(rng)
    cmax = 1.3
    x = O.mlp_features(0, Ws, WL, WR, cmax)
    a, b = 3.7, 0.21
    xs = O.mlp_features(0, _scale_prim(Ws, a, b), _scale_prim(WL, a, b), _scale_prim(WR, a, b), cmax * b)
    assert np.allclose(xs, x, rtol=1e-13, atol=1e-14)
    # a y-face of the state whose (y, z, x) components are the x-face's (x, y, z)
    perm = [0, 3, 1, 2, 6, 4, 5, 7]   # new[v] = old[perm[v]]: u_x' = u_z, u_y' = u_x, u_z' = u_y
    xy = O.mlp_features(1, Ws[:, perm], WL[perm], WR[perm], cmax)
    assert np.array_equal(xy, x)


def test_learned_residual_scales_like_the_flux():
    """Under rho -> a rho, u -> b u, B -> sqrt(a) b B, p -> a b^2 p the features are
    unchanged and the corrections are rescaled by the flux units, so the whole
    learned residual scales like the plain one: (a b, a b^2, sqrt(a) b^2, a b^3)."""
    q = W.blast(nsteps=1)
    q.learned = 1
    q.mlp = _params(11, scale=0.2)
    # smooth nontrivial state
    X = W.cell_centres(q.lo, q.hi, q.root, q.leaves)
    Wp = [1 + 0.3 * np.sin(2 * X[0]), 0.2 * np.cos(3 * X[1]), 0.1 * np.sin(X[2]), 0.05 + 0 * X[0],
          0.5 + 0.1 * X[1], 0.3 * np.cos(X[0]), 0.1 + 0 * X[0], 1 + 0.2 * np.cos(X[0] + X[2])]
    q = W.with_state(q, Wp)
    R = O.residual(q, q.U0)
    q0 = W.Problem(**{**q.__dict__, "learned": 0})
    R0 = O.residual(q0, q.U0)
    assert np.abs(R - R0).max() > 1e-6 * np.abs(R0).max()   # the network changes the residual
    a, b = 2.5, 0.4
    Wsc = [Wp[0] * a] + [w * b for w in Wp[1:4]] + [w * math.sqrt(a) * b for w in Wp[4:7]] + [Wp[7] * a * b * b]
    qs = W.with_state(W.Problem(**{**q.__dict__}), Wsc)
    Rs = O.residual(qs, qs.U0)
    f = np.array([a * b] + [a * b * b] * 3 + [math.sqrt(a) * b * b] * 3 + [a * b ** 3])
    scale = np.abs(R).reshape(8, -1).max(1)
    err = np.abs(Rs - f[:, None, None, None, None] * R).reshape(8, -1).max(1) / (f * scale)
    assert err.max() < 1e-11, err


def test_learned_fallback_replaces_exactly_the_non_physical_blocks():
    """The learned form's fallback: a block whose learned update has a cell with
    rho <= 0 or p <= 0 is recomputed with the plain Rusanov flux; every other
    block keeps its learned update."""
    import copy
    q = W.blast()
    ql = W.Problem(**{**q.__dict__, "learned": 1, "mlp": double_dissipation_net()})
    qn = copy.copy(ql)
    qn.no_fallback = 1
    # the first step: stage 1 stays physical, stage 2 fails next to the jump
    U = q.U0
    dt = 0.8 / O.cfl_smax(q, U)
    Ustar = O.stage(ql, U, U, 0, 0.5 * dt)
    found = False
    for Uin, c in ((U, 0.5 * dt), (Ustar, dt)):
        Uf, fb = O.stage(ql, Uin, U, 0, c, with_fallback_flags=True)
        Un, fbn = O.stage(qn, Uin, U, 0, c, with_fallback_flags=True)
        Up = O.stage(q, Uin, U, 0, c)
        assert not fbn.any()
        bad = ~physical_per_block(q.gamma, Un)
        assert np.array_equal(fb.astype(bool), bad)
        assert np.array_equal(Uf[:, fb == 1], Up[:, fb == 1])
        assert np.array_equal(Uf[:, fb == 0], Un[:, fb == 0])
        found |= bool(fb.any()) and not bool(fb.all())
    assert found, "the test network never made a block non-physical"


def test_learned_fallback_count_over_a_run():
    """The run counts the block-stages that fell back: over one step it is the
    sum of the two stages' flags; a zero network never falls back."""
    q = W.blast()
    ql = W.Problem(**{**q.__dict__, "learned": 1, "mlp": double_dissipation_net()})
    dt = 0.8 / O.cfl_smax(q, q.U0)
    Us, fb1 = O.stage(ql, q.U0, q.U0, 0, 0.5 * dt, with_fallback_flags=True)
    U1, fb2 = O.stage(ql, Us, q.U0, 0, dt, with_fallback_flags=True)
    Ur, _, _, nfb = O.run(ql, q.U0, 1, cfl=0.8, with_fallbacks=True)
    assert nfb == fb1.sum() + fb2.sum() > 0
    assert np.array_equal(Ur, U1)
    qz = W.Problem(**{**q.__dict__, "learned": 1, "mlp": np.zeros(O.MLP_NPARAM)})
    _, _, _, nz = O.run(qz, q.U0, 3, cfl=0.8, with_fallbacks=True)
    assert nz == 0


def test_learned_fallback_rescues_a_stage_the_plain_flux_keeps_physical():
    """Blast with p_in = 1.5 at CFL 0.8: the doubled dissipation makes 8 blocks
    non-physical in the first step's second stage; their plain recompute is
    physical, so the step ends physical, unlike the unguarded learned step."""
    import copy
    q = W.blast(pin=1.5)
    ql = W.Problem(**{**q.__dict__, "learned": 1, "mlp": double_dissipation_net()})
    U, _, _, nfb = O.run(ql, q.U0, 1, cfl=0.8, with_fallbacks=True)
    assert nfb == 8
    assert physical_per_block(q.gamma, U).all()
    qn = copy.copy(ql)
    qn.no_fallback = 1
    Un, _, _ = O.run(qn, q.U0, 1, cfl=0.8)
    assert (~physical_per_block(q.gamma, Un)).sum() == 8


def test_learned_last_stage_only_composes_a_plain_first_stage():
    """With the correction in the last stage only, a midpoint step is the
    plain first stage followed by the learned second stage (bitwise), and it
    differs from the step with the correction in both stages."""
    q = W.blast()
    rng = np.random.default_rng(5)
    P = rng.normal(0, 0.1, size=O.MLP_NPARAM)
    both = W.Problem(**{**q.__dict__, "learned": 1, "mlp": P})
    last = W.Problem(**{**q.__dict__, "learned": 1, "mlp": P, "learned_last_only": 1})
    U = q.U0.reshape(8, q.nb, 8, 8, 8)
    dt = 2e-3
    Us = O.stage(q, U, U, 0, 0.5 * dt)          # plain stage 1
    U1 = O.stage(both, Us, U, 0, dt)            # learned stage 2
    Ul, _, _ = O.run(last, U, 1, dt=dt)
    assert np.array_equal(Ul, U1)
    Ub, _, _ = O.run(both, U, 1, dt=dt)
    assert np.abs(Ub - Ul).max() > 1e-10
    # one-stage scheme: the only stage is the last, so the option changes nothing
    qe = W.Problem(**{**q.__dict__, "rk": W.RK_EULER, "limiter": W.LIM_NONE, "learned": 1, "mlp": P})
    qel = W.Problem(**{**qe.__dict__, "learned_last_only": 1})
    assert np.array_equal(O.run(qe, U, 1, dt=dt)[0], O.run(qel, U, 1, dt=dt)[0])
