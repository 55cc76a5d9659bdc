"""The learned flux correction on the GPU against the CPU oracle.

Network forward and gradient: the GPU rounds inputs, weights and hidden
activations to BF16 and accumulates in FP32; the oracle runs FP64 on the same
BF16-representable weights and inputs.  With 8-bit mantissas per layer the
expected relative difference is a few 2^-8, so the bound is 2e-2 (relative L2
norm), as for any BF16 network against an FP64 evaluation.
"""
import numpy as np
import pytest

from oracle import oracle as O
from paper_2501_06717_gb300 import workloads as W

from learned_nets import double_dissipation_net, physical_per_block

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def B():
    from paper_2501_06717_gb300 import bats
    bats.lib()
    return bats


def bf16(a):
    """Round float32 values to the nearest BF16 (ties to even), from the format:
    keep the top 16 bits after adding half an ulp of the dropped part."""
    u = np.ascontiguousarray(a, dtype=np.float32).view(np.uint32).astype(np.uint64)
    r = ((u + 0x7FFF + ((u >> 16) & 1)) & 0xFFFF0000).astype(np.uint32)
    return r.view(np.float32)


def _net(seed, scale=0.3):
    rng = np.random.default_rng(seed)
    P = rng.normal(0, scale, size=O.MLP_NPARAM).astype(np.float32)
    return bf16(P)


def _relnorm(a, b):
    return float(np.linalg.norm(np.asarray(a, float) - b) / np.linalg.norm(b))


def test_bf16_rounding_helper():
    x = np.array([1.0, 1.00390625, 1.005859375, -2.5], np.float32)  # 1 + 2^-8 is a tie -> even (1.0)
    assert np.array_equal(bf16(x), np.array([1.0, 1.0, 1.0078125, -2.5], np.float32))


def test_network_forward_matches_oracle(B):
    P = _net(1)
    rng = np.random.default_rng(2)
    X = bf16(rng.normal(size=(2000, 40)))
    with_mlp = B.Mlp(P)
    Y = with_mlp.forward(X)
    Yo = np.array([O.mlp_forward(P.astype(np.float64), x.astype(np.float64))[2] for x in X])
    assert _relnorm(Y, Yo) <= 2e-2


def _forward_bf16_reference(P, X):
    """The network in numpy as the kernels evaluate it: BF16 weights and
    inputs, sums in FP64, bias, tanh-form GELU, hidden activations rounded
    to BF16 before the next layer."""
    W1, b1 = P[:2560].reshape(64, 40).astype(float), P[2560:2624].astype(float)
    W2, b2 = P[2624:6720].reshape(64, 64).astype(float), P[6720:6784].astype(float)
    W3, b3 = P[6784:7296].reshape(8, 64).astype(float), P[7296:7304].astype(float)

    def gelu(z):
        return 0.5 * z * (1.0 + np.tanh(0.7978845608028654 * (z + 0.044715 * z ** 3)))

    h1 = bf16(gelu(X.astype(float) @ W1.T + b1)).astype(float)
    h2 = bf16(gelu(h1 @ W2.T + b2)).astype(float)
    return h2 @ W3.T + b3


@pytest.mark.parametrize("n", [1, 127, 128, 129, 200003])
def test_network_forward_ragged_sizes(B, n):
    """The tensor-core forward runs 128-row tiles (persistent CTAs take several
    tiles at the largest size): every row, the ragged last tile included,
    matches the numpy evaluation of the same BF16 network."""
    P = _net(11)
    rng = np.random.default_rng(n)
    X = bf16(rng.normal(size=(n, 40)))
    m = B.Mlp(P)
    Y = m.forward(X)
    m.close()
    Yr = _forward_bf16_reference(P, X)
    assert Y.shape == (n, 8) and np.isfinite(Y).all()
    # a hidden activation may round to the other BF16 neighbour when the two
    # FP32/FP64 sums straddle a rounding boundary: a few 2^-8 per row at most
    assert (np.abs(Y - Yr).max(axis=1) / np.abs(Yr).max()).max() <= 2e-2
    assert _relnorm(Y, Yr) <= 2e-3


@pytest.mark.parametrize("n", [1, 129, 70001])
def test_forward_bf16_equals_forward_bitwise(B, n):
    """The queued entry on pre-rounded BF16 rows gives the synchronous
    forward's outputs bit for bit (the same kernel on the same rows)."""
    import torch
    P = _net(13)
    rng = np.random.default_rng(300 + n)
    X = bf16(rng.normal(size=(n, 40)))
    m = B.Mlp(P)
    Y = m.forward(X)
    Xh = torch.zeros(n, 48, dtype=torch.bfloat16)
    Xh[:, :40] = torch.from_numpy(X).to(torch.bfloat16)
    Xb = Xh.view(torch.int32).cuda()
    Yd = torch.empty(n, 8, device="cuda")
    m.forward_bf16(Xb, Yd)
    m.sync()
    assert np.array_equal(Yd.cpu().numpy().view(np.uint32), Y.view(np.uint32))
    with pytest.raises(B.BatsError):
        m.forward_bf16(Xb.cpu(), Yd)  # host buffers are refused
    m.close()


def test_network_gradient_matches_oracle(B):
    P = _net(3)
    rng = np.random.default_rng(4)
    X = bf16(rng.normal(size=(3000, 40)))
    T = rng.normal(size=(3000, 8)).astype(np.float32)
    m = B.Mlp(P)
    loss, g = m.loss_grad(X, T)
    lo, go = O.mlp_loss_grad(P.astype(np.float64), X.astype(np.float64), T.astype(np.float64))
    assert loss == pytest.approx(lo, rel=1e-2)
    assert _relnorm(g, go) <= 2e-2
    # every parameter group
    starts = np.cumsum([0, 64 * 40, 64, 64 * 64, 64, 8 * 64, 8])
    for a, b in zip(starts[:-1], starts[1:]):
        assert _relnorm(g[a:b], go[a:b]) <= 3e-2, (a, b)


@pytest.mark.parametrize("n", [1, 129, 5000])
def test_gradient_ragged_batches_match_oracle(B, n):
    """The trainer runs 128-row tiles, one CTA per SM: a batch of one row, a
    ragged last tile and a batch spread over many CTAs all give the oracle's
    loss and gradient."""
    P = _net(21)
    rng = np.random.default_rng(100 + n)
    X = bf16(rng.normal(size=(n, 40)))
    T = rng.normal(size=(n, 8)).astype(np.float32)
    m = B.Mlp(P)
    loss, g = m.loss_grad(X, T)
    m.close()
    lo, go = O.mlp_loss_grad(P.astype(np.float64), X.astype(np.float64), T.astype(np.float64))
    assert loss == pytest.approx(lo, rel=1e-2)
    assert _relnorm(g, go) <= 2e-2


@pytest.mark.parametrize("n", [129, 300001])
def test_gradient_is_the_same_bit_for_bit_run_to_run(B, n):
    """Per-CTA partial sums are added in CTA order, never by atomics: the loss
    and gradient of a batch do not change from call to call or handle to
    handle."""
    P = _net(23)
    rng = np.random.default_rng(200 + n)
    X = bf16(rng.normal(size=(n, 40)))
    T = rng.normal(size=(n, 8)).astype(np.float32)
    m = B.Mlp(P)
    l1, g1 = m.loss_grad(X, T)
    l2, g2 = m.loss_grad(X, T)
    m.close()
    m = B.Mlp(P)
    l3, g3 = m.loss_grad(X, T)
    m.close()
    assert l1 == l2 == l3
    assert np.array_equal(g1.view(np.uint32), g2.view(np.uint32))
    assert np.array_equal(g1.view(np.uint32), g3.view(np.uint32))


def test_train_epoch_equals_its_steps_bitwise(B):
    """An epoch on device-resident samples (the minibatch rows gathered by
    index inside the trainer) gives the weights of the same minibatches
    copied and stepped one by one, bit for bit."""
    import torch
    rng = np.random.default_rng(31)
    n, batch = 5000, 1024
    X = bf16(rng.normal(size=(n, 40)))
    T = (0.1 * rng.normal(size=(n, 8))).astype(np.float32)
    perm = rng.permutation(n).astype(np.int64)
    a, b = B.Mlp(seed=3), B.Mlp(seed=3)
    la = a.train_epoch(torch.from_numpy(X).cuda(), torch.from_numpy(T).cuda(), torch.from_numpy(perm).cuda(),
                       batch, 1e-3)
    lb = [b.train_step(np.ascontiguousarray(X[perm[s:s + batch]]), np.ascontiguousarray(T[perm[s:s + batch]]), 1e-3)
          for s in range(0, n - batch + 1, batch)]
    assert la == pytest.approx(float(np.mean(lb)), rel=1e-12)
    assert np.array_equal(a.get_params().view(np.uint32), b.get_params().view(np.uint32))
    a.close()
    b.close()


def test_train_epoch_rejects_bad_inputs(B):
    """Host buffers, a batch larger than the permutation and an index outside
    the sample set are refused (the index is checked before any access)."""
    import torch
    rng = np.random.default_rng(32)
    n = 300
    X = bf16(rng.normal(size=(n, 40)))
    T = rng.normal(size=(n, 8)).astype(np.float32)
    Xd, Td = torch.from_numpy(X).cuda(), torch.from_numpy(T).cuda()
    perm = torch.arange(n, dtype=torch.int64).cuda()
    m = B.Mlp(seed=4)
    with pytest.raises(B.BatsError) as e:
        m.train_epoch(X, T, perm.cpu().numpy(), 100, 1e-3)
    assert e.value.code == B.BATS_ERR_INVALID_ARG
    with pytest.raises(B.BatsError) as e:
        m.train_epoch(Xd, Td, perm, n + 1, 1e-3)
    assert e.value.code == B.BATS_ERR_INVALID_ARG
    bad = perm.clone()
    bad[17] = n
    with pytest.raises(B.BatsError) as e:
        m.train_epoch(Xd, Td, bad, 100, 1e-3)
    assert e.value.code == B.BATS_ERR_INVALID_ARG
    # the handle is still usable
    assert np.isfinite(m.train_epoch(Xd, Td, perm, 100, 1e-3))
    m.close()


def test_training_fits_a_teacher_network(B):
    teacher = _net(5, scale=0.2)
    rng = np.random.default_rng(6)
    X = bf16(rng.normal(size=(8192, 40)))
    T = np.array([O.mlp_forward(teacher.astype(np.float64), x.astype(np.float64))[2] for x in X[:8192]],
                 dtype=np.float32)
    m = B.Mlp(seed=7)
    l0, _ = m.loss_grad(X, T)
    for it in range(400):
        sl = slice((it * 1024) % 8192, (it * 1024) % 8192 + 1024)
        m.train_step(np.ascontiguousarray(X[sl]), np.ascontiguousarray(T[sl]), 3e-3)
    l1, _ = m.loss_grad(X, T)
    assert l1 < 0.2 * l0, (l0, l1)


def test_zero_network_stage_equals_plain_bitwise(B):
    q = W.blast()
    with B.Solver(q) as s:
        s.set_state(0, q.U0)
        s.step(3, 0.8)
        ref = s.get_state(0)
    with B.Solver(q) as s:
        s.set_mlp(np.zeros(B.BATS_MLP_NPARAM, np.float32))
        s.set_state(0, q.U0)
        s.step(3, 0.8)
        assert np.array_equal(s.get_state(0), ref)
        assert s.launch_count() == 3 * (2 + 2 * 3)


@pytest.mark.parametrize("precision", ["fp64", "mixed"])
def test_learned_stage_matches_oracle(B, precision):
    """Both stages learned: FP64 (inputs, network and correction in three
    launches) and mixed (the network fused into the stage kernel on the
    tensor cores) against the oracle, to BF16 accuracy of the network's
    effect."""
    q = W.blast()
    P = _net(8, scale=0.15)
    prec = B.BATS_FP64 if precision == "fp64" else B.BATS_MIXED
    with B.Solver(q, precision=prec) as s:
        s.set_mlp(P)
        s.set_state(0, q.U0)
        s.step_dt(2, 2e-3)
        Ug = s.get_state(0)
    ql = W.Problem(**{**q.__dict__, "learned": 1, "mlp": P.astype(np.float64)})
    Uo, _, _ = O.run(ql, q.U0, 2, dt=2e-3)
    U0, _, _ = O.run(q, q.U0, 2, dt=2e-3)
    scale = np.abs(Uo).reshape(8, -1).max(1)
    err = (np.abs(Ug - Uo).reshape(8, -1).max(1) / scale).max()
    effect = (np.abs(Uo - U0).reshape(8, -1).max(1) / scale).max()
    print("learned stage:", precision, "max scaled error", err, "effect of the network", effect)
    assert effect > 1e-4          # the network does change the solution
    # and the GPU reproduces that change to BF16 accuracy
    assert err <= (3e-2 if precision == "fp64" else 5e-2) * effect


def test_face_data_fluxes_reproduce_the_residual(B):
    """The dumped plain fluxes, differenced on the host, give the oracle's
    residual (no sources: Powell off, no B0)."""
    q = W.orszag_tang()
    with B.Solver(q) as s:
        s.set_state(0, q.U0)
        X, F = s.face_data(0)
    nb = q.nb
    F = F[:, :8].reshape(nb, 3, 64, 9, 8)   # block, direction, line (a + 8 b), f, variable
    dx = 1.0 / 16
    R = np.zeros((8, nb, 8, 8, 8))   # v, block, k, j, i
    for d in range(3):
        dF = (F[:, d, :, 1:, :] - F[:, d, :, :-1, :]) / dx     # block, line, cell along d, v
        dF = dF.reshape(nb, 8, 8, 8, 8)                         # block, b, a, c, v
        if d == 0:
            R -= dF.transpose(4, 0, 1, 2, 3)                    # (b=k, a=j, c=i)
        elif d == 1:
            R -= dF.transpose(4, 0, 1, 3, 2)                    # (b=k, a=i, c=j)
        else:
            R -= dF.transpose(4, 0, 3, 1, 2)                    # (b=j, a=i, c=k)
    Ro = O.residual(q, q.U0)
    scale = np.abs(Ro).reshape(8, -1).max(1)
    scale = np.where(scale > 0, scale, 1.0)  # u_z, B_z: identically zero in this z-invariant state
    assert (np.abs(R - Ro).reshape(8, -1).max(1) / scale).max() <= 1e-12
    # inputs of a uniform state in closed form
    qu = W.Problem("u", (0, 0, 0), (1, 1, 1), (1, 1, 1), W.as_leaf_array([(0, 0, 0, 0)]), (W.BC_PERIODIC,) * 6)
    rho, u, Bv, p = 2.0, np.array([0.3, -0.1, 0.2]), np.array([0.5, 0.2, -0.4]), 1.5
    W.uniform_state(qu, [rho, *u, *Bv, p])
    with B.Solver(qu) as s:
        s.set_state(0, qu.U0)
        Xu, _ = s.face_data(0)
    cf = O.fast_speed(qu.gamma, np.r_[rho, u, Bv, p], Bv, 0)
    c = abs(u[0]) + cf
    face = Xu.reshape(1, 3, 576, 40)[0, 0, 0]
    expect = np.r_[1.0, u / c, Bv / (np.sqrt(rho) * c), p / (rho * c * c)]
    assert np.allclose(face.reshape(5, 8), expect[None, :], rtol=1e-6)


def test_learned_graph_replay_equals_eager(B):
    q = W.blast()
    P = _net(9, scale=0.1)
    outs = []
    for graph in (0, 1):
        with B.Solver(q, precision=B.BATS_MIXED, persistent=1, use_graph=graph) as s:
            s.set_mlp(P)
            s.set_state(0, q.U0)
            s.step(2, 0.8)
            s.step(2, 0.8)
            outs.append(s.get_state(0))
    assert np.array_equal(outs[0], outs[1])


@pytest.mark.parametrize("precision,graph", [("fp64", 0), ("mixed", 0), ("mixed", 1)])
def test_learned_fallback_matches_oracle(B, precision, graph):
    """A network that doubles the dissipation of rho and e1 (weights 0, +-1,
    +-1000: exact in BF16) drives p to about -0.053 in 8 blocks next to the
    jump of a blast with p_in = 1.5 in the first step's second stage; the plain
    recompute gives p >= 0.0166 there and every other block keeps p >= 0.1.
    The decisions are far from the threshold, so the GPU must make the
    oracle's (8 block-stages) and match its (physical) result."""
    q = W.blast(pin=1.5)
    P = double_dissipation_net()
    ql = W.Problem(**{**q.__dict__, "learned": 1, "mlp": P})
    dt = 0.8 / O.cfl_smax(q, q.U0)
    Uo, _, _, nfb = O.run(ql, q.U0, 1, dt=dt, with_fallbacks=True)
    Up, _, _ = O.run(q, q.U0, 1, dt=dt)
    assert nfb == 8
    prec = B.BATS_FP64 if precision == "fp64" else B.BATS_MIXED
    with B.Solver(q, precision=prec, persistent=graph, use_graph=graph) as s:
        s.set_mlp(P.astype(np.float32))
        s.set_state(0, q.U0)
        s.step_dt(1, dt)
        Ug = s.get_state(0)
        assert s.fallbacks() == nfb
    assert physical_per_block(q.gamma, Ug).all()
    scale = np.abs(Uo).reshape(8, -1).max(1)
    err = (np.abs(Ug - Uo).reshape(8, -1).max(1) / scale).max()
    effect = (np.abs(Uo - Up).reshape(8, -1).max(1) / scale).max()
    print("fallback: max scaled error", err, "effect of the network", effect)
    assert effect > 1e-3
    assert err <= 3e-2 * effect


@pytest.mark.parametrize("precision", ["fp64", "mixed"])
def test_learned_last_stage_only_matches_oracle(B, precision):
    """The correction applied in the last stage of each step only (the stage
    whose fluxes make U^{n+1}): GPU against the oracle with the same option,
    to BF16 accuracy of the network's effect, in both precisions."""
    q = W.blast()
    P = _net(8, scale=0.15)
    prec = B.BATS_FP64 if precision == "fp64" else B.BATS_MIXED
    q.learned_last_only = 1
    with B.Solver(q, precision=prec) as s:
        s.set_mlp(P)
        s.set_state(0, q.U0)
        s.step_dt(2, 2e-3)
        Ug = s.get_state(0)
    ql = W.Problem(**{**q.__dict__, "learned": 1, "mlp": P.astype(np.float64)})
    Uo, _, _ = O.run(ql, q.U0, 2, dt=2e-3)
    q.learned_last_only = 0
    U0, _, _ = O.run(q, q.U0, 2, dt=2e-3)
    scale = np.abs(Uo).reshape(8, -1).max(1)
    err = (np.abs(Ug - Uo).reshape(8, -1).max(1) / scale).max()
    effect = (np.abs(Uo - U0).reshape(8, -1).max(1) / scale).max()
    print("learned, last stage only:", precision, "max scaled error", err, "effect", effect)
    assert effect > 1e-4
    assert err <= (3e-2 if precision == "fp64" else 5e-2) * effect


@pytest.mark.parametrize("variant", [0, 1])
def test_gelu_pair_within_its_bound(B, variant):
    """The kernels' GELU (packed FP32 around tanh.approx.f32, BF16 result;
    variant 1 the inference kernel's doubled form, halved) against the exact
    tanh-form GELU: |gelu2 - gelu| <= 0.5 |x| |dt| + the final BF16 rounding
    (2^-8 of the value, 1e-30 floor), with |dt| <= 2e-3, several times the
    hardware tanh's absolute error.  Over [-12, 12] and at the tails (beyond
    the FP32 range of x^2 the argument is +-inf, tanh +-1)."""
    x = np.concatenate([np.linspace(-12, 12, 200001),
                        [-3e19, -40.0, -7.5, 0.0, 1e-3, -1e-3, 7.5, 40.0, 3e19]]).astype(np.float32)
    y = B.bats_debug_gelu(x, variant)
    xd = x.astype(np.float64)
    exact = 0.5 * xd * (1 + np.tanh(0.7978845608028654 * (xd + 0.044715 * xd ** 3)))
    err = np.abs(y - exact)
    bound = 0.5 * np.abs(xd) * 2e-3 + np.abs(exact) * 2.0 ** -8 + 1e-30
    print("GELU pair: largest error / bound", float((err / bound).max()), "at x =", float(x[np.argmax(err / bound)]),
          "largest error", float(err.max()))
    assert np.all(err <= bound), (float((err / bound).max()), float(x[np.argmax(err / bound)]))
    assert np.all(y[x >= 6] == pytest.approx(x[x >= 6].astype(np.float64), rel=2 ** -8))
    assert np.all(np.abs(y[x <= -6]) <= 0.5 * np.abs(xd[x <= -6]) * 2e-3)
