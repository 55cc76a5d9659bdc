"""Pins of the FP64 CPU oracle against facts the paper and the mathematics fix.

Each check would fail on a plausible slip in the oracle: a dropped flux or
source term, a wrong sign, a transposed index or axis, a wrong ghost source.
CPU only.
"""
import math
import os

import numpy as np
import pytest

from oracle import oracle as O
from paper_2501_06717_gb300 import workloads as W

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


def _golden_table(name):
    rows = {}
    with open(os.path.join(GOLDEN, name)) as f:
        for line in f:
            line = line.strip()
            if not line or line.startswith("#"):
                continue
            parts = line.split()
            rows[parts[0]] = [float(x) for x in parts[1:]]
    return rows


def _l1(a, b):
    return float(np.abs(np.asarray(a) - np.asarray(b)).mean())


# --------------------------------------------------------------------------
# Paper values: Eq. 6 fast wave and Table 2 grids


def test_fast_wave_speeds_from_eq6():
    """Section 5.1: with gamma = 5/3 the background V0 has c_s = 0.03,
    c_A = 0.04 and, for k perpendicular to B, c_F = 0.05."""
    g = _golden_table("fast_wave_eq6.txt")
    V0 = np.array(g["V0"])
    gamma = 5.0 / 3.0
    B = V0[4:7]
    cs = O.fast_speed(gamma, V0, np.zeros(3), 0)        # B = 0: sound speed
    assert cs == pytest.approx(g["c_s"][0], rel=1e-12)
    cf_perp = O.fast_speed(gamma, V0, B, 0)             # along k = x, B along y
    assert cf_perp == pytest.approx(g["c_F"][0], rel=1e-12)
    cf_par = O.fast_speed(gamma, V0, B, 1)              # along B: max(c_s, c_A)
    assert cf_par == pytest.approx(g["c_A"][0], rel=1e-12)
    assert g["k"][0] == pytest.approx(math.pi / 16)


@pytest.mark.parametrize("axis", [0, 1, 2])
def test_fast_wave_eigenvector_travels_at_cF(axis):
    """The Eq. 6 amplitude V1 is a fast eigenvector: at small amplitude the
    wave translates at c_F = 0.05, converging at second order."""
    errs = []
    t_end = 160.0
    for n in (32, 64, 128):
        q = W.fast_wave_linear(axis, n, eps=1e-4)
        dx = 32.0 / n
        ns = int(round(t_end / (0.4 * dx / 0.05)))
        dt = t_end / ns
        U, _, t = O.run(q, q.U0, ns, dt=dt)
        ex = W.fast_wave_linear(axis, n, eps=1e-4, t_shift=t).U0
        errs.append(_l1(U[0], ex[0]))
    orders = [math.log2(errs[i] / errs[i + 1]) for i in range(2)]
    assert errs[2] < errs[1] < errs[0]
    assert orders[-1] > 1.8, (errs, orders)


def test_table2_block_counts():
    """Table 2, one GPU: 2*2^(m/3) root blocks per axis, -x-y-z octant
    refined once, 15*2^m blocks; the oracle accepts each tree as 2:1 balanced."""
    with open(os.path.join(GOLDEN, "table2_blocks.txt")) as f:
        rows = [list(map(int, l.split())) for l in f if l.strip() and not l.startswith("#")]
    for m, per_axis, total_root, nb in rows:
        lo, hi, root, leaves = W.fast_wave_leaves(m)
        assert root == (per_axis,) * 3 and per_axis ** 3 == total_root
        assert leaves.shape[0] == nb
        if m <= 6:
            q = W.fast_wave(m)
            assert O.validate(q) == 0


def test_message_sizes_section_4_3():
    """Ghost values a block receives from one neighbour: face 8*8*2 cells,
    edge 8*2*2, corner 2*2*2 (times 8 variables), divided by 4 (face) or 2
    (edge) when the sender is finer and the receiver coarser."""
    g = _golden_table("message_sizes.txt")
    # 2x2x2 roots; the roots touching root (0,0,0) across its +x face, its
    # +x+y edge and its +x+y+z corner are refined once.
    root = (2, 2, 2)
    refined = [(1, 0, 0), (1, 1, 0), (1, 1, 1)]
    leaves = [lf for lf in W.uniform_leaves(root) if lf[1:] not in refined]
    for r in refined:
        leaves += W._children((0,) + r)
    leaves = W.as_leaf_array(leaves)
    q = W.Problem("msg", (0, 0, 0), (1, 1, 1), root, leaves, (W.BC_OUTFLOW,) * 6)
    assert O.validate(q) == 0
    coarse = 0  # leaf (0,0,0,0)
    t, s = O.ghost_info(q, coarse)
    # the +x face neighbours: fine children with local x index 0 (i == 2)
    face_senders = [i for i, lf in enumerate(leaves.tolist()) if lf[0] == 1 and lf[1] == 2 and lf[2] <= 1 and lf[3] <= 1]
    assert len(face_senders) == 4
    for fid in face_senders:
        # each sends one quarter of a face slab: 4*4*2 restricted cells
        assert np.all(t[s == fid] == O.GT_RESTRICT)
        face_cells = 0
        for k in range(2, 10):
            for j in range(2, 10):
                for i in (10, 11):
                    if s[k, j, i] == fid:
                        face_cells += 1
        assert face_cells * 8 == g["face"][1]
    # same-level face neighbour in +y: leaf (0,0,1,0) sends a full face slab
    same = [i for i, lf in enumerate(leaves.tolist()) if lf == [0, 0, 1, 0]][0]
    face_same = sum(1 for k in range(2, 10) for j in (10, 11) for i in range(2, 10) if s[k, j, i] == same)
    assert face_same * 8 == g["face"][0]
    # same-level edge neighbour (0,0,1,1): 8*2*2 cells of the +y+z edge
    edge_same = [i for i, lf in enumerate(leaves.tolist()) if lf == [0, 0, 1, 1]][0]
    ce = sum(1 for k in (10, 11) for j in (10, 11) for i in range(2, 10) if s[k, j, i] == edge_same)
    assert ce * 8 == g["edge"][0]
    # fine edge neighbour across the +x+y edge: half the edge, restricted
    fe = [i for i, lf in enumerate(leaves.tolist()) if lf == [1, 2, 2, 0]][0]
    cfe = sum(1 for k in range(2, 10) for j in (10, 11) for i in (10, 11) if s[k, j, i] == fe)
    assert cfe * 8 == g["edge"][1]
    # fine corner neighbour across +x+y+z: the whole 2x2x2 corner region
    fc = [i for i, lf in enumerate(leaves.tolist()) if lf == [1, 2, 2, 2]][0]
    cfc = sum(1 for k in (10, 11) for j in (10, 11) for i in (10, 11) if s[k, j, i] == fc)
    assert cfc * 8 == g["corner"][1] == g["corner"][0]


# --------------------------------------------------------------------------
# Tree validation


def test_tree_validation():
    root = (2, 2, 2)
    ok = W.as_leaf_array(W.uniform_leaves(root))
    q = W.Problem("v", (0, 0, 0), (1, 1, 1), root, ok, (W.BC_PERIODIC,) * 6)
    assert O.validate(q) == 0
    # a gap
    q.leaves = ok[1:]
    assert O.validate(q) == -1
    # an overlap (a leaf and its child)
    q.leaves = W.as_leaf_array(W.uniform_leaves(root) + [(1, 0, 0, 0)])
    assert O.validate(q) == -1
    # two-level jump across a face: refine (0,0,0,0) twice in one corner
    lv = [lf for lf in W.uniform_leaves(root) if lf != (0, 0, 0, 0)]
    ch = W._children((0, 0, 0, 0))
    lv += [c for c in ch if c != (1, 1, 1, 1)] + W._children((1, 1, 1, 1))
    q.leaves = W.as_leaf_array(lv)
    assert O.validate(q) == -2
    # mixed periodic / non-periodic ends of one axis are rejected
    q.leaves = ok
    q.bc = (W.BC_PERIODIC, W.BC_OUTFLOW, 0, 0, 0, 0)
    assert O.validate(q) == -1


def test_balanced_trees_need_no_deep_prolongation():
    """With 8^3 blocks, 2 ghost layers and face/edge/corner 2:1 balance, no
    prolongation stencil reaches a leaf two levels coarser."""
    trees = [W.random_amr_tree(s, periodic=p) for s in range(4) for p in (True, False)]
    for lv in trees:
        q = W.Problem("t", (0, 0, 0), (1, 1, 1), (3, 3, 3), lv,
                      (W.BC_PERIODIC,) * 6 if lv is trees[0] else (W.BC_OUTFLOW,) * 6)
        q.bc = (W.BC_PERIODIC,) * 6
        if O.validate(q) != 0:
            q.bc = (W.BC_OUTFLOW,) * 6
        assert O.validate(q) == 0
        W.uniform_state(q, [1, 0, 0, 0, 0, 0, 0, 1])
        rng = np.random.default_rng(1)
        U = q.U0 + rng.uniform(0, 0.1, size=q.U0.shape)
        _, deep = O.fill_ghosts(q, U)
        assert deep == 0
    mq = W.magnetosphere(nsteps=1)
    _, deep = O.fill_ghosts(mq, mq.U0)
    assert deep == 0


# --------------------------------------------------------------------------
# Ghost fill


def test_ghost_fill_uniform_periodic_equals_wrapped_array():
    """On a uniform periodic grid every ghost value is the wrap-indexed value
    of the monolithic array (brute force)."""
    root = (3, 2, 2)
    lv = W.as_leaf_array(W.uniform_leaves(root))
    q = W.Problem("wrap", (0, 0, 0), (1, 1, 1), root, lv, (W.BC_PERIODIC,) * 6)
    rng = np.random.default_rng(7)
    U = rng.normal(size=(8, lv.shape[0], 8, 8, 8))
    T, _ = O.fill_ghosts(q, U)
    N = [r * 8 for r in root]
    mono = np.zeros((8, N[2], N[1], N[0]))
    for b, (l, i, j, k) in enumerate(lv.tolist()):
        mono[:, k * 8:(k + 1) * 8, j * 8:(j + 1) * 8, i * 8:(i + 1) * 8] = U[:, b]
    for b, (l, i, j, k) in enumerate(lv.tolist()):
        gk = (np.arange(-2, 10) + k * 8) % N[2]
        gj = (np.arange(-2, 10) + j * 8) % N[1]
        gi = (np.arange(-2, 10) + i * 8) % N[0]
        ref = mono[:, gk][:, :, gj][:, :, :, gi]
        assert np.array_equal(T[:, b], ref)


def _linear_field(q, coef):
    X = W.cell_centres(q.lo, q.hi, q.root, q.leaves)
    U = np.zeros((8,) + X[0].shape)
    for v in range(8):
        U[v] = coef[v, 0] + coef[v, 1] * X[0] + coef[v, 2] * X[1] + coef[v, 3] * X[2]
    return U


def _tile_centres(q):
    """Centre of every tile cell (ghosts included) of every block."""
    lv = q.leaves
    out = []
    off = np.arange(-2, 10) + 0.5
    for a in range(3):
        n = np.array(q.root[a]) * 8 * (2.0 ** lv[:, 0])
        dx = (q.hi[a] - q.lo[a]) / n
        g = lv[:, 1 + a][:, None] * 8 + off[None, :]
        xa = q.lo[a] + g * dx[:, None]
        shape = [lv.shape[0], 1, 1, 1]
        shape[3 - a] = 12
        out.append(np.broadcast_to(xa.reshape(shape), (lv.shape[0], 12, 12, 12)))
    dxs = np.stack([(q.hi[a] - q.lo[a]) / (q.root[a] * 8 * 2.0 ** lv[:, 0]) for a in range(3)], 1)
    return out, dxs


@pytest.mark.parametrize("seed", [0, 1, 2])
def test_ghost_fill_reproduces_linear_fields(seed):
    """Copy, restriction (mean of 8) and prolongation (minmod-limited linear)
    are all exact for a linear field away from the domain edges."""
    lv = W.random_amr_tree(seed, root=(4, 4, 4), periodic=False, frac=0.3)
    q = W.Problem("lin", (0, 0, 0), (1, 1, 1), (4, 4, 4), lv, (W.BC_OUTFLOW,) * 6)
    assert O.validate(q) == 0
    rng = np.random.default_rng(seed)
    coef = rng.normal(size=(8, 4))
    U = _linear_field(q, coef)
    T, _ = O.fill_ghosts(q, U)
    (X, Y, Z), dxs = _tile_centres(q)
    margin = 6.0 * dxs.max(1)[:, None, None, None]
    inside = ((X > margin) & (X < 1 - margin) & (Y > margin) & (Y < 1 - margin) & (Z > margin) & (Z < 1 - margin))
    n_checked = 0
    for v in range(8):
        exact = coef[v, 0] + coef[v, 1] * X + coef[v, 2] * Y + coef[v, 3] * Z
        scale = np.abs(coef[v]).sum()
        err = np.abs(T[v] - exact)[inside]
        assert err.max() <= 1e-13 * scale
        n_checked += err.size
    # the trees do contain resolution changes
    kinds = set()
    for b in range(lv.shape[0]):
        t, _ = O.ghost_info(q, b)
        kinds |= set(np.unique(t).tolist())
    assert {O.GT_COPY, O.GT_RESTRICT, O.GT_PROLONG} <= kinds
    assert n_checked > 0


def test_restriction_is_mean_of_the_eight_children():
    """Every restricted ghost value equals the mean of the 8 fine cells of the
    source leaf that cover it (brute force over the source's interior)."""
    lv = W.random_amr_tree(5, root=(3, 3, 3), periodic=True, frac=0.35)
    q = W.Problem("restr", (0, 0, 0), (1, 1, 1), (3, 3, 3), lv, (W.BC_PERIODIC,) * 6)
    assert O.validate(q) == 0
    rng = np.random.default_rng(3)
    U = rng.uniform(1, 2, size=(8, lv.shape[0], 8, 8, 8))
    T, _ = O.fill_ghosts(q, U)
    L = lv.tolist()
    checked = 0
    for b in range(0, lv.shape[0], 3):
        t, s = O.ghost_info(q, b)
        l, bi, bj, bk = L[b]
        n = [q.root[a] * 8 * 2 ** l for a in range(3)]
        for (kk, jj, ii) in zip(*np.nonzero(t == O.GT_RESTRICT)):
            g = [(bi * 8 + ii - 2) % n[0], (bj * 8 + jj - 2) % n[1], (bk * 8 + kk - 2) % n[2]]
            src = s[kk, jj, ii]
            ls, si, sj, sk = L[src]
            assert ls == l + 1
            fi, fj, fk = 2 * g[0] - si * 8, 2 * g[1] - sj * 8, 2 * g[2] - sk * 8
            ref = U[:, src, fk:fk + 2, fj:fj + 2, fi:fi + 2].reshape(8, 8).mean(1)
            assert np.allclose(T[:, b, kk, jj, ii], ref, rtol=1e-15, atol=0)
            checked += 1
    assert checked > 50


def test_prolongation_preserves_the_coarse_mean():
    """The 8 fine ghost cells prolonged from one coarse cell average to it."""
    lv = W.random_amr_tree(11, root=(3, 3, 3), periodic=True, frac=0.35)
    q = W.Problem("pmean", (0, 0, 0), (1, 1, 1), (3, 3, 3), lv, (W.BC_PERIODIC,) * 6)
    assert O.validate(q) == 0
    rng = np.random.default_rng(5)
    U = rng.uniform(1, 2, size=(8, lv.shape[0], 8, 8, 8))
    T, _ = O.fill_ghosts(q, U)
    L = lv.tolist()
    groups = 0
    for b in range(lv.shape[0]):
        t, s = O.ghost_info(q, b)
        l, bi, bj, bk = L[b]
        n = [q.root[a] * 8 * 2 ** l for a in range(3)]
        cells = {}
        for (kk, jj, ii) in zip(*np.nonzero(t == O.GT_PROLONG)):
            g = ((bi * 8 + ii - 2) % n[0], (bj * 8 + jj - 2) % n[1], (bk * 8 + kk - 2) % n[2])
            cells.setdefault((g[0] >> 1, g[1] >> 1, g[2] >> 1), []).append((kk, jj, ii, s[kk, jj, ii]))
        for gc, members in cells.items():
            if len(members) != 8:
                continue
            src = members[0][3]
            ls, si, sj, sk = L[src]
            ci, cj, ck = gc[0] - si * 8, gc[1] - sj * 8, gc[2] - sk * 8
            coarse = U[:, src, ck, cj, ci]
            mean = np.mean([T[:, b, kk, jj, ii] for kk, jj, ii, _ in members], axis=0)
            assert np.allclose(mean, coarse, rtol=1e-14, atol=0)
            groups += 1
    assert groups > 20


# --------------------------------------------------------------------------
# Stage: exact invariants


UNIFORM_W = [1.3, 0.4, -0.2, 0.3, 0.7, -0.5, 0.25, 0.9]


@pytest.mark.parametrize("limiter", [W.LIM_MINMOD, W.LIM_MC])
@pytest.mark.parametrize("case", ["periodic_amr", "outflow_amr", "inflow_amr_b0"])
def test_uniform_state_preserved_bitwise(limiter, case):
    """A uniform state stays bitwise uniform, across resolution changes, with
    any boundary, limiter, a uniform B0 and the Powell terms on."""
    periodic = case == "periodic_amr"
    lv = W.random_amr_tree(2, root=(3, 3, 3), periodic=periodic, frac=0.3)
    bc = (W.BC_PERIODIC,) * 6 if periodic else (W.BC_OUTFLOW,) * 6
    q = W.Problem(case, (-1, -1, -1), (1, 1, 1), (3, 3, 3), lv, bc, limiter=limiter, powell=1)
    if case == "inflow_amr_b0":
        q.bc = (W.BC_INFLOW, W.BC_OUTFLOW, W.BC_OUTFLOW, W.BC_INFLOW, W.BC_OUTFLOW, W.BC_OUTFLOW)
        q.inflow = np.array(UNIFORM_W)
        q.b0 = W.B0_UNIFORM
        q.b0_param = np.array([0.3, -1.1, 0.6] + [0.0] * 9)
    W.uniform_state(q, UNIFORM_W)
    U, dt, _ = O.run(q, q.U0, 2, cfl=0.8)
    assert dt > 0
    assert np.array_equal(U, q.U0)


@pytest.mark.parametrize("maker", ["orszag_tang", "random_smooth"])
def test_conservation_on_periodic_grids(maker):
    """Without the Powell terms all 8 totals are conserved to round-off on a
    periodic uniform grid (fluxes telescope)."""
    if maker == "orszag_tang":
        q = W.orszag_tang()
    else:
        q = W.random_smooth_grid(27, seed=4)
        q.leaves = W.as_leaf_array(W.uniform_leaves(q.root))
        q = W.with_state(q, _smooth_prims(q))
    U, _, _ = O.run(q, q.U0, 5, cfl=0.8)
    s0 = q.U0.reshape(8, -1).sum(1)
    s1 = U.reshape(8, -1).sum(1)
    scale = np.abs(q.U0).reshape(8, -1).max(1) * q.U0[0].size
    assert np.all(np.abs(s1 - s0) <= 1e-14 * scale), (s1 - s0) / scale
    # the state did change
    assert np.abs(U - q.U0).max() > 1e-3


def _smooth_prims(q):
    X = W.cell_centres(q.lo, q.hi, q.root, q.leaves)
    tp = 2 * math.pi
    x, y, z = X
    return [1 + 0.3 * np.sin(tp * x), 0.5 * np.cos(tp * y), 0.3 * np.sin(tp * z), 0.2 * np.cos(tp * x),
            0.4 * np.sin(tp * x), 0.3, 0.2 * np.cos(tp * y), 1 + 0.2 * np.cos(tp * (x + y))]


def test_powell_conserves_mass_and_balances_sources():
    """With the Powell terms on, mass is still conserved and the change of
    each other total is the cell-volume sum of dt * source (round-off)."""
    q = W.random_smooth_grid(27, seed=9)
    q.leaves = W.as_leaf_array(W.uniform_leaves(q.root))
    q = W.with_state(q, _smooth_prims(q))
    q.powell = 1
    dt = 1e-3
    U1 = O.stage(q, q.U0, q.U0, 0, dt)
    q0 = W.Problem(**{**q.__dict__, "powell": 0})
    U0 = O.stage(q0, q.U0, q.U0, 0, dt)
    d_pow = U1.reshape(8, -1).sum(1) - q.U0.reshape(8, -1).sum(1)
    d_nop = U0.reshape(8, -1).sum(1) - q.U0.reshape(8, -1).sum(1)
    scale = np.abs(q.U0).reshape(8, -1).max(1) * q.U0[0].size
    assert abs(d_pow[0]) <= 1e-14 * scale[0]
    assert np.all(np.abs(d_nop) <= 1e-14 * scale)
    # the Powell source sum is visible and equals the sum of dt*S over cells
    diff = (U1 - U0).reshape(8, -1).sum(1)
    assert np.abs(diff[1:]).max() > 1e-9
    assert np.allclose(d_pow - d_nop, diff, rtol=1e-9, atol=1e-14 * scale.max())


def test_orszag_tang_z_invariant_and_divergence_free_start():
    """The z-invariant Orszag-Tang stays bitwise z-invariant, and its
    discrete div B is zero at t = 0 (B_x depends on y only, B_y on x only),
    so the first stage is the same with or without the Powell terms."""
    q = W.orszag_tang()
    U, _, _ = O.run(q, q.U0, 4, cfl=0.8)
    U5 = U.reshape(8, 2, 2, 2, 8, 8, 8)  # v, bk, bj, bi, k, j, i  (leaves in k, j, i order)
    z = U5.transpose(0, 1, 4, 2, 5, 3, 6).reshape(8, 16, 16, 16)
    assert np.array_equal(z, np.broadcast_to(z[:, :1], z.shape))
    q1 = W.Problem(**{**q.__dict__, "powell": 1})
    a = O.stage(q, q.U0, q.U0, 0, 1e-3)
    b = O.stage(q1, q.U0, q.U0, 0, 1e-3)
    assert np.array_equal(a, b)


def test_blast_symmetries():
    """Point inversion, z mirror and x<->y swap of the blast (B along
    (1,1,0)) hold to round-off on the AMR grid."""
    q = W.blast(nsteps=3)
    U, _, _ = O.run(q, q.U0, 3, cfl=0.8)
    X = W.cell_centres(q.lo, q.hi, q.root, q.leaves)
    key = {}
    for b in range(q.nb):
        for c in range(512):
            k, j, i = c // 64, (c // 8) % 8, c % 8
            key[(round(X[0][b, k, j, i], 12), round(X[1][b, k, j, i], 12), round(X[2][b, k, j, i], 12))] = (b, k, j, i)
    scale = np.abs(U).reshape(8, -1).max(1)
    worst = 0.0
    for (x, y, z), (b, k, j, i) in list(key.items())[::7]:
        u = U[:, b, k, j, i]
        bi = key[(round(-x, 12), round(-y, 12), round(-z, 12))]
        ui = U[(slice(None),) + bi]
        # inversion: scalars and B even, velocity odd
        sgn = np.array([1, -1, -1, -1, 1, 1, 1, 1])
        worst = max(worst, np.max(np.abs(ui - sgn * u) / scale))
        bm = key[(round(x, 12), round(y, 12), round(-z, 12))]
        um = U[(slice(None),) + bm]
        sgn = np.array([1, 1, 1, -1, 1, 1, -1, 1])  # mirror z: u_z and B_z odd (B as a polar vector)
        worst = max(worst, np.max(np.abs(um - sgn * u) / scale))
        bs = key[(round(y, 12), round(x, 12), round(z, 12))]
        us = U[(slice(None),) + bs]
        perm = [0, 2, 1, 3, 5, 4, 6, 7]
        worst = max(worst, np.max(np.abs(us[perm] - u) / scale))
    assert worst < 1e-13, worst


# --------------------------------------------------------------------------
# Convergence to exact linear solutions


def _convergence(make, ns_list, t_end, var_slice, dt_of_n):
    errs = []
    for n in ns_list:
        q = make(n, 0.0)
        steps = int(round(t_end / dt_of_n(n)))
        U, _, t = O.run(q, q.U0, steps, dt=t_end / steps)
        ex = make(n, t).U0
        errs.append(_l1(U[var_slice], ex[var_slice]))
    return errs, [math.log2(errs[i] / errs[i + 1]) for i in range(len(errs) - 1)]


@pytest.mark.parametrize("axis", [0, 1, 2])
def test_alfven_wave_second_order(axis):
    """Linear Alfven wave, one period: L1 error ratio tends to 4 (MC)."""
    errs, orders = _convergence(lambda n, t: W.alfven_wave(axis, n, t_shift=t), (32, 64, 128), 1.0,
                                slice(None), lambda n: 0.4 / n)
    assert errs[0] > errs[1] > errs[2]
    assert orders[-1] >= 1.8, (errs, orders)


@pytest.mark.parametrize("axis", [0, 1, 2])
def test_sound_wave_second_order(axis):
    errs, orders = _convergence(lambda n, t: W.sound_wave(axis, n, t_shift=t), (32, 64, 128), 0.5,
                                slice(None), lambda n: 0.4 / n)
    assert errs[0] > errs[1] > errs[2]
    assert orders[-1] >= 1.8, (errs, orders)


@pytest.mark.parametrize("axis", [0, 2])
def test_powell_terms_advect_divergence(axis):
    """With the Powell 8-wave terms a non-solenoidal B_n(x) on a uniform flow
    is advected with the flow (every variable), converging at second order;
    without them the state does not follow that solution."""
    mk = lambda n, t: W.divb_advection(axis, n, t_shift=t)
    errs, orders = _convergence(mk, (32, 64, 128), 0.25, slice(None), lambda n: 0.3 / n)
    assert errs[0] > errs[1] > errs[2]
    assert orders[-1] >= 1.7, (errs, orders)
    q = W.divb_advection(axis, 128, powell=0)
    steps = int(round(0.25 / (0.3 / 128)))
    U, _, t = O.run(q, q.U0, steps, dt=0.25 / steps)
    ex = W.divb_advection(axis, 128, t_shift=t).U0
    assert _l1(U, ex) > 20 * errs[2]


# --------------------------------------------------------------------------
# Symmetry under axis permutation


@pytest.mark.parametrize("fixed_dt", [True, False])
def test_brio_wu_identical_along_each_axis(fixed_dt):
    """Brio-Wu along x, y and z with cyclically permuted components gives
    bitwise the same profile at a fixed dt; with the CFL dt the 3-term speed
    sum is added in a permuted order, so the runs agree to round-off."""
    prof = []
    for axis in range(3):
        q = W.brio_wu(axis, ncells=64, nsteps=30)
        if fixed_dt:
            U, _, _ = O.run(q, q.U0, q.nsteps, dt=1.1e-3)
        else:
            U, _, _ = O.run(q, q.U0, q.nsteps, cfl=0.8)
        nb = q.nb
        # gather the line along the axis: blocks are ordered k, j, i
        U6 = U.reshape(8, *q.root[::-1], 8, 8, 8)
        full = U6.transpose(0, 1, 4, 2, 5, 3, 6).reshape(8, q.root[2] * 8, q.root[1] * 8, q.root[0] * 8)
        if axis == 0:
            line = full[:, 0, 0, :]
        elif axis == 1:
            line = full[:, 0, :, 0]
        else:
            line = full[:, :, 0, 0]
        # rotate vector components into (n, t1, t2)
        rot = [0, 1 + axis, 1 + (axis + 1) % 3, 1 + (axis + 2) % 3,
               4 + axis, 4 + (axis + 1) % 3, 4 + (axis + 2) % 3, 7]
        prof.append(line[rot])
        # uniform across the transverse directions
        tr = tuple(a for a in (1, 2, 3) if a != 3 - axis)
        assert np.array_equal(full, np.broadcast_to(np.take(np.take(full, [0], tr[0]), [0], tr[1]), full.shape))
    if fixed_dt:
        assert np.array_equal(prof[0], prof[1])
        assert np.array_equal(prof[0], prof[2])
    else:
        assert np.abs(prof[0] - prof[1]).max() <= 1e-14
        assert np.abs(prof[0] - prof[2]).max() <= 1e-14
    assert np.abs(prof[0][0] - prof[0][0][0]).max() > 0.1  # the shock tube evolved


# --------------------------------------------------------------------------
# Split field


def test_split_field_with_uniform_b0_equals_unsplit():
    """With a uniform B0 the split equations are the unsplit ones written
    for B1 = B - B0 and e1 = e - B0.B1 - B0^2/2, so both runs agree to
    round-off (pins every B0 term of the split flux)."""
    q = W.blast(nsteps=3)
    q.powell = 1
    B0 = np.array([0.4, 0.9, -0.3])
    # unsplit: B0 = 0, B = B_total
    U, _, _ = O.run(q, q.U0, 3, cfl=0.8)
    qs = W.Problem(**{**q.__dict__, "b0": W.B0_UNIFORM, "b0_param": np.r_[B0, np.zeros(9)]})
    U1 = q.U0.copy()
    U1[4:7] = q.U0[4:7] - B0[:, None, None, None, None]
    U1[7] = q.U0[7] - np.einsum("c,c...->...", B0, U1[4:7]) - 0.5 * B0 @ B0
    Us, _, _ = O.run(qs, U1, 3, cfl=0.8)
    Bt = Us[4:7] + B0[:, None, None, None, None]
    et = Us[7] + np.einsum("c,c...->...", B0, Us[4:7]) + 0.5 * B0 @ B0
    scale = np.abs(U).reshape(8, -1).max(1)
    assert np.abs(Us[0] - U[0]).max() <= 1e-12 * scale[0]
    assert np.abs(Us[1:4] - U[1:4]).max() <= 1e-12 * scale[1:4].max()
    assert np.abs(Bt - U[4:7]).max() <= 1e-12 * scale[4:7].max()
    assert np.abs(et - U[7]).max() <= 1e-12 * scale[7]
    assert np.abs(U - q.U0).max() > 1e-2


def test_static_dipole_state_is_preserved_bitwise():
    """u = 0, B1 = 0, uniform rho and p in a dipole B0: every flux difference
    and every source vanish exactly."""
    lv = W.random_amr_tree(3, root=(4, 4, 4), periodic=False, frac=0.3)
    q = W.Problem("dip", (-4.0, -4.0, -4.0), (4.0, 4.0, 4.0), (4, 4, 4), lv, (W.BC_OUTFLOW,) * 6,
                  b0=W.B0_DIPOLE, b0_param=np.r_[0.0, 0.0, -30.0, np.zeros(9)], powell=1)
    W.uniform_state(q, [2.0, 0, 0, 0, 0, 0, 0, 0.5])
    U, _, _ = O.run(q, q.U0, 2, dt=1e-3)
    assert np.array_equal(U, q.U0)


def test_b0_correction_cancels_spurious_force_of_a_linear_b0():
    """For a linear B0 with divergence and curl, a uniform B1 at rest is in
    equilibrium of the split system with the B0 correction: the discrete
    stress divergence of the B0-B1 cross terms equals (curl B0) x B1 +
    B1 div B0, which the correction removes (round-off)."""
    root = (2, 2, 2)
    lv = W.as_leaf_array(W.uniform_leaves(root))
    G = np.array([[0.3, 0.0, 0.0], [0.8, -0.1, 0.0], [0.0, 0.0, 0.5]])  # div = 0.7, curl = (0,0,0.8)
    q = W.Problem("linb0", (-1, -1, -1), (1, 1, 1), root, lv, (W.BC_OUTFLOW,) * 6, b0=W.B0_LINEAR,
                  b0_param=np.r_[0.2, 0.1, -0.4, G.reshape(-1)], powell=1)
    W.uniform_state(q, [1.0, 0, 0, 0, 0.6, -0.3, 0.45, 1.0])
    dt = 1e-2
    U = O.stage(q, q.U0, q.U0, 0, dt)
    # interior cells away from the outflow edges (ghosts there are copies)
    inner = U[:, :, 2:6, 2:6, 2:6] - q.U0[:, :, 2:6, 2:6, 2:6]
    assert np.abs(inner).max() <= 1e-13
    # without the correction the momentum would change at O(dt |B1| |G|)
    R = O.residual(q, q.U0)
    assert np.abs(R[:, :, 2:6, 2:6, 2:6]).max() <= 1e-12


# --------------------------------------------------------------------------
# Formulas with textbook values


def test_limiters_textbook_values():
    assert O.limiter(W.LIM_MINMOD, 1.0, 2.0) == 1.0
    assert O.limiter(W.LIM_MINMOD, -3.0, -2.0) == -2.0
    assert O.limiter(W.LIM_MINMOD, -1.0, 2.0) == 0.0
    assert O.limiter(W.LIM_MINMOD, 0.0, 2.0) == 0.0
    assert O.limiter(W.LIM_MC, 1.0, 3.0) == 2.0      # min(2, 6, 2)
    assert O.limiter(W.LIM_MC, 1.0, 1.5) == 1.25     # min(2, 3, 1.25)
    assert O.limiter(W.LIM_MC, -1.0, -10.0) == -2.0
    assert O.limiter(W.LIM_MC, 1.0, -1.0) == 0.0


def test_cfl_closed_form_for_a_uniform_unmagnetised_state():
    """B = 0: the fast speed is the sound speed, so dt = cfl / sum_d
    (|u_d| + c_s)/dx_d."""
    root = (2, 1, 1)
    lv = W.as_leaf_array(W.uniform_leaves(root))
    q = W.Problem("cfl", (0, 0, 0), (2.0, 0.5, 0.25), root, lv, (W.BC_PERIODIC,) * 6)
    rho, u, p = 1.7, np.array([0.3, -1.2, 0.05]), 2.3
    W.uniform_state(q, [rho, *u, 0, 0, 0, p])
    cs = math.sqrt(q.gamma * p / rho)
    dx = np.array([2.0 / 16, 0.5 / 8, 0.25 / 8])
    s = np.sum((np.abs(u) + cs) / dx)
    assert O.cfl_smax(q, q.U0) == pytest.approx(s, rel=1e-14)
    _, dt, _ = O.run(q, q.U0, 1, cfl=0.8)
    assert dt == pytest.approx(0.8 / s, rel=1e-14)


def test_primitive_round_trip():
    rng = np.random.default_rng(0)
    Wp = rng.uniform(0.1, 2, size=(100, 8))
    Wp[:, 1:7] -= 1.0
    U = O.cons_from_prim(5.0 / 3.0, Wp)
    W2 = O.prim_from_cons(5.0 / 3.0, U)
    assert np.allclose(W2, Wp, rtol=1e-12, atol=1e-13)
    # energy definition, Eq. 5, on one hand-computed state
    w1 = np.array([2.0, 1.0, 0.0, 0.0, 0.0, 3.0, 0.0, 1.0])
    u1 = O.cons_from_prim(5.0 / 3.0, w1[None])[0]
    assert u1[7] == pytest.approx(1.0 / (2.0 / 3.0) + 0.5 * 2.0 * 1.0 + 0.5 * 9.0)


def test_dipole_b0_field_values():
    """B0 of the moment m = -M z at the equator is +M z and at the pole -2M z
    (textbook dipole)."""
    q = W.Problem("d", (0, 0, 0), (1, 1, 1), (1, 1, 1), W.as_leaf_array([(0, 0, 0, 0)]), (0,) * 6,
                  b0=W.B0_DIPOLE, b0_param=np.r_[0, 0, -5.0, np.zeros(9)])
    assert np.allclose(O.b0_at(q, [2.0, 0, 0]), [0, 0, 5.0 / 8])
    assert np.allclose(O.b0_at(q, [0, 0, 2.0]), [0, 0, -2 * 5.0 / 8])
