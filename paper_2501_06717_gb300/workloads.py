"""Seeded synthetic workloads: block trees and initial states.

This module generates inputs only.  It builds 2:1-balanced block trees
(8^3-cell blocks, leaves given as ``(level, i, j, k)``) and evaluates initial
primitive states at cell centres, converting them to the conservative
variables with the energy definition e1 = p/(gamma-1) + rho u^2/2 + B1^2/2
(Eq. 5, split field).  It contains none of the solver's arithmetic, and
both the CUDA path and the CPU oracle take its output unchanged.

State arrays are ``[8][n_blocks][8][8][8]`` (variable, block, k, j, i) of
``(rho, rho ux, rho uy, rho uz, B1x, B1y, B1z, e1)``.

Workloads (with their sources):
  * Orszag-Tang vortex on 2x2x2 periodic blocks (16^3 cells).
  * Spherical MHD blast on 4^3 root blocks over [-1,1]^3, one 2:1 level inside
    r < 0.4 (120 leaves), outflow boundaries, MC limiter.
  * Magnetosphere-like run: [-224,32]x[-128,128]^2 R_E, 5 refinement levels
    toward the origin, dipole B0, inner body at 2.5 R_E, solar-wind inflow at
    x = +32 (stand-in for the paper's 1998 event of Section 5.2, whose input
    data are not available).
  * 64 independent periodic grids of uneven size (64..4096 leaves,
    log-uniform, seeded) with smooth random states from Fourier modes k <= 4.
  * The paper's fast-wave test (Section 5.1, Table 2, Eq. 6): root blocks
    2*2^(m/3) per axis on [-32,32]^3, the -x-y-z octant refined once.
  * Linear waves (Alfven, sound, fast, divergence advection) and Brio-Wu
    shock tubes for the oracle's convergence and symmetry checks.
"""
from dataclasses import dataclass, field, replace
import math

import numpy as np

BC_PERIODIC, BC_OUTFLOW, BC_INFLOW = 0, 1, 2
LIM_MINMOD, LIM_MC, LIM_NONE = 0, 1, 2
RK_MIDPOINT, RK_SSP2, RK_EULER = 0, 1, 2
B0_NONE, B0_UNIFORM, B0_DIPOLE, B0_LINEAR = 0, 1, 2, 3
FLUX_RUSANOV, FLUX_HLL, FLUX_LINDE = 0, 1, 2

NC = 8  # cells per block per axis


@dataclass
class Problem:
    name: str
    lo: tuple
    hi: tuple
    root: tuple
    leaves: np.ndarray          # (n, 4) int32: level, i, j, k
    bc: tuple                   # -x, +x, -y, +y, -z, +z
    gamma: float = 5.0 / 3.0
    limiter: int = LIM_MINMOD
    rk: int = RK_MIDPOINT
    b0: int = B0_NONE
    b0_param: np.ndarray = field(default_factory=lambda: np.zeros(12))
    powell: int = 0
    inflow: np.ndarray = field(default_factory=lambda: np.zeros(8))
    body_r: float = 0.0
    body: np.ndarray = field(default_factory=lambda: np.zeros(8))
    cfl: float = 0.8
    nsteps: int = 10
    U0: np.ndarray = None       # [8][nb][8][8][8]
    learned: int = 0
    mlp: np.ndarray = None
    local_dt: int = 0
    reflux: int = 0
    flux: int = 0               # FLUX_RUSANOV, FLUX_HLL or FLUX_LINDE
    learned_last_only: int = 0  # learned form: the correction in the last stage of a step only

    @property
    def nb(self):
        return int(self.leaves.shape[0])

    @property
    def ncells(self):
        return self.nb * NC ** 3


# --------------------------------------------------------------------------
# Trees


def uniform_leaves(root):
    nx, ny, nz = root
    out = [(0, i, j, k) for k in range(nz) for j in range(ny) for i in range(nx)]
    return out


def _children(leaf):
    l, i, j, k = leaf
    return [(l + 1, 2 * i + (o & 1), 2 * j + ((o >> 1) & 1), 2 * k + ((o >> 2) & 1)) for o in range(8)]


def block_box(leaf, lo, hi, root):
    """Lower and upper corner of a leaf's block."""
    l, i, j, k = leaf
    lo = np.asarray(lo, float)
    hi = np.asarray(hi, float)
    n = np.asarray(root, float) * (1 << l)
    w = (hi - lo) / n
    b0 = lo + np.array([i, j, k]) * w
    return b0, b0 + w


def refine_where(leaves, pred, lo, hi, root, max_level):
    """Refine every leaf with level < max_level whose box satisfies pred."""
    out = []
    for lf in leaves:
        if lf[0] < max_level and pred(*block_box(lf, lo, hi, root)):
            out.extend(_children(lf))
        else:
            out.append(lf)
    return out


def balance(leaves, root, periodic):
    """Refine until every pair of leaves touching by a face, edge or corner
    (through periodic wraps) differs by at most one level."""
    S = set(map(tuple, leaves))
    changed = True
    while changed:
        changed = False
        by_level = sorted(S, key=lambda t: -t[0])
        for lf in by_level:
            if lf not in S:
                continue
            l, i, j, k = lf
            nbl = [r << l for r in root]
            for dk in (-1, 0, 1):
                for dj in (-1, 0, 1):
                    for di in (-1, 0, 1):
                        if di == dj == dk == 0:
                            continue
                        p = [i + di, j + dj, k + dk]
                        ok = True
                        for a in range(3):
                            if p[a] < 0 or p[a] >= nbl[a]:
                                if periodic[a]:
                                    p[a] %= nbl[a]
                                else:
                                    ok = False
                        if not ok:
                            continue
                        # covering leaf at a coarser level?
                        for lc in range(l - 1, -1, -1):
                            sh = l - lc
                            c = (lc, p[0] >> sh, p[1] >> sh, p[2] >> sh)
                            if c in S:
                                if lc < l - 1:
                                    S.remove(c)
                                    S.update(_children(c))
                                    changed = True
                                break
    return list(S)


def morton_sort(leaves):
    """Order leaves along a Z-order curve at the finest level."""
    maxl = max(l for l, *_ in leaves)

    def key(lf):
        l, i, j, k = lf
        s = maxl - l
        x, y, z = i << s, j << s, k << s
        code = 0
        for b in range(24):
            code |= ((x >> b) & 1) << (3 * b) | ((y >> b) & 1) << (3 * b + 1) | ((z >> b) & 1) << (3 * b + 2)
        return code

    return sorted(leaves, key=key)


def as_leaf_array(leaves):
    return np.ascontiguousarray(np.array(leaves, dtype=np.int32).reshape(-1, 4))


# --------------------------------------------------------------------------
# Cell centres and state assembly


def cell_centres(lo, hi, root, leaves):
    """Cell-centre coordinates x, y, z, each [nb][8][8][8] (k, j, i)."""
    leaves = np.asarray(leaves).reshape(-1, 4)
    lo = np.asarray(lo, float)
    hi = np.asarray(hi, float)
    root = np.asarray(root)
    nb = leaves.shape[0]
    out = []
    idx = np.arange(NC)
    for a in range(3):
        lev = leaves[:, 0]
        ncell = (root[a] * NC) * (2.0 ** lev)
        dx = (hi[a] - lo[a]) / ncell
        g = leaves[:, 1 + a][:, None] * NC + idx[None, :]
        xa = lo[a] + (g + 0.5) * dx[:, None]
        shape = [nb, 1, 1, 1]
        shape[3 - a] = NC
        out.append(np.broadcast_to(xa.reshape(shape), (nb, NC, NC, NC)).copy())
    return out


def prim_to_cons(W, gamma):
    """W = (rho, ux, uy, uz, B1x, B1y, B1z, p) stacked on axis 0 -> U."""
    rho, ux, uy, uz, bx, by, bz, p = W
    U = np.empty_like(np.asarray(W, dtype=np.float64))
    U[0] = rho
    U[1] = rho * ux
    U[2] = rho * uy
    U[3] = rho * uz
    U[4] = bx
    U[5] = by
    U[6] = bz
    U[7] = p / (gamma - 1.0) + 0.5 * rho * (ux * ux + uy * uy + uz * uz) + 0.5 * (bx * bx + by * by + bz * bz)
    return U


def _finish(prob, W):
    shape = (prob.nb, NC, NC, NC)
    Wa = np.stack([np.broadcast_to(np.asarray(w, dtype=np.float64), shape) for w in W])
    prob.U0 = np.ascontiguousarray(prim_to_cons(Wa, prob.gamma))
    return prob


def uniform_state(prob, W):
    nb = prob.nb
    Wf = np.empty((8, nb, NC, NC, NC))
    for v in range(8):
        Wf[v] = W[v]
    return _finish(prob, Wf)


# --------------------------------------------------------------------------
# Workloads


def orszag_tang(nsteps=10):
    """3-D (z-invariant) Orszag-Tang vortex on 2x2x2 periodic blocks of 8^3."""
    root = (2, 2, 2)
    lo, hi = (0.0, 0.0, 0.0), (1.0, 1.0, 1.0)
    leaves = as_leaf_array(uniform_leaves(root))
    prob = Problem("orszag_tang", lo, hi, root, leaves, (BC_PERIODIC,) * 6, gamma=5.0 / 3.0,
                   limiter=LIM_MINMOD, cfl=0.8, nsteps=nsteps)
    x, y, z = cell_centres(lo, hi, root, leaves)
    tp = 2.0 * math.pi
    rho = np.full_like(x, 25.0 / (36.0 * math.pi))
    p = np.full_like(x, 5.0 / (12.0 * math.pi))
    s4 = math.sqrt(4.0 * math.pi)
    W = [rho, -np.sin(tp * y), np.sin(tp * x), np.zeros_like(x),
         -np.sin(tp * y) / s4, np.sin(2.0 * tp * x) / s4, np.zeros_like(x), p]
    return _finish(prob, W)


def blast(resolution=1, nsteps=100, limiter=LIM_MC, pin=10.0, centre=(0.0, 0.0, 0.0), bdir=(1.0, 1.0, 0.0),
          roots_per_axis=4):
    """Spherical MHD blast on [-1,1]^3: root blocks refined once where the
    block intersects r < 0.4; resolution=2 (4) refines every leaf once (twice)
    more."""
    root = (roots_per_axis,) * 3
    lo, hi = (-1.0,) * 3, (1.0,) * 3
    leaves = uniform_leaves(root)

    def hits(b0, b1):
        q = np.clip(0.0, b0, b1)  # nearest point of the box to the origin
        return float(np.sqrt(np.sum(q * q))) < 0.4

    leaves = refine_where(leaves, hits, lo, hi, root, 1)
    if resolution not in (1, 2, 4):
        raise ValueError("blast: resolution must be 1, 2 or 4")
    for _ in range({1: 0, 2: 1, 4: 2}[resolution]):
        leaves = [c for lf in leaves for c in _children(lf)]
    leaves = balance(leaves, root, (False,) * 3)
    leaves = as_leaf_array(morton_sort(leaves))
    prob = Problem("blast" if resolution == 1 else "blast_x%d" % resolution, lo, hi, root, leaves, (BC_OUTFLOW,) * 6,
                   gamma=5.0 / 3.0, limiter=limiter, cfl=0.8, nsteps=nsteps)
    x, y, z = cell_centres(lo, hi, root, leaves)
    r = np.sqrt((x - centre[0]) ** 2 + (y - centre[1]) ** 2 + (z - centre[2]) ** 2)
    bd = np.asarray(bdir, float)
    bd = bd / np.linalg.norm(bd)
    one = np.ones_like(x)
    p = np.where(r < 0.1, pin, 0.1)
    W = [one, 0 * one, 0 * one, 0 * one, bd[0] * one, bd[1] * one, bd[2] * one, p]
    return _finish(prob, W)


# magnetosphere units: length R_E, density amu/cm^3, velocity km/s,
# B in sqrt(mu0 * 1 amu/cm^3) * 1 km/s, pressure amu/cm^3 (km/s)^2
_AMU = 1.66053906660e-27
_KB = 1.380649e-23
_MU0 = 4.0e-7 * math.pi
B_UNIT_NT = math.sqrt(_MU0 * _AMU * 1e6) * 1e3 * 1e9   # ~0.0457 nT
KT_UNIT_K = _AMU * 1e6 / _KB                          # temperature of 1 amu (km/s)^2 / k_B, in K


def magnetosphere_leaves():
    root = (4, 4, 4)
    lo, hi = (-224.0, -128.0, -128.0), (32.0, 128.0, 128.0)
    leaves = uniform_leaves(root)
    for lev in range(5):
        R = 150.0 / (2 ** lev)

        def near(b0, b1, R=R):
            q = np.clip(0.0, b0, b1)
            return float(np.sqrt(np.sum(q * q))) < R

        leaves = refine_where(leaves, near, lo, hi, root, lev + 1)
    leaves = balance(leaves, root, (False,) * 3)
    return lo, hi, root, as_leaf_array(morton_sort(leaves))


def magnetosphere(nsteps=200):
    lo, hi, root, leaves = magnetosphere_leaves()
    n_sw, u_sw, T_sw, bz_nT = 5.0, -400.0, 1.0e5, -5.0
    p_sw = n_sw * T_sw / KT_UNIT_K
    rho_body, T_body = 28.0, 2.5e4
    p_body = rho_body * T_body / KT_UNIT_K
    inflow = np.array([n_sw, u_sw, 0.0, 0.0, 0.0, 0.0, bz_nT / B_UNIT_NT, p_sw])
    body = np.array([rho_body, 0.0, 0.0, 0.0, 0.0, 0.0, 0.0, p_body])
    b0p = np.zeros(12)
    b0p[2] = -31000.0 / B_UNIT_NT  # dipole moment along -z: B0 = +31000 nT z at the equator, r = 1
    bc = (BC_OUTFLOW, BC_INFLOW, BC_OUTFLOW, BC_OUTFLOW, BC_OUTFLOW, BC_OUTFLOW)
    prob = Problem("magnetosphere", lo, hi, root, leaves, bc, gamma=5.0 / 3.0, limiter=LIM_MINMOD,
                   b0=B0_DIPOLE, b0_param=b0p, powell=1, inflow=inflow, body_r=2.5, body=body,
                   cfl=0.8, nsteps=nsteps)
    x, y, z = cell_centres(lo, hi, root, leaves)
    inb = (x * x + y * y + z * z) < 2.5 * 2.5
    W = [np.where(inb, body[v], inflow[v]) * np.ones_like(x) for v in range(8)]
    return _finish(prob, W)


def fast_wave_leaves(m):
    """Table 2, one GPU: 2*2^(m/3) root blocks per axis on [-32,32]^3 and the
    -x-y-z octant refined once: 15 * 2^m leaves."""
    if m % 3:
        raise ValueError("m must be a multiple of 3")
    n = 2 * 2 ** (m // 3)
    root = (n, n, n)
    lo, hi = (-32.0,) * 3, (32.0,) * 3
    leaves = uniform_leaves(root)
    leaves = refine_where(leaves, lambda b0, b1: bool(np.all(b1 <= 0.0)), lo, hi, root, 1)
    leaves = balance(leaves, root, (True,) * 3)
    return lo, hi, root, as_leaf_array(morton_sort(leaves))


FAST_WAVE_V0 = np.array([1.0, 0.0, 0.0, 0.005, 0.0, 0.04, 0.0, 0.00054])
FAST_WAVE_V1 = np.array([0.1, 0.005, 0.0, 0.0, 0.0, 0.004, 0.0, 0.00009])


def fast_wave(m=6, nsteps=500, amplitude=1.0):
    """Eq. 6: V = V0 + V1 cos(k.x), k = (pi/16, 0, 0), periodic."""
    lo, hi, root, leaves = fast_wave_leaves(m)
    prob = Problem("fast_wave_m%d" % m, lo, hi, root, leaves, (BC_PERIODIC,) * 6, gamma=5.0 / 3.0,
                   limiter=LIM_MINMOD, cfl=0.8, nsteps=nsteps)
    x, y, z = cell_centres(lo, hi, root, leaves)
    c = np.cos(math.pi / 16.0 * x)
    W = [FAST_WAVE_V0[v] + amplitude * FAST_WAVE_V1[v] * c for v in range(8)]
    return _finish(prob, W)


def _axis_coords(lo, hi, root, leaves):
    """Per-block cell-centre coordinates along each axis: 3 arrays [nb][8]."""
    leaves = np.asarray(leaves).reshape(-1, 4)
    out = []
    for a in range(3):
        dx = (hi[a] - lo[a]) / ((root[a] * NC) * (2.0 ** leaves[:, 0]))
        g = leaves[:, 1 + a][:, None] * NC + np.arange(NC)[None, :]
        out.append(lo[a] + (g + 0.5) * dx[:, None])
    return out


def _fourier(rng, xs, nmodes=8, kmax=4):
    """Sum of seeded cosine modes a cos(2 pi k.x + phi) with integer wave
    vectors |k_i| <= kmax on the unit cube, evaluated at cell centres from the
    per-axis coordinates xs (the modes are separable: e^{i k.x} is a product
    of per-axis factors).  Returns (value, gradient (3), amplitude sum,
    gradient bound), arrays [nb][8][8][8]."""
    nb = xs[0].shape[0]
    val = np.zeros((nb, NC, NC, NC))
    grad = [np.zeros((nb, NC, NC, NC)) for _ in range(3)]
    asum = 0.0
    gsum = 0.0
    for _ in range(nmodes):
        k = rng.integers(-kmax, kmax + 1, size=3)
        if not np.any(k):
            k[0] = 1
        a = rng.uniform(0.2, 1.0)
        ph = rng.uniform(0, 2 * math.pi)
        ex = np.exp(2j * math.pi * k[0] * xs[0])
        ey = np.exp(2j * math.pi * k[1] * xs[1])
        ez = np.exp(2j * math.pi * k[2] * xs[2]) * np.exp(1j * ph)
        E = (ez[:, :, None] * ey[:, None, :])[:, :, :, None] * ex[:, None, None, :]
        val += a * E.real
        s = -a * 2 * math.pi * E.imag
        for c in range(3):
            if k[c]:
                grad[c] += s * k[c]
        asum += a
        gsum += a * 2 * math.pi * float(np.abs(k).max())
    return val, grad, asum, gsum


def random_smooth_grid(n_target, seed):
    """One periodic unit-cube grid with about n_target leaves: root blocks
    4^3, 8^3 or 16^3, then leaves refined (up to 2 levels) inside seeded
    spheres until the count reaches n_target, then 2:1 balanced; smooth random
    state (rho, p in [0.5, 2], |u_i| <= 1, B = curl A with |B_i| <= 1)."""
    rng = np.random.default_rng(seed)
    r = 4 if n_target < 512 else (8 if n_target < 4096 else 16)
    root = (r, r, r)
    lo, hi = (0.0,) * 3, (1.0,) * 3
    L = np.array(uniform_leaves(root), dtype=np.int64)
    guard = 0
    while L.shape[0] < n_target and guard < 200:
        guard += 1
        cen = rng.uniform(0, 1, size=3)
        rad = rng.uniform(0.05, 0.25)
        maxl = int(rng.integers(1, 3))
        # nearest point of each leaf's box to the sphere centre (unit cube)
        w = 1.0 / (r * (2.0 ** L[:, 0]))
        b0 = L[:, 1:] * w[:, None]
        q = np.clip(cen[None, :], b0, b0 + w[:, None]) - cen[None, :]
        hit = (np.sqrt((q * q).sum(1)) < rad) & (L[:, 0] < maxl)
        n_new = L.shape[0] + 7 * int(hit.sum())
        if n_new > n_target * 1.25 and L.shape[0] > n_target * 0.5:
            continue
        kids = L[hit]
        ch = np.repeat(kids, 8, axis=0)
        o = np.tile(np.arange(8), kids.shape[0])
        ch[:, 0] += 1
        ch[:, 1] = 2 * ch[:, 1] + (o & 1)
        ch[:, 2] = 2 * ch[:, 2] + ((o >> 1) & 1)
        ch[:, 3] = 2 * ch[:, 3] + ((o >> 2) & 1)
        L = np.concatenate([L[~hit], ch])
    leaves = balance([tuple(int(v) for v in lf) for lf in L], root, (True,) * 3)
    leaves = as_leaf_array(morton_sort(leaves))
    prob = Problem("random_smooth", lo, hi, root, leaves, (BC_PERIODIC,) * 6, gamma=5.0 / 3.0,
                   limiter=LIM_MINMOD, cfl=0.8, nsteps=20)
    xs = _axis_coords(lo, hi, root, leaves)
    srho, _, a1, _ = _fourier(rng, xs)
    sp, _, a2, _ = _fourier(rng, xs)
    rho = 1.25 + 0.75 * srho / a1
    p = 1.25 + 0.75 * sp / a2
    u = []
    for _ in range(3):
        s, _, a, _ = _fourier(rng, xs)
        u.append(s / a)
    A = [_fourier(rng, xs) for _ in range(3)]
    # B = curl A, normalised by a bound on each component's magnitude
    bx = A[2][1][1] - A[1][1][2]
    by = A[0][1][2] - A[2][1][0]
    bz = A[1][1][0] - A[0][1][1]
    bnorm = A[0][3] + A[1][3] + A[2][3]
    W = [rho, u[0], u[1], u[2], bx / bnorm, by / bnorm, bz / bnorm, p]
    return _finish(prob, W)


def _smooth_grid_job(args):
    return random_smooth_grid(*args)


def batched_grids(n_grids=64, seed=20250112, lo_blocks=64, hi_blocks=4096, processes=None, first=None):
    """n_grids independent grids with log-uniform leaf targets in
    [lo_blocks, hi_blocks] (only the first `first` of them are built when
    given).  Each grid depends only on its own seed, so the result does not
    depend on `processes` (a spawn-context pool when > 1)."""
    rng = np.random.default_rng(seed)
    targets = np.exp(rng.uniform(math.log(lo_blocks), math.log(hi_blocks), size=n_grids)).astype(int)
    jobs = [(int(t), seed * 1000 + i) for i, t in enumerate(targets)]
    if first is not None:
        jobs = jobs[:first]
    if processes and processes > 1:
        import multiprocessing as mp
        with mp.get_context("spawn").Pool(processes) as pool:
            return pool.map(_smooth_grid_job, jobs, chunksize=1)
    return [random_smooth_grid(*j) for j in jobs]


def _line_problem(name, axis, ncells, transverse_blocks=1, bc=BC_PERIODIC, length=1.0, gamma=5.0 / 3.0,
                  limiter=LIM_MINMOD):
    if ncells % NC:
        raise ValueError("ncells must be a multiple of 8")
    root = [transverse_blocks] * 3
    root[axis] = ncells // NC
    lo = [0.0] * 3
    hi = [length * transverse_blocks * NC / ncells] * 3
    hi[axis] = length
    bcs = [BC_PERIODIC] * 6
    bcs[2 * axis] = bc
    bcs[2 * axis + 1] = bc
    leaves = as_leaf_array(uniform_leaves(tuple(root)))
    return Problem(name, tuple(lo), tuple(hi), tuple(root), leaves, tuple(bcs), gamma=gamma, limiter=limiter)


def _axis_vec(axis, n, t1, t2):
    v = [0.0, 0.0, 0.0]
    v[axis] = n
    v[(axis + 1) % 3] = t1
    v[(axis + 2) % 3] = t2
    return v


def alfven_wave(axis, ncells, amplitude=1e-6, limiter=LIM_MC, t_shift=0.0):
    """Linear Alfven wave along `axis`: rho = 1, p = 1, B = B_n = 1,
    du_t1 = A cos(2 pi s), dB_t1 = -sqrt(rho) du_t1, travelling at v_A = 1.
    t_shift evaluates the exact solution at time t."""
    prob = _line_problem("alfven", axis, ncells, limiter=limiter)
    X = cell_centres(prob.lo, prob.hi, prob.root, prob.leaves)
    s = X[axis] - t_shift
    du = amplitude * np.cos(2 * math.pi * s)
    one = np.ones_like(s)
    u = _axis_vec(axis, 0 * one, du, 0 * one)
    B = _axis_vec(axis, one, -du, 0 * one)
    W = [one, u[0], u[1], u[2], B[0], B[1], B[2], one]
    return _finish(prob, W)


def sound_wave(axis, ncells, amplitude=1e-6, limiter=LIM_MC, t_shift=0.0):
    """Linear sound wave, B = 0, rho = 1, c_s = 1 (p = 1/gamma)."""
    prob = _line_problem("sound", axis, ncells, limiter=limiter)
    g = prob.gamma
    X = cell_centres(prob.lo, prob.hi, prob.root, prob.leaves)
    s = X[axis] - t_shift
    d = amplitude * np.cos(2 * math.pi * s)
    one = np.ones_like(s)
    u = _axis_vec(axis, d, 0 * one, 0 * one)
    W = [one + d, u[0], u[1], u[2], 0 * one, 0 * one, 0 * one, one / g + d]
    return _finish(prob, W)


def fast_wave_linear(axis, ncells, eps=1e-3, limiter=LIM_MC, t_shift=0.0):
    """Eq. 6 background and eigenvector, scaled by eps, along `axis` over one
    wavelength (32 length units, as k = pi/16); travels at c_F = 0.05."""
    prob = _line_problem("fast_linear", axis, ncells, length=32.0, limiter=limiter)
    X = cell_centres(prob.lo, prob.hi, prob.root, prob.leaves)
    s = X[axis] - 0.05 * t_shift
    c = eps * np.cos(math.pi / 16.0 * s)
    V0, V1 = FAST_WAVE_V0, FAST_WAVE_V1
    one = np.ones_like(s)
    u = _axis_vec(axis, V0[1] + V1[1] * c, V0[2] + V1[2] * c, V0[3] + V1[3] * c)
    B = _axis_vec(axis, V0[4] + V1[4] * c, V0[5] + V1[5] * c, V0[6] + V1[6] * c)
    W = [V0[0] + V1[0] * c, u[0], u[1], u[2], B[0], B[1], B[2], V0[7] + V1[7] * c]
    return _finish(prob, W)


def divb_advection(axis, ncells, amplitude=1e-3, speed=1.0, t_shift=0.0, powell=1):
    """Uniform rho, p and flow u_n = speed with a non-solenoidal normal field
    B_n = 1 + A sin(2 pi s): with the Powell terms every quantity is advected
    at the flow speed."""
    prob = _line_problem("divb_advection", axis, ncells, limiter=LIM_MC)
    prob.powell = powell
    X = cell_centres(prob.lo, prob.hi, prob.root, prob.leaves)
    s = X[axis] - speed * t_shift
    one = np.ones_like(s)
    bn = one + amplitude * np.sin(2 * math.pi * s)
    u = _axis_vec(axis, speed * one, 0 * one, 0 * one)
    B = _axis_vec(axis, bn, 0 * one, 0 * one)
    W = [one, u[0], u[1], u[2], B[0], B[1], B[2], one]
    return _finish(prob, W)


def entropy_wave(axis, ncells, amplitude=0.2, speed=1.0, t_shift=0.0, limiter=LIM_MC):
    """A density wave rho = 1 + A sin(2 pi s) carried by the uniform flow
    u_n = speed at uniform pressure 1 and B = (0.3, 0.2, 0.1): an exact
    solution that moves at the flow speed."""
    prob = _line_problem("entropy_wave", axis, ncells, limiter=limiter)
    X = cell_centres(prob.lo, prob.hi, prob.root, prob.leaves)
    s = X[axis] - speed * t_shift
    one = np.ones_like(s)
    u = _axis_vec(axis, speed * one, 0 * one, 0 * one)
    B = _axis_vec(axis, 0.3 * one, 0.2 * one, 0.1 * one)
    W = [one + amplitude * np.sin(2 * math.pi * s), u[0], u[1], u[2], B[0], B[1], B[2], one]
    return _finish(prob, W)


def brio_wu(axis, ncells=64, nsteps=40):
    """Brio-Wu shock tube along `axis` (gamma = 2): rho 1 | 0.125,
    p 1 | 0.1, B_t 1 | -1, B_n = 0.75, outflow ends."""
    prob = _line_problem("brio_wu", axis, ncells, bc=BC_OUTFLOW, gamma=2.0, limiter=LIM_MINMOD)
    prob.nsteps = nsteps
    X = cell_centres(prob.lo, prob.hi, prob.root, prob.leaves)
    left = X[axis] < 0.5
    one = np.ones_like(X[0])
    rho = np.where(left, 1.0, 0.125)
    p = np.where(left, 1.0, 0.1)
    bt = np.where(left, 1.0, -1.0)
    B = _axis_vec(axis, 0.75 * one, bt, 0 * one)
    W = [rho, 0 * one, 0 * one, 0 * one, B[0], B[1], B[2], p]
    return _finish(prob, W)


def random_amr_tree(seed, root=(3, 3, 3), periodic=True, max_level=2, frac=0.3):
    """Random 2:1-balanced tree: leaves picked at random and refined, twice."""
    rng = np.random.default_rng(seed)
    leaves = uniform_leaves(root)
    for _ in range(max_level):
        pick = rng.uniform(size=len(leaves)) < frac
        new = []
        for lf, p in zip(leaves, pick):
            new.extend(_children(lf) if p and lf[0] < max_level else [lf])
        leaves = balance(new, root, (periodic,) * 3)
    return as_leaf_array(morton_sort(leaves))


def with_state(prob, W):
    """Copy of prob with the initial state from primitive fields W."""
    q = replace(prob)
    return _finish(q, W)
