"""Training pairs made by the solver, GPU training, and evaluation of the
learned flux correction.

Pairs.  A blast variant is run on the fine grid (every leaf of the coarse grid
refined once).  At a snapshot U_f^n the state is restricted to the coarse grid
(U_c^n, mean of the 8 children) and, with the coarse CFL step dt_c:
  * coarse: the network inputs and the plain Rusanov flux of the midpoint
    stage-2 input U_c* = U_c^n + (dt_c/2) R(U_c^n), face by face;
  * fine: two steps of dt_c/2 from U_f^n; the stage-2 fluxes of each fine step
    on the four fine faces that make up each coarse face.
The coarse face's target flux is the mean over the 4 sub-faces and 2 fine
steps (with the midpoint scheme a step's net flux is its stage-2 flux), and the
network's target is (target - Rusanov) rotated into the face frame and divided
by the flux units of the face (rho_ref c_ref, rho_ref c_ref^2,
sqrt(rho_ref) c_ref^2, rho_ref c_ref^3).

Training: Adam on the GPU, minibatches of face samples; the pairs stay on the
device and each epoch is one library call (bats_mlp_train_epoch).

Evaluation: the coarse grid with and without the network against the fine run
restricted to the coarse grid, at the same time and fixed dt; and (evaluate_4x)
the coarse runs and the plain fine run against a run at 4x restricted to the
coarse grid, which places the learned coarse run between the plain coarse and
the plain fine resolution.
"""
import math

import numpy as np

from . import bats as B
from . import workloads as W


def blast_variant(seed, resolution):
    """Blast with the centre offset by up to 0.1, inner pressure in [3, 30]
    and a random field direction (seeded)."""
    rng = np.random.default_rng(seed)
    centre = tuple(rng.uniform(-0.1, 0.1, 3))
    pin = float(rng.uniform(3.0, 30.0))
    bdir = tuple(rng.normal(size=3))
    return W.blast(resolution=resolution, pin=pin, centre=centre, bdir=bdir)


def children_map(coarse, fine):
    """C[b, o] = index of the fine leaf that is child o (= ox + 2 oy + 4 oz) of
    coarse leaf b."""
    pos = {tuple(lf): i for i, lf in enumerate(fine.leaves.tolist())}
    C = np.zeros((coarse.nb, 8), np.int64)
    for b, (l, i, j, k) in enumerate(coarse.leaves.tolist()):
        for o in range(8):
            C[b, o] = pos[(l + 1, 2 * i + (o & 1), 2 * j + ((o >> 1) & 1), 2 * k + ((o >> 2) & 1))]
    return C


def restrict_state(Uf, C):
    """Mean of each coarse cell's 8 fine children: [8][nbf][8][8][8] -> [8][nbc][8][8][8]."""
    nbc = C.shape[0]
    Uc = np.zeros((8, nbc, 8, 8, 8))
    for o in range(8):
        ox, oy, oz = o & 1, (o >> 1) & 1, o >> 2
        ch = Uf[:, C[:, o]].reshape(8, nbc, 4, 2, 4, 2, 4, 2).mean(axis=(3, 5, 7))
        Uc[:, :, oz * 4:(oz + 1) * 4, oy * 4:(oy + 1) * 4, ox * 4:(ox + 1) * 4] = ch
    return Uc


def _fine_face_index(C):
    """For every coarse face (block, d, line = a + 8 b, f) the indices of its 4
    fine sub-faces in the fine face arrays: [nbc * 1728, 4]."""
    nbc = C.shape[0]
    b, d, line, f = np.meshgrid(np.arange(nbc), np.arange(3), np.arange(64), np.arange(9), indexing="ij")
    b, d, line, f = (x.reshape(-1) for x in (b, d, line, f))
    a, bb = line % 8, line // 8
    od = (f >= 4).astype(np.int64)
    fl = 2 * f - 8 * od
    oa, ob = (a >= 4).astype(np.int64), (bb >= 4).astype(np.int64)
    lo_ax = np.where(d == 0, 1, 0)
    hi_ax = np.where(d == 2, 1, 2)
    out = np.zeros((b.size, 4), np.int64)
    for s in range(4):
        ea, eb = s & 1, s >> 1
        o_axis = np.zeros((b.size, 3), np.int64)
        o_axis[np.arange(b.size), d] = od
        o_axis[np.arange(b.size), lo_ax] = oa
        o_axis[np.arange(b.size), hi_ax] = ob
        o = o_axis[:, 0] + 2 * o_axis[:, 1] + 4 * o_axis[:, 2]
        child = C[b, o]
        fa, fb = 2 * (a % 4) + ea, 2 * (bb % 4) + eb
        out[:, s] = (child * 3 + d) * 576 + (fa + 8 * fb) * 9 + fl
    return out


def _rotation(nbc):
    """Per coarse face, the x/y/z component index of each face-frame component."""
    d = np.broadcast_to(np.arange(3)[None, :, None], (nbc, 3, 576)).reshape(-1)
    d1, d2 = (d + 1) % 3, (d + 2) % 3
    return np.stack([0 * d, 1 + d, 1 + d1, 1 + d2, 4 + d, 4 + d1, 4 + d2, 7 + 0 * d], axis=1)


def fine_face_index(Cs):
    """For every coarse face, the indices of its fine sub-faces r^2 levels of
    refinement down (Cs: the children maps of each refinement, coarse first):
    [nbc * 1728, 4^len(Cs)]."""
    idx = _fine_face_index(Cs[0])
    for C in Cs[1:]:
        nxt = _fine_face_index(C)
        idx = nxt[idx].reshape(idx.shape[0], -1)
    return idx


def targets(Fc, Ffs, Cs):
    """Normalised face-frame targets from the coarse dump Fc (n x 10) and the
    fine stage-2 dumps Ffs of the fine substeps (one per substep, the fine
    grid len(Cs) refinements down): the mean over the substeps and the fine
    sub-faces of each coarse face, minus the coarse Rusanov flux."""
    idx = fine_face_index(Cs)
    tgt = sum(F[idx, :8].mean(axis=1) for F in Ffs) / len(Ffs)
    dF = tgt - Fc[:, :8]
    rot = _rotation(Cs[0].shape[0])
    dF = np.take_along_axis(dF, rot, axis=1)
    rho, c = Fc[:, 8], Fc[:, 9]
    sc = np.stack([rho * c] + [rho * c * c] * 3 + [np.sqrt(rho) * c * c] * 3 + [rho * c ** 3], axis=1)
    return dF / sc


def make_pairs(variants, snapshots=(6, 14), cfl=0.8, keep=0.3, seed=0, precision=B.BATS_FP64, factor=2):
    """Training pairs from the blast variants (list of seeds), with targets
    from the plain solver at `factor` (2 or 4) times the coarse resolution
    (snapshots are counted in fine steps of the 2x run and scaled with the
    factor).  Returns (X, Y), float32, n x 40 and n x 8."""
    if factor not in (2, 4):
        raise ValueError("factor must be 2 or 4")
    rng = np.random.default_rng(seed)
    Xs, Ys = [], []
    nsub = factor
    for vs in variants:
        coarse, fine = blast_variant(vs, 1), blast_variant(vs, factor)
        if factor == 2:
            Cs = [children_map(coarse, fine)]
        else:
            mid = blast_variant(vs, 2)
            Cs = [children_map(coarse, mid), children_map(mid, fine)]
        with B.Solver(fine, precision=precision) as sf, B.Solver(coarse, precision=precision) as sc:
            Uf = fine.U0
            sf.set_state(0, Uf)
            done = 0
            for snap0 in snapshots:
                snap = snap0 * factor // 2
                if snap > done:
                    sf.step(snap - done, cfl)
                    done = snap
                Uf = sf.get_state(0)
                Uc = Uf
                for C in reversed(Cs):
                    Uc = restrict_state(Uc, C)
                sc.set_state(0, Uc)
                dtc = sc.dt(0, cfl)
                Xc, Fc = sc.face_data(0, stage_input=1, dt=dtc)
                Ffs = []
                for _ in range(nsub):
                    _, Ff = sf.face_data(0, stage_input=1, dt=dtc / nsub, with_inputs=False)
                    Ffs.append(Ff)
                    sf.step_dt(1, dtc / nsub)
                Y = targets(Fc, Ffs, Cs)
                sel = rng.uniform(size=Y.shape[0]) < keep
                ok = np.isfinite(Y).all(axis=1) & np.isfinite(Xc).all(axis=1)
                Xs.append(Xc[sel & ok])
                Ys.append(Y[sel & ok].astype(np.float32))
                # the fine run continues from the end of the substeps
                Uf = sf.get_state(0)
                sf.set_state(0, Uf)
                done += nsub
    return np.concatenate(Xs).astype(np.float32), np.concatenate(Ys).astype(np.float32)


def train(X, Y, epochs=4, batch=8192, lr=1e-3, seed=0, log=None):
    """Adam on the GPU; returns (params float32, per-epoch mean loss).  The
    minibatches of an epoch are consecutive slices of a seeded permutation of
    the samples (a ragged rest is left out)."""
    import torch
    rng = np.random.default_rng(seed)
    m = B.Mlp(seed=seed)
    hist = []
    n = X.shape[0]
    Xd = torch.from_numpy(np.ascontiguousarray(X, dtype=np.float32)).cuda()
    Yd = torch.from_numpy(np.ascontiguousarray(Y, dtype=np.float32)).cuda()
    torch.cuda.synchronize()
    for ep in range(epochs):
        perm = torch.from_numpy(rng.permutation(n).astype(np.int64)).cuda()
        torch.cuda.synchronize()
        hist.append(m.train_epoch(Xd, Yd, perm, batch, lr))
        if log:
            log("epoch %d loss %.4e" % (ep, hist[-1]))
    P = m.get_params()
    m.close()
    return P, hist


def evaluate(params, nsteps=16, cfl=0.8, precision=B.BATS_FP64, dt_safety=0.5):
    """Errors of the coarse run with and without the network against the fine
    run restricted to the coarse grid (the exact blast: centre 0, p_in 10,
    B along (1,1,0)), after nsteps coarse steps of a fixed dt.  Returns
    (plain error, learned error), each the mean over the 8 variables of
    ||U - U_ref||_1 / ||U_ref - U_0||_1."""
    coarse, fine = W.blast(), W.blast(resolution=2)
    C = children_map(coarse, fine)
    Uc0 = restrict_state(fine.U0, C)
    with B.Solver(coarse, precision=precision) as s:
        s.set_state(0, Uc0)
        dtc = dt_safety * s.dt(0, cfl)
        s.step_dt(nsteps, dtc)
        U_plain = s.get_state(0)
    with B.Solver(coarse, precision=precision) as s:
        s.set_mlp(params)
        s.set_state(0, Uc0)
        s.step_dt(nsteps, dtc)
        U_learn = s.get_state(0)
    with B.Solver(fine, precision=precision) as s:
        s.set_state(0, fine.U0)
        s.step_dt(2 * nsteps, 0.5 * dtc)
        U_ref = restrict_state(s.get_state(0), C)

    def err(U):
        e = np.abs(U - U_ref).reshape(8, -1).sum(1)
        d = np.abs(U_ref - Uc0).reshape(8, -1).sum(1)
        keep = d > 1e-12 * np.abs(U_ref).reshape(8, -1).sum(1)
        return float(np.mean(e[keep] / d[keep]))

    return err(U_plain), err(U_learn)


def evaluate_4x(params, nsteps=16, cfl=0.8, precision=B.BATS_FP64, dt_safety=0.5, last_only=0):
    """Errors against the plain run at 4x (every coarse leaf refined twice,
    7,680 blocks) restricted to the coarse grid, on the exact blast from the 4x
    initial state restricted to each resolution, fixed dt (dt_c, dt_c / 2,
    dt_c / 4).  Returns {"plain_1x", "learned_1x", "plain_2x"}, each the mean
    over the 8 variables of ||U - U_ref||_1 / ||U_ref - U_0||_1."""
    coarse, fine, fine4 = W.blast(), W.blast(resolution=2), W.blast(resolution=4)
    C12, C24 = children_map(coarse, fine), children_map(fine, fine4)
    U2_0 = restrict_state(fine4.U0, C24)
    U1_0 = restrict_state(U2_0, C12)
    with B.Solver(coarse, precision=precision) as s:
        s.set_state(0, U1_0)
        dtc = dt_safety * s.dt(0, cfl)
        s.step_dt(nsteps, dtc)
        U_plain = s.get_state(0)
    coarse_l = W.Problem(**{**coarse.__dict__, "learned_last_only": int(last_only)})
    with B.Solver(coarse_l, precision=precision) as s:
        s.set_mlp(params)
        s.set_state(0, U1_0)
        s.step_dt(nsteps, dtc)
        U_learn = s.get_state(0)
    with B.Solver(fine, precision=precision) as s:
        s.set_state(0, U2_0)
        s.step_dt(2 * nsteps, 0.5 * dtc)
        U_2x = restrict_state(s.get_state(0), C12)
    with B.Solver(fine4, precision=precision) as s:
        s.set_state(0, fine4.U0)
        s.step_dt(4 * nsteps, 0.25 * dtc)
        U_ref = restrict_state(restrict_state(s.get_state(0), C24), C12)

    def err(U):
        e = np.abs(U - U_ref).reshape(8, -1).sum(1)
        d = np.abs(U_ref - U1_0).reshape(8, -1).sum(1)
        keep = d > 1e-12 * np.abs(U_ref).reshape(8, -1).sum(1)
        return float(np.mean(e[keep] / d[keep]))

    return {"plain_1x": err(U_plain), "learned_1x": err(U_learn), "plain_2x": err(U_2x)}
