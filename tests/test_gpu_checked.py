"""The checked build (-DBATS_CHECKED: every kernel index tested against its
range; an index outside it raises an error instead of an access) over every
code path of the stage: both precisions, first and second order, SSP-RK2 and
one-stage stepping, local time steps, refluxing, the HLL flux, the inner body
with a dipole B0, batched grids, the learned correction, the ghost-fill and
residual debug views.  No index may leave its range, and the checked library
must give the normal library's results (FP64 form to 1e-12, mixed form to its
parity tolerance 1e-5).  The checked runs happen in a child
process (one library per process, chosen by BATS_LIB)."""
import os
import subprocess
import sys

import numpy as np
import pytest

HERE = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, os.path.dirname(HERE))


def _cases():
    from paper_2501_06717_gb300 import workloads as W
    lv = W.random_amr_tree(5, root=(3, 3, 3), periodic=False, frac=0.3)
    amr = W.Problem("amr", (-1, -1, -1), (1, 1, 1), (3, 3, 3), lv,
                    (W.BC_INFLOW,) + (W.BC_OUTFLOW,) * 5, powell=1, limiter=W.LIM_MC)
    amr.inflow = np.array([1.0, 0.9, 0.0, -0.1, 0.3, 0.0, 0.0, 0.3])
    X = W.cell_centres(amr.lo, amr.hi, amr.root, amr.leaves)
    amr = W.with_state(amr, [1 + 0.2 * np.sin(3 * X[1]), 0.6 + 0.3 * np.cos(2 * X[2]), 0.1 * np.sin(2 * X[0]),
                             -0.1 + 0 * X[0], 0.3 + 0 * X[0], 0.2 * np.sin(2 * X[0]), 0.2 * np.cos(2 * X[1]),
                             0.3 + 0.1 * np.cos(2 * (X[1] + X[2]))])
    per = W.random_amr_tree(6, root=(3, 3, 3), periodic=True, frac=0.3)
    rfx = W.Problem("reflux", (0, 0, 0), (1, 1, 1), (3, 3, 3), per, (W.BC_PERIODIC,) * 6, limiter=W.LIM_MINMOD)
    X = W.cell_centres(rfx.lo, rfx.hi, rfx.root, rfx.leaves)
    tp = 2 * np.pi
    rfx = W.with_state(rfx, [1 + 0.3 * np.sin(tp * X[0]), 0.4 * np.cos(tp * X[1]), 0.2 * np.sin(tp * X[2]),
                             0.1 + 0 * X[0], 0.3 * np.sin(tp * X[1]), 0.2 + 0 * X[0], 0.1 * np.cos(tp * X[0]),
                             1 + 0.2 * np.cos(tp * (X[0] + X[1]))])
    rfx.reflux = 1
    out = []
    for prec in (0, 1):
        out.append(("amr", prec, amr, {}))
        out.append(("amr_hll", prec, amr, {"flux": W.FLUX_HLL}))
        out.append(("amr_ssp", prec, amr, {"rk": W.RK_SSP2}))
        out.append(("amr_euler_first_order", prec, amr, {"rk": W.RK_EULER, "limiter": W.LIM_NONE}))
        out.append(("amr_lts", prec, amr, {"local_dt": 1, "limiter": W.LIM_NONE}))
        out.append(("reflux", prec, rfx, {}))
        out.append(("magnetosphere", prec, None, {}))
    return out


def _run_all(out_path):
    """Every case through the library that BATS_LIB names; results to an npz."""
    from paper_2501_06717_gb300 import bats as B
    from paper_2501_06717_gb300 import workloads as W
    res = {}
    mag = W.magnetosphere()
    for name, prec, q, opts in _cases():
        q = mag if q is None else q
        q = W.Problem(**{**q.__dict__, **opts})
        key = "%s_%d" % (name, prec)
        with B.Solver(q, precision=prec) as s:
            s.set_state(0, q.U0)
            s.step(2, 0.5)
            res[key] = s.get_state(0)
            if name == "amr":
                s.set_state(0, q.U0)
                res[key + "_residual"] = s.residual(0)
                res[key + "_ghosts"] = s.fill_ghosts_w(0) if prec == 1 else s.fill_ghosts(0)
    # batched grids in one launch, persistent, from a CUDA graph
    probs = [W.Problem(**{**c[2].__dict__}) for c in _cases()[:1]] + [W.orszag_tang()]
    for p in probs:
        p.limiter, p.powell = W.LIM_MC, 1
    with B.Solver(probs, precision=1, persistent=1, blocks_per_cta=2, use_graph=1) as s:
        s.set_states()
        s.step(2, 0.5)
        s.step(2, 0.5)
        res["batched_0"] = s.get_state(0)
        res["batched_1"] = s.get_state(1)
    # the learned correction (a small fixed network)
    rng = np.random.default_rng(3)
    P = (rng.normal(0, 0.1, size=B.BATS_MLP_NPARAM)).astype(np.float32)
    q = W.blast()
    for prec in (0, 1):
        with B.Solver(q, precision=prec) as s:
            s.set_mlp(P)
            s.set_state(0, q.U0)
            s.step_dt(2, 2e-3)
            res["learned_%d" % prec] = s.get_state(0)
    np.savez(out_path, **res)


@pytest.mark.gpu
def test_checked_build_finds_no_index_out_of_range_and_matches(tmp_path):
    from paper_2501_06717_gb300 import build as BLD
    lib = BLD.build(checked=True)
    ref_path = str(tmp_path / "ref.npz")
    chk_path = str(tmp_path / "checked.npz")
    env = dict(os.environ)
    env.pop("BATS_LIB", None)
    subprocess.run([sys.executable, __file__, ref_path], check=True, env=env, timeout=1200)
    env["BATS_LIB"] = lib
    r = subprocess.run([sys.executable, __file__, chk_path], env=env, timeout=1800, capture_output=True, text=True)
    assert r.returncode == 0, r.stdout[-2000:] + r.stderr[-4000:]
    ref = np.load(ref_path)
    chk = np.load(chk_path)
    assert sorted(ref.files) == sorted(chk.files)
    for k in ref.files:
        a, b = ref[k], chk[k]
        s = np.abs(a).reshape(8, -1).max(1) if a.shape[0] == 8 else np.abs(a).max()
        s = np.where(np.asarray(s) > 0, s, 1.0)
        err = (np.abs(a - b).reshape(8, -1).max(1) / s).max() if a.shape[0] == 8 else np.abs(a - b).max() / s
        # FP64 form: the same arithmetic; mixed form: the extra checks may make
        # the compiler fuse FP32 multiply-adds differently, a 1e-7 effect
        mixed = k.endswith("_1") or k.startswith("batched") or "_1_" in k
        assert err <= (1e-5 if mixed else 1e-12), (k, err)


if __name__ == "__main__":
    _run_all(sys.argv[1])
