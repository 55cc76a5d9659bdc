"""ctypes wrapper around the plain FP64 CPU oracle (``oracle.c``).

TEST INFRASTRUCTURE ONLY: the tests, ``__graft_entry__.smoke()`` and the
benchmark's CPU-baseline leg may use this module; the product path never
does.  It shares no code with the CUDA path and imports nothing from the
package.

A *problem* is any object with the attributes ``lo, hi, root, leaves, bc,
inflow, body_r, body, gamma, limiter, rk, b0, b0_param, powell`` (and
optionally ``learned``/``mlp``), with the state arrays laid out
``[8][n_blocks][8][8][8]`` (variable, block, k, j, i), conservative
variables ``(rho, rho u, B1, e1)``.
"""
import ctypes
import os
import subprocess

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "oracle.c")
_BUILD = os.path.join(_HERE, "_build")
_LIB_PATH = os.path.join(_BUILD, "liboracle.so")

MLP_IN, MLP_H, MLP_OUT = 40, 64, 8
MLP_NPARAM = MLP_H * MLP_IN + MLP_H + MLP_H * MLP_H + MLP_H + MLP_OUT * MLP_H + MLP_OUT

GT_INTERIOR, GT_COPY, GT_RESTRICT, GT_PROLONG, GT_INFLOW = range(5)


def build(force=False):
    """Compile oracle.c into _build/liboracle.so (no FMA contraction, OpenMP)."""
    os.makedirs(_BUILD, exist_ok=True)
    if (not force and os.path.exists(_LIB_PATH)
            and os.path.getmtime(_LIB_PATH) >= os.path.getmtime(_SRC)):
        return _LIB_PATH
    tmp = _LIB_PATH + ".tmp%d" % os.getpid()
    cmd = ["gcc", "-O2", "-std=c11", "-fopenmp", "-ffp-contract=off", "-fPIC", "-shared",
           "-o", tmp, _SRC, "-lm"]
    subprocess.run(cmd, check=True)
    os.replace(tmp, _LIB_PATH)
    return _LIB_PATH


class _Desc(ctypes.Structure):
    _fields_ = [
        ("lo", ctypes.c_double * 3),
        ("hi", ctypes.c_double * 3),
        ("root", ctypes.c_int32 * 3),
        ("n_leaves", ctypes.c_int32),
        ("leaves", ctypes.POINTER(ctypes.c_int32)),
        ("bc", ctypes.c_int32 * 6),
        ("inflow", ctypes.c_double * 8),
        ("body_r", ctypes.c_double),
        ("body", ctypes.c_double * 8),
        ("gamma", ctypes.c_double),
        ("limiter", ctypes.c_int32),
        ("rk", ctypes.c_int32),
        ("b0", ctypes.c_int32),
        ("powell", ctypes.c_int32),
        ("b0_param", ctypes.c_double * 12),
        ("learned", ctypes.c_int32),
        ("no_fallback", ctypes.c_int32),
        ("mlp", ctypes.POINTER(ctypes.c_double)),
        ("local_dt", ctypes.c_int32),
        ("reflux", ctypes.c_int32),
        ("flux", ctypes.c_int32),
        ("learned_last_only", ctypes.c_int32),
    ]


_lib = None


def lib():
    global _lib
    if _lib is None:
        _lib = ctypes.CDLL(build())
        D = ctypes.POINTER(_Desc)
        dp = ctypes.POINTER(ctypes.c_double)
        ip = ctypes.POINTER(ctypes.c_int32)
        lp = ctypes.POINTER(ctypes.c_long)
        _lib.or_validate.argtypes = [D]
        _lib.or_fill_ghosts.argtypes = [D, dp, dp, lp]
        _lib.or_ghost_info.argtypes = [D, ctypes.c_int, ip, ip]
        _lib.or_residual.argtypes = [D, dp, dp]
        _lib.or_stage.argtypes = [D, dp, dp, dp, ctypes.c_int, ctypes.c_double]
        _lib.or_stage_ex.argtypes = [D, dp, dp, dp, ctypes.c_int, ctypes.c_double, dp, ip]
        _lib.or_local_dt.argtypes = [D, dp, ctypes.c_double, dp]
        _lib.or_cfl_smax.argtypes = [D, dp, dp]
        _lib.or_run.argtypes = [D, dp, ctypes.c_int, ctypes.c_double, ctypes.c_double, dp, dp]
        _lib.or_run_ex.argtypes = [D, dp, ctypes.c_int, ctypes.c_double, ctypes.c_double, dp, dp, lp]
        _lib.or_fast_speed.argtypes = [ctypes.c_double, dp, dp, ctypes.c_int]
        _lib.or_fast_speed.restype = ctypes.c_double
        _lib.or_prim_from_cons.argtypes = [ctypes.c_double, dp, dp, ctypes.c_long]
        _lib.or_cons_from_prim.argtypes = [ctypes.c_double, dp, dp, ctypes.c_long]
        _lib.or_b0_at.argtypes = [D, dp, dp]
        _lib.or_limiter.argtypes = [ctypes.c_int, ctypes.c_double, ctypes.c_double]
        _lib.or_limiter.restype = ctypes.c_double
        _lib.or_numerical_flux.argtypes = [D, ctypes.c_int, dp, dp, dp, dp]
        _lib.or_numerical_flux_contact.argtypes = [D, ctypes.c_int, dp, dp, dp, ctypes.c_double, dp]
        _lib.or_num_threads.restype = ctypes.c_int
        _lib.or_set_threads.argtypes = [ctypes.c_int]
        _lib.or_mlp_forward.argtypes = [dp, dp, dp, dp, dp]
        _lib.or_mlp_features.argtypes = [ctypes.c_int, dp, dp, dp, ctypes.c_double, dp]
        _lib.or_mlp_loss_grad.argtypes = [dp, dp, dp, ctypes.c_long, dp]
        _lib.or_mlp_loss_grad.restype = ctypes.c_double
        _lib.or_gelu.argtypes = [ctypes.c_double]
        _lib.or_gelu.restype = ctypes.c_double
    return _lib


def _dp(a):
    return a.ctypes.data_as(ctypes.POINTER(ctypes.c_double))


def _ip(a):
    return a.ctypes.data_as(ctypes.POINTER(ctypes.c_int32))


class _Bound:
    """Keeps the numpy buffers a descriptor points to alive."""

    def __init__(self, prob):
        self.leaves = np.ascontiguousarray(prob.leaves, dtype=np.int32).reshape(-1, 4)
        d = _Desc()
        d.lo[:] = [float(x) for x in prob.lo]
        d.hi[:] = [float(x) for x in prob.hi]
        d.root[:] = [int(x) for x in prob.root]
        d.n_leaves = self.leaves.shape[0]
        d.leaves = _ip(self.leaves)
        d.bc[:] = [int(x) for x in prob.bc]
        d.inflow[:] = [float(x) for x in np.asarray(prob.inflow, dtype=np.float64).reshape(8)]
        d.body_r = float(prob.body_r)
        d.body[:] = [float(x) for x in np.asarray(prob.body, dtype=np.float64).reshape(8)]
        d.gamma = float(prob.gamma)
        d.limiter = int(prob.limiter)
        d.rk = int(prob.rk)
        d.b0 = int(prob.b0)
        d.powell = int(prob.powell)
        d.b0_param[:] = [float(x) for x in np.asarray(prob.b0_param, dtype=np.float64).reshape(12)]
        learned = int(getattr(prob, "learned", 0) or 0)
        mlp = getattr(prob, "mlp", None)
        self.mlp = None
        if learned and mlp is not None:
            self.mlp = np.ascontiguousarray(mlp, dtype=np.float64).reshape(MLP_NPARAM)
            d.learned = 1
            d.mlp = _dp(self.mlp)
        else:
            d.learned = 0
        d.no_fallback = int(getattr(prob, "no_fallback", 0) or 0)
        d.local_dt = int(getattr(prob, "local_dt", 0) or 0)
        d.reflux = int(getattr(prob, "reflux", 0) or 0)
        d.flux = int(getattr(prob, "flux", 0) or 0)
        d.learned_last_only = int(getattr(prob, "learned_last_only", 0) or 0)
        self.desc = d
        self.nb = d.n_leaves

    def ref(self):
        return ctypes.byref(self.desc)


def _check(rc, what):
    if rc != 0:
        raise ValueError("oracle %s failed with code %d" % (what, rc))


def _state(prob, U, nb):
    U = np.ascontiguousarray(U, dtype=np.float64)
    if U.size != 8 * nb * 512:
        raise ValueError("state has %d values, expected %d" % (U.size, 8 * nb * 512))
    return U


def validate(prob):
    """0 when the leaves tile the domain and are 2:1 balanced, else an error code."""
    b = _Bound(prob)
    return lib().or_validate(b.ref())


def fill_ghosts(prob, U):
    """Padded tiles [8][nb][12][12][12] with all ghost cells filled, and the
    number of prolongations that needed a source two or more levels coarser."""
    b = _Bound(prob)
    U = _state(prob, U, b.nb)
    T = np.zeros((8, b.nb, 12, 12, 12))
    deep = ctypes.c_long(0)
    _check(lib().or_fill_ghosts(b.ref(), _dp(U), _dp(T), ctypes.byref(deep)), "fill_ghosts")
    return T, deep.value


def ghost_info(prob, block):
    b = _Bound(prob)
    t = np.zeros((12, 12, 12), dtype=np.int32)
    s = np.zeros((12, 12, 12), dtype=np.int32)
    _check(lib().or_ghost_info(b.ref(), int(block), _ip(t), _ip(s)), "ghost_info")
    return t, s


def residual(prob, U):
    b = _Bound(prob)
    U = _state(prob, U, b.nb)
    R = np.zeros_like(U)
    _check(lib().or_residual(b.ref(), _dp(U), _dp(R)), "residual")
    return R.reshape(8, b.nb, 8, 8, 8)


def stage(prob, Uin, Ubase, kind, c, with_fallback_flags=False, dtc=None):
    """One stage; dtc (per cell, [nb][512]) makes the coefficient of cell i
    c * dtc[i] (local time stepping).  with_fallback_flags also returns, per
    block, 1 where the learned update was replaced by the plain one."""
    b = _Bound(prob)
    Uin = _state(prob, Uin, b.nb)
    Ubase = _state(prob, Ubase, b.nb)
    Uout = np.zeros_like(Uin)
    fb = np.zeros(b.nb, dtype=np.int32)
    dp_ = None
    if dtc is not None:
        dtc = np.ascontiguousarray(dtc, dtype=np.float64).reshape(b.nb * 512)
        dp_ = _dp(dtc)
    _check(lib().or_stage_ex(b.ref(), _dp(Uin), _dp(Ubase), _dp(Uout), int(kind), float(c), dp_, _ip(fb)), "stage")
    Uout = Uout.reshape(8, b.nb, 8, 8, 8)
    return (Uout, fb) if with_fallback_flags else Uout


def local_dt(prob, U, cfl):
    """Per-cell time steps dt_i = cfl / s_i, [nb][512] (0 in body cells)."""
    b = _Bound(prob)
    U = _state(prob, U, b.nb)
    out = np.zeros(b.nb * 512)
    _check(lib().or_local_dt(b.ref(), _dp(U), float(cfl), _dp(out)), "local_dt")
    return out.reshape(b.nb, 512)


def cfl_smax(prob, U):
    b = _Bound(prob)
    U = _state(prob, U, b.nb)
    s = ctypes.c_double(0.0)
    _check(lib().or_cfl_smax(b.ref(), _dp(U), ctypes.byref(s)), "cfl_smax")
    return s.value


def run(prob, U, nsteps, cfl=None, dt=None, with_fallbacks=False):
    """Advance n steps; returns (U, last dt, elapsed time) and, with
    with_fallbacks, the number of block-stages that fell back to the plain flux."""
    b = _Bound(prob)
    U = np.array(_state(prob, U, b.nb), copy=True)
    dtl = ctypes.c_double(0.0)
    tt = ctypes.c_double(0.0)
    nfb = ctypes.c_long(0)
    c = float(cfl) if cfl is not None else -1.0
    fdt = float(dt) if dt is not None else 0.0
    if c <= 0.0 and not fdt > 0.0:
        raise ValueError("need cfl > 0 or a fixed dt > 0")
    _check(lib().or_run_ex(b.ref(), _dp(U), int(nsteps), c, fdt, ctypes.byref(dtl), ctypes.byref(tt),
                           ctypes.byref(nfb)), "run")
    out = (U.reshape(8, b.nb, 8, 8, 8), dtl.value, tt.value)
    return out + (nfb.value,) if with_fallbacks else out


def fast_speed(gamma, W, B, direction):
    W = np.ascontiguousarray(W, dtype=np.float64).reshape(8)
    B = np.ascontiguousarray(B, dtype=np.float64).reshape(3)
    return lib().or_fast_speed(float(gamma), _dp(W), _dp(B), int(direction))


def prim_from_cons(gamma, U):
    """U [..., 8] -> W [..., 8] (last axis = variable)."""
    U = np.ascontiguousarray(U, dtype=np.float64)
    W = np.zeros_like(U)
    lib().or_prim_from_cons(float(gamma), _dp(U), _dp(W), U.size // 8)
    return W


def cons_from_prim(gamma, W):
    W = np.ascontiguousarray(W, dtype=np.float64)
    U = np.zeros_like(W)
    lib().or_cons_from_prim(float(gamma), _dp(W), _dp(U), W.size // 8)
    return U


def b0_at(prob, x):
    b = _Bound(prob)
    x = np.ascontiguousarray(x, dtype=np.float64).reshape(3)
    out = np.zeros(3)
    lib().or_b0_at(b.ref(), _dp(x), _dp(out))
    return out


def limiter(kind, a, b):
    return lib().or_limiter(int(kind), float(a), float(b))


def num_threads():
    return lib().or_num_threads()


def set_threads(n):
    lib().or_set_threads(int(n))


def numerical_flux(prob, direction, WL, WR, B0=(0.0, 0.0, 0.0), contact=None):
    """The numerical flux (prob.flux: Rusanov, HLL or Linde) through a face
    along `direction` between the primitive face states WL and WR; `contact`
    scales the Linde flux's restored contact part (0: HLL)."""
    b = _Bound(prob)
    WL = np.ascontiguousarray(WL, dtype=np.float64).reshape(8)
    WR = np.ascontiguousarray(WR, dtype=np.float64).reshape(8)
    B0 = np.ascontiguousarray(B0, dtype=np.float64).reshape(3)
    out = np.zeros(8)
    if contact is None:
        lib().or_numerical_flux(b.ref(), int(direction), _dp(WL), _dp(WR), _dp(B0), _dp(out))
    else:
        lib().or_numerical_flux_contact(b.ref(), int(direction), _dp(WL), _dp(WR), _dp(B0), float(contact),
                                        _dp(out))
    return out


def mlp_forward(params, x):
    P = np.ascontiguousarray(params, dtype=np.float64).reshape(MLP_NPARAM)
    x = np.ascontiguousarray(x, dtype=np.float64).reshape(MLP_IN)
    h1 = np.zeros(MLP_H)
    h2 = np.zeros(MLP_H)
    y = np.zeros(MLP_OUT)
    lib().or_mlp_forward(_dp(P), _dp(x), _dp(h1), _dp(h2), _dp(y))
    return h1, h2, y


def mlp_loss_grad(params, X, T):
    """MSE loss (1/(8n)) sum (y - t)^2 and its gradient (FP64 backprop)."""
    P = np.ascontiguousarray(params, dtype=np.float64).reshape(MLP_NPARAM)
    X = np.ascontiguousarray(X, dtype=np.float64).reshape(-1, MLP_IN)
    T = np.ascontiguousarray(T, dtype=np.float64).reshape(-1, MLP_OUT)
    g = np.zeros(MLP_NPARAM)
    loss = lib().or_mlp_loss_grad(_dp(P), _dp(X), _dp(T), X.shape[0], _dp(g))
    return loss, g


def gelu(x):
    return lib().or_gelu(float(x))


def mlp_features(direction, Wstencil, WL, WR, cmax):
    """The 40 normalised inputs of one face (see oracle.c)."""
    Ws = np.ascontiguousarray(Wstencil, dtype=np.float64).reshape(32)
    WL = np.ascontiguousarray(WL, dtype=np.float64).reshape(8)
    WR = np.ascontiguousarray(WR, dtype=np.float64).reshape(8)
    x = np.zeros(MLP_IN)
    lib().or_mlp_features(int(direction), _dp(Ws), _dp(WL), _dp(WR), float(cmax), _dp(x))
    return x
