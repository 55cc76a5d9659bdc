"""Thin ctypes binding of libbats (``include/bats.h``), same names as the C ABI.

Argument marshalling only: every step of the solver runs in the CUDA
library.  There is no fallback: if ``_build/libbats.so`` is missing, loading
raises.  Arrays may be numpy arrays (host) or torch tensors (host or
device); device tensors are passed to the library as device pointers.
"""
import ctypes
import os

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
# BATS_LIB selects another build of the same library (the checked build in
# the tests)
LIB_PATH = os.environ.get("BATS_LIB") or os.path.join(_HERE, "_build", "libbats.so")

BATS_OK = 0
BATS_ERR_INVALID_ARG = -1
BATS_ERR_UNBALANCED_TREE = -2
BATS_ERR_OUT_OF_MEMORY = -3
BATS_ERR_CUDA = -4
BATS_ERR_NONPHYSICAL = -5
BATS_ERR_TIMEOUT = -6
BATS_ERR_NOT_TRAINED = -7

BATS_BC_PERIODIC, BATS_BC_OUTFLOW, BATS_BC_INFLOW = 0, 1, 2
BATS_LIM_MINMOD, BATS_LIM_MC, BATS_LIM_NONE = 0, 1, 2
BATS_RK_MIDPOINT, BATS_RK_SSP2, BATS_RK_EULER = 0, 1, 2
BATS_FP64, BATS_MIXED = 0, 1
BATS_B0_NONE, BATS_B0_UNIFORM, BATS_B0_DIPOLE, BATS_B0_LINEAR = 0, 1, 2, 3
BATS_FLUX_RUSANOV, BATS_FLUX_HLL, BATS_FLUX_LINDE = 0, 1, 2
BATS_PHASE_STAGE, BATS_PHASE_DT, BATS_PHASE_TOTAL, BATS_NUM_PHASES = 0, 1, 2, 3


class bats_grid_desc(ctypes.Structure):
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
    ]


class bats_physics(ctypes.Structure):
    _fields_ = [
        ("gamma", ctypes.c_double),
        ("limiter", ctypes.c_int32),
        ("rk", ctypes.c_int32),
        ("precision", ctypes.c_int32),
        ("b0", ctypes.c_int32),
        ("b0_param", ctypes.c_double * 12),
        ("powell", ctypes.c_int32),
        ("learned", ctypes.c_int32),
        ("persistent", ctypes.c_int32),
        ("blocks_per_cta", ctypes.c_int32),
        ("ctas_per_sm", ctypes.c_int32),
        ("use_graph", ctypes.c_int32),
        ("local_dt", ctypes.c_int32),
        ("reflux", ctypes.c_int32),
        ("flux", ctypes.c_int32),
        ("learned_last_only", ctypes.c_int32),
    ]


class BatsError(RuntimeError):
    def __init__(self, code, msg):
        super().__init__("libbats error %d: %s" % (code, msg))
        self.code = code


_lib = None


def lib():
    """Load libbats.so (raises if it has not been built)."""
    global _lib
    if _lib is not None:
        return _lib
    if not os.path.exists(LIB_PATH):
        raise RuntimeError("libbats.so is not built (%s); run __graft_entry__.build()" % LIB_PATH)
    L = ctypes.CDLL(LIB_PATH)
    vp = ctypes.c_void_p
    dp = ctypes.c_void_p  # host or device double*
    L.bats_create.argtypes = [ctypes.POINTER(bats_grid_desc), ctypes.c_int, ctypes.POINTER(bats_physics), vp,
                              ctypes.POINTER(vp)]
    L.bats_destroy.argtypes = [vp]
    L.bats_destroy.restype = None
    L.bats_last_error.argtypes = [vp]
    L.bats_last_error.restype = ctypes.c_char_p
    L.bats_set_state.argtypes = [vp, ctypes.c_int, dp, ctypes.c_size_t]
    L.bats_get_state.argtypes = [vp, ctypes.c_int, dp, ctypes.c_size_t]
    L.bats_set_states.argtypes = [vp, dp, ctypes.c_size_t]
    L.bats_get_states.argtypes = [vp, dp, ctypes.c_size_t]
    L.bats_step.argtypes = [vp, ctypes.c_int, ctypes.c_double, ctypes.POINTER(ctypes.c_double)]
    L.bats_step_dt.argtypes = [vp, ctypes.c_int, ctypes.c_double, ctypes.POINTER(ctypes.c_double)]
    L.bats_get_dt.argtypes = [vp, ctypes.c_int, ctypes.c_double, ctypes.POINTER(ctypes.c_double)]
    L.bats_get_time.argtypes = [vp, ctypes.c_int, ctypes.POINTER(ctypes.c_double)]
    L.bats_get_timings.argtypes = [vp, ctypes.POINTER(ctypes.c_double), ctypes.c_int]
    L.bats_debug_fill_ghosts.argtypes = [vp, ctypes.c_int, dp, ctypes.c_size_t]
    L.bats_debug_fill_ghosts_w.argtypes = [vp, ctypes.c_int, dp, ctypes.c_size_t]
    L.bats_debug_residual.argtypes = [vp, ctypes.c_int, dp, ctypes.c_size_t]
    L.bats_debug_wait_timeout.argtypes = [vp]
    L.bats_set_launch.argtypes = [vp, ctypes.c_int, ctypes.c_int, ctypes.c_int, ctypes.c_int]
    L.bats_set_staging.argtypes = [vp, ctypes.c_int]
    L.bats_fp64_fma_rate.argtypes = [vp, ctypes.POINTER(ctypes.c_double)]
    L.bats_get_staging.argtypes = [vp]
    L.bats_get_staging.restype = ctypes.c_int
    L.bats_get_launch_count.argtypes = [vp, ctypes.POINTER(ctypes.c_longlong)]
    L.bats_get_fallbacks.argtypes = [vp, ctypes.POINTER(ctypes.c_longlong)]
    L.bats_debug_check_conversions.argtypes = [vp, vp, ctypes.c_int, vp, vp]
    L.bats_debug_gelu.argtypes = [vp, ctypes.c_int, ctypes.c_int, vp]
    L.bats_set_mlp.argtypes = [vp, vp]
    L.bats_debug_face_data.argtypes = [vp, ctypes.c_int, ctypes.c_int, ctypes.c_double, vp, vp, ctypes.c_size_t]
    L.bats_mlp_create.argtypes = [vp, ctypes.c_uint64, vp, ctypes.POINTER(vp)]
    L.bats_mlp_destroy.argtypes = [vp]
    L.bats_mlp_destroy.restype = None
    L.bats_mlp_set_params.argtypes = [vp, vp]
    L.bats_mlp_get_params.argtypes = [vp, vp]
    L.bats_mlp_forward.argtypes = [vp, vp, ctypes.c_int64, vp]
    L.bats_mlp_forward_bf16.argtypes = [vp, vp, ctypes.c_int64, vp]
    L.bats_mlp_sync.argtypes = [vp]
    L.bats_mlp_loss_grad.argtypes = [vp, vp, vp, ctypes.c_int64, vp, ctypes.POINTER(ctypes.c_double)]
    L.bats_mlp_train_step.argtypes = [vp, vp, vp, ctypes.c_int64, ctypes.c_float, ctypes.POINTER(ctypes.c_double)]
    L.bats_mlp_train_epoch.argtypes = [vp, vp, vp, ctypes.c_int64, vp, ctypes.c_int64, ctypes.c_int64,
                                       ctypes.c_float, ctypes.POINTER(ctypes.c_double)]
    L.bats_step_noalloc.argtypes = [ctypes.POINTER(bats_grid_desc), ctypes.POINTER(bats_physics), dp,
                                    ctypes.c_size_t, ctypes.c_int, ctypes.c_double, ctypes.c_double,
                                    ctypes.POINTER(ctypes.c_double), vp, ctypes.c_char_p, ctypes.c_size_t]
    _lib = L
    return L


def _ptr_and_size(a):
    """(pointer as int, number of elements) of a numpy array or torch tensor."""
    if hasattr(a, "data_ptr"):
        if not a.is_contiguous():
            raise ValueError("tensor must be contiguous")
        return a.data_ptr(), a.numel()
    if not (isinstance(a, np.ndarray) and a.flags.c_contiguous):
        raise ValueError("array must be a C-contiguous numpy array or torch tensor")
    return a.ctypes.data, a.size


def _check(h, rc):
    if rc != BATS_OK:
        msg = lib().bats_last_error(h)
        raise BatsError(rc, msg.decode() if msg else "")


# --------------------------------------------------------------------------
# Descriptors from workload problems


class _Grids:
    """ctypes array of bats_grid_desc and the leaf arrays it points to."""

    def __init__(self, problems):
        self.leaves = []
        self.arr = (bats_grid_desc * len(problems))()
        for d, p in zip(self.arr, problems):
            lv = np.ascontiguousarray(p.leaves, dtype=np.int32).reshape(-1, 4)
            self.leaves.append(lv)
            d.lo[:] = [float(x) for x in p.lo]
            d.hi[:] = [float(x) for x in p.hi]
            d.root[:] = [int(x) for x in p.root]
            d.n_leaves = lv.shape[0]
            d.leaves = lv.ctypes.data_as(ctypes.POINTER(ctypes.c_int32))
            d.bc[:] = [int(x) for x in p.bc]
            d.inflow[:] = [float(x) for x in np.asarray(p.inflow, float).reshape(8)]
            d.body_r = float(p.body_r)
            d.body[:] = [float(x) for x in np.asarray(p.body, float).reshape(8)]


def physics_from(problem, precision=BATS_FP64, persistent=0, blocks_per_cta=1, ctas_per_sm=0, use_graph=0):
    ph = bats_physics()
    ph.gamma = float(problem.gamma)
    ph.limiter = int(problem.limiter)
    ph.rk = int(problem.rk)
    ph.precision = int(precision)
    ph.b0 = int(problem.b0)
    ph.b0_param[:] = [float(x) for x in np.asarray(problem.b0_param, float).reshape(12)]
    ph.powell = int(problem.powell)
    ph.learned = int(getattr(problem, "learned", 0) or 0)
    ph.persistent = int(persistent)
    ph.blocks_per_cta = int(blocks_per_cta)
    ph.ctas_per_sm = int(ctas_per_sm)
    ph.use_graph = int(use_graph)
    ph.local_dt = int(getattr(problem, "local_dt", 0) or 0)
    ph.reflux = int(getattr(problem, "reflux", 0) or 0)
    ph.flux = int(getattr(problem, "flux", 0) or 0)
    ph.learned_last_only = int(getattr(problem, "learned_last_only", 0) or 0)
    return ph


# --------------------------------------------------------------------------
# Same-name wrappers of the C ABI


def bats_create(problems, phys, stream=None):
    """problems: list of workload problems (grid descriptors); phys: bats_physics.
    stream: a torch.cuda.Stream, a raw cudaStream_t int, or None."""
    g = _Grids(problems)
    h = ctypes.c_void_p()
    s = None
    if stream is not None:
        s = ctypes.c_void_p(stream.cuda_stream if hasattr(stream, "cuda_stream") else int(stream))
    rc = lib().bats_create(g.arr, len(problems), ctypes.byref(phys), s, ctypes.byref(h))
    if rc != BATS_OK:
        msg = lib().bats_last_error(None)
        raise BatsError(rc, msg.decode() if msg else "")
    return h


def bats_destroy(h):
    lib().bats_destroy(h)


def bats_last_error(h):
    m = lib().bats_last_error(h)
    return m.decode() if m else ""


def bats_set_state(h, grid, U):
    p, n = _ptr_and_size(U)
    _check(h, lib().bats_set_state(h, int(grid), p, n))


def bats_get_state(h, grid, out):
    p, n = _ptr_and_size(out)
    _check(h, lib().bats_get_state(h, int(grid), p, n))
    return out


def bats_set_states(h, U):
    p, n = _ptr_and_size(U)
    _check(h, lib().bats_set_states(h, p, n))


def bats_get_states(h, out):
    p, n = _ptr_and_size(out)
    _check(h, lib().bats_get_states(h, p, n))
    return out


def bats_step(h, n, cfl):
    t = ctypes.c_double(0.0)
    _check(h, lib().bats_step(h, int(n), float(cfl), ctypes.byref(t)))
    return t.value


def bats_step_dt(h, n, dt):
    t = ctypes.c_double(0.0)
    _check(h, lib().bats_step_dt(h, int(n), float(dt), ctypes.byref(t)))
    return t.value


def bats_get_dt(h, grid, cfl):
    d = ctypes.c_double(0.0)
    _check(h, lib().bats_get_dt(h, int(grid), float(cfl), ctypes.byref(d)))
    return d.value


def bats_get_time(h, grid):
    t = ctypes.c_double(0.0)
    _check(h, lib().bats_get_time(h, int(grid), ctypes.byref(t)))
    return t.value


def bats_get_timings(h):
    ms = (ctypes.c_double * BATS_NUM_PHASES)()
    _check(h, lib().bats_get_timings(h, ms, BATS_NUM_PHASES))
    return list(ms)


def bats_debug_fill_ghosts(h, grid, out):
    p, n = _ptr_and_size(out)
    _check(h, lib().bats_debug_fill_ghosts(h, int(grid), p, n))
    return out


def bats_debug_fill_ghosts_w(h, grid, out):
    p, n = _ptr_and_size(out)
    _check(h, lib().bats_debug_fill_ghosts_w(h, int(grid), p, n))
    return out


def bats_debug_wait_timeout(h):
    _check(h, lib().bats_debug_wait_timeout(h))


def bats_debug_residual(h, grid, out):
    p, n = _ptr_and_size(out)
    _check(h, lib().bats_debug_residual(h, int(grid), p, n))
    return out


def bats_set_launch(h, persistent, blocks_per_cta, ctas_per_sm, use_graph):
    _check(h, lib().bats_set_launch(h, int(persistent), int(blocks_per_cta), int(ctas_per_sm), int(use_graph)))


def bats_set_staging(h, tma):
    _check(h, lib().bats_set_staging(h, int(tma)))


def bats_get_staging(h):
    return lib().bats_get_staging(h)


def bats_fp64_fma_rate(stream=None):
    """FP64 FMA throughput of the current device in GFLOP/s (2 flops per FMA)."""
    g = ctypes.c_double(0.0)
    s = None
    if stream is not None:
        s = ctypes.c_void_p(stream.cuda_stream if hasattr(stream, "cuda_stream") else int(stream))
    _check(None, lib().bats_fp64_fma_rate(s, ctypes.byref(g)))
    return g.value


def bats_get_launch_count(h):
    n = ctypes.c_longlong(0)
    _check(h, lib().bats_get_launch_count(h, ctypes.byref(n)))
    return n.value


def bats_get_fallbacks(h):
    n = ctypes.c_longlong(0)
    _check(h, lib().bats_get_fallbacks(h, ctypes.byref(n)))
    return n.value


def bats_debug_check_conversions(f, d):
    f = np.ascontiguousarray(f, dtype=np.float32)
    d = np.ascontiguousarray(d, dtype=np.float64)
    n = min(f.size, d.size)
    o1 = np.zeros(n, np.float64)
    o2 = np.zeros(n, np.float32)
    rc = lib().bats_debug_check_conversions(f.ctypes.data, d.ctypes.data, n, o1.ctypes.data, o2.ctypes.data)
    if rc != BATS_OK:
        raise BatsError(rc, "conversion check failed")
    return o1, o2


def bats_debug_gelu(x, variant=0):
    x = np.ascontiguousarray(x, dtype=np.float32)
    y = np.zeros_like(x)
    rc = lib().bats_debug_gelu(x.ctypes.data, int(x.size), int(variant), y.ctypes.data)
    if rc != BATS_OK:
        raise BatsError(rc, "GELU check failed")
    return y


BATS_MLP_NPARAM = 7304


def bats_set_mlp(h, params):
    """Install network weights (float32, BATS_MLP_NPARAM) and turn the learned
    form on; None turns it off."""
    if params is None:
        _check(h, lib().bats_set_mlp(h, None))
        return
    if not hasattr(params, "data_ptr"):
        params = np.ascontiguousarray(params, dtype=np.float32)
    p, n = _ptr_and_size(params)
    if n != BATS_MLP_NPARAM:
        raise ValueError("expected %d parameters" % BATS_MLP_NPARAM)
    _check(h, lib().bats_set_mlp(h, p))


def bats_debug_face_data(h, grid, nblocks, stage_input=0, dt=0.0, X=None, F=None, with_inputs=True):
    """Network inputs (n_faces x 40 float32, or None) and F (n_faces x 10
    float64: the plain Rusanov flux, rho_ref, c_ref) of every face of grid
    `grid`."""
    nf = nblocks * 3 * 576
    if X is None and with_inputs:
        X = np.zeros((nf, 40), np.float32)
    if F is None:
        F = np.zeros((nf, 10), np.float64)
    px = _ptr_and_size(X)[0] if X is not None else None
    pf, _ = _ptr_and_size(F)
    _check(h, lib().bats_debug_face_data(h, int(grid), int(stage_input), float(dt), px, pf, nf))
    return X, F


class Mlp:
    """The trainer: FP32 master weights + Adam state on the device."""

    def __init__(self, params=None, seed=0, stream=None):
        self.h = ctypes.c_void_p()
        s = None
        if stream is not None:
            s = ctypes.c_void_p(stream.cuda_stream if hasattr(stream, "cuda_stream") else int(stream))
        buf = None
        if params is not None:
            buf = np.ascontiguousarray(params, dtype=np.float32)
        rc = lib().bats_mlp_create(buf.ctypes.data if buf is not None else None, int(seed), s, ctypes.byref(self.h))
        if rc != BATS_OK:
            raise BatsError(rc, "bats_mlp_create failed")

    def close(self):
        if self.h:
            lib().bats_mlp_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def _rc(self, rc, what):
        if rc != BATS_OK:
            raise BatsError(rc, what)

    def set_params(self, params):
        buf = np.ascontiguousarray(params, dtype=np.float32)
        self._rc(lib().bats_mlp_set_params(self.h, buf.ctypes.data), "set_params")

    def get_params(self):
        out = np.zeros(BATS_MLP_NPARAM, np.float32)
        self._rc(lib().bats_mlp_get_params(self.h, out.ctypes.data), "get_params")
        return out

    def forward(self, X):
        X = X if hasattr(X, "data_ptr") else np.ascontiguousarray(X, dtype=np.float32)
        px, n = _ptr_and_size(X)
        n //= 40
        Y = np.zeros((n, 8), np.float32)
        self._rc(lib().bats_mlp_forward(self.h, px, n, Y.ctypes.data), "forward")
        return Y

    def forward_bf16(self, Xb, Y):
        """Queues Y = network(Xb) on the handle's stream: Xb (n x 24 int32
        words of BF16 pairs) and Y (n x 8 float32) device tensors."""
        px, n = _ptr_and_size(Xb)
        py, ny = _ptr_and_size(Y)
        if n % 24 or ny != (n // 24) * 8:
            raise ValueError("Xb must be n x 24 words and Y n x 8 floats")
        self._rc(lib().bats_mlp_forward_bf16(self.h, px, n // 24, py), "forward_bf16")

    def sync(self):
        self._rc(lib().bats_mlp_sync(self.h), "sync")

    def loss_grad(self, X, T):
        X = X if hasattr(X, "data_ptr") else np.ascontiguousarray(X, dtype=np.float32)
        T = T if hasattr(T, "data_ptr") else np.ascontiguousarray(T, dtype=np.float32)
        px, n = _ptr_and_size(X)
        pt, _ = _ptr_and_size(T)
        g = np.zeros(BATS_MLP_NPARAM, np.float32)
        loss = ctypes.c_double(0.0)
        self._rc(lib().bats_mlp_loss_grad(self.h, px, pt, n // 40, g.ctypes.data, ctypes.byref(loss)), "loss_grad")
        return loss.value, g

    def train_step(self, X, T, lr):
        px, n = _ptr_and_size(X)
        pt, _ = _ptr_and_size(T)
        loss = ctypes.c_double(0.0)
        self._rc(lib().bats_mlp_train_step(self.h, px, pt, n // 40, float(lr), ctypes.byref(loss)), "train_step")
        return loss.value

    def train_epoch(self, X, T, perm, batch, lr):
        """Adam steps over minibatches perm[s*batch:(s+1)*batch] of the rows of
        X (n x 40) and T (n x 8); X, T and perm (int64) are device tensors.
        Returns the mean loss of the steps."""
        px, n = _ptr_and_size(X)
        pt, _ = _ptr_and_size(T)
        pp, npm = _ptr_and_size(perm)
        loss = ctypes.c_double(0.0)
        self._rc(lib().bats_mlp_train_epoch(self.h, px, pt, n // 40, pp, npm, int(batch), float(lr),
                                            ctypes.byref(loss)), "train_epoch")
        return loss.value


BATS_NOALLOC_MAX_BLOCKS = 128
BATS_NOALLOC_MAX_MAP_ENTRIES = 16384


def bats_step_noalloc(problem, phys, U, steps, cfl=None, dt=None, stream=None):
    """Advance one grid held in the caller's buffer U (numpy array or torch
    tensor, host or device; overwritten) without any device allocation; see
    include/bats.h.  Returns the elapsed time."""
    g = _Grids([problem])
    p, n = _ptr_and_size(U)
    t = ctypes.c_double(0.0)
    buf = ctypes.create_string_buffer(256)
    s = None
    if stream is not None:
        s = ctypes.c_void_p(stream.cuda_stream if hasattr(stream, "cuda_stream") else int(stream))
    rc = lib().bats_step_noalloc(g.arr, ctypes.byref(phys), p, n, int(steps),
                                 float(cfl) if cfl else -1.0, float(dt) if dt else 0.0,
                                 ctypes.byref(t), s, buf, len(buf))
    if rc != BATS_OK:
        raise BatsError(rc, buf.value.decode())
    return t.value


# --------------------------------------------------------------------------
# Convenience wrapper


class Solver:
    """One handle over one or more workload problems (batched when several)."""

    def __init__(self, problems, precision=BATS_FP64, persistent=0, blocks_per_cta=1, ctas_per_sm=0,
                 use_graph=0, stream=None):
        if not isinstance(problems, (list, tuple)):
            problems = [problems]
        self.problems = list(problems)
        self.precision = int(precision)
        self.phys = physics_from(self.problems[0], precision, persistent, blocks_per_cta, ctas_per_sm, use_graph)
        self.h = bats_create(self.problems, self.phys, stream)

    def close(self):
        if self.h is not None:
            bats_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def __enter__(self):
        return self

    def __exit__(self, *exc):
        self.close()

    def set_state(self, grid, U):
        if isinstance(U, np.ndarray):
            U = np.ascontiguousarray(U, dtype=np.float64)
        bats_set_state(self.h, grid, U)

    def set_states(self):
        for g, p in enumerate(self.problems):
            self.set_state(g, p.U0)

    def get_state(self, grid=0):
        p = self.problems[grid]
        out = np.zeros((8, p.nb, 8, 8, 8))
        return bats_get_state(self.h, grid, out)

    def step(self, n, cfl):
        return bats_step(self.h, n, cfl)

    def step_dt(self, n, dt):
        return bats_step_dt(self.h, n, dt)

    def dt(self, grid=0, cfl=0.8):
        return bats_get_dt(self.h, grid, cfl)

    def time(self, grid=0):
        return bats_get_time(self.h, grid)

    def fill_ghosts(self, grid=0):
        p = self.problems[grid]
        out = np.zeros((8, p.nb, 12, 12, 12))
        return bats_debug_fill_ghosts(self.h, grid, out)

    def fill_ghosts_w(self, grid=0):
        p = self.problems[grid]
        out = np.zeros((8, p.nb, 12, 12, 12))
        return bats_debug_fill_ghosts_w(self.h, grid, out)

    def residual(self, grid=0):
        p = self.problems[grid]
        out = np.zeros((8, p.nb, 8, 8, 8))
        return bats_debug_residual(self.h, grid, out)

    def set_mlp(self, params):
        bats_set_mlp(self.h, params)

    def face_data(self, grid=0, stage_input=0, dt=0.0, with_inputs=True):
        return bats_debug_face_data(self.h, grid, self.problems[grid].nb, stage_input, dt, with_inputs=with_inputs)

    def set_staging(self, tma):
        bats_set_staging(self.h, tma)

    def staging(self):
        return bats_get_staging(self.h)

    def set_launch(self, persistent=0, blocks_per_cta=1, ctas_per_sm=0, use_graph=0):
        bats_set_launch(self.h, persistent, blocks_per_cta, ctas_per_sm, use_graph)

    def timings(self):
        return bats_get_timings(self.h)

    def launch_count(self):
        return bats_get_launch_count(self.h)

    def fallbacks(self):
        return bats_get_fallbacks(self.h)
