"""The C-ABI library: it builds, loads and exports every entry point that
include/bats.h declares; descriptor validation needs no GPU.  CPU only."""
import ctypes
import os
import re

import numpy as np
import pytest

from paper_2501_06717_gb300 import workloads as W

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
HEADER = os.path.join(ROOT, "include", "bats.h")


@pytest.fixture(scope="module")
def libbats():
    from paper_2501_06717_gb300 import bats
    from paper_2501_06717_gb300 import build as B
    if not os.path.exists(bats.LIB_PATH):
        B.build()
    return bats


def _declared():
    src = open(HEADER).read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    return sorted(set(re.findall(r"\b(bats_[a-z_]+)\s*\(", src)))


def test_library_exports_every_declared_entry_point(libbats):
    names = _declared()
    assert "bats_create" in names and "bats_step" in names and len(names) >= 12
    L = ctypes.CDLL(libbats.LIB_PATH)
    missing = [n for n in names if not hasattr(L, n)]
    assert not missing, missing


def test_header_enumerations_match_the_binding_and_workloads(libbats):
    src = open(HEADER).read()
    enums = dict((k, int(v)) for k, v in re.findall(r"\b(BATS_[A-Z0-9_]+)\s*=\s*(-?\d+)", src))
    codes = dict((k, int(v)) for k, v in re.findall(r"#define\s+(BATS_[A-Z_]+)\s+\(?(-?\d+)\)?", src))
    for k, v in {**enums, **codes}.items():
        assert getattr(libbats, k) == v, k
    assert enums["BATS_BC_INFLOW"] == W.BC_INFLOW and enums["BATS_LIM_MC"] == W.LIM_MC
    assert enums["BATS_B0_LINEAR"] == W.B0_LINEAR and enums["BATS_RK_SSP2"] == W.RK_SSP2
    assert enums["BATS_LIM_NONE"] == W.LIM_NONE and enums["BATS_RK_EULER"] == W.RK_EULER
    assert enums["BATS_FLUX_HLL"] == W.FLUX_HLL and enums["BATS_FLUX_RUSANOV"] == W.FLUX_RUSANOV


def _create_code(libbats, prob):
    try:
        h = libbats.bats_create([prob], libbats.physics_from(prob))
    except libbats.BatsError as e:
        return e.code, str(e)
    libbats.bats_destroy(h)
    return 0, ""


def test_create_rejects_bad_trees_before_touching_the_gpu(libbats):
    """Validation happens on the host before any CUDA call, so these run
    without a GPU."""
    root = (2, 2, 2)
    ok = W.as_leaf_array(W.uniform_leaves(root))
    q = W.Problem("v", (0, 0, 0), (1, 1, 1), root, ok, (W.BC_PERIODIC,) * 6)
    # a gap
    q.leaves = ok[1:]
    assert _create_code(libbats, q)[0] == libbats.BATS_ERR_UNBALANCED_TREE
    # a leaf and its child
    q.leaves = W.as_leaf_array(W.uniform_leaves(root) + [(1, 0, 0, 0)])
    assert _create_code(libbats, q)[0] == libbats.BATS_ERR_UNBALANCED_TREE
    # a two-level jump
    lv = [lf for lf in W.uniform_leaves(root) if lf != (0, 0, 0, 0)]
    ch = W._children((0, 0, 0, 0))
    lv += [c for c in ch if c != (1, 1, 1, 1)] + W._children((1, 1, 1, 1))
    q.leaves = W.as_leaf_array(lv)
    code, msg = _create_code(libbats, q)
    assert code == libbats.BATS_ERR_UNBALANCED_TREE and "level" in msg
    # the two-level jump across a periodic wrap only
    lv = [lf for lf in W.uniform_leaves((3, 1, 1)) if lf != (0, 0, 0, 0)]
    ch = W._children((0, 0, 0, 0))
    lv += [c for c in ch if c != (1, 0, 0, 0)] + W._children((1, 0, 0, 0))
    q2 = W.Problem("wrap", (0, 0, 0), (3, 1, 1), (3, 1, 1), W.as_leaf_array(lv), (W.BC_PERIODIC,) * 6)
    assert _create_code(libbats, q2)[0] == libbats.BATS_ERR_UNBALANCED_TREE
    # periodic on one side only; leaf outside the domain; bad gamma
    q.leaves = ok
    q.bc = (W.BC_PERIODIC, W.BC_OUTFLOW, 0, 0, 0, 0)
    assert _create_code(libbats, q)[0] == libbats.BATS_ERR_INVALID_ARG
    q.bc = (W.BC_PERIODIC,) * 6
    q.leaves = W.as_leaf_array([(0, 0, 0, 0), (0, 5, 0, 0)])
    assert _create_code(libbats, q)[0] == libbats.BATS_ERR_INVALID_ARG
    q.leaves = ok
    q.gamma = 1.0
    assert _create_code(libbats, q)[0] == libbats.BATS_ERR_INVALID_ARG


def test_create_error_message_is_kept(libbats):
    root = (2, 2, 2)
    q = W.Problem("v", (0, 0, 0), (1, 1, 1), root, W.as_leaf_array(W.uniform_leaves(root))[1:],
                  (W.BC_PERIODIC,) * 6)
    code, msg = _create_code(libbats, q)
    assert code < 0 and "tile" in libbats.bats_last_error(None)


def test_binding_refuses_to_run_without_the_library(tmp_path, monkeypatch):
    """No CPU fallback: a missing libbats.so raises on first use."""
    from paper_2501_06717_gb300 import bats
    monkeypatch.setattr(bats, "_lib", None)
    monkeypatch.setattr(bats, "LIB_PATH", str(tmp_path / "missing.so"))
    with pytest.raises(RuntimeError, match="not built"):
        bats.lib()


def test_create_rejects_bad_options_and_empty_grids(libbats):
    """Unknown enumerations, refluxing or the HLL or Linde flux with the
    learned correction, and an empty leaf list are refused on the host, before
    any CUDA call."""
    root = (2, 2, 2)
    q = W.Problem("v", (0, 0, 0), (1, 1, 1), root, W.as_leaf_array(W.uniform_leaves(root)), (W.BC_PERIODIC,) * 6)
    for field, bad in (("limiter", 3), ("rk", 3), ("local_dt", 2), ("flux", 3), ("flux", -1)):
        ph = libbats.physics_from(q)
        setattr(ph, field, bad)
        with pytest.raises(libbats.BatsError) as e:
            libbats.bats_create([q], ph)
        assert e.value.code == libbats.BATS_ERR_INVALID_ARG, field
    ph = libbats.physics_from(q)
    ph.reflux = 1
    ph.learned = 1
    with pytest.raises(libbats.BatsError) as e:
        libbats.bats_create([q], ph)
    assert e.value.code == libbats.BATS_ERR_INVALID_ARG and "reflux" in str(e.value)
    for flux in (libbats.BATS_FLUX_HLL, libbats.BATS_FLUX_LINDE):
        ph = libbats.physics_from(q)
        ph.flux = flux
        ph.learned = 1
        with pytest.raises(libbats.BatsError) as e:
            libbats.bats_create([q], ph)
        assert e.value.code == libbats.BATS_ERR_INVALID_ARG and "Rusanov" in str(e.value)
    q.leaves = np.zeros((0, 4), np.int32)
    assert _create_code(libbats, q)[0] == libbats.BATS_ERR_INVALID_ARG
