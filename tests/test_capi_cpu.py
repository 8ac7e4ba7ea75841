"""CPU checks of the boundary: the CUDA library builds, loads and exports every entry point
include/lbm.h declares (no compute call: there is no GPU here), and the Python binding's
parameter struct matches the header's layout."""
import ctypes
import os
import re

import pytest

from paper_1712_07028_gb300 import build as B
from paper_1712_07028_gb300 import workloads as W

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _declared():
    src = open(os.path.join(ROOT, "include", "lbm.h")).read()
    return sorted(set(re.findall(r"^(?:int|const char\*)\s+(lbm_\w+)\(", src, re.M)))


@pytest.fixture(scope="module")
def built():
    try:
        return B.build()
    except (RuntimeError, FileNotFoundError) as e:
        pytest.skip("nvcc unavailable: %s" % e)


def test_library_exports_every_declared_symbol(built):
    lib = ctypes.CDLL(built)
    names = _declared()
    assert len(names) >= 15
    missing = [n for n in names if not hasattr(lib, n)]
    assert not missing, missing
    from paper_1712_07028_gb300 import lbm
    assert sorted(lbm.EXPORTS) == names


def test_params_layout_matches_header(built):
    from paper_1712_07028_gb300 import lbm
    # 12 int32 fields, then 7 doubles, then open_top, hydrostatic and split_every (padded to 8)
    assert ctypes.sizeof(lbm.Params) == 12 * 4 + 7 * 8 + 4 * 4
    assert lbm.Params.tau.offset == 48
    assert lbm.Params.open_top.offset == 104 and lbm.Params.hydrostatic.offset == 108
    assert lbm.Params.split_every.offset == 112


def test_arena_size_and_argument_checks(built):
    """lbm_arena_bytes needs no GPU: sizes scale with the grid, bad parameters are refused"""
    from paper_1712_07028_gb300 import lbm
    L = lbm.load()
    p = lbm.make_params(W.column_c0())
    n = ctypes.c_size_t()
    assert L.lbm_arena_bytes(ctypes.byref(p), ctypes.byref(n)) == 0
    assert n.value > 19 * 2 * 4 * 32 ** 3
    p16 = lbm.make_params(W.Workload(name="x", nx=32, ny=32, nz=32, storage="f16dev"))
    n16 = ctypes.c_size_t()
    assert L.lbm_arena_bytes(ctypes.byref(p16), ctypes.byref(n16)) == 0
    assert n16.value < n.value
    for field, bad in (("nx", 2), ("tau", 0.5), ("n_substeps", 0), ("storage", 7), ("max_spheres", 0)):
        q = lbm.make_params(W.column_c0())
        setattr(q, field, bad)
        assert L.lbm_arena_bytes(ctypes.byref(q), ctypes.byref(n)) == lbm.LBM_EINVAL, field
    assert L.lbm_strerror(-4) == b"density became non-positive or NaN"
    # face kinds: free-slip accepted; an open top needs a non-periodic z axis; the hydrostatic
    # start needs the open top
    ok = lbm.make_params(W.rising_bubble("B"))
    assert L.lbm_arena_bytes(ctypes.byref(ok), ctypes.byref(n)) == 0
    for field, bad in (("bc", 3), ("open_top", 2), ("hydrostatic", 2)):
        q = lbm.make_params(W.rising_bubble("B"))
        if field == "bc":
            q.bc[0] = bad
        else:
            setattr(q, field, bad)
        assert L.lbm_arena_bytes(ctypes.byref(q), ctypes.byref(n)) == lbm.LBM_EINVAL, field
    q = lbm.make_params(W.rising_bubble("B"))
    q.bc[2] = 1
    assert L.lbm_arena_bytes(ctypes.byref(q), ctypes.byref(n)) == lbm.LBM_EINVAL
    q = lbm.make_params(W.rising_bubble("B"))
    q.open_top = 0
    assert L.lbm_arena_bytes(ctypes.byref(q), ctypes.byref(n)) == lbm.LBM_EINVAL
    # splitting: a negative interval is refused; the labels (4 B a cell) and the part table
    # are in the arena only when bubbles split
    q = lbm.make_params(W.column_c0())
    q.split_every = -1
    assert L.lbm_arena_bytes(ctypes.byref(q), ctypes.byref(n)) == lbm.LBM_EINVAL
    q.split_every = 5
    ns = ctypes.c_size_t()
    assert L.lbm_arena_bytes(ctypes.byref(q), ctypes.byref(ns)) == 0
    q.split_every = 0
    assert L.lbm_arena_bytes(ctypes.byref(q), ctypes.byref(n)) == 0
    assert ns.value >= n.value + 4 * 32 ** 3
    assert L.lbm_strerror(lbm.LBM_ESPLIT).startswith(b"a bubble could not be split")


def test_sim_refuses_without_gpu(built):
    import torch
    if torch.cuda.is_available():
        pytest.skip("a GPU is present")
    from paper_1712_07028_gb300 import lbm
    with pytest.raises(RuntimeError):
        lbm.Sim(W.column_c0())
