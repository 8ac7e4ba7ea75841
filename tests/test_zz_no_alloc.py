"""The allocation-free bubble-volume entry point (for callers that cannot call cudaMalloc)
against the volumes lbm_step computes, through the C ABI, on two calls in a row."""
import ctypes

import numpy as np
import pytest

from paper_1712_07028_gb300 import workloads as W

pytestmark = pytest.mark.gpu


def _noalloc(L, st, n_cells, nb, out, stream):
    return L.lbm_bubble_volumes_noalloc(ctypes.c_void_p(st["flags"].data_ptr()), ctypes.c_void_p(st["owner"].data_ptr()),
                                        ctypes.c_void_p(st["phi"].data_ptr()), n_cells, nb,
                                        ctypes.c_void_p(out.data_ptr()), stream)


def test_bubble_volumes_noalloc_matches_step():
    import torch
    assert torch.cuda.is_available()
    from paper_1712_07028_gb300 import lbm
    L = lbm.load()
    wl = W.column_c0()
    wl.sphere_mode = W.SPHERES_FIXED   # no covering after the step's bubble model
    sim = lbm.Sim(wl)
    nb = len(wl.bubbles)
    stream = ctypes.c_void_p(torch.cuda.current_stream().cuda_stream)
    for _ in range(2):
        sim.step(7)
        st = sim.export_state()
        out = torch.full((nb,), -1.0, dtype=torch.float64, device="cuda")
        assert _noalloc(L, st, sim.N, nb, out, stream) == lbm.LBM_OK
        torch.cuda.synchronize()
        _, V, _ = sim.bubbles()
        got = out.cpu().numpy()
        assert np.all(got > 100.0)
        assert np.abs(got - V).max() <= 1e-9 * np.abs(V).max(), (got, V)
    assert _noalloc(L, st, sim.N, 1025, out, stream) == lbm.LBM_EINVAL


def test_bubble_volumes_noalloc_per_id_after_a_merge():
    """two bubbles touching from the start merge (one root): the entry point's volumes are per
    id, and their sum over the root's ids is the merged volume lbm_bubbles reports"""
    import torch
    from paper_1712_07028_gb300 import lbm
    L = lbm.load()
    wl = W.Workload(name="two", nx=24, ny=16, nz=16, tau=0.7, g=(0, 0, 0), sphere_mode=W.SPHERES_FIXED,
                    bubbles=[W.Bubble((7.0, 8.0, 8.0), 4.0), W.Bubble((15.0, 8.0, 8.0), 4.0)])
    sim = lbm.Sim(wl)
    stream = ctypes.c_void_p(torch.cuda.current_stream().cuda_stream)
    for _ in range(2):
        sim.step(3)
        roots, _ = sim.bubble_roots()
        assert list(roots) == [0, 0]
        st = sim.export_state()
        out = torch.full((2,), -1.0, dtype=torch.float64, device="cuda")
        assert _noalloc(L, st, sim.N, 2, out, stream) == lbm.LBM_OK
        torch.cuda.synchronize()
        got = out.cpu().numpy()
        _, V, _ = sim.bubbles()
        assert np.all(got > 10.0)   # both ids carry cells: two parts of one bubble
        assert abs(got.sum() - V[0]) <= 1e-9 * V[0] and V[1] == V[0], (got, V)
