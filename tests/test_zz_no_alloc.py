"""The allocation-free bubble-volume entry point (for callers that cannot call cudaMalloc)
against the volumes lbm_step computes, through the C ABI, on two calls in a row."""
import ctypes

import numpy as np
import pytest

from paper_1712_07028_gb300 import workloads as W

pytestmark = pytest.mark.gpu


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
        rc = L.lbm_bubble_volumes_noalloc(ctypes.c_void_p(st["flags"].data_ptr()), ctypes.c_void_p(st["owner"].data_ptr()),
                                          ctypes.c_void_p(st["phi"].data_ptr()), sim.N, nb,
                                          ctypes.c_void_p(out.data_ptr()), stream)
        assert rc == lbm.LBM_OK
        torch.cuda.synchronize()
        _, V, _ = sim.bubbles()
        got = out.cpu().numpy()
        assert np.all(got > 100.0)
        assert np.abs(got - V).max() <= 1e-9 * np.abs(V).max(), (got, V)
    too_many = L.lbm_bubble_volumes_noalloc(ctypes.c_void_p(st["flags"].data_ptr()), ctypes.c_void_p(st["owner"].data_ptr()),
                                            ctypes.c_void_p(st["phi"].data_ptr()), sim.N, 1025,
                                            ctypes.c_void_p(out.data_ptr()), stream)
    assert too_many == lbm.LBM_EINVAL
