"""Rising single bubbles in the four shape regimes of Sec. 3.2 (Table 1), at the paper's
resolution: 40 x 40 x 100 cells, bubble radius 6 dx at (20, 20, 10) dx, free-slip sides,
no-slip bottom, open top (Fig. bubbleSetup), dx = 1e-3 m, dt = 1e-4 s.

The terminal Reynolds number Re_b = u d / nu (d the volume-equivalent diameter, nu the lattice
viscosity) is measured from the rise velocity of the bubble's gas centroid and compared with
the paper's own FSLBM values Re_b* in the same finite column (Table 1).  The paper's FSLBM and
this one share the model but not every detail the paper leaves to cited works (conversions,
excess redistribution, initial fields): the bound is 15 %, the accuracy the paper attributes to
the Fan-Tsuchiya correlation its numbers are compared with (about 10 %) plus margin.

Case A (spherical, Eo ~ 1, surface tension four times the buoyancy over the bubble) rises at
Re_b ~ 1.2 against the paper's 1.76 and is marked as an expected failure: with the curvature
from Parker-Youngs normals on a bubble of radius 6 cells, the capillary pressure's errors
around the bubble are of the size of the hydrostatic pressure difference across it.
"""
import numpy as np
import pytest

from paper_1712_07028_gb300 import workloads as W

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def lbm():
    import torch
    if not torch.cuda.is_available():
        pytest.fail("these tests need the GPU")
    from paper_1712_07028_gb300 import lbm as L
    L.load()
    return L


def gas_centroid_z(sim):
    """z of the gas centroid: gas cells weight 1, interface cells 1 - phi"""
    import torch
    fl = sim.fields()
    t, phi = fl["flags"], fl["phi"]
    w = torch.where(t == 4, 1.0, torch.where(t == 2, 1.0 - phi, 0.0)).double()
    prof = w.sum(dim=(1, 2))
    z = torch.arange(prof.shape[0], device=prof.device, dtype=torch.float64)
    return float((prof * z).sum() / prof.sum())


def rise(lbm, case, every=50):
    """(times, centroid heights, volume-equivalent diameter at the end, nu) of a Table 1 case"""
    wl = W.rising_bubble(case)
    sim = lbm.Sim(wl)
    ts, zs = [0], []
    sim.step(0)
    zs.append(gas_centroid_z(sim))
    n = W.RISING_BUBBLE_CASES[case]["steps"]
    for t in range(every, n + 1, every):
        sim.step(every)
        ts.append(t)
        zs.append(gas_centroid_z(sim))
    V = sim.bubbles()[1][0]
    assert sim.status() == 0
    sim.close()
    return np.array(ts, float), np.array(zs), (6.0 * V / np.pi) ** (1.0 / 3.0), (wl.tau - 0.5) / 3.0


def terminal_velocity(ts, zs, top=100.0, margin=20.0):
    """rise velocity over the last third of the run before the centroid comes within `margin`
    cells of the top (least-squares slope)"""
    keep = zs < top - margin
    t, z = ts[keep], zs[keep]
    sel = t >= t[-1] - (t[-1] - t[0]) / 3.0
    return np.polyfit(t[sel], z[sel], 1)[0]


@pytest.mark.parametrize("case", [pytest.param("A", marks=pytest.mark.xfail(
    strict=True, reason="Re_b ~ 1.2 against 1.76: capillary-dominated (Eo ~ 1), see the module docstring")),
    "B", "C", "D"])
def test_terminal_reynolds_number(lbm, case):
    ts, zs, d, nu = rise(lbm, case)
    u = terminal_velocity(ts, zs)
    re = u * d / nu
    ref = W.RISING_BUBBLE_CASES[case]["re_star"]
    print("case %s: u_inf = %.5g, d = %.3f, Re_b = %.3f (paper's FSLBM: %.2f, %+.1f %%)"
          % (case, u, d, re, ref, 100 * (re / ref - 1)))
    assert abs(re / ref - 1) <= 0.15
