"""Bubble splitting on the GPU (a bubble is one connected gas region, Sec. 2.2; reading R39)
against the oracle and against what splitting must leave behind.

The workload: a small bubble rising into a larger one in a 20x20x56 column (g = 3e-4): the
two merge, and the thin gas necks of the merged region pinch off and touch again over the
following steps, so merges and splits repeat.  Bubbles split every step.
"""
import numpy as np
import pytest

import oracle
from paper_1712_07028_gb300 import workloads as W
from tests import gpu_util as U

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def lbm():
    import torch
    if not torch.cuda.is_available():
        pytest.fail("these tests need the GPU")
    from paper_1712_07028_gb300 import lbm as L
    L.load()
    oracle.build()
    return L


def _pinch(split_every=1, max_bubbles=8):
    return W.Workload(name="pinch", nx=20, ny=20, nz=56, tau=0.7, g=(0, 0, -3e-4), sphere_mode=W.SPHERES_FIXED,
                      bubbles=[W.Bubble((10.0, 10.0, 24.0), 6.0), W.Bubble((10.0, 10.0, 12.0), 3.5)],
                      split_every=split_every, max_bubbles=max_bubbles)


def test_split_leaves_every_bubble_one_connected_region(lbm):
    """after every step each bubble id's gas and interface cells form exactly one
    D3Q19-connected region (scipy's 18-connectivity labelling), every id with cells is a root
    within the table, the total gas mass sum rho_g V over them is conserved, and merges and
    splits both happened"""
    ndimage = pytest.importorskip("scipy.ndimage")
    st3 = ndimage.generate_binary_structure(3, 2)
    wl = _pinch()
    sim = lbm.Sim(wl)
    sim.step(0)
    V0, V, rg = sim.bubbles()
    mg0 = float((rg[:2] * V[:2]).sum())
    for k in range(600):
        sim.step(1)
        ex = sim.export_state()
        flags = ex["flags"].cpu().numpy()
        owner = ex["owner"].cpu().numpy()
        act = (flags & (oracle.GAS | oracle.IFACE)) != 0
        live = np.unique(owner[act])
        assert live.min() >= 0 and live.max() < wl.max_bubbles, (k, live)
        roots, _ = sim.bubble_roots()
        _, V, rg = sim.bubbles()
        for b in live:
            assert roots[b] == b, (k, b)
            assert ndimage.label(act & (owner == b), st3)[1] == 1, (k, b)
        mg = float(sum(rg[b] * V[b] for b in live))
        assert abs(mg - mg0) <= 1e-9 * mg0, (k, mg, mg0)
        assert sim.status() == 0, k
    n_ids, n_splits = sim.bubble_splits()
    _, n_merges = sim.bubble_roots()
    print("pinch-off: %d merges, %d splits, ids in use %d" % (n_merges, n_splits, n_ids))
    assert n_merges >= 2 and n_splits >= 2 and n_ids <= wl.max_bubbles


def test_split_steps_match_the_oracle(lbm):
    """the first split steps of the run, one step each from the GPU's state before it, against
    the oracle: the same cells convert (away from a threshold), the split parts take the same
    ids, and every id's gas density agrees"""
    wl = _pinch()
    sim = lbm.Sim(wl)
    sim.step(0)
    prev = U.gpu_state(sim)
    checked = 0
    for k in range(600):
        sim.step(1)
        cur = U.gpu_state(sim)
        if cur["n_splits"] > prev["n_splits"]:
            o = U.oracle_from_state(wl, prev)
            o.step(1)
            same = cur["flags"] == o.flag
            assert np.all(same | U.dilate(o.near > 0, 1)), (k, "types")
            gas = ((cur["flags"] & (oracle.GAS | oracle.IFACE)) != 0) & same
            assert (cur["owner"][gas] == o.owner[gas]).all(), (k, "ids")
            assert o.scal[oracle.SC_NSPLIT] == cur["n_splits"] - prev["n_splits"], k
            live = np.unique(cur["owner"][gas])
            assert np.allclose(cur["rho_g"][live], o.rho_gas[live], rtol=1e-6), (k, cur["rho_g"][live], o.rho_gas[live])
            checked += 1
            if checked == 2:
                break
        prev = cur
    assert checked == 2


def test_bubble_across_a_periodic_face_is_not_split(lbm):
    """a bubble centred on a periodic face: its cells on both sides of the grid are neighbours
    through the wrap, so splitting every step leaves it one bubble"""
    wl = W.Workload(name="wrap", nx=24, ny=14, nz=14, tau=0.7, g=(0, 0, 0), bc=(W.PERIODIC, W.WALL, W.WALL),
                    sphere_mode=W.SPHERES_FIXED, bubbles=[W.Bubble((0.0, 7.0, 7.0), 4.0)],
                    split_every=1, max_bubbles=4)
    sim = lbm.Sim(wl)
    sim.step(20)
    ex = sim.export_state()
    flags, owner = ex["flags"].cpu().numpy(), ex["owner"].cpu().numpy()
    assert sim.bubble_splits() == (1, 0)
    assert (owner[(flags & (oracle.GAS | oracle.IFACE)) != 0] == 0).all()
    assert sim.status() == 0
