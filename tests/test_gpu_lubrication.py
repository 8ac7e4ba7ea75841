"""GPU parity of the lubrication correction (Sec. 2.3, Eq. lubrication) with the FP64 oracle:
free spheres approaching head-on so that they spend steps closer than Delta_c = 2/3 of a cell,
one pair starting below the floor 0.2 Delta_c; the single-block sub-step kernel (a few
spheres) and the per-sub-step kernels (more than 1024 spheres) both."""
import numpy as np
import pytest

import oracle
from paper_1712_07028_gb300 import workloads as W
from tests import gpu_util as U

pytestmark = pytest.mark.gpu

DC = 2.0 / 3.0


@pytest.fixture(scope="module")
def lbm():
    import torch
    if not torch.cuda.is_available():
        pytest.fail("these tests need the GPU")
    from paper_1712_07028_gb300 import lbm as L
    L.load()
    return L


def _pairs_box():
    """two pairs of free spheres r=3 (density 1.5) in a walled liquid box, no gravity: pair A
    starts 0.5 apart (inside Delta_c) closing at 0.006 cells per step, pair B starts 0.12
    apart (below the 0.2 Delta_c floor) closing at 0.002"""
    sph = [W.Sphere((8.0, 12.0, 12.0), 3.0, 1.5, (0.003, 0.0, 0.0)),
           W.Sphere((14.5, 12.05, 11.98), 3.0, 1.5, (-0.003, 0.0, 0.0)),
           W.Sphere((27.0, 12.0, 12.0), 3.0, 1.5, (0.001, 0.0, 0.0), (0.0, 0.0, 0.002)),
           W.Sphere((33.12, 11.97, 12.02), 3.0, 1.5, (-0.001, 0.0005, 0.0))]
    return W.Workload(name="lubrication_pairs", nx=42, ny=24, nz=24, tau=0.6, g=(0.0, 0.0, 0.0),
                      sphere_mode=W.SPHERES_FREE, spheres=sph)


def _gaps(x, R):
    d = np.linalg.norm(x[1] - x[0]), np.linalg.norm(x[3] - x[2])
    return d[0] - 2 * R, d[1] - 2 * R


def test_lubrication_pairs_lockstep_against_oracle(lbm):
    """60 steps side by side; both pairs stay inside Delta_c, pair B below the floor.  The two
    runs share every FP64 sphere operation; they differ through the momentum exchange, whose
    FP32 link sums differ from the oracle's by dF <~ 1e-6 |F| each step (the force pin below).
    That difference accumulates: du <= N dF / m and dx <= N^2 / 2 dF / m over N steps; with
    |F| ~ 1e-3, m = 170 (r = 3, density 1.5) and N = 60 that allows du ~ 4e-10 and dx ~ 1e-8
    (coherent worst case).  Bounds: positions 1e-7, velocities and angular velocities 1e-8,
    the lubrication force of the last sub-step Fl 1e-5 relative to its largest component (it
    follows the relative velocity and the gap: 1/h - 1/Delta_c moves with dx / h^2)"""
    wl = _pairs_box()
    sim = lbm.Sim(wl)
    o = oracle.Sim(wl)
    below_floor = inside = 0
    worst = {"x": 0.0, "u": 0.0, "w": 0.0, "Fl": 0.0}
    for k in range(60):
        sim.step(1)
        o.step(1)
        x, u, w = sim.spheres()
        Fl = sim.lubrication()
        xo = o.sph[:4, oracle.S_X:oracle.S_X + 3]
        uo = o.sph[:4, oracle.S_U:oracle.S_U + 3]
        wo = o.sph[:4, oracle.S_W:oracle.S_W + 3]
        Flo = o.sph[:4, oracle.S_FLUB:oracle.S_FLUB + 3]
        worst["x"] = max(worst["x"], float(np.abs(x - xo).max()))
        worst["u"] = max(worst["u"], float(np.abs(u - uo).max()))
        worst["w"] = max(worst["w"], float(np.abs(w - wo).max()))
        worst["Fl"] = max(worst["Fl"], float(np.abs(Fl - Flo).max() / max(1e-12, np.abs(Flo).max())))
        ga, gb = _gaps(xo, 3.0)
        inside += int(ga < DC) + int(gb < DC)
        below_floor += int(gb < 0.2 * DC)
        assert np.abs(Flo).max() > 0.0   # lubrication acts in every step
    print("lubrication lockstep, worst differences: %s; pair-steps inside Delta_c %d, below the floor %d"
          % (worst, inside, below_floor))
    assert worst["x"] <= 1e-7 and worst["u"] <= 1e-8 and worst["w"] <= 1e-8, worst
    assert worst["Fl"] <= 1e-5, worst
    assert inside == 120 and below_floor >= 10
    # after 60 lockstep steps: the link-sum budget of the lockstep force test (1e-5 relative)
    F, T = sim.forces()
    Fo, To = o.forces
    assert np.abs(F - Fo).max() <= 1e-5 * np.abs(Fo).max() + 1e-9
    assert np.abs(T - To).max() <= 1e-5 * np.abs(To).max() + 1e-9
    assert sim.status() == 0


@pytest.mark.parametrize("pre", [0, 25, 50])
def test_lubrication_pairs_one_step_from_gpu_state(lbm, pre):
    """one step of the oracle from the GPU's own state: positions 1e-9, velocities, angular
    velocities and Fl element-wise (1e-12 absolute for u, w: the same FP64 arithmetic on the same
    inputs up to the FP32 momentum exchange)"""
    wl = _pairs_box()
    sim = lbm.Sim(wl)
    sim.step(pre)
    st0 = U.gpu_state(sim)
    o = U.oracle_from_state(wl, st0, near_tol=1e-5)
    sim.step(1)
    o.step(1)
    x, u, w = sim.spheres()
    Fl = sim.lubrication()
    Flo = o.sph[:4, oracle.S_FLUB:oracle.S_FLUB + 3]
    assert np.abs(x - o.positions).max() <= 1e-9
    assert np.abs(u - o.sph[:4, oracle.S_U:oracle.S_U + 3]).max() <= 1e-9
    assert np.abs(w - o.sph[:4, oracle.S_W:oracle.S_W + 3]).max() <= 1e-9
    assert np.abs(Fl - Flo).max() <= 1e-6 * np.abs(Flo).max()
    assert np.abs(Flo[:2]).max() > 0 and np.abs(Flo[2:]).max() > 0
    F, T = sim.forces()
    Fo, To = o.forces
    assert np.abs(F - Fo).max() <= 1e-6 * max(1e-3, np.abs(Fo).max())
    assert np.abs(T - To).max() <= 1e-6 * max(1e-1, np.abs(To).max())


def _many_spheres():
    """1331 free spheres r=1.5 on an 11^3 lattice of spacing 5.8 in a 64^3 walled liquid box
    (more than the 1024 the single-block sub-step kernel takes), six of them moved to within
    0.2-0.6 of a neighbour and set approaching it"""
    sph = []
    for k in range(11):
        for j in range(11):
            for i in range(11):
                sph.append(W.Sphere((3.5 + 5.8 * i, 3.5 + 5.8 * j, 3.5 + 5.8 * k), 1.5, 1.5))
    idx = lambda i, j, k: i + 11 * (j + 11 * k)
    for (i, j, k), gap in (((2, 3, 4), 0.55), ((6, 6, 6), 0.3), ((8, 1, 9), 0.15)):
        a, b = idx(i, j, k), idx(i + 1, j, k)
        xa = sph[a].x
        sph[b] = W.Sphere((xa[0] + 3.0 + gap, xa[1] + 0.03, xa[2] - 0.02), 1.5, 1.5, (-0.002, 0.0, 0.0))
        sph[a] = W.Sphere(xa, 1.5, 1.5, (0.002, 0.0, 0.0))
    return W.Workload(name="many_spheres_lubrication", nx=64, ny=64, nz=64, tau=0.6, g=(0.0, 0.0, -1e-5),
                      sphere_mode=W.SPHERES_FREE, spheres=sph)


def test_lubrication_many_spheres_against_oracle(lbm):
    """more than 1024 spheres (the per-sub-step kernels): 30 steps side by side, positions,
    velocities and Fl of every sphere against the oracle (the lockstep bounds of the pair test
    above); the three close pairs feel lubrication every step"""
    wl = _many_spheres()
    sim = lbm.Sim(wl)
    o = oracle.Sim(wl)
    n = len(wl.spheres)
    for k in range(30):
        sim.step(1)
        o.step(1)
        if k % 10 == 9:
            x, u, w = sim.spheres()
            Fl = sim.lubrication()
            Flo = o.sph[:n, oracle.S_FLUB:oracle.S_FLUB + 3]
            assert np.abs(x - o.positions).max() <= 1e-7
            assert np.abs(u - o.sph[:n, oracle.S_U:oracle.S_U + 3]).max() <= 1e-8
            assert np.abs(w - o.sph[:n, oracle.S_W:oracle.S_W + 3]).max() <= 1e-8
            assert np.abs(Fl - Flo).max() <= 1e-5 * np.abs(Flo).max()
            assert int((np.abs(Flo).max(axis=1) > 0).sum()) == 6
    assert sim.status() == 0
