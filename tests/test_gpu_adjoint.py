"""The hand-written adjoint of the frozen liquid window (through the C ABI) against the
oracle's tangent-linear gradient, the oracle's finite differences in the initial state, and
finite differences of the GPU forward itself on the 96^3 periodic sphere array.

J = sum over the window's steps of jdir . (total momentum-exchange force on the spheres)
(Eqs. netforce, momentum_transfer); parameters tau (lambda_+ = -1/tau, lambda_- from the
magic relation) and the body force g (Guo forcing).

Tolerances.  The GPU runs the forward and the reverse sweep in FP32 (PDFs stored as FP32
deviations); the oracle is FP64 (on the 96^3 window through a stored golden value, written by a
script that runs only the oracle).  A reverse step's rounding error is a few FP32 ulps of the
adjoint variables, which are O(|jdir|) and grow at most linearly over the window, so over T
steps the gradient is good to about T x 1e-6 relative to its largest component: the bound is
2e-4 relative for the 40-step windows here.  The GPU's own finite differences carry the FP32
rounding noise of J divided by the step h, bounded at 1e-2 relative below.
"""
import numpy as np
import pytest

import oracle
from paper_1712_07028_gb300 import workloads as W
from tests import gpu_util as U

pytestmark = pytest.mark.gpu

G0 = (2e-5, -1e-5, 5e-6)


@pytest.fixture(scope="module")
def lbm():
    import torch
    if not torch.cuda.is_available():
        pytest.fail("these tests need the GPU")
    from paper_1712_07028_gb300 import lbm as L
    L.load()
    oracle.build()
    return L


def _walled(tau=0.7, g=G0):
    """14x12x13 walled box, two fixed spheres, one with a surface velocity (moving wall)"""
    return W.Workload(name="adjoint_walls", nx=14, ny=12, nz=13, tau=tau, g=g, bc=(W.WALL,) * 3,
                      sphere_mode=W.SPHERES_FIXED,
                      spheres=[W.Sphere((5.3, 6.1, 6.2), 2.5, 1.5, (0.002, 0.0, -0.001), (0.0, 0.001, 0.0)),
                               W.Sphere((10.2, 5.7, 6.4), 2.0, 1.5)])


def _periodic(tau=0.65, g=(1e-5, 3e-6, -2e-6)):
    """16x14x15 periodic box, a sphere across the corner of the periodic images and one spinning"""
    return W.Workload(name="adjoint_periodic", nx=16, ny=14, nz=15, tau=tau, g=g, bc=(W.PERIODIC,) * 3,
                      sphere_mode=W.SPHERES_FIXED,
                      spheres=[W.Sphere((0.7, 13.2, 1.4), 3.0, 1.5),
                               W.Sphere((8.4, 6.6, 8.1), 2.5, 1.5, (0.0, 0.0, 0.0), (0.0, 0.0, 0.002))])


def _started(lbm, wl):
    sim = lbm.Sim(wl)
    sim.step(0)
    return sim


def _oracle_gradient(wl, st, n, jdir):
    """(J, dJ/dtau, dJ/dg) of the oracle's tangent-linear window from a GPU state"""
    J, dtau = U.oracle_from_state(wl, st).tangent_window(n, dtau=1.0, jdir=jdir)
    dg = np.array([U.oracle_from_state(wl, st).tangent_window(n, dg=e, jdir=jdir)[1] for e in np.eye(3)])
    return J, dtau, dg


@pytest.mark.parametrize("case", ["walls", "periodic"])
@pytest.mark.parametrize("jdir", [(1.0, 0.0, 0.0), (0.3, -0.5, 0.8)])
def test_adjoint_matches_oracle_tangent(lbm, case, jdir):
    from paper_1712_07028_gb300 import adjoint as A
    wl = _walled() if case == "walls" else _periodic()
    n = 40
    sim = _started(lbm, wl)
    st = U.gpu_state(sim)
    J, dtau, dg = A.window_gradient(sim, n, jdir, every=7)   # ragged last segment
    Jo, dtau_o, dg_o = _oracle_gradient(wl, st, n, jdir)
    assert abs(J - Jo) <= 1e-5 * abs(Jo) + 1e-9, (J, Jo)
    scale = max(abs(dtau_o), np.abs(dg_o).max())
    assert scale > 0
    tol = 2e-4
    assert abs(dtau - dtau_o) <= tol * abs(dtau_o) + 1e-7 * scale, (dtau, dtau_o)
    assert np.abs(dg - dg_o).max() <= tol * np.abs(dg_o).max(), (dg, dg_o)


def test_state_adjoint_matches_oracle_differences(lbm):
    """dJ/df*(0) . v against central differences of the FP64 oracle along v (the transposed
    streaming, wall and moving-sphere bounce-back and the rho0 term of Eq. bbrule)"""
    from paper_1712_07028_gb300 import adjoint as A
    wl = _walled()
    n, jdir = 12, (0.2, 0.9, -0.4)
    sim = _started(lbm, wl)
    st = U.gpu_state(sim)
    J, ck = A.forward_window(sim, n, jdir, every=5)
    _, _, lam0 = A.backward_window(sim, n, jdir, 5, ck)
    lam0 = lam0.cpu().numpy().astype(np.float64)
    liq = (st["flags"] & oracle.LIQ) != 0
    rng = np.random.default_rng(7)
    v = rng.standard_normal((19,) + liq.shape) * liq[None]
    h = 1e-4

    def J_at(sign):
        s2 = dict(st, f=st["f"].astype(np.float64) + sign * h * v)
        return U.oracle_from_state(wl, s2).window_objective(n, jdir)

    fd = (J_at(1) - J_at(-1)) / (2 * h)
    ad = float((lam0 * v).sum())
    assert abs(ad - fd) <= 1e-4 * abs(fd), (ad, fd)


def test_frozen_forward_is_the_step(lbm):
    """the replay step of the backward pass reproduces lbm_step on the frozen window"""
    import torch
    wl = _periodic()
    sim = _started(lbm, wl)
    sim.step(5)
    f0 = sim.export_state()["f"]
    f1 = torch.empty_like(f0)
    sim.forward_frozen(f0, f1)
    sim.step(1)
    ref = sim.export_state()["f"]
    liq = (sim.export_state()["flags"] & 1) != 0
    d = (f1 - ref).abs()[:, liq].max().item()
    assert d <= 2e-7, d


def test_checkpoint_interval_does_not_change_the_gradient(lbm):
    from paper_1712_07028_gb300 import adjoint as A
    wl = _walled()
    res = []
    for every in (1, 6, 30):
        sim = _started(lbm, wl)
        res.append(A.window_gradient(sim, 30, (1.0, 0.0, 0.0), every=every))
    for J, dtau, dg in res[1:]:
        # J itself comes from the forward's force reduction, whose FP32 per-warp partial sums
        # follow the boundary-list order (built with atomics): equal to ~1e-10 relative
        assert abs(J - res[0][0]) <= 1e-8 * abs(res[0][0])
        assert abs(dtau - res[0][1]) <= 1e-5 * abs(res[0][1])
        assert np.abs(dg - res[0][2]).max() <= 1e-5 * np.abs(res[0][2]).max()


def test_adjoint_rejects_unfrozen_windows(lbm):
    from paper_1712_07028_gb300 import adjoint as A
    wl = W.column_c0()   # a bubble: cells may change type
    sim = _started(lbm, wl)
    f = sim.export_state()["f"]
    with pytest.raises(lbm.LBMError) as e:
        sim.forward_frozen(f, f.clone())
    assert e.value.code == lbm.LBM_ESTATE
    with pytest.raises(lbm.LBMError):
        A.window_gradient(sim, 3)


def _golden_c2():
    """the FP64 oracle's tangent-linear gradient of the 96^3 window (tests/golden, written by
    make_c2_window_gradient.py from the oracle alone)"""
    import os
    vals = {}
    for line in open(os.path.join(os.path.dirname(__file__), "golden", "c2_window_gradient.txt")):
        if line.strip() and not line.startswith("#"):
            k, v = line.split()
            vals[k] = float(v)
    return vals["J"], vals["dJ_dtau"], np.array([vals["dJ_dgx"], vals["dJ_dgy"], vals["dJ_dgz"]])


def test_autograd_window_c2_against_oracle_and_finite_differences(lbm):
    """96^3 periodic array of 27 spheres, 500-step window, checkpoints every 50, through
    torch.autograd: J and its gradient against the FP64 oracle's tangent-linear window
    (1e-5 and 1e-3 relative: FP32 forward and reverse over 500 steps, T x 1e-6), and against
    central differences of the GPU forward evaluated by the same Function at shifted
    parameters (1e-2: the FP32 rounding noise of J over the step h)"""
    import torch
    from paper_1712_07028_gb300 import adjoint as A
    wl = W.periodic_array_c2()
    n, every, jdir = 500, 50, (1.0, 0.0, 0.0)
    sim = _started(lbm, wl)
    f0 = sim.export_state()["f"].clone()
    tau = torch.tensor(wl.tau, dtype=torch.float64, requires_grad=True)
    g = torch.tensor(wl.g, dtype=torch.float64, requires_grad=True)
    J = A.LBMWindow.apply(tau, g, f0, sim, n, jdir, every)
    J.backward()
    Jo, dtau_o, dg_o = _golden_c2()
    print("C2 window: J %.10g (oracle %.10g); dJ/dtau %.6g (%.6g); dJ/dg %s (%s)"
          % (J.item(), Jo, tau.grad.item(), dtau_o, g.grad.numpy(), dg_o))
    assert abs(J.item() - Jo) <= 1e-5 * abs(Jo)
    assert abs(tau.grad.item() - dtau_o) <= 1e-3 * abs(dtau_o)
    assert abs(g.grad[0].item() - dg_o[0]) <= 1e-3 * abs(dg_o[0])
    assert np.abs(g.grad.numpy() - dg_o).max() <= 1e-3 * np.abs(dg_o).max()

    def J_of(tau_, g_):
        with torch.no_grad():
            return A.LBMWindow.apply(torch.tensor(tau_, dtype=torch.float64), torch.tensor(g_, dtype=torch.float64),
                                     f0, sim, n, jdir, n).item()

    ht = 1e-3
    fd_tau = (J_of(wl.tau + ht, wl.g) - J_of(wl.tau - ht, wl.g)) / (2 * ht)
    hg = 1e-6
    fd_g = np.array([(J_of(wl.tau, np.add(wl.g, np.eye(3)[k] * hg)) - J_of(wl.tau, np.subtract(wl.g, np.eye(3)[k] * hg)))
                     / (2 * hg) for k in range(3)])
    assert abs(J.item() - J_of(wl.tau, wl.g)) <= 1e-8 * abs(J.item())
    assert abs(tau.grad.item() - fd_tau) <= 1e-2 * abs(fd_tau), (tau.grad.item(), fd_tau)
    assert np.abs(g.grad.numpy() - fd_g).max() <= 1e-2 * np.abs(fd_g).max(), (g.grad.numpy(), fd_g)


def test_set_params_and_import_reproduce_a_fresh_simulation(lbm):
    """J of a window after lbm_set_params + lbm_import_state equals J of a simulation created
    with those parameters (the same state); the objective accumulated on the device equals the
    per-step sum of the forces read to the host"""
    from paper_1712_07028_gb300 import adjoint as A
    wl = _periodic()
    n, jdir = 25, (0.4, -0.3, 0.9)
    sim = _started(lbm, wl)
    f0 = sim.export_state()["f"].clone()
    J0, _ = A.forward_window(sim, n, jdir, 10)
    tau2, g2 = wl.tau + 0.07, (2e-5, -4e-6, 1e-6)
    sim.set_params(tau2, g2)
    sim.import_state(f0)
    J1, _ = A.forward_window(sim, n, jdir, 10)
    w2 = _periodic(tau=tau2, g=g2)
    fresh = _started(lbm, w2)
    Jf = 0.0
    for _ in range(n):
        fresh.step(1)
        F, _ = fresh.forces()
        Jf += float(F.sum(axis=0) @ np.asarray(jdir))
    assert abs(J1 - Jf) <= 1e-9 * abs(Jf), (J1, Jf)
    assert abs(J1 - J0) > 1e-3 * abs(J0)   # the parameters changed the window
    sim.set_params(wl.tau, wl.g)
    sim.import_state(f0)
    J0b, _ = A.forward_window(sim, n, jdir, 10)
    assert abs(J0b - J0) <= 1e-9 * abs(J0)
