"""The hand-written adjoint of the frozen liquid window (through the C ABI) against the
oracle's tangent-linear gradient, the oracle's finite differences in the initial state, and
finite differences of the GPU forward itself on the 96^3 periodic sphere array.

J = sum over the window's steps of jdir . (total momentum-exchange force on the spheres)
(Eqs. netforce, momentum_transfer); parameters tau (lambda_+ = -1/tau, lambda_- from the
magic relation) and the body force g (Guo forcing).

Tolerances.  The GPU runs the forward and the reverse sweep in FP32 (PDFs stored as FP32
deviations); the oracle is FP64.  A reverse step's rounding error is a few FP32 ulps of the
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


def test_autograd_window_vs_gpu_finite_differences_c2(lbm):
    """96^3 periodic array of 27 spheres, 500-step window, checkpoints every 50: the gradient
    of the summed drag through torch.autograd against central differences of the GPU forward"""
    import torch
    from paper_1712_07028_gb300 import adjoint as A
    wl = W.periodic_array_c2()
    n, every, jdir = 500, 50, (1.0, 0.0, 0.0)
    sim = _started(lbm, wl)
    tau = torch.tensor(wl.tau, dtype=torch.float64, requires_grad=True)
    g = torch.tensor(wl.g, dtype=torch.float64, requires_grad=True)
    J = A.LBMWindow.apply(tau, g, sim, n, jdir, every)
    J.backward()

    def J_of(tau_, g_):
        w2 = W.periodic_array_c2()
        w2.tau, w2.g = tau_, tuple(g_)
        return A.forward_window(_started(lbm, w2), n, jdir, n)[0]

    ht = 1e-3
    fd_tau = (J_of(wl.tau + ht, wl.g) - J_of(wl.tau - ht, wl.g)) / (2 * ht)
    hg = 1e-6
    fd_g = []
    for k in range(3):
        e = np.eye(3)[k] * hg
        fd_g.append((J_of(wl.tau, np.add(wl.g, e)) - J_of(wl.tau, np.subtract(wl.g, e))) / (2 * hg))
    fd_g = np.array(fd_g)
    assert abs(J.item() - J_of(wl.tau, wl.g)) <= 1e-8 * abs(J.item())
    assert abs(tau.grad.item() - fd_tau) <= 1e-2 * abs(fd_tau), (tau.grad.item(), fd_tau)
    gg = g.grad.numpy()
    assert np.abs(gg - fd_g).max() <= 1e-2 * np.abs(fd_g).max(), (gg, fd_g)
