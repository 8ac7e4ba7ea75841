"""The C oracle's sweep against the independent push-form NumPy transcription on tiny grids
(every feature of step 1 on: walls and periodic axes, gravity, a translating and rotating
sphere, a gas bubble with interface cells, surface tension), to 1e-12."""
import numpy as np
import pytest

from tests import bruteforce_numpy as bf

CASES = {
    "walls_bubble_sphere": dict(nx=9, ny=8, nz=10, tau=0.7, g=(1e-4, -2e-4, -3e-4), bc=(0, 0, 0), sigma=0.0,
                                bubbles=[(4, 4, 3, 2.4)],
                                spheres=[(4.3, 3.8, 7.1, 1.8, 1.5, 0.02, -0.01, 0.015, 0.01, -0.02, 0.03)]),
    "periodic_sphere": dict(nx=7, ny=8, nz=7, tau=0.9, g=(2e-4, 0, 1e-4), bc=(1, 1, 1), sigma=0.0, bubbles=[],
                            spheres=[(0.4, 3.9, 6.2, 2.1, 1.5, -0.01, 0.02, 0.0, 0.0, 0.01, -0.02)]),
    "mixed_bc_tension": dict(nx=10, ny=9, nz=9, tau=0.6, g=(0, 0, -1e-4), bc=(1, 0, 0), sigma=5e-3,
                             bubbles=[(5, 4, 4, 2.6)],
                             spheres=[(8.0, 4.0, 6.0, 1.5, 1.5, 0.0, 0.0, 0.02, 0.02, 0.0, 0.0)]),
}


@pytest.mark.parametrize("name", sorted(CASES))
def test_sweep_matches_push_transcription(orc, name):
    cfg = dict(CASES[name])
    s = orc.Sim(sphere_mode=0, **cfg)
    rng = np.random.default_rng(11)
    act = (s.flag & (orc.LIQ | orc.IFACE)) != 0
    s.f *= np.where(act, 1 + 0.02 * (rng.random(s.f.shape) - 0.5), 1)
    if cfg["sigma"] > 0:
        s.kappa[:] = np.where(s.flag == orc.IFACE, -0.3 + 0.1 * rng.random(s.kappa.shape), 0)
    p = {"nx": cfg["nx"], "ny": cfg["ny"], "nz": cfg["nz"], "tau": cfg["tau"], "g": cfg["g"], "bc": cfg["bc"],
         "sigma": cfg["sigma"]}
    checked = 0
    for it in range(3):
        spheres = [{"x": s.sph[a, orc.S_X:orc.S_X + 3].copy(), "u": s.sph[a, orc.S_U:orc.S_U + 3].copy(),
                    "w": s.sph[a, orc.S_W:orc.S_W + 3].copy()} for a in range(s.p.nsph)]
        rho_gas = s.bub[:, orc.B_RHOG].copy()
        pre_flag = s.flag.copy()
        fb, mb, pb, Fb, Tb = bf.sweep(p, s.f.copy(), s.flag.copy(), s.m.copy(), s.phi.copy(), s.owner.copy(),
                                      s.kappa.copy(), spheres, rho_gas)
        s.step(1)
        F, T = s.forces
        assert np.abs(F - Fb).max() < 1e-12 and np.abs(T - Tb).max() < 1e-12
        untouched = (s.mark == 0) & ((pre_flag & (orc.LIQ | orc.IFACE)) != 0)
        assert np.abs((s.f - fb) * untouched).max() < 1e-12, it
        iface = untouched & (pre_flag == orc.IFACE) & (s.flag == orc.IFACE)
        assert np.abs((s.m - mb) * iface).max() < 1e-12
        assert np.abs((s.phi - pb) * iface).max() < 1e-12
        checked += int(untouched.sum()) + int(iface.sum())
        if cfg["sigma"] > 0:
            s.kappa[:] = np.where(s.flag == orc.IFACE, s.kappa, 0)
    assert checked > 500
    if cfg["bubbles"]:
        assert (pre_flag == orc.IFACE).sum() > 10
