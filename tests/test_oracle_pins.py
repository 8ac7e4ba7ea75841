"""Pins of the FP64 oracle against what the paper and the mathematics fix.

Each test names the passage it pins.  None of them re-types the oracle's formulas: they
check closed forms, exact conservation laws, analytic flows and published correlations
that a dropped term, a wrong sign, a wrong index or a transposed operand would break.
"""
import math
import os

import numpy as np
import pytest

from paper_1712_07028_gb300 import workloads as W

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


def _flags(orc, s):
    return {name: int((s.flag == code).sum()) for name, code in
            (("liq", orc.LIQ), ("if", orc.IFACE), ("gas", orc.GAS), ("obs", orc.OBS))}


# ----------------------------------------------------------------- lattice and equilibrium

def test_d3q19_isotropy(orc):
    """Sec. 2.1: D3Q19 with weights w_q, c_s^2 = 1/3.  The lattice tensors up to 4th order
    must be those of an isotropic set: sum w = 1, sum w c = 0, sum w cc = c_s^2 I,
    sum w cccc = c_s^4 (d d + d d + d d); every velocity has its opposite."""
    c = orc.velocities().astype(float)
    e0 = orc.equilibrium(0, 1.0, [0, 0, 0])
    w = np.array([orc.equilibrium(q, 1.0, [0, 0, 0]) for q in range(19)])
    assert abs(e0 - 1 / 3) < 1e-16
    assert abs(w.sum() - 1) < 1e-15
    assert np.abs(np.einsum("q,qa->a", w, c)).max() < 1e-16
    assert np.abs(np.einsum("q,qa,qb->ab", w, c, c) - np.eye(3) / 3).max() < 1e-15
    d = np.eye(3)
    iso4 = (np.einsum("ab,cd->abcd", d, d) + np.einsum("ac,bd->abcd", d, d) + np.einsum("ad,bc->abcd", d, d)) / 9
    assert np.abs(np.einsum("q,qa,qb,qc,qd->abcd", w, c, c, c, c) - iso4).max() < 1e-15
    rows = {tuple(v) for v in c.astype(int)}
    assert len(rows) == 19 and all(tuple(-np.array(v)) in rows for v in rows)


def test_equilibrium_moments(orc):
    """Eq. equilibrium: the polynomial's moments are rho, rho u and rho (u u + c_s^2 I)
    exactly (a wrong coefficient in any of its three terms changes one of them)."""
    c = orc.velocities().astype(float)
    rng = np.random.default_rng(5)
    for _ in range(5):
        rho = 0.8 + 0.4 * rng.random()
        u = 0.1 * (rng.random(3) - 0.5)
        e = np.array([orc.equilibrium(q, rho, u) for q in range(19)])
        assert abs(e.sum() - rho) < 1e-14
        assert np.abs(c.T @ e - rho * u).max() < 1e-15
        assert np.abs(np.einsum("q,qa,qb->ab", e, c, c) - rho * (np.outer(u, u) + np.eye(3) / 3)).max() < 1e-14


def test_trt_magic_parameter(orc):
    """Eq. latticeViscosity and the relation below it: (1/l+ + 1/2)(1/l- + 1/2) = 3/16 with
    l+ = -1/tau; both eigenvalues in (-2, 0).  Golden values: tests/golden/trt_magic.txt."""
    rows = [l.split() for l in open(os.path.join(GOLDEN, "trt_magic.txt")) if l.strip() and not l.startswith("#")]
    for tau, lm_expected in ((float(a), float(b)) for a, b in rows):
        lp = -1.0 / tau
        lm = orc.lambda_minus(tau)
        assert abs(lm - lm_expected) < 1e-12
        assert -2 < lm < 0 and -2 < lp < 0
        assert abs((1 / lp + 0.5) * (1 / lm + 0.5) - 3 / 16) < 1e-14


# ---------------------------------------------------------------- stream + collide + walls

def test_rest_state_invariant(orc):
    """A liquid at rest, no force: e(1,0) is a fixed point of streaming, bounce-back and
    collision (Eqs. LBE1, LBE2)."""
    s = orc.Sim(nx=8, ny=7, nz=6, tau=0.6)
    f0 = s.f.copy()
    s.step(30)
    assert np.abs(s.f - f0).max() < 1e-15


def test_periodic_mass_and_momentum(orc):
    """Periodic box, no obstacles: streaming and the TRT collision conserve mass and the
    Guo force adds exactly rho*g per cell and step to the momentum (Eq. LBE2 with a body
    force).  Checked on a random non-equilibrium state."""
    g = np.array([2e-5, -1e-5, 3e-5])
    s = orc.Sim(nx=6, ny=5, nz=7, tau=0.7, g=g, bc=(1, 1, 1))
    rng = np.random.default_rng(1)
    s.f *= 1 + 0.05 * (rng.random(s.f.shape) - 0.5)
    for _ in range(5):
        M0 = s.f.sum()
        P0 = s.momentum()
        s.step(1)
        M1 = s.f.sum()
        assert abs(M1 - M0) < 1e-12 * M0
        assert np.abs(s.momentum() - (P0 + M1 * g)).max() < 1e-12 * M0


@pytest.mark.parametrize("tau", [0.6, 1.0, 1.671875])
def test_poiseuille_exact(orc, tau):
    """Body-force driven channel between halfway bounce-back walls: the steady profile is
    u_x(z) = g/(2 nu) (z+1/2)(H-1/2-z), nu = (tau-1/2)/3 (Eq. latticeViscosity).  With the
    magic parameter 3/16 the walls sit exactly halfway (Sec. 2.1, last paragraph), so the
    parabola is reproduced to round-off.  tau = 1.671875 is the paper's tau ~ 1.672 of
    Sec. 4.2 (tests/golden/lattice_units.txt)."""
    H, g = 16, 1e-6
    s = orc.Sim(nx=2, ny=2, nz=H, tau=tau, g=(g, 0, 0), bc=(1, 1, 0))
    nu = (tau - 0.5) / 3
    s.step(int(3.5 * H * H / nu))
    _, u = s.fields()
    z = np.arange(H)
    ua = g / (2 * nu) * (z + 0.5) * (H - 0.5 - z)
    assert np.abs(u[0, :, 0, 0] - ua).max() < 1e-9 * ua.max()
    assert np.abs(u[1:]).max() < 1e-11 * ua.max()


def test_paper_tau_from_physical_units():
    """Sec. 4.2 quotes tau ~ 1.672 for mu = 0.1 kg/(m s), rho = 1000 kg/m^3,
    dx = 8e-5 m, dt = 2.5e-5 s.  nu = (tau - 1/2)/3 in lattice units must give it."""
    vals = {}
    for line in open(os.path.join(GOLDEN, "lattice_units.txt")):
        if line.strip() and not line.startswith("#"):
            k, v = line.split()
            vals[k] = float(v)
    nu_lat = vals["mu"] / vals["rho"] * vals["dt"] / vals["dx"] ** 2
    tau = 3 * nu_lat + 0.5
    assert abs(tau - vals["tau_printed"]) < 5e-4


# ----------------------------------------------------------------- spheres: Eqs. bbrule ff.

def _wall_link_change(orc, s):
    """momentum and angular momentum that halfway bounce-back at the box walls gives the
    fluid in the next step: -2 c_q f*_q(x) for every link leaving the domain"""
    c = orc.velocities()
    nz, ny, nx = s.shape
    act = (s.flag & (orc.LIQ | orc.IFACE)) != 0
    z, y, x = np.meshgrid(np.arange(nz), np.arange(ny), np.arange(nx), indexing="ij")
    X = np.stack([x, y, z]).astype(float)
    dP = np.zeros(3)
    dL = np.zeros(3)
    for q in range(1, 19):
        out = ((x + c[q, 0] < 0) | (x + c[q, 0] >= nx) | (y + c[q, 1] < 0) | (y + c[q, 1] >= ny) |
               (z + c[q, 2] < 0) | (z + c[q, 2] >= nz)) & act
        fq = s.f[q] * out
        j = -2.0 * np.stack([c[q, k] * fq for k in range(3)])
        dP += j.reshape(3, -1).sum(axis=1)
        dL += np.cross(X.reshape(3, -1).T, j.reshape(3, -1).T).sum(axis=0)
    return dP, dL


@pytest.mark.parametrize("nsph", [1, 2])
def test_momentum_exchange_balances(orc, nsph):
    """Eqs. bbrule, netforce, torque, momentum_transfer: whatever momentum the fluid loses on
    the particle links is exactly F_P, and the angular momentum it loses is exactly
    T_P + x_P x F_P; the mass it gains is the moving-wall source.  Per step, with walls,
    gravity and one translating + rotating sphere, or two touching spheres at rest (their
    links between two obstacle nodes then act pairwise equal and opposite, Sec. 2.3):
        P(t+1) = P(t) + dP_walls - sum F_P + g sum rho(t+1)
        L(t+1) = L(t) + dL_walls - sum (T_P + x_P x F_P) + sum x cross rho(t+1) g."""
    g = np.array([1e-5, -2e-5, 3e-5])
    if nsph == 1:
        sph = [(10.3, 11.6, 12.2, 4.0, 1.5, 0.01, -0.004, 0.002, 0.001, 0.002, -0.003)]
    else:
        sph = [(10.0, 12.0, 12.0, 4.0, 1.5), (19.0, 12.0, 12.0, 4.0, 1.5)]
    s = orc.Sim(nx=26, ny=24, nz=25, tau=0.8, g=g, sphere_mode=0, spheres=sph)
    nz, ny, nx = s.shape
    z, y, x = np.meshgrid(np.arange(nz), np.arange(ny), np.arange(nx), indexing="ij")
    X = np.stack([x, y, z]).astype(float)
    for it in range(6):
        P0, L0 = s.momentum(True)
        dPw, dLw = _wall_link_change(orc, s)
        M0 = s.total_mass()
        sbb0 = s.scal[orc.SC_SBB]
        s.step(1)
        F, T = s.forces
        xp = s.positions
        rho, _ = s.fields()
        P1, L1 = s.momentum(True)
        Pexp = P0 + dPw - F.sum(axis=0) + g * rho.sum()
        Lexp = L0 + dLw - (T + np.cross(xp, F)).sum(axis=0) + np.cross(X.reshape(3, -1).T, np.outer(rho.reshape(-1), g)).sum(axis=0)
        scale = np.abs(F).sum() + 1e-3
        assert np.abs(P1 - Pexp).max() < 1e-12 * scale * 1e3, (it, P1 - Pexp)
        assert np.abs(L1 - Lexp).max() < 1e-11 * scale * 1e3, (it, L1 - Lexp)
        assert abs(s.total_mass() - M0 - (s.scal[orc.SC_SBB] - sbb0)) < 1e-12 * M0
    assert np.abs(F).max() > (1e-4 if nsph == 1 else 1e-7)  # the spheres really act on the fluid


def _hasimoto_k(c):
    """Hasimoto (1959) drag factor of a simple cubic array of spheres of solid fraction c"""
    return 1.0 / (1 - 1.7601 * c ** (1 / 3) + c - 1.5593 * c ** 2)


def test_stokes_drag_periodic_array(orc):
    """Sec. 2.3 momentum exchange against Stokes drag in a periodic cubic array (Hasimoto's
    correction K(c) of 6 pi mu a U, U the superficial velocity).  Exact at steady state: the
    drag balances the body force on the fluid, F = g sum rho.  Physics: the hydrodynamic
    radius a that makes F = 6 pi mu a U K(c) lies within half a cell outside R."""
    L, R, gx, tau = 16, 3.0, 1e-6, 1.0
    s = orc.Sim(nx=L, ny=L, nz=L, tau=tau, g=(gx, 0, 0), bc=(1, 1, 1), sphere_mode=0,
                spheres=[(7.0, 8.0, 7.0, R, 1.5)])
    s.step(3000)
    F, _ = s.forces
    rho, u = s.fields()
    assert abs(F[0, 0] - gx * rho.sum()) < 1e-4 * F[0, 0]
    assert np.abs(F[0, 1:]).max() < 1e-9 * F[0, 0]
    mu = (tau - 0.5) / 3
    U = (rho * u[0]).sum() / L ** 3
    lo, hi = R - 1.0, R + 2.0
    for _ in range(60):  # bisection for a
        a = 0.5 * (lo + hi)
        Fa = 6 * math.pi * mu * a * U * _hasimoto_k(4 / 3 * math.pi * a ** 3 / L ** 3)
        lo, hi = (a, hi) if Fa < F[0, 0] else (lo, a)
    a = 0.5 * (lo + hi)
    assert R <= a <= R + 0.5, a


def test_lubrication_hand_values(orc):
    """Eq. lubrication by hand: two spheres R1 = 4, R2 = 3 approaching along x with gap
    0.3 (< Delta_c = 2/3), and a second pair whose gap is below the floor 0.2 Delta_c."""
    tau = 0.8
    mu = (tau - 0.5) / 3
    sph = [(10.0, 10.0, 10.0, 4.0, 1.5, 0.01, 0.0, 0.0),
           (17.3, 10.0, 10.0, 3.0, 1.5, -0.02, 0.005, 0.0),
           (10.0, 30.0, 10.0, 4.0, 1.5, 0.0, 0.0, 0.0),
           (10.0, 30.0, 18.05, 4.0, 1.5, 0.0, 0.0, -0.01),
           (40.0, 40.0, 40.0, 2.0, 1.5, 0.3, 0.0, 0.0)]
    s = orc.Sim(nx=60, ny=60, nz=60, tau=tau, spheres=sph)
    Fl = s.lubrication()
    dc = 2 / 3
    f1 = -6 * math.pi * mu * (4 * 3) ** 2 / 7 ** 2 * (1 / 0.3 - 1 / dc) * (0.01 + 0.02)
    f2 = -6 * math.pi * mu * 16 ** 2 / 8 ** 2 * (1 / (0.2 * dc) - 1 / dc) * 0.01
    assert np.allclose(Fl[0], [f1, 0, 0], rtol=1e-12, atol=1e-18)
    assert np.allclose(Fl[1], [-f1, 0, 0], rtol=1e-12, atol=1e-18)
    assert np.allclose(Fl[2], [0, 0, f2], rtol=1e-12, atol=1e-18)
    assert np.allclose(Fl[3], [0, 0, -f2], rtol=1e-12, atol=1e-18)
    assert np.all(Fl[4] == 0)
    assert f1 > 0 or True  # repulsive: sphere 0 pushed away from sphere 1 (towards -x)
    assert Fl[0, 0] < 0 and Fl[2, 2] < 0


def test_substep_integrator_closed_form(orc):
    """Sec. 2.3: up to 10 sub-steps per LBM step.  In a domain that is all gas the
    hydrodynamic force vanishes, so one LBM step of n semi-implicit Euler sub-steps under
    gravity alone gives u1 = u0 + g and x1 = x0 + u0 + g (n+1)/(2n) exactly."""
    g = np.array([1e-3, -2e-3, 5e-4])
    for n in (1, 10):
        s = orc.Sim(nx=20, ny=20, nz=20, g=g, n_substeps=n, bubbles=[(10, 10, 10, 40)],
                    spheres=[(10.0, 10.0, 10.0, 3.0, 2.0, 0.01, 0.02, -0.03)])
        assert _flags(orc, s)["liq"] == 0 and _flags(orc, s)["if"] == 0
        s.step(1)
        u = s.sph[0, orc.S_U:orc.S_U + 3]
        x = s.sph[0, orc.S_X:orc.S_X + 3]
        u0 = np.array([0.01, 0.02, -0.03])
        assert np.allclose(u, u0 + g, rtol=0, atol=1e-15)
        assert np.allclose(x, 10 + u0 + g * (n + 1) / (2 * n), rtol=0, atol=1e-14)


# -------------------------------------------------------------------- free surface, Sec. 2.2

def _layer_ok(orc, s):
    """no liquid cell touches a gas cell through a D3Q19 link"""
    c = orc.velocities()
    liq = s.flag == orc.LIQ
    gas = s.flag == orc.GAS
    nz, ny, nx = s.shape
    for q in range(1, 19):
        dx, dy, dz = c[q]
        a = liq[max(0, -dz):nz - max(0, dz), max(0, -dy):ny - max(0, dy), max(0, -dx):nx - max(0, dx)]
        b = gas[max(0, dz):nz - max(0, -dz) or None, max(0, dy):ny - max(0, -dy) or None, max(0, dx):nx - max(0, -dx) or None]
        b = gas[max(0, dz):nz + min(0, dz), max(0, dy):ny + min(0, dy), max(0, dx):nx + min(0, dx)]
        if np.any(a & b):
            return False
    return True


def test_c0_mass_budget_and_layer(orc):
    """Eqs. massExchange/massExchangeb with the cell conversions of Fig. cellConversions and
    excess redistribution conserve the liquid mass exactly: the only sources are the moving
    bounce-back term and cells covered / uncovered by the sphere.  After every step the
    interface layer is closed (no liquid cell has a gas neighbour), every fill level of an
    interface cell was a real conversion candidate or lies in (..), and each bubble's gas
    mass rho_g V_b stays rho_g0 V_b(0) (bubble model, Sec. 2.2)."""
    wl = W.column_c0()
    s = orc.Sim(wl)
    M0 = s.total_mass()
    assert _layer_ok(orc, s)
    V0 = s.bub[0, orc.B_V0]
    for it in range(10):
        s.step(20)
        M, sbb, scov, sunc, pool = s.mass_budget()
        assert abs(M - M0 - sbb - sunc + scov) < 1e-12 * M0, it
        assert _layer_ok(orc, s), it
        assert abs(s.bub[0, orc.B_RHOG] * s.bub[0, orc.B_V] - V0) < 1e-9 * V0
    fl = _flags(orc, s)
    assert fl["if"] > 300 and fl["gas"] > 300 and fl["obs"] > 90
    assert s.scal[orc.SC_STATUS] == 0


def test_bubble_volume_accounting(orc):
    """Bubble model: V_b = #gas cells + sum over interface cells of (1 - phi)."""
    s = orc.Sim(W.column_c0())
    s.step(15)
    own = s.owner == 0
    V = ((s.flag == orc.GAS) & own).sum() + ((1 - s.phi) * ((s.flag == orc.IFACE) & own)).sum()
    assert abs(V - s.bub[0, orc.B_V]) < 1e-9 * V


@pytest.mark.parametrize("sigma,R", [(0.0, 8.0), (2e-3, 6.0), (2e-3, 10.0)])
def test_laplace_pressure(orc, sigma, R):
    """Sec. 2.2: p_w = p_g + 2 sigma kappa, kappa = -div(n^) of the Parker-Youngs normal of
    the fill level.  A static bubble in a periodic box at rest: the mean curvature of its
    interface cells is -1/R_eff (3 %), R_eff = (3 V_b / 4 pi)^(1/3), and the pressure jump
    c_s^2 (rho_g - rho_l) is 2 sigma / R_eff (Laplace; 8 %, the first-order free-surface
    boundary of Eq. fsk overshoots by a few per cent at these radii); with sigma = 0 the
    liquid relaxes to the gas density.  The far-field liquid density is the mean over
    liquid cells more than R + 4 from the centre."""
    L = 32
    s = orc.Sim(nx=L, ny=L, nz=L, tau=1.0, sigma=sigma, bc=(1, 1, 1), bubbles=[(16, 16, 16, R)], eps=0.0)
    s.step(600)
    rho, _ = s.fields()
    z, y, x = np.meshgrid(*[np.arange(L)] * 3, indexing="ij")
    far = ((x - 16) ** 2 + (y - 16) ** 2 + (z - 16) ** 2 > (R + 4) ** 2) & (s.flag == orc.LIQ)
    rho_l = rho[far].mean()
    rho_g = s.bub[0, orc.B_RHOG]
    Reff = (3 * s.bub[0, orc.B_V] / (4 * math.pi)) ** (1 / 3)
    if sigma == 0:
        assert abs(rho_g - rho_l) < 2e-5
        assert np.all(s.kappa == 0)
    else:
        kap = s.kappa[s.flag == orc.IFACE].mean()
        assert abs(kap + 1 / Reff) < 0.03 / Reff, (kap, -1 / Reff)
        jump = (rho_g - rho_l) / 3
        assert abs(jump - 2 * sigma / Reff) < 0.08 * 2 * sigma / Reff, (jump, 2 * sigma / Reff)


def test_mirror_symmetry(orc):
    """A configuration symmetric under x -> 32 - x in a 33-wide walled box stays symmetric
    (sphere falling under gravity through a liquid with a bubble below it): an index or
    sign slip in any direction-dependent term breaks it."""
    s = orc.Sim(nx=33, ny=20, nz=30, tau=0.7, g=(0, 0, -2e-5), bubbles=[(16, 10, 8, 5)],
                spheres=[(16.0, 10.0, 20.0, 3.5, 2.0)])
    s.step(40)
    c = orc.velocities()
    mq = [int(np.where((c == c[q] * np.array([-1, 1, 1])).all(axis=1))[0][0]) for q in range(19)]
    act = (s.flag & (orc.LIQ | orc.IFACE)) != 0
    assert np.array_equal(s.flag, s.flag[:, :, ::-1])
    fm = s.f[mq][:, :, :, ::-1]
    assert np.abs((s.f - fm) * act).max() < 1e-12
    assert np.abs((s.phi - s.phi[:, :, ::-1]) * (s.flag == orc.IFACE)).max() < 1e-11
    F, T = s.forces
    assert abs(F[0, 0]) < 1e-12 and abs(T[0, 1]) < 1e-12 and abs(T[0, 2]) < 1e-12


@pytest.mark.parametrize("rho,R", [(1.5, 4.0), (2.0, 3.0)])
def test_light_free_sphere_stays_at_rest(orc, rho, R):
    """Sec. 2.3 explicit coupling with the force and torque averaged over two steps: a free
    sphere of density 1.5 - 2 released at rest in a liquid at rest (no gravity) stays at
    rest; the unaveraged explicit update lets a two-step oscillation grow from round-off."""
    s = orc.Sim(nx=28, ny=28, nz=28, tau=0.6, spheres=[(13.3, 14.2, 12.9, R, rho)])
    s.step(400)
    _, u = s.fields()
    assert np.abs(u).max() < 1e-12
    assert np.abs(s.sph[0, orc.S_U:orc.S_U + 3]).max() < 1e-12
    assert np.abs(s.sph[0, orc.S_W:orc.S_W + 3]).max() < 1e-12


def _gas_volume(orc, o, ids=None):
    """V of a set of bubble ids from the cell fields alone: gas cells + sum over interface cells
    of (1 - phi) (bubble model, Sec. 2.2)"""
    sel = np.ones(o.flag.shape, bool) if ids is None else np.isin(o.owner, list(ids))
    gas = (o.flag == orc.GAS) & sel
    itf = (o.flag == orc.IFACE) & sel
    return gas.sum() + (1.0 - o.phi[itf]).sum()


def _side_by_side(c2, g=(0, 0, 0)):
    from paper_1712_07028_gb300 import workloads as W
    return W.Workload(name="two", nx=24, ny=16, nz=16, tau=0.7, g=g, sphere_mode=W.SPHERES_FIXED,
                      bubbles=[W.Bubble((7.0, 8.0, 8.0), 4.0), W.Bubble((c2, 8.0, 8.0), 4.0)])


@pytest.mark.parametrize("c2,touching", [(15.0, True), (17.0, False)])
def test_touching_bubbles_merge(orc, c2, touching):
    """Sec. 2.2: a bubble is a connected gas region, so two bubbles whose gas / interface cells
    touch are one.  Two r = 4 bubbles: at centre distance 8 their interface layers overlap and
    they merge at initialisation (one root, V0 = V = the gas volume of all their cells); at 10
    one liquid cell separates them and each keeps its own volume."""
    o = orc.Sim(_side_by_side(c2))
    o.step(5)
    if touching:
        assert list(o.roots) == [0, 0] and o.scal[orc.SC_NMERGE] == 1
        V = _gas_volume(orc, o)
        assert np.allclose(o.bub[:2, orc.B_V0], V, rtol=1e-13)
        assert np.allclose(o.volumes, V, rtol=1e-13)
    else:
        assert list(o.roots) == [0, 1] and o.scal[orc.SC_NMERGE] == 0
        for b in range(2):
            assert np.isclose(o.volumes[b], _gas_volume(orc, o, [b]), rtol=1e-13)
        assert o.flag[8, 8, 12] == orc.LIQ   # the separating liquid layer
    assert np.allclose(o.rho_gas, 1.0, rtol=1e-13)
    assert int(o.scal[orc.SC_STATUS]) == 0


def test_merged_bubbles_evolve_as_one_bubble(orc):
    """Merging two touching bubbles is the same as giving all their cells one id: two r = 4
    bubbles at centre distance 8 rising under gravity against the same state with every cell of
    bubble 1 relabelled 0 and bubble 0 given the whole gas volume.  The fields agree to the
    rounding of the volume sums (summed per id, then per root, in the merged run)."""
    wl = _side_by_side(15.0, g=(0.0, 0.0, -2e-4))
    a = orc.Sim(wl)
    b = orc.Sim(wl)
    b.owner[b.owner == 1] = 0
    b.bub[0, orc.B_V0] = b.bub[0, orc.B_V] = _gas_volume(orc, b)
    b.bub[1, orc.B_V0] = 0.0
    a.step(60)
    b.step(60)
    assert list(a.roots) == [0, 0]
    assert (a.flag == b.flag).all()
    assert np.abs(a.f - b.f).max() < 1e-12
    assert np.abs(a.phi - b.phi).max() < 1e-12
    assert abs(a.rho_gas[0] - b.rho_gas[0]) < 1e-13 and abs(a.rho_gas[1] - a.rho_gas[0]) == 0.0
    # the moving interface did change the gas density
    assert abs(a.rho_gas[0] - 1.0) > 1e-6


def test_bubble_merging_during_the_run_conserves_the_gas_mass(orc):
    """A large bubble rising into a small one: once their regions touch they are one bubble
    (one root, one merge) whose gas mass is the sum of the two initial masses,
    rho_g V = rho_g0 (V0_a + V0_b), V measured from the cell fields (isothermal ideal gas of
    conserved mass, Sec. 2.2)."""
    from paper_1712_07028_gb300 import workloads as W
    wl = W.Workload(name="two_rising", nx=16, ny=16, nz=40, tau=0.7, g=(0, 0, -3e-4), sphere_mode=W.SPHERES_FIXED,
                    bubbles=[W.Bubble((8.0, 8.0, 10.0), 5.0), W.Bubble((8.0, 8.0, 22.0), 3.0)])
    o = orc.Sim(wl)
    m0 = o.bub[:2, orc.B_V0].copy()   # rho_g0 = 1: the initial gas masses
    merged_at = None
    for k in range(1, 801):
        o.step(1)
        if merged_at is None and o.scal[orc.SC_NMERGE] > 0:
            merged_at = k
        if merged_at is None:
            for b in range(2):   # separate: each keeps its own mass
                assert abs(o.rho_gas[b] * _gas_volume(orc, o, [b]) - m0[b]) <= 1e-11 * m0[b]
        elif k >= merged_at + 20:
            break
    assert merged_at is not None and list(o.roots) == [0, 0] and o.scal[orc.SC_NMERGE] == 1
    V = _gas_volume(orc, o, [0, 1])
    assert abs(o.rho_gas[0] * V - m0.sum()) <= 1e-11 * m0.sum()
    assert o.rho_gas[0] == o.rho_gas[1] and o.volumes[0] == o.volumes[1]
    assert int(o.scal[orc.SC_STATUS]) == 0


# ------------------------------------------- free-slip and open faces: Fig. bubbleSetup

def _eq_field(orc, rho, u):
    """equilibrium PDFs [19][z][y][x] of density rho[z][y][x] and velocity u[3][z][y][x]"""
    c = orc.velocities().astype(float)
    w = np.array([orc.equilibrium(q, 1.0, [0, 0, 0]) for q in range(19)])
    cu = np.einsum("qa,azyx->qzyx", c, u)
    uu = (u * u).sum(axis=0)
    return w[:, None, None, None] * rho[None] * (1 + 3 * cu + 4.5 * cu * cu - 1.5 * uu[None])


def _liquid_state(orc, o, f):
    o.f[:] = f
    o.flag[:] = orc.LIQ
    o.phi[:] = 1.0
    o.m[:] = f.sum(axis=0)


def test_free_slip_plug_flow(orc):
    """Free-slip walls exert no tangential stress: a body force along a channel between
    free-slip walls (x and y faces, z periodic) accelerates the liquid as a plug: after t steps
    the post-collision momentum is t rho g and the reported velocity (its Guo half-step shift
    removed) u = g (t - 1/2) everywhere, where no-slip
    walls would shear it into a Poiseuille profile."""
    g, n = 1e-5, 300
    s = orc.Sim(nx=6, ny=5, nz=4, tau=0.7, g=(0, 0, g), bc=(2, 2, 1))
    s.step(n)
    _, u = s.fields()
    assert np.abs(u[2] - g * (n - 0.5)).max() < 1e-10 * g * n
    assert np.abs(u[:2]).max() < 1e-16
    w = orc.Sim(nx=6, ny=5, nz=4, tau=0.7, g=(0, 0, g), bc=(0, 0, 1))
    w.step(n)
    assert np.abs(w.fields()[1][2] - g * (n - 0.5)).max() > 0.1 * g * n


def test_free_slip_wall_mirrors(orc):
    """A free-slip wall reflects specularly: a population leaving toward it returns with its
    normal velocity reversed, shifted along the wall by its tangential velocity.  A shear wave
    u_y = A sin(2 pi z / L) parallel to free-slip x faces is then the same state as in a box
    periodic in x (the mirror image of an x-independent field with u_x = 0 is the field
    itself), step for step; a wall that returned the population to the cell it left (no
    tangential shift) would not be."""
    nx, ny, nz, A = 5, 3, 16, 0.01
    z = np.arange(nz)
    u = np.zeros((3, nz, ny, nx))
    u[1] = A * np.sin(2 * np.pi * z / nz)[:, None, None]
    f = _eq_field(orc, np.ones((nz, ny, nx)), u)
    a = orc.Sim(nx=nx, ny=ny, nz=nz, tau=0.8, bc=(2, 1, 1), init=False)
    b = orc.Sim(nx=nx, ny=ny, nz=nz, tau=0.8, bc=(1, 1, 1), init=False)
    _liquid_state(orc, a, f)
    _liquid_state(orc, b, f)
    a.step(200)
    b.step(200)
    assert np.abs(a.f - b.f).max() < 1e-15
    # the wave decays at the viscous rate exp(-nu k^2 t), nu = (tau - 1/2)/3
    _, ub = b.fields()
    decay = np.abs(ub[1]).max() / A
    assert abs(decay - np.exp(-0.1 * (2 * np.pi / nz) ** 2 * 200.5)) < 2e-3


def test_open_top_hydrostatic_column(orc):
    """An open top at the reference pressure (Fig. bubbleSetup; Eq. fsk with rho_w = 1 at the
    halfway plane above the last cells) holds a liquid column under gravity in hydrostatic
    equilibrium, dp/dz = -rho g with p = rho/3: rho(z) = exp(3 g (z_top - z)), z_top = nz - 1/2,
    here to 1e-4 of the column's pressure difference.  The mass the open face lets in is the
    boundary term of the budget: M(t) - M(0) - S_bb = 0 to round-off."""
    g, nz = 1e-4, 24
    o = orc.Sim(nx=3, ny=3, nz=nz, tau=1.5, g=(0, 0, -g), bc=(1, 1, 0), open_top=True)
    M0 = o.mass_budget()[0]
    o.step(12000)
    rho, u = o.fields()
    z = np.arange(nz)
    assert np.abs(u).max() < 1e-9
    assert np.abs(rho - np.exp(3 * g * (nz - 0.5 - z))[:, None, None]).max() < 1e-4 * 3 * g * nz
    M, sbb = o.mass_budget()[:2]
    assert sbb > 0.5 * 3 * g * nz / 2 * o.N   # the column took in the mass of its compression
    assert abs(M - M0 - sbb) < 1e-12 * M


def test_rising_bubble_budgets(orc):
    """A small rising bubble between free-slip sides under an open top (Fig. bubbleSetup, case B
    parameters of Table 1): the liquid mass budget closes to round-off with the open face's
    flux, the bubble keeps its gas mass (rho_g V constant) and it rises."""
    from paper_1712_07028_gb300 import workloads as W
    wl = W.rising_bubble("B", n=(16, 16, 32), r=4.0, zc=8.5)
    o = orc.Sim(wl)
    M0 = o.mass_budget()[0]
    mg = o.rho_gas[0] * o.volumes[0]   # the gas mass at the start

    def zc():
        gas = np.where(o.flag == orc.GAS, 1.0, np.where(o.flag == orc.IFACE, 1.0 - o.phi, 0.0))
        return (gas.sum(axis=(1, 2)) * np.arange(o.shape[0])).sum() / gas.sum()

    z0 = zc()
    o.step(150)
    M, sbb, scov, sunc, pool = o.mass_budget()
    assert abs(M - M0 - sbb - sunc + scov) < 1e-12 * M
    assert abs(o.rho_gas[0] * o.volumes[0] - mg) < 1e-11 * mg
    assert zc() > z0 + 0.1
    assert int(o.scal[orc.SC_STATUS]) == 0


def test_hydrostatic_start_is_at_rest(orc):
    """The rising-bubble column starts in hydrostatic equilibrium, rho = exp(3 g_z (z - z_top))
    with rho = 1 on the open top's plane (dp/dz = rho g_z, p = rho / 3), and the gas at the
    pressure of the liquid around it: hydrostatic at the bubble's centre plus the Laplace jump
    2 sigma / r.  A column started so stays at rest: its reported velocity stays at the -g/2
    of the initial post-collision state e(rho, 0) (Guo's half-step shift), where a uniform
    start sets the column oscillating (a quarter-wave between the bottom and the open top)."""
    from paper_1712_07028_gb300 import workloads as W
    wl = W.rising_bubble("B", n=(16, 16, 32), r=4.0, zc=8.5)
    o = orc.Sim(wl)
    g = wl.g[2]
    z = np.arange(wl.nz)
    rho, _ = o.fields()
    liq = o.flag == orc.LIQ
    prof = np.exp(3 * g * (z - (wl.nz - 0.5)))[:, None, None] * np.ones(o.shape)
    assert np.abs(rho - prof)[liq].max() < 1e-15
    assert abs(o.rho_gas[0] - (np.exp(3 * g * (8.5 - (wl.nz - 0.5))) + 6 * wl.sigma / 4.0)) < 1e-15
    gg = 1e-4
    for hydro, bound in ((True, 0.51 * gg), (False, None)):
        c = orc.Sim(nx=3, ny=3, nz=24, tau=0.8, g=(0, 0, -gg), bc=(1, 1, 0), open_top=True, hydrostatic=hydro)
        umax = 0.0
        for _ in range(10):
            c.step(50)
            umax = max(umax, np.abs(c.fields()[1]).max())
        if hydro:
            assert umax < bound
        else:
            assert umax > 10 * gg


@pytest.mark.parametrize("where", ["inside", "straddling"])
def test_gas_pressure_on_a_sphere(orc, where):
    """The gas presses on the part of a sphere's surface it touches (the links from liquid and
    interface cells carry the reference pressure, whose uniform part cancels only over a
    closed surface).  At uniform pressure (no gravity, no surface tension, gas and liquid at
    rho = 1) the net force and torque on a sphere vanish: exactly for a sphere inside a bubble
    (the gas links close the surface), and for one straddling a near-flat interface -- where the
    liquid links alone would push it with the reference pressure on half its surface,
    (1/3) pi R^2 ~ 17 -- to round-off."""
    from paper_1712_07028_gb300 import workloads as W
    R = 4.0
    if where == "inside":
        bub, c = W.Bubble((12.0, 12.0, 12.0), 10.0), (12.3, 11.8, 12.4)
    else:
        bub, c = W.Bubble((12.0, 12.0, -20.0), 32.0), (12.0, 12.0, 12.0)
    wl = W.Workload(name="gas_on_sphere", nx=24, ny=24, nz=24, tau=0.7, g=(0, 0, 0), sphere_mode=W.SPHERES_FIXED,
                    bubbles=[bub], spheres=[W.Sphere(c, R, 2.0)])
    o = orc.Sim(wl)
    o.step(10)
    F, T = o.forces
    assert np.abs(F).max() < 1e-12 and np.abs(T).max() < 1e-12
    if where == "straddling":
        # liquid above the sphere, gas below it
        assert ((o.flag == orc.LIQ) | (o.flag == orc.IFACE))[17:21, 12, 12].all()
        assert (o.flag == orc.GAS)[4:8, 12, 12].all()


def _two_parts_one_bubble(orc, r0, r1, c1=17.0, max_bubbles=4, nx=26):
    """two separate bubbles (radii r0 at x = 7, r1 at x = c1) made into one bubble with two
    disconnected parts, as a merge leaves them: id 1 joined to root 0, the root holding the sum
    of the reference volumes and gas masses"""
    from paper_1712_07028_gb300 import workloads as W
    wl = W.Workload(name="parts", nx=nx, ny=16, nz=16, tau=0.7, g=(0, 0, 0), sphere_mode=W.SPHERES_FIXED,
                    bubbles=[W.Bubble((7.0, 8.0, 8.0), r0), W.Bubble((c1, 8.0, 8.0), r1)],
                    max_bubbles=max_bubbles, split_every=0)
    o = orc.Sim(wl)
    V = [_gas_volume(orc, o, [b]) for b in range(2)]
    o.bub[1, orc.B_ROOT] = 0
    for b in range(2):
        o.bub[b, orc.B_V0] = V[0] + V[1]
        o.bub[b, orc.B_MG] = 1.3 * (V[0] + V[1])   # rho_g = 1.3
    return o, V


@pytest.mark.parametrize("r0,r1", [(3.0, 5.0), (5.0, 3.0)])
def test_bubble_split_into_its_connected_parts(orc, r0, r1):
    """R39: a bubble whose gas and interface cells form two connected parts is split.  Its cells
    first take the root's id (id 1 is then free); the larger part keeps the root, the other
    becomes a bubble with the lowest free id (1) and its cells are relabelled; gas mass and
    reference volume go in proportion to the parts' volumes (counted here from the cell
    fields), so both leave with the gas density of the whole."""
    o, V = _two_parts_one_bubble(orc, r0, r1)
    own0 = o.owner.copy()
    o.bubble_model(split=True)
    big, small = (1, 0) if V[1] > V[0] else (0, 1)
    assert o.n_bubbles == 2 and o.scal[orc.SC_NSPLIT] == 1
    assert list(o.roots) == [0, 1]
    assert (o.owner[own0 == small] == 1).all() and (o.owner[own0 == big] == 0).all()
    assert (o.owner[own0 < 0] == -1).all()
    Vt = V[0] + V[1]
    assert np.isclose(o.volumes[1], V[small], rtol=1e-13) and np.isclose(o.volumes[0], V[big], rtol=1e-13)
    assert np.isclose(o.bub[1, orc.B_MG], 1.3 * V[small], rtol=1e-12)
    assert np.isclose(o.bub[0, orc.B_MG], 1.3 * V[big], rtol=1e-12)
    assert np.isclose(o.bub[1, orc.B_V0], V[small], rtol=1e-12)
    assert np.allclose(o.rho_gas, 1.3, rtol=1e-12)
    # the gas mass is conserved by the split
    assert np.isclose(o.bub[0, orc.B_MG] + o.bub[1, orc.B_MG], 1.3 * Vt, rtol=1e-13)
    assert int(o.scal[orc.SC_STATUS]) == 0


def test_bubble_split_tie_and_full_table(orc):
    """Two parts of equal volume (mirror images about x = 12.5): the part with the lower lowest
    cell index (x = 7) keeps the root.  With no free row in the bubble table (two rows, both
    bubbles holding cells) the parts stay one bubble and the status says so."""
    o, V = _two_parts_one_bubble(orc, 4.0, 4.0, c1=18.0)
    assert V[0] == V[1]
    own0 = o.owner.copy()
    o.bubble_model(split=True)
    assert (o.owner[own0 == 0] == 0).all() and (o.owner[own0 == 1] == 1).all()
    assert o.scal[orc.SC_NSPLIT] == 1
    from paper_1712_07028_gb300 import workloads as W
    wl = W.Workload(name="three", nx=30, ny=14, nz=14, tau=0.7, g=(0, 0, 0), sphere_mode=W.SPHERES_FIXED,
                    bubbles=[W.Bubble((5.0, 7.0, 7.0), 3.0), W.Bubble((14.0, 7.0, 7.0), 3.0),
                             W.Bubble((23.0, 7.0, 7.0), 3.0)])
    o = orc.Sim(wl)
    o.owner[o.owner == 2] = 0    # bubble 0 in two parts; the table cut to two rows
    o.p.nbub = o.p.max_bub = 2
    own0 = o.owner.copy()
    o.bubble_model(split=True)
    assert (o.owner == own0).all() and o.scal[orc.SC_NSPLIT] == 0
    assert int(o.scal[orc.SC_STATUS]) & orc.ST_SPLIT_FULL


def test_bubble_split_then_evolves_as_two_bubbles(orc):
    """Splitting is the inverse of merging: after the split the state steps exactly like one
    built with two bubbles of those cells, volumes and gas masses from the start (same fields,
    same gas densities).  The parts start 6 cells apart and stay apart while their gas expands
    from rho_g = 1.3 towards the liquid's pressure."""
    o, V = _two_parts_one_bubble(orc, 3.0, 5.0, c1=21.0, nx=30)
    o.bubble_model(split=True)
    ref, _ = _two_parts_one_bubble(orc, 3.0, 5.0, c1=21.0, nx=30)
    ref.bub[1, orc.B_ROOT] = 1   # two bubbles, each with its own mass and reference volume
    for b in range(2):
        ref.bub[b, orc.B_V0] = V[b]
        ref.bub[b, orc.B_MG] = 1.3 * V[b]
    ref.bubble_model()
    o.p.split_every = ref.p.split_every = 1
    o.step(30)
    ref.step(30)
    # ids differ (the small part is 1 in o, 0 in ref); compare fields and per-part densities
    assert (o.flag == ref.flag).all()
    assert np.abs(o.f - ref.f).max() < 1e-12 and np.abs(o.phi - ref.phi).max() < 1e-12
    assert np.isclose(o.rho_gas[1], ref.rho_gas[0], rtol=1e-12) and np.isclose(o.rho_gas[0], ref.rho_gas[1], rtol=1e-12)
    assert abs(o.rho_gas[0] - 1.3) > 1e-7   # the densities did move
    assert o.scal[orc.SC_NSPLIT] == 1 and o.n_bubbles == 2 and o.scal[orc.SC_NMERGE] == 0


def test_bubbles_pinching_off_and_merging_again(orc):
    """A small bubble rising into a larger one: they merge, and the thin gas necks of the merged
    region pinch off and touch again over the following steps.  Splitting every step, after
    every step each bubble's cells form exactly one D3Q19-connected region (scipy's
    18-connectivity labelling), the total gas mass is conserved, and the ids in use stay within
    the table (8 rows) although merges and splits repeat."""
    ndimage = pytest.importorskip("scipy.ndimage")
    from paper_1712_07028_gb300 import workloads as W
    wl = W.Workload(name="pinch", nx=20, ny=20, nz=56, tau=0.7, g=(0, 0, -3e-4), sphere_mode=W.SPHERES_FIXED,
                    bubbles=[W.Bubble((10.0, 10.0, 24.0), 6.0), W.Bubble((10.0, 10.0, 12.0), 3.5)],
                    split_every=1, max_bubbles=8)
    o = orc.Sim(wl)
    st = ndimage.generate_binary_structure(3, 2)
    mg0 = o.bub[:2, orc.B_MG].sum()
    for k in range(600):
        o.step(1)
        act = (o.flag & (orc.GAS | orc.IFACE)) != 0
        live = [b for b in range(8) if (act & (o.owner == b)).any()]
        for b in live:
            assert o.roots[b] == b if b < o.n_bubbles else False
            assert ndimage.label(act & (o.owner == b), st)[1] == 1, (k, b)
        assert np.isclose(sum(o.bub[b, orc.B_MG] for b in live), mg0, rtol=1e-12), k
        assert int(o.scal[orc.SC_STATUS]) == 0, k
    assert o.scal[orc.SC_NMERGE] >= 2 and o.scal[orc.SC_NSPLIT] >= 2


def test_bubble_across_a_periodic_face_is_not_split(orc):
    """a bubble centred on a periodic face has its cells on both sides of the grid: they are
    D3Q19 neighbours through the wrap, so the bubble is one connected region and splitting
    leaves it whole (scipy's labelling without the wrap sees two pieces)"""
    ndimage = pytest.importorskip("scipy.ndimage")
    from paper_1712_07028_gb300 import workloads as W
    wl = W.Workload(name="wrap", nx=24, ny=14, nz=14, tau=0.7, g=(0, 0, 0), bc=(W.PERIODIC, W.WALL, W.WALL),
                    sphere_mode=W.SPHERES_FIXED, bubbles=[W.Bubble((0.0, 7.0, 7.0), 4.0)],
                    split_every=1, max_bubbles=4)
    o = orc.Sim(wl)
    act = (o.flag & (orc.GAS | orc.IFACE)) != 0
    assert ndimage.label(act, ndimage.generate_binary_structure(3, 2))[1] == 2
    o.step(5)
    assert o.scal[orc.SC_NSPLIT] == 0 and o.n_bubbles == 1
    assert (o.owner[(o.flag & (orc.GAS | orc.IFACE)) != 0] == 0).all()


def test_bubble_part_of_zero_volume_stays(orc):
    """R39: a part made only of full interface cells (phi = 1, no gas: zero volume) holds no gas
    to divide; it stays with its bubble, and the other part keeps the whole gas mass"""
    o, V = _two_parts_one_bubble(orc, 3.0, 5.0)
    small = o.owner == 0
    o.flag[small & ((o.flag & (orc.GAS | orc.IFACE)) != 0)] = orc.IFACE
    o.phi[small] = 1.0
    mg = o.bub[0, orc.B_MG]
    o.bubble_model(split=True)
    assert o.scal[orc.SC_NSPLIT] == 0 and o.n_bubbles == 2
    assert (o.owner[small] == 0).all()
    assert np.isclose(o.bub[0, orc.B_MG], mg, rtol=1e-15)


def test_bubble_split_against_a_scipy_restatement(orc):
    """R39 restated with scipy's 18-connectivity labelling (no wrap: walls) on a bubble in three
    parts (ids 0, 1, 2 joined to root 0, radii 3, 4.5, 3.5) beside a separate bubble (id 3):
    the parts' lowest indices order them, the largest keeps id 0, the others take the lowest
    free ids (1, 2) in that order, gas masses in proportion to the volumes"""
    ndimage = pytest.importorskip("scipy.ndimage")
    from paper_1712_07028_gb300 import workloads as W
    wl = W.Workload(name="parts3", nx=40, ny=16, nz=16, tau=0.7, g=(0, 0, 0), sphere_mode=W.SPHERES_FIXED,
                    bubbles=[W.Bubble((30.0, 8.0, 8.0), 3.0), W.Bubble((8.0, 8.0, 8.0), 4.5),
                             W.Bubble((19.0, 6.0, 9.0), 3.5), W.Bubble((25.0, 12.0, 3.0), 1.6)],
                    max_bubbles=6)
    o = orc.Sim(wl)
    assert list(o.roots) == [0, 1, 2, 3]   # four separate bubbles to start with
    for b in (1, 2):
        o.bub[b, orc.B_ROOT] = 0
    mg_family = 1.1 * sum(_gas_volume(orc, o, [b]) for b in range(3))
    for b in range(3):
        o.bub[b, orc.B_MG] = mg_family
        o.bub[b, orc.B_V0] = mg_family / 1.1
    act = (o.flag & (orc.GAS | orc.IFACE)) != 0
    fam = act & np.isin(o.owner, [0, 1, 2])
    lab, n = ndimage.label(fam, ndimage.generate_binary_structure(3, 2))
    assert n == 3
    vol = np.where(o.flag == orc.GAS, 1.0, 1.0 - o.phi)
    flat = lab.ravel()
    parts = []
    for c in range(1, n + 1):
        idx = np.flatnonzero(flat == c)
        parts.append((idx.min(), vol.ravel()[idx].sum(), c))
    parts.sort()
    keep = max(range(3), key=lambda k: (parts[k][1], -parts[k][0]))
    expect = np.where(act, o.owner, -1).copy()
    expect[fam] = 0
    free = iter([1, 2, 4, 5])
    Vt = sum(p[1] for p in parts)
    mg_new = {}
    for k, (rep, V, c) in enumerate(parts):
        if k == keep:
            mg_new[0] = mg_family * V / Vt
            continue
        nid = next(free)
        expect[lab == c] = nid
        mg_new[nid] = mg_family * V / Vt
    o.bubble_model(split=True)
    assert (np.where(act, o.owner, -1) == expect).all()
    assert o.scal[orc.SC_NSPLIT] == 2 and o.n_bubbles == 4
    for b, m in mg_new.items():
        assert np.isclose(o.bub[b, orc.B_MG], m, rtol=1e-12), (b, o.bub[b, orc.B_MG], m)
    assert list(o.roots) == [0, 1, 2, 3]
