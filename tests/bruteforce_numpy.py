"""Brute-force NumPy transcription of the sweep (step 1) on tiny grids -- test infrastructure.

Written in *push* form, per link, independently of the C oracle (which pulls): every
post-collision f*_q(y) of an active cell y travels to y + c_q, and what happens there
decides where it lands (Eq. LBE1; halfway bounce-back at walls; Eq. bbrule at sphere
links; Eq. fsk where the target is gas); the gas at rest reflected from a sphere's surface
presses on the sphere.  Mass exchange (Eqs. massExchange/b) is taken
per interface link.  The collision is the TRT operator of Eq. LBE2 written with explicit
even/odd parts and the Guo force, which acts on the liquid mass (rho g in a liquid cell, phi rho g
in an interface cell, phi its fill level after the mass exchange).  Cell conversions are not
transcribed here.
"""
import numpy as np

LIQ, IFACE, GAS, OBS = 1, 2, 4, 8

C = np.array([[0, 0, 0], [1, 0, 0], [-1, 0, 0], [0, 1, 0], [0, -1, 0], [0, 0, 1], [0, 0, -1],
              [1, 1, 0], [-1, -1, 0], [1, -1, 0], [-1, 1, 0], [1, 0, 1], [-1, 0, -1], [1, 0, -1],
              [-1, 0, 1], [0, 1, 1], [0, -1, -1], [0, 1, -1], [0, -1, 1]])
WQ = np.array([1 / 3] + [1 / 18] * 6 + [1 / 36] * 12)
OPP = np.array([int(np.where((C == -C[q]).all(axis=1))[0][0]) for q in range(19)])


def _target(p, x, y, z, c):
    """cell reached from (x,y,z) along c, or None beyond a wall"""
    n = [p["nx"], p["ny"], p["nz"]]
    t = [x + c[0], y + c[1], z + c[2]]
    for k in range(3):
        if t[k] < 0 or t[k] >= n[k]:
            if not p["bc"][k]:
                return None
            t[k] %= n[k]
    return tuple(t)


def _mind(p, a, b):
    n = [p["nx"], p["ny"], p["nz"]]
    d = np.array(a, float) - np.array(b, float)
    for k in range(3):
        if p["bc"][k]:
            d[k] -= n[k] * np.round(d[k] / n[k])
    return d


def sweep(p, f, flag, m, phi, owner, kappa, spheres, rho_gas):
    """one sweep; f is [19][z][y][x]; spheres: list of dicts x,u,w.  Returns
    (f_new, m_new, phi_new, F, T) with F, T the momentum-exchange sums per sphere."""
    nz, ny, nx = flag.shape
    g = np.array(p["g"], float)
    fin = np.full_like(f, np.nan)
    F = np.zeros((len(spheres), 3))
    T = np.zeros((len(spheres), 3))
    dm = np.zeros_like(m)
    act = (flag & (LIQ | IFACE)) != 0
    rho0 = f.sum(axis=0)
    gw0 = np.where(flag & IFACE, phi, 1.0)   # the force the last collision applied
    u0 = (np.einsum("qk,qzyx->kzyx", C, f) - 0.5 * rho0 * gw0 * g[:, None, None, None]) / np.where(act, rho0, 1)
    for z in range(nz):
        for y in range(ny):
            for x in range(nx):
                if flag[z, y, x] & GAS and len(spheres):   # the gas at rest presses on spheres
                    for q in range(1, 19):
                        t = _target(p, x, y, z, C[q])
                        if t is not None and flag[t[2], t[1], t[0]] & OBS:
                            k = owner[t[2], t[1], t[0]]
                            dj = 2 * WQ[q] * rho_gas[owner[z, y, x]] * C[q]
                            F[k] += dj
                            T[k] += np.cross(_mind(p, (x, y, z), spheres[k]["x"]), dj)
                if not act[z, y, x]:
                    continue
                for q in range(19):
                    v = f[q, z, y, x]
                    t = _target(p, x, y, z, C[q])
                    if t is None:                              # wall
                        fin[OPP[q], z, y, x] = v
                        continue
                    tx, ty, tz = t
                    ft = flag[tz, ty, tx]
                    if ft & (LIQ | IFACE):
                        fin[q, tz, ty, tx] = v
                        if flag[z, y, x] & IFACE and q > 0:     # mass leaving y towards t
                            if ft & LIQ:
                                dm[z, y, x] -= v
                                pass
                            else:
                                dm[z, y, x] -= 0.5 * (phi[z, y, x] + phi[tz, ty, tx]) * v
                        if ft & IFACE and q > 0 and flag[z, y, x] & (LIQ | IFACE):
                            if flag[z, y, x] & LIQ:
                                dm[tz, ty, tx] += v
                            else:
                                dm[tz, ty, tx] += 0.5 * (phi[z, y, x] + phi[tz, ty, tx]) * v
                    elif ft & OBS:                             # moving wall, link midpoint
                        S = spheres[owner[tz, ty, tx]]
                        xw = np.array([x, y, z], float) + 0.5 * C[q]
                        uw = np.array(S["u"]) + np.cross(S["w"], _mind(p, xw, S["x"]))
                        back = v - 6 * WQ[q] * rho0[z, y, x] * (C[q] @ uw)
                        fin[OPP[q], z, y, x] = back
                        dj = C[q] * v - C[OPP[q]] * back
                        F[owner[tz, ty, tx]] += dj
                        T[owner[tz, ty, tx]] += np.cross(_mind(p, (x, y, z), S["x"]), dj)
                    else:                                      # gas
                        rw = rho_gas[owner[tz, ty, tx]] + 6 * p["sigma"] * kappa[z, y, x]
                        uu = u0[:, z, y, x]
                        ep = WQ[q] * rw * (1 + 4.5 * (C[q] @ uu) ** 2 - 1.5 * (uu @ uu))
                        fin[OPP[q], z, y, x] = -v + 2 * ep
    lp = -1 / p["tau"]
    lm = 1 / ((3 / 16) / (1 / lp + 0.5) - 0.5)
    fout = np.zeros_like(f)
    m_new = m.copy()
    phi_new = phi.copy()
    for z in range(nz):
        for y in range(ny):
            for x in range(nx):
                if not act[z, y, x]:
                    continue
                fi = fin[:, z, y, x]
                rho = fi.sum()
                gc = g
                if flag[z, y, x] & IFACE:
                    m_new[z, y, x] = m[z, y, x] + dm[z, y, x]
                    phi_new[z, y, x] = m_new[z, y, x] / rho
                    gc = g * phi_new[z, y, x]
                u = (C.T @ fi + 0.5 * rho * gc) / rho
                e = WQ * rho * (1 + 3 * (C @ u) + 4.5 * (C @ u) ** 2 - 1.5 * (u @ u))
                G = WQ * rho * ((3 * (C - u) + 9 * np.outer(C @ u, np.ones(3)) * C) @ gc)
                fp, fm = 0.5 * (fi + fi[OPP]), 0.5 * (fi - fi[OPP])
                ep, em = 0.5 * (e + e[OPP]), 0.5 * (e - e[OPP])
                Gp, Gm = 0.5 * (G + G[OPP]), 0.5 * (G - G[OPP])
                fout[:, z, y, x] = fi + lp * (fp - ep) + lm * (fm - em) + (1 + lp / 2) * Gp + (1 + lm / 2) * Gm
    return fout, m_new, phi_new, F, T
