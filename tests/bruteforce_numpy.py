"""Brute-force NumPy transcription of the sweep (step 1) on tiny grids -- test infrastructure.

Written in *push* form, per link, independently of the C oracle (which pulls): every
post-collision f*_q(y) of an active cell y travels to y + c_q, and what happens there
decides where it lands (Eq. LBE1; halfway bounce-back at walls; Eq. bbrule at sphere
links; Eq. fsk where the target is gas); the gas at rest reflected from a sphere's surface
presses on the sphere.  Mass exchange (Eqs. massExchange/b) is taken
per interface link.  The collision is the TRT operator of Eq. LBE2 written with explicit
even/odd parts and the Guo force, which acts on the liquid mass (rho g in a liquid cell, phi rho g
in an interface cell, phi its fill level after the mass exchange).

The cell conversions (Sec. 2.2, Fig. cellConversions) and the covering / uncovering of cells
by moved spheres with the refill of uncovered cells (Sec. 2.3) are transcribed below in set
form: whole-grid masks combined by neighbour shifts, where the oracle walks cells one by one.
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


# ------------------------------------------------------------------ conversions (set form)

def _nb(a, c, bc, fill):
    """b[z, y, x] = a at the neighbour (x, y, z) + c; `fill` where that lies beyond a wall"""
    out = a
    for axis, k in ((2, 0), (1, 1), (0, 2)):   # array axes (z, y, x) hold coordinates (x, y, z) reversed
        d = int(c[k])
        if d == 0:
            continue
        out = np.roll(out, -d, axis=axis)
        if not bc[k]:
            out = out.copy()
            idx = [slice(None)] * 3
            idx[axis] = slice(-1, None) if d > 0 else slice(0, 1)
            out[tuple(idx)] = fill
    return out


def _any_nb(mask, bc):
    """cells with at least one D3Q19 neighbour in mask"""
    out = np.zeros_like(mask)
    for q in range(1, 19):
        out |= _nb(mask, C[q], bc, False)
    return out


def _density(f):
    return f.sum(axis=0)


def _velocity(p, f, flag, phi):
    """the velocity the last collision used: (sum c f - rho gw g / 2) / rho, gw the fill level
    of an interface cell, 1 otherwise"""
    rho = f.sum(axis=0)
    gw = np.where(flag == IFACE, phi, 1.0)
    g = np.array(p["g"], float)
    return (np.einsum("qk,qzyx->kzyx", C, f) - 0.5 * rho * gw * g[:, None, None, None]) / np.where(rho != 0, rho, 1)


def _equilibrium(rho, u):
    """e_q(rho, u) for every q, [19] + shape of rho"""
    cu = np.einsum("qk,k...->q...", C, u)
    uu = (u * u).sum(axis=0)
    return WQ.reshape((19,) + (1,) * np.ndim(rho)) * rho * (1 + 3 * cu + 4.5 * cu ** 2 - 1.5 * uu)


def _fill_seen(flag, phi):
    """the fill level the interface normal sees: phi at interface cells, 0 at gas, 1 at
    liquid and obstacle cells"""
    return np.where(flag == IFACE, phi, np.where(flag == GAS, 0.0, 1.0))


def _normal(bc, flag, phi):
    """Parker-Youngs gradient of the fill level at every cell: the central difference along
    each axis, summed over the 3 x 3 cross-section with weights [1,2,1] x [1,2,1], over 32;
    beyond a wall the fill level is 1"""
    fs = _fill_seen(flag, phi)
    wt = {-1: 1.0, 0: 2.0, 1: 1.0}
    n = np.zeros((3,) + flag.shape)
    for k in range(3):
        others = [a for a in range(3) if a != k]
        for a in (-1, 0, 1):
            for b in (-1, 0, 1):
                cp = [0, 0, 0]
                cp[others[0]], cp[others[1]] = a, b
                cm = list(cp)
                cp[k], cm[k] = 1, -1
                n[k] += wt[a] * wt[b] * (_nb(fs, cp, bc, 1.0) - _nb(fs, cm, bc, 1.0))
    return n / 32.0


def conversions(p, f, flag, m, phi, owner, eps=0.0):
    """interface / liquid / gas conversions of one step on the sweep's result (f holds
    f*(t+1), phi and m its fill levels and masses).  Returns (f, flag, m, phi, owner, pool,
    stats) with pool the excess no neighbour could take and stats the branches taken."""
    bc = p["bc"]
    shape = flag.shape
    f, flag0, m, phi, owner = f.copy(), flag.copy(), m.copy(), phi.copy(), owner.copy()
    iface, gas, liq = flag0 == IFACE, flag0 == GAS, flag0 == LIQ
    # an interface cell fills at phi >= 1 + eps, or when no gas cell is beside it (it is then no
    # boundary of the liquid towards the gas); else it empties at phi <= -eps
    filled = iface & (~_any_nb(gas, bc) | (phi >= 1 + eps))
    emptied = iface & ~filled & (phi <= -eps)
    # filling wins: a filled neighbour keeps an emptied cell an interface cell, and turns gas
    # neighbours into new interface cells
    near_filled = _any_nb(filled, bc)
    emptied &= ~near_filled
    newif = gas & near_filled
    # liquid beside an emptied cell becomes interface, with its whole density as mass and the
    # smallest bubble id among the emptied cells beside it
    fromliq = liq & _any_nb(emptied, bc)
    rho = _density(f)
    u = _velocity(p, f, flag0, phi)
    big = np.iinfo(np.int64).max
    own_e = np.full(shape, big, np.int64)
    for q in range(1, 19):
        cand = _nb(np.where(emptied & (owner >= 0), owner, big), C[q], bc, big)
        own_e = np.minimum(own_e, cand)
    m[fromliq] = rho[fromliq]
    owner[fromliq] = np.where(own_e[fromliq] == big, -1, own_e[fromliq])
    # new interface cells: equilibrium of the mean density and velocity of the neighbours that
    # carry PDFs and do not empty; no mass
    src = ((flag0 == LIQ) | (flag0 == IFACE)) & ~emptied
    cnt = np.zeros(shape)
    rsum = np.zeros(shape)
    usum = np.zeros((3,) + shape)
    for q in range(1, 19):
        cnt += _nb(src.astype(float), C[q], bc, 0.0)
        rsum += _nb(np.where(src, rho, 0.0), C[q], bc, 0.0)
        for k in range(3):
            usum[k] += _nb(np.where(src, u[k], 0.0), C[q], bc, 0.0)
    rb = np.where(cnt > 0, rsum / np.maximum(cnt, 1), 1.0)
    ub = np.where(cnt > 0, usum / np.maximum(cnt, 1), 0.0)
    feq = _equilibrium(rb, ub)
    f[:, newif] = feq[:, newif]
    m[newif] = 0.0
    # excess mass of each converting cell to the cells beside it that are interface cells after
    # the step, weighted along the normal into the gas n_g = -grad phi: a filled cell by
    # max(0, n_g . c), an emptied one by max(0, -n_g . c); equal shares if every weight is 0;
    # the global pool if no such cell is beside it
    ng = -_normal(bc, flag0, phi)
    conv = filled | emptied
    recv_mask = (iface & ~conv) | newif | fromliq
    received = np.zeros(shape, bool)
    pool = 0.0
    stats = {"filled": int(filled.sum()), "emptied": int(emptied.sum()), "newif": int(newif.sum()),
             "fromliq": int(fromliq.sum()), "weighted": 0, "uniform": 0, "pooled": 0,
             "no_gas_filled": int((iface & ~_any_nb(gas, bc)).sum())}
    nz, ny, nx = shape
    for idx in np.flatnonzero(conv.ravel()):   # in the order of the cells' linear index
        z, y, x = np.unravel_index(idx, shape)
        if filled[z, y, x]:
            mex = m[z, y, x] - rho[z, y, x]
            m[z, y, x] = rho[z, y, x]
        else:
            mex = m[z, y, x]
            m[z, y, x] = 0.0
        recs, ws = [], []
        for q in range(1, 19):
            t = _target(p, x, y, z, C[q])
            if t is None or not recv_mask[t[2], t[1], t[0]]:
                continue
            nc = float(ng[:, z, y, x] @ C[q])
            ws.append(max(nc, 0.0) if filled[z, y, x] else max(-nc, 0.0))
            recs.append((t[2], t[1], t[0]))
        if not recs:
            pool += mex
            stats["pooled"] += 1
            continue
        W = sum(ws)
        stats["weighted" if W > 0 else "uniform"] += 1
        for r, w in zip(recs, ws):
            m[r] += mex * (w / W) if W > 0 else mex / len(recs)
            received[r] = True
    flag = flag0.copy()
    flag[filled] = LIQ
    owner[filled] = -1
    flag[emptied] = GAS
    flag[newif | fromliq] = IFACE
    upd = (newif | fromliq | received) & (flag == IFACE)
    phi[upd] = m[upd] / _density(f)[upd]
    return f, flag, m, phi, owner, pool, stats


# ------------------------------------------------------- cover / uncover and refill (set form)

def covered_by(p, spheres, shape):
    """the lowest id of the spheres whose centre is within R of each cell (|x - x_P|^2 <= R^2,
    nearest periodic image), -1 where none is"""
    nz, ny, nx = shape
    zz, yy, xx = np.meshgrid(np.arange(nz), np.arange(ny), np.arange(nx), indexing="ij")
    L = (nx, ny, nz)
    own = np.full(shape, -1, np.int64)
    for a in reversed(range(len(spheres))):
        S = spheres[a]
        d2 = np.zeros(shape)
        for k, cc in enumerate((xx, yy, zz)):
            d = cc - S["x"][k]
            if p["bc"][k]:
                d = d - L[k] * np.round(d / L[k])
            d2 += d * d
        own[d2 <= S["r"] ** 2] = a
    return own


def cover_uncover(p, f, flag, m, phi, owner, spheres):
    """cells that the spheres at their current centres cover become their obstacle cells (a
    covered liquid cell's density, an interface cell's mass goes to S_cover); obstacle cells
    no sphere covers any more are refilled from the neighbours that are neither obstacle nor
    refilled themselves: all gas -> gas (the first gas neighbour's bubble); gas and liquid /
    interface -> interface with mass phi_mean rho_mean; else liquid; PDFs e(rho_mean,
    u_P + w_P x (x - x_P)) of the sphere that left.  Returns (f, flag, m, phi, owner, S_cover,
    S_uncover, stats)."""
    bc = p["bc"]
    shape = flag.shape
    f, flag, m, phi, owner = f.copy(), flag.copy(), m.copy(), phi.copy(), owner.copy()
    nown = covered_by(p, spheres, shape)
    obs = flag == OBS
    uncov = obs & (nown < 0)
    keep = obs & (nown >= 0)
    owner[keep] = nown[keep]
    cov = ~obs & (nown >= 0)
    rho = _density(f)
    s_cover = float(rho[cov & (flag == LIQ)].sum() + m[cov & (flag == IFACE)].sum())
    flag[cov] = OBS
    owner[cov] = nown[cov]
    s_uncover = 0.0
    stats = {"covered": int(cov.sum()), "uncovered": int(uncov.sum()), "to_gas": 0, "to_iface": 0, "to_liq": 0}
    new = {}
    for idx in np.flatnonzero(uncov.ravel()):
        z, y, x = np.unravel_index(idx, shape)
        gas_own, ngas, rhos, phis = None, 0, [], []
        for q in range(1, 19):
            t = _target(p, x, y, z, C[q])
            if t is None:
                continue
            tz, ty, tx = t[2], t[1], t[0]
            if flag[tz, ty, tx] == OBS or uncov[tz, ty, tx]:
                continue
            if flag[tz, ty, tx] == GAS:
                ngas += 1
                if gas_own is None:
                    gas_own = owner[tz, ty, tx]
            else:
                rhos.append(rho[tz, ty, tx])
                phis.append(phi[tz, ty, tx] if flag[tz, ty, tx] == IFACE else 1.0)
        S = spheres[owner[z, y, x]]
        r = _mind(p, (x, y, z), S["x"])
        uf = np.array(S["u"], float) + np.cross(S["w"], r)
        if not rhos and ngas:
            new[(z, y, x)] = (GAS, gas_own, 0.0, 0.0, None)
            stats["to_gas"] += 1
            continue
        rb = float(np.mean(rhos)) if rhos else 1.0
        fe = _equilibrium(np.array(rb), uf)
        if ngas:
            pb = float(np.mean(phis))
            new[(z, y, x)] = (IFACE, gas_own, pb * rb, pb, fe)
            s_uncover += pb * rb
            stats["to_iface"] += 1
        else:
            new[(z, y, x)] = (LIQ, -1, rb, 1.0, fe)
            s_uncover += rb
            stats["to_liq"] += 1
    for (z, y, x), (t, o, mm, ph, fe) in new.items():
        flag[z, y, x], owner[z, y, x], m[z, y, x], phi[z, y, x] = t, o, mm, ph
        if fe is not None:
            f[:, z, y, x] = fe
    return f, flag, m, phi, owner, s_cover, s_uncover, stats
