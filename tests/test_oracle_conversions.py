"""Pins of the oracle's cell conversions (Sec. 2.2, Fig. cellConversions, with the readings
for the details the paper delegates: filling wins, layer closure, new interface cells from the
equilibrium of their neighbours' mean, excess mass along the interface normal, interface cells
without gas turn liquid) and of its covering / uncovering of cells by moved spheres with the
refill of uncovered cells (Sec. 2.3):

  - against the independent set-form NumPy transcription (tests/bruteforce_numpy.py) on
    random states of tiny grids, every field to 1e-12, every branch taken;
  - against values worked out by hand on a flat interface: a filled cell, an emptied cell,
    equal shares when every normal weight vanishes, the global pool, and an uncovered cell
    with a known mix of neighbours (its type, bubble, fill level, mass and PDFs).
"""
import numpy as np
import pytest

from tests import bruteforce_numpy as bf

LIQ, IFACE, GAS, OBS = 1, 2, 4, 8
W = np.array([1 / 3] + [1 / 18] * 6 + [1 / 36] * 12)


def _eq(rho, u):
    c = bf.C
    cu = c @ np.asarray(u, float)
    return W * rho * (1 + 3 * cu + 4.5 * cu ** 2 - 1.5 * float(np.dot(u, u)))


def _sim(orc, shape, bc, g=(0.0, 0.0, 0.0), eps=0.0, spheres=(), sphere_mode=2, nbub=3):
    nz, ny, nx = shape
    s = orc.Sim(nx=nx, ny=ny, nz=nz, bc=bc, g=g, eps=eps, sphere_mode=sphere_mode,
                bubbles=[(0.0, 0.0, 0.0, 1.0)] * nbub, spheres=spheres, init=False)
    return s


def _random_state(rng, s, p_types=(0.4, 0.32, 0.22, 0.06)):
    shape = s.shape
    s.flag[:] = rng.choice([LIQ, IFACE, GAS, OBS], p=p_types, size=shape).astype(np.uint8)
    rho = 1.0 + 0.05 * (rng.random(shape) - 0.5)
    u = 0.02 * (rng.random((3,) + shape) - 0.5)
    cu = np.einsum("qk,kzyx->qzyx", bf.C, u)
    s.f[:] = W[:, None, None, None] * rho * (1 + 3 * cu + 4.5 * cu ** 2 - 1.5 * (u * u).sum(0))
    s.f[:] *= 1 + 0.02 * (rng.random(s.f.shape) - 0.5)
    iface = s.flag == IFACE
    s.phi[:] = np.where(iface, rng.uniform(-0.35, 1.35, shape), np.where(s.flag == GAS, 0.0, 1.0))
    s.m[:] = np.where(iface, s.phi * s.f.sum(0) + 0.01 * (rng.random(shape) - 0.5), 0.0)
    s.owner[:] = np.where(iface | (s.flag == GAS), rng.integers(0, 3, shape), -1)


CONV_CASES = [("walls", (7, 6, 8), (0, 0, 0), (0.0, 0.0, -1e-4), 0.0, 1),
              ("periodic", (6, 7, 6), (1, 1, 1), (2e-4, 0.0, 1e-4), 0.0, 2),
              ("mixed_eps", (8, 7, 6), (1, 0, 0), (0.0, 1e-4, -2e-4), 0.05, 3),
              ("walls_dense_gas", (6, 6, 7), (0, 1, 0), (0.0, 0.0, 0.0), 0.0, 4)]


def _liquid_mass(fl, m, f):
    """liquid mass of a state: density of liquid cells, mass of interface cells"""
    return float(np.where(fl == LIQ, f.sum(0), np.where(fl == IFACE, m, 0.0)).sum())


def _conversions_vs_transcription(orc, s, bc, g=(0.0, 0.0, 0.0), eps=0.0, name=""):
    """run the oracle's conversions on s and the transcription on a copy; compare everything;
    return the transcription's branch counts"""
    nz, ny, nx = s.shape
    p = {"nx": nx, "ny": ny, "nz": nz, "g": g, "bc": bc}
    f0, fl0, m0, ph0, ow0 = s.f.copy(), s.flag.copy(), s.m.copy(), s.phi.copy(), s.owner.copy()
    fb, flb, mb, phb, owb, poolb, st = bf.conversions(p, f0, fl0, m0, ph0, ow0.astype(np.int64), eps=eps)
    pool0 = s.scal[orc.SC_POOL]
    s.conversions()
    assert np.array_equal(s.flag, flb), name
    gi = (flb == IFACE) | (flb == GAS)
    assert np.array_equal(s.owner[gi], owb[gi]), name
    act = (flb == LIQ) | (flb == IFACE)
    assert np.abs(s.f - fb)[:, act].max() < 1e-12, name
    assert np.abs(s.m - mb)[act].max() < 1e-12, name
    if (flb == IFACE).any():
        assert np.abs(s.phi - phb)[flb == IFACE].max() < 1e-12, name
    assert abs(s.scal[orc.SC_POOL] - pool0 - poolb) < 1e-12, name
    # the conversions move mass between cells and the pool, never create or destroy it
    assert abs(_liquid_mass(s.flag, s.m, s.f) + s.scal[orc.SC_POOL] - _liquid_mass(fl0, m0, f0) - pool0) < 1e-11, name
    return st


def test_conversions_match_set_transcription(orc):
    """random types, fill levels, masses and PDFs: the oracle's conversions and the set-form
    transcription agree on types, bubble ids, masses, fill levels, PDFs and the pool (1e-12),
    and both conserve the liquid mass plus the pool; across the cases every branch occurs
    (filled and emptied cells, filled-wins, new interface cells, liquid turned interface,
    weighted / pooled excess, interface cells without gas; equal shares in the hand-built
    case below, which runs through the same comparison)"""
    seen = {}
    for name, shape, bc, g, eps, seed in CONV_CASES:
        rng = np.random.default_rng(seed)
        s = _sim(orc, shape, bc, g=g, eps=eps)
        types = (0.35, 0.3, 0.3, 0.05) if name == "walls_dense_gas" else (0.4, 0.32, 0.22, 0.06)
        _random_state(rng, s, types)
        st = _conversions_vs_transcription(orc, s, bc, g, eps, name)
        for k, v in st.items():
            seen[k] = seen.get(k, 0) + v
    for k in ("filled", "emptied", "newif", "fromliq", "weighted", "pooled", "no_gas_filled"):
        assert seen[k] > 0, (k, seen)


def _flat_interface(orc, shape=(7, 7, 7), g=(0.0, 0.0, 0.0)):
    """liquid below z = 3, interface cells (fill 0.5) at z = 3, gas (bubble 0) above; every
    cell at rest at the density 1 + 0.01 x with velocity (0.001 y, 0, 0)"""
    s = _sim(orc, shape, (0, 0, 0), g=g)
    nz, ny, nx = shape
    z = np.arange(nz)[:, None, None] * np.ones(shape)
    x = np.arange(nx)[None, None, :] * np.ones(shape)
    y = np.arange(ny)[None, :, None] * np.ones(shape)
    s.flag[:] = np.where(z < 3, LIQ, np.where(z == 3, IFACE, GAS)).astype(np.uint8)
    for idx in np.ndindex(shape):
        s.f[(slice(None),) + idx] = _eq(1 + 0.01 * x[idx], (0.001 * y[idx], 0.0, 0.0))
    s.phi[:] = np.where(z < 3, 1.0, np.where(z == 3, 0.5, 0.0))
    s.m[:] = np.where(z == 3, 0.5 * s.f.sum(0), 0.0)
    s.owner[:] = np.where(z >= 3, 0, -1)
    return s


def test_filled_cell_on_a_flat_interface_by_hand(orc):
    """a filled cell (3,3,3) in a flat interface layer: the Parker-Youngs gradient there is
    (0, 0, -1/2) (16 (0 - 1) / 32 along z, symmetric in x and y), so the normal into the gas is
    +z/2 and its excess m - rho goes in equal fifths to the five gas cells above it (weight 1/2
    each), which become interface cells; the in-plane interface cells get nothing.  The new
    interface cell above it takes the equilibrium of the mean density and velocity of its five
    neighbours in the layer: density 1.03, velocity (0.003, 0, 0)"""
    s = _flat_interface(orc)
    rho = 1.03   # at x = 3
    s.m[3, 3, 3], s.phi[3, 3, 3] = rho + 0.2, 1.2
    st = _conversions_vs_transcription(orc, s, (0, 0, 0), name="filled by hand")
    assert st["filled"] == 1 and st["newif"] == 5 and st["weighted"] == 1
    assert s.flag[3, 3, 3] == LIQ and s.owner[3, 3, 3] == -1 and abs(s.m[3, 3, 3] - rho) < 1e-15
    up = [(4, 3, 3), (4, 3, 4), (4, 3, 2), (4, 4, 3), (4, 2, 3)]   # (z, y, x): c = (0,0,1), (+-1,0,1), (0,+-1,1)
    for c in up:
        assert s.flag[c] == IFACE and s.owner[c] == 0
        assert abs(s.m[c] - 0.04) < 1e-14, (c, s.m[c])
    # the cell straight above: neighbours in the layer at x = 2, 3, 3, 3, 4 and y = 3, 3, 2, 4, 3
    assert np.abs(s.f[:, 4, 3, 3] - _eq(1.03, (0.003, 0.0, 0.0))).max() < 1e-15
    assert abs(s.phi[4, 3, 3] - 0.04 / 1.03) < 1e-14
    # in-plane interface neighbours: weight 0, fill level unchanged
    for c in [(3, 3, 2), (3, 3, 4), (3, 2, 3), (3, 4, 3), (3, 2, 2), (3, 4, 4), (3, 2, 4), (3, 4, 2)]:
        assert s.flag[c] == IFACE and abs(s.phi[c] - 0.5) < 1e-15
    assert (s.flag[5:] == GAS).all() and s.scal[orc.SC_POOL] == 0.0
    assert (s.flag == IFACE).sum() == 7 * 7 - 1 + 5


def test_emptied_cell_on_a_flat_interface_by_hand(orc):
    """an emptied cell (3,3,3): its five liquid neighbours below turn interface with their
    density as mass and its bubble id; its (negative) mass goes along -n_g = -z/2 to them in
    equal fifths; it becomes gas"""
    s = _flat_interface(orc)
    s.m[3, 3, 3], s.phi[3, 3, 3] = -0.1, -0.1
    st = _conversions_vs_transcription(orc, s, (0, 0, 0), name="emptied by hand")
    assert st["emptied"] == 1 and st["fromliq"] == 5 and st["weighted"] == 1
    assert s.flag[3, 3, 3] == GAS and s.m[3, 3, 3] == 0.0
    down = [(2, 3, 3), (2, 3, 4), (2, 3, 2), (2, 4, 3), (2, 2, 3)]
    for c in down:
        r = 1 + 0.01 * c[2]
        assert s.flag[c] == IFACE and s.owner[c] == 0
        assert abs(s.m[c] - (r - 0.02)) < 1e-14 and abs(s.phi[c] - (r - 0.02) / r) < 1e-14
    assert (s.flag[4:] == GAS).all() and s.scal[orc.SC_POOL] == 0.0


def test_equal_shares_and_pool_by_hand(orc):
    """(a) an interface cell with no gas neighbour is filled whatever its fill level; with a
    vanishing normal (liquid all round but two interface cells at +-x, each beside a gas cell)
    its excess goes in equal halves to those two; (b) a filled cell with no interface
    neighbour at all gives its excess to the global pool"""
    s = _sim(orc, (7, 7, 9), (0, 0, 0))
    s.flag[:] = LIQ
    s.f[:] = W[:, None, None, None]
    s.phi[:] = 1.0
    s.owner[:] = -1
    for x in (2, 4):
        s.flag[3, 3, x], s.phi[3, 3, x], s.m[3, 3, x], s.owner[3, 3, x] = IFACE, 0.5, 0.5, 0
    for x in (1, 5):
        s.flag[3, 3, x], s.phi[3, 3, x], s.owner[3, 3, x] = GAS, 0.0, 0
    s.flag[3, 3, 3], s.phi[3, 3, 3], s.m[3, 3, 3], s.owner[3, 3, 3] = IFACE, 0.7, 0.7, 0
    s.flag[3, 3, 7], s.phi[3, 3, 7], s.m[3, 3, 7], s.owner[3, 3, 7] = IFACE, 0.8, 1.25, 0   # no gas, no interface beside it
    st = _conversions_vs_transcription(orc, s, (0, 0, 0), name="equal shares and pool by hand")
    assert st["uniform"] == 1 and st["pooled"] == 1 and st["no_gas_filled"] == 2
    assert s.flag[3, 3, 3] == LIQ and abs(s.m[3, 3, 3] - 1.0) < 1e-15
    for x in (2, 4):
        assert s.flag[3, 3, x] == IFACE and abs(s.m[3, 3, x] - 0.35) < 1e-15 and abs(s.phi[3, 3, x] - 0.35) < 1e-15
    assert s.flag[3, 3, 7] == LIQ and abs(s.scal[orc.SC_POOL] - 0.25) < 1e-15


COVER_CASES = [("walls", (9, 8, 10), (0, 0, 0), 5, (0.45, 0.3, 0.25, 0.0)),
               ("periodic", (8, 9, 8), (1, 1, 1), 6, (0.45, 0.3, 0.25, 0.0)),
               ("mixed", (10, 8, 9), (0, 1, 0), 7, (0.45, 0.3, 0.25, 0.0)),
               ("mostly_gas", (9, 9, 9), (0, 0, 1), 8, (0.04, 0.04, 0.92, 0.0))]


def test_cover_uncover_matches_set_transcription(orc):
    """random types around spheres that moved by up to 0.9 cells (obstacle cells stamped at
    the old centres): the oracle and the transcription agree on covered and uncovered cells,
    their types, bubble / sphere ids, masses, fill levels and refilled PDFs, and S_cover,
    S_uncover (1e-12); every refill type occurs"""
    seen = {}
    for name, shape, bc, seed, types in COVER_CASES:
        rng = np.random.default_rng(seed)
        nz, ny, nx = shape
        sph = []
        for a in range(3):
            x = tuple(float(rng.uniform(1.5, n - 2.5)) for n in (nx, ny, nz))
            sph.append((*x, float(rng.uniform(1.2, 2.2)), 1.5, *(rng.uniform(-0.05, 0.05, 3)), *(rng.uniform(-0.05, 0.05, 3))))
        s = _sim(orc, shape, bc, spheres=sph)
        _random_state(rng, s, types)
        p = {"nx": nx, "ny": ny, "nz": nz, "bc": bc}
        old = [{"x": np.array(sp[:3]), "r": sp[3]} for sp in sph]
        own_old = bf.covered_by(p, old, shape)
        s.flag[own_old >= 0] = OBS
        s.owner[own_old >= 0] = own_old[own_old >= 0]
        for a in range(3):   # the move
            s.sph[a, orc.S_X:orc.S_X + 3] += rng.uniform(-0.9, 0.9, 3)
        new = [{"x": s.sph[a, orc.S_X:orc.S_X + 3].copy(), "r": s.sph[a, orc.S_R], "u": s.sph[a, orc.S_U:orc.S_U + 3].copy(),
                "w": s.sph[a, orc.S_W:orc.S_W + 3].copy()} for a in range(3)]
        f0, fl0, m0, ph0, ow0 = s.f.copy(), s.flag.copy(), s.m.copy(), s.phi.copy(), s.owner.copy()
        fb, flb, mb, phb, owb, scb, sub, st = bf.cover_uncover(p, f0, fl0, m0, ph0, ow0.astype(np.int64), new)
        s.cover_uncover()
        assert np.array_equal(s.flag, flb), name
        keep = flb != LIQ
        assert np.array_equal(s.owner[keep], owb[keep]), name
        act = (flb == LIQ) | (flb == IFACE)
        assert np.abs(s.f - fb)[:, act].max() < 1e-12, name
        assert np.abs(s.m - mb)[act].max() < 1e-12 and np.abs(s.phi - phb)[flb == IFACE].max() < 1e-12, name
        assert abs(s.scal[orc.SC_SCOV] - scb) < 1e-12 and abs(s.scal[orc.SC_SUNC] - sub) < 1e-12, name
        for k, v in st.items():
            seen[k] = seen.get(k, 0) + v
    for k in ("covered", "uncovered", "to_gas", "to_iface", "to_liq"):
        assert seen[k] > 0, (k, seen)


def test_uncovered_cell_by_hand(orc):
    """a sphere of radius 1/2 moves from (3,3,3) to (4,3,3) in a flat interface layer (liquid
    below z = 3 at density 1.02, interface at z = 3 with fill 0.4 and density 0.99, gas above):
    the cell it leaves has 7 interface, 5 liquid and 5 gas neighbours (the 18th is the sphere),
    so it becomes an interface cell of the first gas neighbour's bubble (q order: straight up,
    bubble 1), fill (7 0.4 + 5) / 12 = 0.65, mass 0.65 rho_mean with rho_mean =
    (7 0.99 + 5 1.02) / 12, PDFs e(rho_mean, u_P + w_P x (x - x_P)) = e(rho_mean, (0.5, -0.2, 0));
    the cell it enters loses its interface mass 0.4 0.99 to S_cover"""
    s = _sim(orc, (7, 7, 7), (0, 0, 0), spheres=[(4.0, 3.0, 3.0, 0.5, 1.5, 0.5, 0.0, 0.0, 0.0, 0.0, 0.2)])
    z = np.arange(7)[:, None, None] * np.ones((7, 7, 7))
    s.flag[:] = np.where(z < 3, LIQ, np.where(z == 3, IFACE, GAS)).astype(np.uint8)
    rho = np.where(z < 3, 1.02, 0.99)
    s.f[:] = W[:, None, None, None] * rho
    s.phi[:] = np.where(z < 3, 1.0, np.where(z == 3, 0.4, 0.0))
    s.m[:] = np.where(z == 3, 0.4 * 0.99, 0.0)
    s.owner[:] = np.where(z >= 3, 0, -1)
    s.owner[4, 3, 3] = 1
    s.flag[3, 3, 3], s.owner[3, 3, 3] = OBS, 0
    s.cover_uncover()
    rb = (7 * 0.99 + 5 * 1.02) / 12
    assert s.flag[3, 3, 3] == IFACE and s.owner[3, 3, 3] == 1
    assert abs(s.phi[3, 3, 3] - 0.65) < 1e-15 and abs(s.m[3, 3, 3] - 0.65 * rb) < 1e-15
    assert np.abs(s.f[:, 3, 3, 3] - _eq(rb, (0.5, -0.2, 0.0))).max() < 1e-15
    assert s.flag[3, 3, 4] == OBS and s.owner[3, 3, 4] == 0
    assert abs(s.scal[orc.SC_SCOV] - 0.4 * 0.99) < 1e-15 and abs(s.scal[orc.SC_SUNC] - 0.65 * rb) < 1e-15


@pytest.mark.parametrize("where,expect", [("liquid", LIQ), ("gas", GAS)])
def test_uncovered_cell_type_by_hand(orc, where, expect):
    """the same move deep in the liquid (no gas neighbour) refills a liquid cell of the mean
    density (bubble id -1, mass rho_mean); deep in the gas (no liquid or interface neighbour)
    a gas cell of its first gas neighbour's bubble"""
    s = _sim(orc, (7, 7, 7), (0, 0, 0), spheres=[(4.0, 3.0, 3.0, 0.5, 1.5, 0.1, 0.0, 0.0, 0.0, 0.0, 0.0)])
    t = LIQ if where == "liquid" else GAS
    s.flag[:] = t
    s.f[:] = W[:, None, None, None] * 1.01
    s.phi[:] = 1.0 if t == LIQ else 0.0
    s.owner[:] = -1 if t == LIQ else 2
    s.flag[3, 3, 3], s.owner[3, 3, 3] = OBS, 0
    s.cover_uncover()
    assert s.flag[3, 3, 3] == expect
    if expect == LIQ:
        assert s.owner[3, 3, 3] == -1 and abs(s.m[3, 3, 3] - 1.01) < 1e-15
        assert np.abs(s.f[:, 3, 3, 3] - _eq(1.01, (0.1, 0.0, 0.0))).max() < 1e-15
    else:
        assert s.owner[3, 3, 3] == 2 and s.m[3, 3, 3] == 0.0 and s.scal[orc.SC_SUNC] == 0.0
