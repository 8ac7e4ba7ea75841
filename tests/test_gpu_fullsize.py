"""Parity at the full sizes of the large columns, in the launch configuration the benchmark
times (CUDA-graph replay, each bulk sweep overlapping the previous step's end-of-step
kernels): after some steps, one more step is checked cell by cell against the FP64 oracle
on samples it can compute one at a time.

A sampled cell's post-collision PDFs depend only on its own and its 18 neighbours' PDFs and
types (and, next to a sphere, on the sphere's state), so the oracle steps a small crop of the
GPU's state around it: a 3^3 all-liquid block for a bulk cell, a box around a whole sphere
(its links, its momentum-exchange force) or around two neighbouring spheres (cells between
them link to both), a 9^3 block around an interface cell, among them cells that convert in
the checked step (types, PDFs, masses and fill levels compared in the central 3^3, which
the crop's walls cannot reach within one step: a conversion looks two cells further, its
excess three).  The crop's own walls are seen only by cells that are not compared, except
where they coincide with the domain's walls.  The bubbles' volumes are checked against a
count from the exported fields (gas cells + sum of 1 - phi over interface cells).

Tolerances: the oracle starts from the GPU's stored values, so the difference is the GPU's
FP32 arithmetic (a few 1e-8 on deviations of order 1e-2) plus, with FP16 deviation storage,
the rounding of the stored result to FP16 (half an ulp of 2^-7 .. 2^-6 sized deviations:
below 4e-6).
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


def _axis_range(c, n, periodic, lo_ext, hi_ext):
    """indices of a crop axis around c; at a domain wall the crop stops at the wall"""
    lo, hi = c - lo_ext, c + hi_ext
    if not periodic:
        if lo < 0:
            hi, lo = hi - lo, 0
        if hi > n - 1:
            lo, hi = lo - (hi - (n - 1)), n - 1
        lo = max(lo, 0)
    return np.arange(lo, hi + 1) % n, c - lo


def _crop(wl, st, center, ext):
    """(z, y, x) index arrays of a crop of half-width ext around center (x, y, z) and the
    center's position in it"""
    ix, ox = _axis_range(center[0], wl.nx, wl.bc[0], ext, ext)
    iy, oy = _axis_range(center[1], wl.ny, wl.bc[1], ext, ext)
    iz, oz = _axis_range(center[2], wl.nz, wl.bc[2], ext, ext)
    return (iz, iy, ix), (ox, oy, oz)


def _gather(arr, idx, lead=0):
    iz, iy, ix = idx
    if lead:
        return arr[:, iz[:, None, None], iy[None, :, None], ix[None, None, :]]
    return arr[iz[:, None, None], iy[None, :, None], ix[None, None, :]]


def _oracle_crop_step(wl, f, flags, owner, spheres, mass=None, phi=None, rho_gas=None, share=0.0):
    """one oracle step of a crop: f [19][z][y][x] deviations (FP64), types, owners; spheres
    as (x, u, w, R, rho, F, T) in crop coordinates; with interface cells their masses and fill
    levels, every bubble id's gas density and the pool share each interface cell gets this
    step.  Returns the oracle (near_tol 1e-5: the cells it logs near a threshold)."""
    nz, ny, nx = flags.shape
    nb = len(rho_gas) if rho_gas is not None else 0
    o = oracle.Sim(nx=nx, ny=ny, nz=nz, tau=wl.tau, g=wl.g, bc=(W.WALL,) * 3, sphere_mode=wl.sphere_mode,
                   n_substeps=wl.n_substeps, near_tol=1e-5, bubbles=[(0.0, 0.0, 0.0, 1.0)] * nb,
                   spheres=[(s[0][0], s[0][1], s[0][2], s[3], s[4]) for s in spheres], init=False)
    o.f[:] = f + U.WEIGHTS[:, None, None, None]
    o.flag[:] = flags
    o.owner[:] = owner
    if mass is None:
        o.m[:] = np.where(flags == oracle.LIQ, o.f.sum(axis=0), 0.0)
        o.phi[:] = np.where(flags == oracle.LIQ, 1.0, 0.0)
    else:
        o.m[:] = np.where(flags == oracle.IFACE, mass, np.where(flags == oracle.LIQ, o.f.sum(axis=0), 0.0))
        o.phi[:] = np.where(flags == oracle.IFACE, phi, np.where(flags == oracle.GAS, 0.0, 1.0))
    for b in range(nb):
        o.bub[b, oracle.B_RHOG] = rho_gas[b]
        o.bub[b, oracle.B_V] = o.bub[b, oracle.B_V0] = 1.0
        o.bub[b, oracle.B_MG] = rho_gas[b]
    # the excess pool reaches each interface cell as the same share
    o.scal[oracle.SC_POOL] = share * float((flags == oracle.IFACE).sum())
    for a, s in enumerate(spheres):
        o.sph[a, oracle.S_U:oracle.S_U + 3] = s[1]
        o.sph[a, oracle.S_W:oracle.S_W + 3] = s[2]
        o.sph[a, oracle.S_F:oracle.S_F + 3] = s[5]
        o.sph[a, oracle.S_T:oracle.S_T + 3] = s[6]
        o.sph[a, oracle.S_HASP] = 1.0
    assert o.step(1) & 1 == 0
    return o


def _box(wl, lo, hi):
    """(z, y, x) index arrays of the box [lo, hi] (x, y, z), or None if it leaves the domain"""
    if any(lo[k] < 0 or hi[k] > (wl.nx, wl.ny, wl.nz)[k] - 1 for k in range(3)):
        return None
    return np.arange(lo[2], hi[2] + 1), np.arange(lo[1], hi[1] + 1), np.arange(lo[0], hi[0] + 1)


def _workload(name, storage):
    return W.column_c3(storage) if name == "c3" else W.column_c4(storage)


def _bubble_volumes_from_fields(flags, owner, phi, nbub):
    """V_b = gas cells of b + sum over b's interface cells of (1 - phi), FP64 on the host"""
    import torch
    V = np.zeros(nbub)
    gas = flags == oracle.GAS
    ifc = flags == oracle.IFACE
    for b in range(nbub):
        own = owner == b
        V[b] = float((gas & own).sum().item()) + float((1.0 - phi[ifc & own].double()).sum().item())
    return V


@pytest.mark.parametrize("name,storage,tol", [("c3", "f32", 2e-6), ("c3", "f16dev", 6e-6), ("c4", "f16dev", 6e-6)])
def test_fullsize_sampled_cells_against_oracle(lbm, name, storage, tol):
    import torch
    wl = _workload(name, storage)
    sim = lbm.Sim(wl)
    sim.step(240)   # the bubbles' interfaces convert cells every few steps by now
    ex = sim.export_state()
    flags_d = ex["flags"]
    nbub = len(wl.bubbles)
    V0, V, rg = sim.bubbles()
    # the bubble model at full size: volumes from the cells, gas density = gas mass / volume
    Vf = _bubble_volumes_from_fields(flags_d, ex["owner"], ex["phi"], nbub)
    assert np.abs(V - Vf).max() <= 1e-9 * V.max(), (V, Vf)
    assert np.abs(rg * V - wl.rho_g0 * V0).max() <= 1e-12 * V0.max()
    share = sim.mass_budget()[4]
    n_if = int((flags_d == oracle.IFACE).sum().item())
    share = share / n_if if n_if else 0.0
    # bulk samples: liquid cells whose 3^3 block is liquid (walls count as liquid here)
    liq = (flags_d == oracle.LIQ).float()[None, None]
    allliq = -torch.nn.functional.max_pool3d(-torch.nn.functional.pad(liq, (1, 1, 1, 1, 1, 1), value=1.0), 3, 1)[0, 0] > 0.5
    del liq
    rng = np.random.default_rng(11)
    cand = np.stack([rng.integers(0, n, 20000) for n in (wl.nz, wl.ny, wl.nx)], axis=1)
    keep = allliq[tuple(torch.as_tensor(cand[:, k], device=allliq.device) for k in range(3))].cpu().numpy()
    pick = cand[keep][:192]
    # and cells on every domain face, edge and corner (walls on all six faces)
    extra = []
    for z in (0, wl.nz // 2, wl.nz - 1):
        for y in (0, wl.ny // 2, wl.ny - 1):
            for x in (0, 1, wl.nx // 2, wl.nx - 1):
                if bool(allliq[z, y, x]):
                    extra.append((z, y, x))
    pick = np.concatenate([pick, np.array(extra, dtype=pick.dtype).reshape(-1, 3)])
    f_pre = ex["f"]
    crops = []
    for z, y, x in pick:
        idx, cen = _crop(wl, None, (int(x), int(y), int(z)), 1)
        t_idx = tuple(torch.as_tensor(a, device=f_pre.device) for a in idx)
        f = _gather(f_pre, t_idx, lead=1).double().cpu().numpy()
        fl = _gather(flags_d, t_idx).cpu().numpy()
        crops.append(((int(x), int(y), int(z)), cen, f, fl))
    # sphere samples: single spheres with no other sphere centre within 2R + 3, and pairs of
    # spheres closer than that, in boxes (R + 3 around each sphere) holding only liquid and
    # obstacle cells; the spheres of all obstacle cells in the box go to the oracle (a compared
    # cell, one cell inside the box, links only to cells of the box); force, torque and new
    # centre are compared for the sampled spheres, whose links all lie inside
    xs, us, ws = sim.spheres()
    Fs, Ts = sim.forces()
    owner_d = ex["owner"]
    R = wl.spheres[0].r
    ext = int(R) + 3
    from scipy.spatial import cKDTree
    tree = cKDTree(xs)
    near = tree.query_ball_point(xs, 2 * R + 3)
    sph_crops = []
    n_single = n_pair = 0
    for a in rng.permutation(len(xs)):
        if n_single >= 6 and n_pair >= 4:
            break
        group = sorted(near[a])
        if len(group) == 1 and n_single < 6:
            pass
        elif len(group) == 2 and n_pair < 4 and a == group[0]:
            pass
        else:
            continue
        cs = np.rint(xs[group]).astype(int)
        idx = _box(wl, cs.min(axis=0) - ext, cs.max(axis=0) + ext)
        if idx is None:
            continue
        t_idx = tuple(torch.as_tensor(v, device=f_pre.device) for v in idx)
        fl = _gather(flags_d, t_idx).cpu().numpy()
        ow = _gather(owner_d, t_idx).cpu().numpy()
        if not np.isin(fl, (oracle.LIQ, oracle.OBS)).all():
            continue
        f = _gather(f_pre, t_idx, lead=1).double().cpu().numpy()
        origin = np.array([idx[2][0], idx[1][0], idx[0][0]], float)
        ids = list(group) + sorted(set(int(v) for v in np.unique(ow[fl == oracle.OBS])) - set(group))
        pos = {b: j for j, b in enumerate(ids)}
        ow_local = np.full(fl.shape, -1, np.int32)
        for b, j in pos.items():
            ow_local[(fl == oracle.OBS) & (ow == b)] = j
        sph_crops.append((group, ids, f, fl, ow_local, [xs[b] - origin for b in ids], idx, origin))
        if len(group) == 1:
            n_single += 1
        else:
            n_pair += 1
    mass_d, phi_d = ex["mass"], ex["phi"]
    del allliq
    torch.cuda.empty_cache()
    sim.step(1)
    ex1 = sim.export_state()
    f_post = ex1["f"]
    F1, T1 = sim.forces()
    x1, _, _ = sim.spheres()
    # interface samples: 9^3 blocks (before the step) without obstacle cells, around cells whose
    # type the step changed (conversions) and around other interface cells; if the step changed
    # none, the next step is taken (at most 12 more)
    pre = {"f": f_pre, "flags": flags_d, "owner": owner_d, "mass": mass_d, "phi": phi_d}
    post = ex1
    for attempt in range(13):
        changed = torch.nonzero((pre["flags"] != post["flags"]) & ((pre["flags"] == oracle.IFACE) | (post["flags"] == oracle.IFACE)))
        if len(changed) or attempt == 12:
            break
        pre = post
        _, _, rg = sim.bubbles()
        n_if = int((pre["flags"] == oracle.IFACE).sum().item())
        share = sim.mass_budget()[4] / n_if if n_if else 0.0
        sim.step(1)
        post = sim.export_state()
    ifc = torch.nonzero(pre["flags"] == oracle.IFACE)
    cands = [tuple(int(v) for v in changed[k]) for k in rng.permutation(len(changed))[:200]]
    cands += [tuple(int(v) for v in ifc[k]) for k in rng.permutation(len(ifc))[:400]]
    if_crops = []
    for z, y, x in cands:
        idx = _box(wl, (x - 4, y - 4, z - 4), (x + 4, y + 4, z + 4))
        if idx is None:
            continue
        t_idx = tuple(torch.as_tensor(v, device=f_pre.device) for v in idx)
        fl = _gather(pre["flags"], t_idx).cpu().numpy()
        if (fl == oracle.OBS).any():
            continue
        if_crops.append(((x, y, z), idx, _gather(pre["f"], t_idx, lead=1).double().cpu().numpy(), fl,
                         _gather(pre["owner"], t_idx).cpu().numpy(), _gather(pre["mass"], t_idx).double().cpu().numpy(),
                         _gather(pre["phi"], t_idx).double().cpu().numpy()))
        if len(if_crops) >= 24:
            break
    del ex, f_pre, flags_d, owner_d, mass_d, phi_d, pre
    torch.cuda.empty_cache()
    worst = 0.0
    for (x, y, z), cen, f, fl in crops:
        o = _oracle_crop_step(wl, f, fl, np.full(fl.shape, -1, np.int32), [])
        gpu = f_post[:, z, y, x].double().cpu().numpy()
        ref = o.f[:, cen[2], cen[1], cen[0]] - U.WEIGHTS
        worst = max(worst, np.abs(gpu - ref).max())
    print("%s %s: %d bulk samples, max |df| = %.3g" % (name, storage, len(crops), worst))
    assert worst <= tol, worst
    assert n_single >= 2 and n_pair >= 2, ("too few isolated spheres or pairs to sample", n_single, n_pair)
    for group, ids, f, fl, ow, xc, idx, origin in sph_crops:
        sp = [(xc[j], us[b], ws[b], R, wl.spheres[0].rho, Fs[b], Ts[b]) for j, b in enumerate(ids)]
        o = _oracle_crop_step(wl, f, fl, ow, sp)
        t_idx = tuple(torch.as_tensor(v, device=f_post.device) for v in idx)
        gpu = _gather(f_post, t_idx, lead=1).double().cpu().numpy()
        # liquid cells that are liquid after the oracle's step too, inside the crop's rim
        inner = np.zeros(fl.shape, bool)
        inner[1:-1, 1:-1, 1:-1] = True
        cmp = inner & (fl == oracle.LIQ) & (o.flag == oracle.LIQ)
        df = np.abs(gpu - (o.f - U.WEIGHTS[:, None, None, None]))[:, cmp].max()
        Fo, To = o.forces
        dF = max(np.abs(F1[b] - Fo[j]).max() for j, b in enumerate(group))
        dx = max(np.abs(x1[b] - origin - o.positions[j]).max() for j, b in enumerate(group))
        print("%s %s spheres %s (%d more in the box): max |df| = %.3g, |dF| = %.3g of |F| = %.3g, |dx| = %.3g" % (
            name, storage, list(group), len(ids) - len(group), df, dF, np.abs(Fo[:len(group)]).max(), dx))
        assert df <= tol, (group, df)
        for j, b in enumerate(group):
            # both sides sum the same stored values: FP32 per cell, FP64 over cells
            assert np.abs(F1[b] - Fo[j]).max() <= 1e-5 * max(1e-3, np.abs(Fo[j]).max())
            assert np.abs(T1[b] - To[j]).max() <= 1e-5 * max(1e-2, np.abs(To[j]).max())
        assert dx <= 1e-9
    # interface blocks: the central 3^3 after one step (types, PDFs, masses, fill levels)
    f_post, flags1, mass1, phi1 = post["f"], post["flags"], post["mass"], post["phi"]
    n_conv = n_cmp = 0
    worst_f = worst_m = 0.0
    for (x, y, z), idx, f, fl, ow, ms, ph in if_crops:
        o = _oracle_crop_step(wl, f, fl, ow, [], mass=ms, phi=ph, rho_gas=rg, share=share)
        t_idx = tuple(torch.as_tensor(v[3:6], device=f_post.device) for v in idx)
        gfl = _gather(flags1, t_idx).cpu().numpy()
        ofl = o.flag[3:6, 3:6, 3:6]
        near = U.dilate(o.near > 0, 1)[3:6, 3:6, 3:6]
        mism = gfl != ofl
        assert not np.any(mism & ~near), ((x, y, z), gfl, ofl)
        if mism.any():
            continue
        n_conv += int((fl[3:6, 3:6, 3:6] != ofl).sum())
        act = (ofl == oracle.LIQ) | (ofl == oracle.IFACE)
        gf = _gather(f_post, t_idx, lead=1).double().cpu().numpy()
        worst_f = max(worst_f, float(np.abs(gf - (o.f[:, 3:6, 3:6, 3:6] - U.WEIGHTS[:, None, None, None]))[:, act].max()))
        ii = ofl == oracle.IFACE
        if ii.any():
            gm = _gather(mass1, t_idx).double().cpu().numpy()
            gp = _gather(phi1, t_idx).double().cpu().numpy()
            worst_m = max(worst_m, float(np.abs(gm - o.m[3:6, 3:6, 3:6])[ii].max()),
                          float(np.abs(gp - o.phi[3:6, 3:6, 3:6])[ii].max()))
        n_cmp += 1
    print("%s %s: %d interface blocks compared (%d cells converted in them), max |df| = %.3g, max |dm|, |dphi| = %.3g"
          % (name, storage, n_cmp, n_conv, worst_f, worst_m))
    assert n_cmp >= 12 and n_conv >= 1, (n_cmp, n_conv)
    assert worst_f <= tol and worst_m <= max(tol, 2e-6), (worst_f, worst_m)
    assert sim.status() == 0
    sim.close()
