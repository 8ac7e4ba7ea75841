"""Parity at the full sizes of the large columns, in the launch configuration the benchmark
times (CUDA-graph replay, each bulk sweep overlapping the previous step's end-of-step
kernels): after some steps, one more step is checked cell by cell against the FP64 oracle
on samples it can compute one at a time.

A sampled cell's post-collision PDFs depend only on its own and its 18 neighbours' PDFs and
types (and, next to a sphere, on the sphere's state), so the oracle steps a small crop of the
GPU's state around it: a 3^3 all-liquid block for a bulk cell, a box around a whole sphere
(its links, its momentum-exchange force).  The crop's own walls are seen only by cells that
are not compared, except where they coincide with the domain's walls.

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


def _oracle_crop_step(wl, f, flags, owner, spheres):
    """one oracle step of a crop: f [19][z][y][x] deviations (FP64), types, owners; spheres
    as (x, u, w, R, rho, F, T) in crop coordinates.  Returns the oracle."""
    nz, ny, nx = flags.shape
    o = oracle.Sim(nx=nx, ny=ny, nz=nz, tau=wl.tau, g=wl.g, bc=(W.WALL,) * 3, sphere_mode=wl.sphere_mode,
                   n_substeps=wl.n_substeps,
                   spheres=[(s[0][0], s[0][1], s[0][2], s[3], s[4]) for s in spheres], init=False)
    o.f[:] = f + U.WEIGHTS[:, None, None, None]
    o.flag[:] = flags
    o.owner[:] = owner
    o.m[:] = np.where(flags == oracle.LIQ, o.f.sum(axis=0), 0.0)
    o.phi[:] = np.where(flags == oracle.LIQ, 1.0, 0.0)
    for a, s in enumerate(spheres):
        o.sph[a, oracle.S_U:oracle.S_U + 3] = s[1]
        o.sph[a, oracle.S_W:oracle.S_W + 3] = s[2]
        o.sph[a, oracle.S_F:oracle.S_F + 3] = s[5]
        o.sph[a, oracle.S_T:oracle.S_T + 3] = s[6]
        o.sph[a, oracle.S_HASP] = 1.0
    assert o.step(1) == 0
    return o


def _workload(name, storage):
    return W.column_c3(storage) if name == "c3" else W.column_c4(storage)


@pytest.mark.parametrize("name,storage,tol", [("c3", "f32", 2e-6), ("c3", "f16dev", 6e-6), ("c4", "f16dev", 6e-6)])
def test_fullsize_sampled_cells_against_oracle(lbm, name, storage, tol):
    import torch
    wl = _workload(name, storage)
    sim = lbm.Sim(wl)
    sim.step(60)
    ex = sim.export_state()
    flags_d = ex["flags"]
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
    # sphere samples: spheres with no other sphere centre within 2R + 3 and only liquid and
    # their own obstacle cells in a box of half-width R + 3 around them
    xs, us, ws = sim.spheres()
    Fs, Ts = sim.forces()
    owner_d = ex["owner"]
    R = wl.spheres[0].r
    ext = int(R) + 3
    from scipy.spatial import cKDTree
    L = np.array([wl.nx, wl.ny, wl.nz], float)
    tree = cKDTree(xs)
    near = tree.query_ball_point(xs, 2 * R + 3)
    sph_crops = []
    for a in rng.permutation(len(xs)):
        if len(sph_crops) >= 6:
            break
        if len(near[a]) > 1:
            continue
        c = np.rint(xs[a]).astype(int)
        if np.any(c - ext < 0) or np.any(c + ext > L.astype(int) - 1):
            continue
        idx, cen = _crop(wl, None, tuple(int(v) for v in c), ext)
        t_idx = tuple(torch.as_tensor(v, device=f_pre.device) for v in idx)
        fl = _gather(flags_d, t_idx).cpu().numpy()
        ow = _gather(owner_d, t_idx).cpu().numpy()
        ok_types = np.isin(fl, (oracle.LIQ, oracle.OBS)).all()
        if not ok_types or np.any((fl == oracle.OBS) & (ow != a)):
            continue
        f = _gather(f_pre, t_idx, lead=1).double().cpu().numpy()
        origin = np.array([idx[2][0], idx[1][0], idx[0][0]], float)
        sph_crops.append((a, f, fl, np.where(fl == oracle.OBS, 0, -1).astype(np.int32), xs[a] - origin, idx))
    del ex, f_pre, flags_d, owner_d, allliq
    torch.cuda.empty_cache()
    sim.step(1)
    ex1 = sim.export_state()
    f_post = ex1["f"]
    F1, T1 = sim.forces()
    worst = 0.0
    for (x, y, z), cen, f, fl in crops:
        o = _oracle_crop_step(wl, f, fl, np.full(fl.shape, -1, np.int32), [])
        gpu = f_post[:, z, y, x].double().cpu().numpy()
        ref = o.f[:, cen[2], cen[1], cen[0]] - U.WEIGHTS
        worst = max(worst, np.abs(gpu - ref).max())
    print("%s %s: %d bulk samples, max |df| = %.3g" % (name, storage, len(crops), worst))
    assert worst <= tol, worst
    assert len(sph_crops) >= 2, "no isolated sphere to sample"
    for a, f, fl, ow, xc, idx in sph_crops:
        sp = (xc, us[a], ws[a], R, wl.spheres[0].rho, Fs[a], Ts[a])
        o = _oracle_crop_step(wl, f, fl, ow, [sp])
        t_idx = tuple(torch.as_tensor(v, device=f_post.device) for v in idx)
        gpu = _gather(f_post, t_idx, lead=1).double().cpu().numpy()
        # liquid cells that are liquid after the oracle's step too, inside the crop's rim
        inner = np.zeros(fl.shape, bool)
        inner[1:-1, 1:-1, 1:-1] = True
        cmp = inner & (fl == oracle.LIQ) & (o.flag == oracle.LIQ)
        df = np.abs(gpu - (o.f - U.WEIGHTS[:, None, None, None]))[:, cmp].max()
        Fo, To = o.forces
        print("%s %s sphere %d: max |df| = %.3g, |dF| = %.3g of |F| = %.3g" % (
            name, storage, a, df, np.abs(F1[a] - Fo[0]).max(), np.abs(Fo[0]).max()))
        assert df <= tol, (a, df)
        # both sides sum the same stored values: FP32 per cell, FP64 over cells
        assert np.abs(F1[a] - Fo[0]).max() <= 1e-5 * max(1e-3, np.abs(Fo[0]).max())
        assert np.abs(T1[a] - To[0]).max() <= 1e-5 * max(1e-2, np.abs(To[0]).max())
    assert sim.status() == 0
    sim.close()
