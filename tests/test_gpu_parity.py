"""Parity of the CUDA library (through the C ABI) with the FP64 oracle.

Tolerances: after 200 steps of the 32^3 bubble/sphere column, max |d rho| <= 1e-5,
max |d u| <= 1e-6, |d phi| <= 1e-5, cell types identical except at cells the oracle logged
within 1e-4 of a conversion threshold and their D3Q19 neighbours (the cells such a conversion
converts with it; rho/u/phi then compared away from every mismatch), total
mass drift <= 1e-6 relative per 1000 FP32 steps.  One-step parity from a state copied out of
the GPU isolates each step with tight bounds.  FP16 / BF16 deviation storage is reported
against the same oracle with looser, stated bounds.
"""
import ctypes
import math

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
    return L


def _liquid(n=24, g=(1e-5, -2e-5, 3e-5), bc=(0, 0, 0), tau=0.6, spheres=(), mode=W.SPHERES_FIXED, storage="f32"):
    wl = W.liquid_box(n, bc=bc, g=g, tau=tau)
    wl.spheres = list(spheres)
    wl.sphere_mode = mode
    wl.storage = storage
    return wl


def test_liquid_box_walls_gravity(lbm):
    """stream + TRT + Guo + halfway walls: 100 steps of a walled box under an oblique body force"""
    wl = _liquid()
    sim = lbm.Sim(wl)
    sim.step(100)
    o = oracle.Sim(wl)
    o.step(100)
    drho, du, n = U.compare_fields(o, U.gpu_state(sim))
    assert n == wl.cells
    assert drho <= 1e-6 and du <= 1e-7, (drho, du)


def test_poiseuille_gpu(lbm):
    """body-force channel: the GPU reproduces the analytic parabola (Sec. 2.1 magic TRT)"""
    H, g, tau = 16, 1e-6, 1.0
    wl = W.Workload(name="channel", nx=4, ny=4, nz=H, tau=tau, g=(g, 0, 0), bc=(1, 1, 0))
    sim = lbm.Sim(wl)
    nu = (tau - 0.5) / 3
    sim.step(int(3.5 * H * H / nu))
    u = sim.fields()["u"].cpu().numpy()
    z = np.arange(H)
    ua = g / (2 * nu) * (z + 0.5) * (H - 0.5 - z)
    assert np.abs(u[0, :, 1, 1] - ua).max() < 2e-5 * ua.max()


@pytest.mark.parametrize("nsph", [1, 2])
def test_sphere_links_forces(lbm, nsph):
    """moving-wall bounce-back and momentum exchange (Eqs. bbrule, netforce, torque) with a
    translating + rotating sphere, or two touching ones (links between obstacle nodes).
    Bound 1e-5 relative, from the FP32 error budget of a link sum: the FP32 state differs from
    the FP64 oracle's by eps_f ~ 5e-10 per PDF after 10-30 steps (the field check below:
    |d rho| ~ 1e-8 over 19 PDFs); F and T sum N_l = 1098 links (r = 4), each with 2 eps_f,
    so |dF| lies between sqrt(N_l) 2 eps_f ~ 3e-8 (incoherent) and N_l 2 eps_f ~ 1e-6 (coherent),
    i.e. 3e-7 .. 1e-4 of the |F| ~ 0.01 - 0.1 here; measured up to 1.3e-6 relative"""
    if nsph == 1:
        sph = [W.Sphere((10.3, 11.6, 12.2), 4.0, 1.5, (0.01, -0.004, 0.002), (0.001, 0.002, -0.003))]
    else:
        sph = [W.Sphere((10.0, 12.0, 12.0), 4.0, 1.5, (0.004, 0, 0), (0, 0, 0.001)),
               W.Sphere((19.0, 12.0, 12.0), 4.0, 1.5, (-0.003, 0.001, 0), (0.001, 0, 0))]
    wl = _liquid(n=26, spheres=sph)
    sim = lbm.Sim(wl)
    o = oracle.Sim(wl)
    for k in range(3):
        sim.step(10)
        o.step(10)
        F, T = sim.forces()
        Fo, To = o.forces
        assert np.abs(F - Fo).max() <= 1e-5 * np.abs(Fo).max() + 1e-9, (F, Fo)
        assert np.abs(T - To).max() <= 1e-5 * np.abs(To).max() + 1e-8, (T, To)
    drho, du, _ = U.compare_fields(o, U.gpu_state(sim))
    assert drho <= 1e-6 and du <= 1e-7, (drho, du)


def _one_step_check(lbm, wl, pre_steps, f_tol, phi_tol):
    sim = lbm.Sim(wl)
    sim.step(pre_steps)
    st0 = U.gpu_state(sim)
    o = U.oracle_from_state(wl, st0, near_tol=1e-5)
    sim.step(1)
    o.step(1)
    st1 = U.gpu_state(sim)
    flags_o = o.flag
    mism = st1["flags"] != flags_o
    near = U.dilate(o.near > 0, 1)
    assert not np.any(mism & ~near), "type mismatch away from a threshold at %s" % (np.argwhere(mism & ~near)[:5],)
    keep = ~U.dilate(mism, 2)
    act = ((st1["flags"] & 3) != 0) & ((flags_o & 3) != 0) & keep
    df = np.abs(st1["f"].astype(np.float64) + U.WEIGHTS[:, None, None, None] - o.f)[:, act].max() if act.any() else 0.0
    iface = (st1["flags"] == oracle.IFACE) & (flags_o == oracle.IFACE) & keep
    dphi = np.abs(st1["phi"] - o.phi)[iface].max() if iface.any() else 0.0
    dm = np.abs(st1["mass"] - o.m)[iface].max() if iface.any() else 0.0
    assert df <= f_tol, df
    assert dphi <= phi_tol and dm <= phi_tol, (dphi, dm)
    if wl.spheres:
        Fo, To = o.forces
        # the links' deviation parts are summed from FP32 per cell (~1e-8 per component over a
        # sphere's few hundred links), the torque with arms of a few cells
        assert np.abs(st1["F"] - Fo).max() <= 1e-6 * max(1e-3, np.abs(Fo).max())
        assert np.abs(st1["T"] - To).max() <= 1e-6 * max(1e-1, np.abs(To).max())
        assert np.abs(st1["sx"] - o.positions).max() <= 1e-9
    if wl.bubbles:
        assert np.abs(st1["rho_g"] - o.rho_gas).max() <= 1e-6
    return int(mism.sum()), int(act.sum())


@pytest.mark.parametrize("pre", [0, 1, 40, 150])
def test_one_step_from_gpu_state_c0(lbm, pre):
    """every part of one step, isolated: the oracle steps the GPU's own state once"""
    _one_step_check(lbm, W.column_c0(), pre, 2e-6, 2e-6)


def test_one_step_moving_sphere_near_surface(lbm):
    """a sphere prescribed to cross the free surface: cover / uncover and refill next to
    interface cells, from the GPU's state"""
    wl = W.Workload(name="cross", nx=28, ny=26, nz=30, tau=0.7, g=(0, 0, -1e-5), bubbles=[W.Bubble((14, 13, 18), 7.0)],
                    spheres=[W.Sphere((14.2, 13.1, 8.6), 3.5, 2.0, (0.0, 0.0, 0.05))], sphere_mode=W.SPHERES_PRESCRIBED)
    for pre in (3, 20, 45):
        _one_step_check(lbm, wl, pre, 2e-6, 2e-6)


def _r27_compare(o, st):
    """mismatching types only at cells the oracle logged near a threshold or at their D3Q19
    neighbours (which a conversion there converts too); rho/u/phi compared away (distance > 2)
    from every mismatch"""
    mism = st["flags"] != o.flag
    near = U.dilate(o.near > 0, 1)
    assert not np.any(mism & ~near), np.argwhere(mism & ~near)[:5]
    keep = ~U.dilate(mism, 2)
    drho, du, n = U.compare_fields(o, st, keep)
    iface = (st["flags"] == oracle.IFACE) & (o.flag == oracle.IFACE) & keep
    dphi = np.abs(st["phi"] - o.phi)[iface].max() if iface.any() else 0.0
    return drho, du, dphi, int(mism.sum()), int((~keep).sum())


def test_c0_200_steps(lbm):
    """the 32^3 column (bubble r=6, falling sphere r=3), 200 steps, FP32 vs FP64, run side by
    side: cell types are compared after every step; a type that differs at some step must be
    at (or next to) a cell the oracle logged within 1e-4 of a threshold; rho, u and phi are
    compared at the end away (distance > 2) from every cell that ever differed"""
    wl = W.column_c0()
    sim = lbm.Sim(wl)
    o = oracle.Sim(wl)
    ever = np.zeros(o.shape, bool)
    for k in range(wl.steps):
        sim.step(1)
        o.step(1)
        fl = sim.fields()["flags"].cpu().numpy()
        mism = fl != o.flag
        assert not np.any(mism & ~U.dilate(o.near > 0, 1)), (k, np.argwhere(mism & ~U.dilate(o.near > 0, 1))[:5])
        ever |= mism
    st = U.gpu_state(sim)
    keep = ~U.dilate(ever, 2)
    drho, du, n = U.compare_fields(o, st, keep)
    iface = (st["flags"] == oracle.IFACE) & (o.flag == oracle.IFACE) & keep
    dphi = np.abs(st["phi"] - o.phi)[iface].max() if iface.any() else 0.0
    print("C0 200 steps: max|drho|=%.3g max|du|=%.3g max|dphi|=%.3g cells that ever differed=%d excluded=%d"
          % (drho, du, dphi, int(ever.sum()), int((~keep).sum())))
    assert drho <= 1e-5 and du <= 1e-6 and dphi <= 1e-5
    Fo, To = o.forces
    assert np.abs(st["F"] - Fo).max() <= 1e-3 * np.abs(Fo).max() + 1e-7
    assert np.abs(st["sx"] - o.positions).max() <= 1e-6


@pytest.mark.parametrize("wl_name", ["c0", "cross"])
def test_overlapped_steps_equal_serial_steps(lbm, wl_name):
    """lbm_step overlaps each step's bulk sweep with the previous step's end-of-step kernels
    and sweeps the cells those kernels touched again afterwards; a query in between runs the
    pending kernels first, so querying after every step gives the plain serial order.  Both
    orders must give the same state (the force sums' atomic order aside)."""
    if wl_name == "c0":
        wl, n = W.column_c0(), 200
    else:
        wl = W.Workload(name="cross", nx=28, ny=26, nz=30, tau=0.7, g=(0, 0, -1e-5),
                        bubbles=[W.Bubble((14, 13, 18), 7.0)],
                        spheres=[W.Sphere((14.2, 13.1, 8.6), 3.5, 2.0, (0.0, 0.0, 0.05))],
                        sphere_mode=W.SPHERES_PRESCRIBED)
        n = 120
    a = lbm.Sim(wl)
    a.step(n)
    b = lbm.Sim(wl)
    for _ in range(n):
        b.step(1)
        assert b.status() == 0
    sa, sb = U.gpu_state(a), U.gpu_state(b)
    assert np.array_equal(sa["flags"], sb["flags"])
    act = (sa["flags"] & 3) != 0
    df = np.abs(sa["f"] - sb["f"])[:, act].max()
    dm = np.abs(sa["mass"] - sb["mass"])[act].max()
    print("%s: overlapped vs serial after %d steps: max|df|=%.3g max|dm|=%.3g" % (wl_name, n, df, dm))
    assert df <= 1e-6 and dm <= 1e-6
    # the sphere forces' FP32 partial sums follow the boundary-list order, which atomics set:
    # free spheres agree to round-off of their displacement, not bit for bit
    disp = np.abs(sb["sx"] - np.array([s.x for s in wl.spheres])).max()
    assert np.abs(sa["sx"] - sb["sx"]).max() <= 1e-5 * disp + 1e-9


def test_c0_mass_drift(lbm):
    """total mass drift <= 1e-6 relative per 1000 FP32 steps (budget terms in FP64)"""
    wl = W.column_c0()
    sim = lbm.Sim(wl)
    sim.step(1)
    M0, b0, c0, u0, _ = sim.mass_budget()
    sim.step(1000)
    M, b, c, u, _ = sim.mass_budget()
    drift = abs((M - M0) - (b - b0) - (u - u0) + (c - c0)) / M0
    print("C0 mass drift over 1000 steps: %.3g" % drift)
    assert drift <= 1e-6
    assert sim.status() == 0


@pytest.mark.parametrize("storage,tol", [("f16dev", (2e-3, 2e-4, 5e-3)), ("bf16dev", (2e-2, 2e-3, 5e-2))])
def test_c0_reduced_storage(lbm, storage, tol):
    """PDFs stored as FP16 / BF16 deviations from w_q, collisions in FP32: error against the
    FP64 oracle after 200 steps of the column (reported; bounded loosely)"""
    wl = W.column_c0()
    wl.storage = storage
    sim = lbm.Sim(wl)
    sim.step(wl.steps)
    o = oracle.Sim(W.column_c0())
    o.step(wl.steps)
    st = U.gpu_state(sim)
    mism = st["flags"] != o.flag
    keep = ~U.dilate(mism, 2)
    drho, du, _ = U.compare_fields(o, st, keep)
    print("%s C0 200 steps: max|drho|=%.3g max|du|=%.3g mismatches=%d" % (storage, drho, du, int(mism.sum())))
    assert drho <= tol[0] and du <= tol[1]
    assert mism.mean() <= tol[2]


def test_c1_full_size_one_step(lbm):
    """the 128^3 column of 64 spheres at full size, after steps replayed through the CUDA
    graph the benchmark times: one step against the oracle from the GPU's state"""
    _one_step_check(lbm, W.column_c1(), 40, 2e-6, 2e-6)


def test_status_unstable(lbm):
    """a body force far beyond the scheme's stability makes densities non-positive: the
    status word reports it and lbm_forces returns LBM_EUNSTABLE (no GPU fault involved)"""
    wl = _liquid(n=12, g=(0.0, 0.0, -0.5), tau=0.51, spheres=[W.Sphere((6.0, 6.0, 6.0), 2.0, 1.5)])
    sim = lbm.Sim(wl)
    sim.step(300)
    assert sim.status() & lbm.S_UNSTABLE
    with pytest.raises(lbm.LBMError) as e:
        sim.forces()
    assert e.value.code == lbm.LBM_EUNSTABLE


def test_abi_argument_errors(lbm):
    L = lbm.load()
    p = lbm.make_params(_liquid(n=8))
    p.nx = 2
    nbytes = ctypes.c_size_t()
    assert L.lbm_arena_bytes(ctypes.byref(p), ctypes.byref(nbytes)) == lbm.LBM_EINVAL
    sim = lbm.Sim(_liquid(n=8))
    sim.step(1)
    c = np.zeros(3)
    assert L.lbm_add_bubble(sim.ctx, c.ctypes.data_as(ctypes.POINTER(ctypes.c_double)), 2.0, None) == lbm.LBM_ESTATE
    assert L.lbm_step(sim.ctx, -1) == lbm.LBM_EINVAL


def _ctx_one_by_one(lbm, wl):
    """a context built through the ABI with one lbm_add_sphere call per sphere (Sim uses the batch
    call); returns (ctx, arena) on the current stream"""
    import torch
    L = lbm.load()
    p = lbm.make_params(wl)
    nbytes = ctypes.c_size_t()
    assert L.lbm_arena_bytes(ctypes.byref(p), ctypes.byref(nbytes)) == 0
    arena = torch.empty(nbytes.value, dtype=torch.uint8, device="cuda")
    ctx = ctypes.c_void_p()
    stream = torch.cuda.current_stream().cuda_stream
    assert L.lbm_init(ctypes.byref(p), ctypes.c_void_p(arena.data_ptr()), nbytes.value, ctypes.c_void_p(stream), ctypes.byref(ctx)) == 0
    dp = lambda v: np.ascontiguousarray(v, dtype=np.float64).ctypes.data_as(ctypes.POINTER(ctypes.c_double))
    for b in wl.bubbles:
        c = np.array(b.c, dtype=np.float64)
        assert L.lbm_add_bubble(ctx, c.ctypes.data_as(ctypes.POINTER(ctypes.c_double)), float(b.r), None) == 0
    for k, s in enumerate(wl.spheres):
        x, u, w = (np.array(v, dtype=np.float64) for v in (s.x, s.u, s.w))
        i = ctypes.c_int(-1)
        assert L.lbm_add_sphere(ctx, x.ctypes.data_as(ctypes.POINTER(ctypes.c_double)), float(s.r), float(s.rho),
                                u.ctypes.data_as(ctypes.POINTER(ctypes.c_double)),
                                w.ctypes.data_as(ctypes.POINTER(ctypes.c_double)), ctypes.byref(i)) == 0
        assert i.value == k
    return ctx, arena


def test_add_spheres_batch_matches_one_by_one(lbm):
    """lbm_add_spheres (the binding's path) adds the table lbm_add_sphere adds sphere by sphere:
    the two contexts step alike (to round-off: the sphere sums are FP64 atomics, whose order
    varies from run to run); a batch with one bad sphere adds none of them, and a batch after the
    first step is refused"""
    import torch
    L = lbm.load()
    wl = _sphere_bed(60)
    a = lbm.Sim(wl)
    ctx, arena = _ctx_one_by_one(lbm, wl)
    a.step(5)
    assert L.lbm_step(ctx, 5) == 0
    n = len(wl.spheres)
    xa, xb = np.zeros((n, 3)), np.zeros((n, 3))
    pd = ctypes.POINTER(ctypes.c_double)
    for ctx_, x in ((a.ctx, xa), (ctx, xb)):
        assert L.lbm_spheres(ctx_, x.ctypes.data_as(pd), None, None, n) == 0
    torch.cuda.synchronize()
    assert np.abs(xa - xb).max() <= 1e-12
    fa = torch.empty((19,) + a.shape, dtype=torch.float32, device="cuda")
    fb = torch.empty_like(fa)
    assert L.lbm_export_state(a.ctx, ctypes.c_void_p(fa.data_ptr()), None, None, None, None, None) == 0
    assert L.lbm_export_state(ctx, ctypes.c_void_p(fb.data_ptr()), None, None, None, None, None) == 0
    torch.cuda.synchronize()
    assert (fa - fb).abs().max().item() <= 1e-6
    # a refused batch adds nothing; after the first step every batch is refused
    wl2 = _sphere_bed(0)
    p = lbm.make_params(wl2, max_spheres=8)
    nbytes = ctypes.c_size_t()
    assert L.lbm_arena_bytes(ctypes.byref(p), ctypes.byref(nbytes)) == 0
    arena2 = torch.empty(nbytes.value, dtype=torch.uint8, device="cuda")
    ctx2 = ctypes.c_void_p()
    assert L.lbm_init(ctypes.byref(p), ctypes.c_void_p(arena2.data_ptr()), nbytes.value,
                      ctypes.c_void_p(torch.cuda.current_stream().cuda_stream), ctypes.byref(ctx2)) == 0
    c = np.array([[20.0, 20.0, 20.0], [40.0, 40.0, 40.0]])
    r, rho = np.array([4.0, -1.0]), np.array([1.5, 1.5])
    vp = lambda v: ctypes.c_void_p(v.ctypes.data)
    first = ctypes.c_int(-1)
    assert L.lbm_add_spheres(ctx2, 2, vp(c), vp(r), vp(rho), None, None, ctypes.byref(first)) == lbm.LBM_EINVAL
    r[1] = 4.0
    assert L.lbm_add_spheres(ctx2, 9, vp(np.zeros((9, 3))), vp(np.full(9, 4.0)), vp(np.full(9, 1.5)), None, None, None) == lbm.LBM_EINVAL
    assert L.lbm_add_spheres(ctx2, 2, vp(c), vp(r), vp(rho), None, None, ctypes.byref(first)) == 0
    assert first.value == 0
    assert L.lbm_step(ctx2, 1) == 0
    assert L.lbm_add_spheres(ctx2, 1, vp(c), vp(r), vp(rho), None, None, None) == lbm.LBM_ESTATE
    for x in (ctx, ctx2):
        L.lbm_destroy(x)
    torch.cuda.synchronize()


def test_launch_count(lbm):
    wl = W.column_c0()
    sim = lbm.Sim(wl)
    sim.step(1)
    n1 = sim.launches()
    sim.step(10)
    assert (sim.launches() - n1) % 10 == 0 and sim.launches() > n1


def _two_bubbles(c2=None, g=0.0):
    if c2 is not None:   # side by side at rest
        return W.Workload(name="two", nx=24, ny=16, nz=16, tau=0.7, g=(0, 0, 0), sphere_mode=W.SPHERES_FIXED,
                          bubbles=[W.Bubble((7.0, 8.0, 8.0), 4.0), W.Bubble((c2, 8.0, 8.0), 4.0)])
    # a large bubble rising into a small one
    return W.Workload(name="two_rising", nx=16, ny=16, nz=40, tau=0.7, g=(0, 0, -g), sphere_mode=W.SPHERES_FIXED,
                      bubbles=[W.Bubble((8.0, 8.0, 10.0), 5.0), W.Bubble((8.0, 8.0, 22.0), 3.0)])


def _gas_volume(st, ids):
    """V of a set of bubble ids from exported cell fields: gas cells + sum over interface cells
    of (1 - phi), in FP64"""
    sel = np.isin(st["owner"], list(ids))
    return float(((st["flags"] == oracle.GAS) & sel).sum() + (1.0 - st["phi"][(st["flags"] == oracle.IFACE) & sel].astype(np.float64)).sum())


@pytest.mark.parametrize("c2,touching", [(15.0, True), (17.0, False)])
def test_touching_bubbles_merge_like_the_oracle(lbm, c2, touching):
    """bubbles whose gas / interface cells touch from the start are one bubble (Sec. 2.2):
    the same roots, merge count, V0, V and rho_g as the oracle's"""
    wl = _two_bubbles(c2)
    sim = lbm.Sim(wl)
    sim.step(5)
    o = oracle.Sim(wl)
    o.step(5)
    roots, nm = sim.bubble_roots()
    assert list(roots) == list(o.roots) == ([0, 0] if touching else [0, 1])
    assert nm == o.scal[oracle.SC_NMERGE] == (1 if touching else 0)
    V0, V, rg = sim.bubbles()
    # FP32 fill levels summed in FP64 on both sides of the comparison
    assert np.abs(V0 - o.bub[:2, oracle.B_V0]).max() <= 1e-5 * V0.max()
    assert np.abs(V - o.volumes).max() <= 1e-5 * V.max()
    assert np.abs(rg - o.rho_gas).max() <= 1e-6
    assert sim.status() == 0
    st = U.gpu_state(sim)
    for r in set(roots):
        ids = [b for b in range(2) if roots[b] == r]
        assert abs(V[r] - _gas_volume(st, ids)) <= 1e-9 * V[r]


def _bubble_lattice(n, sp, r, chains):
    """n^3 bubbles of radius r on a periodic lattice of spacing sp; with chains the lattice is
    stretched to 2 sp across x, so that only x-neighbours touch (one chain of n bubbles per
    (y, z))"""
    spy = 2 * sp if chains else sp
    L = (n * sp, n * spy, n * spy)
    bubs = [W.Bubble((sp * i + sp / 2 - 0.5, spy * j + spy / 2 - 0.5, spy * k + spy / 2 - 0.5), r)
            for k in range(n) for j in range(n) for i in range(n)]
    return W.Workload(name="lattice", nx=L[0], ny=L[1], nz=L[2], tau=0.7, g=(0, 0, 0), bc=(W.PERIODIC,) * 3,
                      sphere_mode=W.SPHERES_FIXED, bubbles=bubs)


def test_bubble_chains_merge_at_initialisation(lbm):
    """64 chains of 8 touching bubbles each (512 bubbles, 512 touching pairs): every chain is
    one bubble rooted at its smallest id, as the oracle's; its V0 is the chain's gas volume"""
    wl = _bubble_lattice(8, 3, 1.6, chains=True)
    sim = lbm.Sim(wl)
    sim.step(0)
    roots, nm = sim.bubble_roots()
    n = 8
    expect = np.array([(b // n) * n for b in range(n ** 3)])   # ids run along x fastest
    assert (roots == expect).all()
    assert nm == n ** 3 - n ** 2
    o = oracle.Sim(wl)
    assert (o.roots == expect).all() and o.scal[oracle.SC_NMERGE] == nm
    V0, V, rg = sim.bubbles()
    st = U.gpu_state(sim)
    for c in range(0, n ** 3, n * 7):   # a sample of the chains
        v = _gas_volume(st, range(c, c + n))
        assert abs(V0[c] - v) <= 1e-9 * v and (V0[c:c + n] == V0[c]).all() and (V[c:c + n] == V0[c]).all()
    assert np.abs(V0 - o.bub[: n ** 3, oracle.B_V0]).max() <= 1e-5 * V0.max()
    assert (rg == 1.0).all() and sim.status() == 0


def test_merge_table_overflow_is_reported(lbm):
    """a packed lattice where every bubble touches its 18 D3Q19 neighbours: 1944 distinct pairs
    meet at once, more than the merge table holds: the state is flagged (LBM_S_MERGE) and the
    calls that read it return LBM_EMERGE"""
    wl = _bubble_lattice(6, 3, 1.5, chains=False)
    sim = lbm.Sim(wl)
    sim.step(0)
    assert sim.status() & lbm.S_MERGE
    with pytest.raises(lbm.LBMError) as e:
        sim.forces()
    assert e.value.code == lbm.LBM_EMERGE


def test_bubbles_merging_during_the_run_like_the_oracle(lbm):
    """a large bubble rising into a small one: the step at which they merge agrees with the
    oracle's to a few steps (FP32 vs FP64 conversions near the threshold); after it they are one
    bubble whose gas mass is the sum of the two initial masses (rho_g V = rho_g0 (V0_a + V0_b),
    V from the exported cells), with the oracle's gas density"""
    wl = _two_bubbles(g=3e-4)
    sim = lbm.Sim(wl)
    o = oracle.Sim(wl)
    sim.step(0)
    m0 = sim.bubbles()[0].copy()   # rho_g0 = 1
    first_gpu = first_orc = None
    for k in range(1, 801):
        sim.step(1)
        o.step(1)
        if first_gpu is None and sim.bubble_roots()[1] > 0:
            first_gpu = k
        if first_orc is None and o.scal[oracle.SC_NMERGE] > 0:
            first_orc = k
        if first_gpu is not None and first_orc is not None:
            break
    print("bubbles merge: GPU step %s, oracle step %s" % (first_gpu, first_orc))
    assert first_orc is not None and first_gpu is not None
    assert abs(first_gpu - first_orc) <= 5
    sim.step(20)
    o.step(20)
    roots, nm = sim.bubble_roots()
    assert list(roots) == [0, 0] and nm == 1
    V0, V, rg = sim.bubbles()
    assert V0[0] == V0[1] and abs(V0[0] - m0.sum()) <= 1e-12 * m0.sum()
    st = U.gpu_state(sim)
    Vf = _gas_volume(st, [0, 1])
    assert abs(rg[0] * Vf - m0.sum()) <= 1e-9 * m0.sum()
    assert rg[0] == rg[1]
    # two runs 600 steps apart from their common start (FP32 against FP64, conversions near
    # the thresholds): the merged bubble's volume, and so its gas density, agree to 1e-4
    assert abs(rg[0] - o.rho_gas[0]) <= 1e-4
    assert sim.status() == 0


def test_one_step_from_merged_state(lbm):
    """every part of one step with two merged bubbles rising: the oracle steps the GPU's own
    merged state once (roots, V0 and rho_g copied over)"""
    wl = _two_bubbles(15.0)
    wl.g = (0.0, 0.0, -2e-4)
    _one_step_check(lbm, wl, 30, 2e-6, 2e-6)


# ------------------------------------------- free-slip sides, open top (Fig. bubbleSetup)

def _rising_small(at_wall=False):
    """case B parameters of Table 1 in a 16 x 16 x 32 column, bubble r = 4; with at_wall the
    bubble is centred 3 cells from an x face, so its interface crosses the free-slip wall"""
    wl = W.rising_bubble("B", n=(16, 16, 32), r=4.0, zc=8.5)
    if at_wall:
        wl.bubbles = [W.Bubble((2.5, 7.5, 8.5), 4.0)]
        wl.name = "rising_at_wall"
    return wl


@pytest.mark.parametrize("at_wall", [False, True])
@pytest.mark.parametrize("pre", [0, 60, 150])
def test_one_step_free_slip_open_top(lbm, at_wall, pre):
    """every part of one step with free-slip sides and an open top, from the GPU's state:
    specular links (with mass exchange, and gas or interface sources across the wall), the
    open face's pressure links and its mass flux"""
    _one_step_check(lbm, _rising_small(at_wall), pre, 2e-6, 2e-6)


@pytest.mark.parametrize("at_wall", [False, True])
def test_rising_bubble_steps_like_the_oracle(lbm, at_wall):
    """the small rising bubble, 200 steps side by side (as the 32^3 column's test): types after
    every step (differences only at or next to cells near a threshold), rho, u, phi at the end
    away from them, the gas density and the mass budget (the open face's flux included)"""
    wl = _rising_small(at_wall)
    sim = lbm.Sim(wl)
    o = oracle.Sim(wl)
    ever = np.zeros(o.shape, bool)
    for k in range(200):
        sim.step(1)
        o.step(1)
        fl = sim.fields()["flags"].cpu().numpy()
        mism = fl != o.flag
        assert not np.any(mism & ~U.dilate(o.near > 0, 1)), (k, np.argwhere(mism & ~U.dilate(o.near > 0, 1))[:5])
        ever |= mism
    st = U.gpu_state(sim)
    keep = ~U.dilate(ever, 2)
    drho, du, n = U.compare_fields(o, st, keep)
    iface = (st["flags"] == oracle.IFACE) & (o.flag == oracle.IFACE) & keep
    dphi = np.abs(st["phi"] - o.phi)[iface].max() if iface.any() else 0.0
    print("%s 200 steps: max|drho|=%.3g max|du|=%.3g max|dphi|=%.3g differed=%d"
          % (wl.name, drho, du, dphi, int(ever.sum())))
    assert drho <= 1e-5 and du <= 1e-6 and dphi <= 1e-5
    assert abs(st["rho_g"][0] - o.rho_gas[0]) <= 1e-6
    # the open face's flux per link is a difference of two FP32 deviations of nearly equal
    # size (the column is in hydrostatic equilibrium): its sum over 200 steps agrees to ~1e-3
    M, sbb, scov, sunc, pool = sim.mass_budget()
    Mo, sbbo = o.mass_budget()[:2]
    assert abs(sbb - sbbo) <= 2e-3 * abs(sbbo)
    assert sim.status() == 0


@pytest.mark.parametrize("where", ["inside", "straddling"])
def test_one_step_sphere_touching_gas(lbm, where):
    """a free sphere inside a bubble, or straddling a bubble's interface, under gravity: the gas
    pressure on its dry surface (the GPU's pass over the spheres flagged beside interface cells
    or gas) against the oracle's, from the GPU's state"""
    if where == "inside":
        bub, c = W.Bubble((12.0, 12.0, 12.0), 10.0), (12.3, 11.8, 12.4)
    else:
        bub, c = W.Bubble((12.0, 12.0, -20.0), 32.0), (12.0, 12.0, 12.0)
    wl = W.Workload(name="sphere_gas_" + where, nx=24, ny=24, nz=24, tau=0.7, g=(0, 0, -1e-5),
                    sphere_mode=W.SPHERES_FREE, bubbles=[bub], spheres=[W.Sphere(c, 4.0, 2.0)])
    for pre in (0, 15):
        _one_step_check(lbm, wl, pre, 2e-6, 2e-6)


# ------------------------------------------------------------ degenerate and ragged inputs

def test_smallest_grid(lbm):
    """the smallest grid the ABI takes (3^3, every cell at a wall), liquid under gravity:
    40 steps against the oracle"""
    wl = W.Workload(name="min3", nx=3, ny=3, nz=3, tau=0.8, g=(1e-4, -2e-4, 3e-4), sphere_mode=W.SPHERES_FIXED)
    sim = lbm.Sim(wl)
    o = oracle.Sim(wl)
    sim.step(40)
    o.step(40)
    drho, du, _ = U.compare_fields(o, U.gpu_state(sim))
    assert drho <= 1e-6 and du <= 1e-7, (drho, du)
    assert sim.status() == 0


def test_all_gas_domain(lbm):
    """a bubble larger than the box: no liquid and no interface cell at all; the steps have
    nothing to stream, convert or cover, and the bubble keeps the box's volume"""
    wl = W.Workload(name="all_gas", nx=8, ny=7, nz=9, tau=0.7, g=(0, 0, -1e-4), sphere_mode=W.SPHERES_FIXED,
                    bubbles=[W.Bubble((4.0, 3.0, 4.0), 30.0)])
    sim = lbm.Sim(wl)
    sim.step(10)
    fl = sim.fields()["flags"].cpu().numpy()
    o = oracle.Sim(wl)
    o.step(10)
    assert (fl == oracle.GAS).all() and (o.flag == oracle.GAS).all()
    V0, V, rg = sim.bubbles()
    assert V[0] == wl.cells and abs(o.volumes[0] - wl.cells) < 1e-12
    assert sim.status() == 0


@pytest.mark.parametrize("pre", [0, 25])
def test_ragged_grid_one_step(lbm, pre):
    """a grid of odd sizes (37 x 29 x 23: partial thread blocks in x, a boundary list that
    ends inside a block) with a bubble and a free sphere, one step from the GPU's state"""
    wl = W.Workload(name="ragged", nx=37, ny=29, nz=23, tau=0.65, g=(0, 0, -1e-5),
                    bubbles=[W.Bubble((18.0, 14.0, 9.0), 5.0)],
                    spheres=[W.Sphere((9.0, 8.0, 16.0), 3.0, 1.8)])
    _one_step_check(lbm, wl, pre, 2e-6, 2e-6)


def _sphere_bed(nsph):
    """64x64x96 column, a bubble r=8 and nsph free spheres r=4 (seed 5)"""
    dims = (64, 64, 96)
    bubbles = [W.Bubble((32.0, 32.0, 20.0), 8.0)]
    spheres = W.place_spheres(W.SplitMix64(5), nsph, 4, 1.5, dims, bubbles)
    return W.Workload(name="bed%d" % nsph, nx=64, ny=64, nz=96, tau=0.6, g=(0.0, 0.0, -2e-5), bubbles=bubbles,
                      spheres=spheres)


def test_lean_boundary_kernel_runs_and_steps_like_the_oracle(lbm):
    """enough spheres that the liquid cells beside them (about 4 pi (R+1)^2 each) outnumber one
    round of the general boundary kernel: they get their own kernels -- the classification of
    their links after the list pass, the lean sweep of the cells with links into one sphere, the
    full sweep of the others -- three more launches per step than with fewer spheres; and a step
    from the GPU's state matches the oracle's"""
    def per_step(wl):
        sim = lbm.Sim(wl)
        sim.step(1)
        n1 = sim.launches()
        sim.step(10)
        return (sim.launches() - n1) // 10

    assert per_step(_sphere_bed(150)) == per_step(_sphere_bed(100)) + 3
    for pre in (0, 30):
        _one_step_check(lbm, _sphere_bed(150), pre, 2e-6, 2e-6)
