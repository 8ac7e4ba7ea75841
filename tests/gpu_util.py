"""Helpers of the GPU parity tests: moving a state between the CUDA library and the oracle,
and comparing them under the tolerances of the method (test infrastructure)."""
import numpy as np

import oracle
from paper_1712_07028_gb300 import workloads as W


# lattice weights of the D3Q19 order shared by the C ABI and the oracle (q = 0 rest, 1..6
# faces, 7..18 edges): the export hands out f - w_q
WEIGHTS = np.array([1 / 3] + [1 / 18] * 6 + [1 / 36] * 12)


def gpu_state(sim):
    """the CUDA library's full state as NumPy (FP64 where the oracle wants it)"""
    st = {k: v.cpu().numpy() for k, v in sim.export_state().items()}
    fl = sim.fields()
    st["rho"] = fl["rho"].cpu().numpy().astype(np.float64)
    st["u"] = fl["u"].cpu().numpy().astype(np.float64)
    x, u, w = sim.spheres()
    V0, V, rg = sim.bubbles()
    roots, n_merges = sim.bubble_roots()
    n_ids, n_splits = sim.bubble_splits()
    M, sbb, scov, sunc, pool = sim.mass_budget()
    F, T = sim.forces()
    st.update(sx=x, su=u, sw=w, V0=V0, V=V, rho_g=rg, roots=roots, n_merges=n_merges, n_ids=n_ids, n_splits=n_splits, pool=pool, F=F, T=T, steps=sim.steps_done)
    return st


def oracle_from_state(wl: W.Workload, st, near_tol=1e-5):
    """an oracle simulation started from a state copied out of the CUDA library"""
    o = oracle.Sim(wl, init=False, near_tol=near_tol)
    o.f[:] = st["f"].astype(np.float64) + WEIGHTS[:, None, None, None]
    o.flag[:] = st["flags"]
    o.m[:] = st["mass"].astype(np.float64)
    o.phi[:] = st["phi"].astype(np.float64)
    o.owner[:] = st["owner"]
    o.kappa[:] = st["kappa"].astype(np.float64)
    for b in range(len(st["V0"])):   # (with splitting: every row of the table)
        o.bub[b, oracle.B_V0] = st["V0"][b]
        o.bub[b, oracle.B_V] = st["V"][b]
        o.bub[b, oracle.B_RHOG] = st["rho_g"][b]
        o.bub[b, oracle.B_ROOT] = st["roots"][b]
        o.bub[b, oracle.B_MG] = st["rho_g"][b] * st["V"][b]   # the conserved gas mass
    o.scal[oracle.SC_NBUB] = st["n_ids"]
    for a in range(len(wl.spheres)):
        o.sph[a, oracle.S_X:oracle.S_X + 3] = st["sx"][a]
        o.sph[a, oracle.S_U:oracle.S_U + 3] = st["su"][a]
        o.sph[a, oracle.S_W:oracle.S_W + 3] = st["sw"][a]
        # this step's force becomes the oracle's previous-step force for the two-step average
        o.sph[a, oracle.S_F:oracle.S_F + 3] = st["F"][a]
        o.sph[a, oracle.S_T:oracle.S_T + 3] = st["T"][a]
        o.sph[a, oracle.S_HASP] = 1.0 if st["steps"] > 0 else 0.0
    o.scal[oracle.SC_POOL] = st["pool"]
    return o


def dilate(mask, r, periodic=(False, False, False)):
    """cells within D3Q19 distance r (r steps along D3Q19 links) of mask"""
    c = oracle.velocities()
    out = mask.copy()
    for _ in range(r):
        nxt = out.copy()
        for q in range(1, 19):
            sh = np.roll(out, shift=(c[q, 2], c[q, 1], c[q, 0]), axis=(0, 1, 2))
            # rolled-in wrap across a wall axis is not a neighbour; trimming it only widens
            nxt |= sh
        out = nxt
    return out


def compare_fields(orc_sim, st, active_mask=None):
    """max |d rho|, max |d u| over cells active in both (GPU moments from lbm_fields, computed
    on the device from the stored deviations), and the number of cells compared"""
    rho_o, u_o = orc_sim.fields()
    act = ((st["flags"] & (oracle.LIQ | oracle.IFACE)) != 0) & ((orc_sim.flag & (oracle.LIQ | oracle.IFACE)) != 0)
    if active_mask is not None:
        act &= active_mask
    if not act.any():
        return 0.0, 0.0, 0
    drho = np.abs(st["rho"] - rho_o)[act].max()
    du = np.abs(st["u"] - u_o)[:, act].max()
    return drho, du, int(act.sum())
