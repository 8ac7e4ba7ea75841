"""FP64 CPU oracle of the free-surface LBM with moving spheres -- TEST INFRASTRUCTURE.

Only ``tests/``, ``__graft_entry__.smoke()`` and the CPU-baseline leg of ``bench.py`` may
import this package.  It loads ``fslbm_oracle.c`` compiled with gcc (``build()``) through
ctypes; the state lives in NumPy arrays owned here, so any state (including one copied
out of the CUDA library) can be stepped by the oracle.
"""
from __future__ import annotations

import ctypes
import os
import subprocess

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "fslbm_oracle.c")
_LIBPATH = os.path.join(_HERE, "_build", "liboracle_fslbm.so")
_lib = None

# the oracle's cell-type codes and record layouts (fslbm_oracle.c)
LIQ, IFACE, GAS, OBS = 1, 2, 4, 8
S_X, S_U, S_W, S_R, S_RHO, S_F, S_T, S_FLUB, S_FP, S_TP, S_HASP, S_LEN = 0, 3, 6, 9, 10, 11, 14, 17, 20, 23, 26, 32
B_C, B_R, B_V0, B_V, B_RHOG, B_ROOT, B_MG, B_LEN = 0, 3, 4, 5, 6, 7, 8, 10
FACE_WALL, FACE_SLIP, FACE_OPEN = 0, 1, 2
SC_POOL, SC_NIF, SC_SBB, SC_SCOV, SC_SUNC, SC_STEPS, SC_STATUS, SC_NMERGE, SC_NBUB, SC_NSPLIT, SC_LEN = (
    0, 1, 2, 3, 4, 5, 6, 7, 8, 9, 16)
ST_UNSTABLE, ST_BUBBLE_GONE, ST_SPLIT_FULL = 1, 2, 4


def build(force: bool = False) -> str:
    """compile the oracle with gcc (plain C11, no FMA contraction so x86 and Arm agree)"""
    os.makedirs(os.path.dirname(_LIBPATH), exist_ok=True)
    if force or not os.path.exists(_LIBPATH) or os.path.getmtime(_LIBPATH) < os.path.getmtime(_SRC):
        tmp = _LIBPATH + ".tmp%d" % os.getpid()
        subprocess.check_call(["gcc", "-O2", "-std=c11", "-ffp-contract=off", "-fPIC", "-shared",
                               "-o", tmp, _SRC, "-lm"])
        os.replace(tmp, _LIBPATH)
    return _LIBPATH


class _Params(ctypes.Structure):
    _fields_ = [("nx", ctypes.c_int32), ("ny", ctypes.c_int32), ("nz", ctypes.c_int32),
                ("bc", ctypes.c_int32 * 3), ("n_substeps", ctypes.c_int32), ("sphere_mode", ctypes.c_int32),
                ("nbub", ctypes.c_int32), ("nsph", ctypes.c_int32),
                ("tau", ctypes.c_double), ("g", ctypes.c_double * 3), ("sigma", ctypes.c_double),
                ("rho_g0", ctypes.c_double), ("eps", ctypes.c_double), ("near_tol", ctypes.c_double),
                ("face", ctypes.c_int32 * 6), ("hydrostatic", ctypes.c_int32),
                ("max_bub", ctypes.c_int32), ("split_every", ctypes.c_int32)]


_P = ctypes.POINTER
class _State(ctypes.Structure):
    _fields_ = [("f", _P(ctypes.c_double)), ("ft", _P(ctypes.c_double)),
                ("flag", _P(ctypes.c_uint8)), ("mark", _P(ctypes.c_uint8)),
                ("m", _P(ctypes.c_double)), ("phi", _P(ctypes.c_double)), ("phit", _P(ctypes.c_double)),
                ("kappa", _P(ctypes.c_double)), ("owner", _P(ctypes.c_int32)), ("nown", _P(ctypes.c_int32)),
                ("near", _P(ctypes.c_int32)), ("bub", _P(ctypes.c_double)), ("sph", _P(ctypes.c_double)),
                ("scal", _P(ctypes.c_double))]


def lib():
    global _lib
    if _lib is None:
        _lib = ctypes.CDLL(build())
        pp, ps = ctypes.POINTER(_Params), ctypes.POINTER(_State)
        _lib.orc_init.argtypes = [pp, ps]
        _lib.orc_step.argtypes = [pp, ps, ctypes.c_int]
        _lib.orc_fields.argtypes = [pp, ps, _P(ctypes.c_double), _P(ctypes.c_double)]
        _lib.orc_total_mass.argtypes = [pp, ps]
        _lib.orc_total_mass.restype = ctypes.c_double
        _lib.orc_equilibrium.argtypes = [ctypes.c_int, ctypes.c_double, _P(ctypes.c_double)]
        _lib.orc_equilibrium.restype = ctypes.c_double
        _lib.orc_lambda_minus.argtypes = [ctypes.c_double]
        _lib.orc_lambda_minus.restype = ctypes.c_double
        _lib.orc_lubrication.argtypes = [pp, ps, _P(ctypes.c_double)]
        _lib.orc_curvature.argtypes = [pp, ps]
        _lib.orc_bubble_model.argtypes = [pp, ps]
        _lib.orc_bubble_model_split.argtypes = [pp, ps]
        _lib.orc_velocity.argtypes = [ctypes.c_int, ctypes.c_int]
        _lib.orc_conversions.argtypes = [pp, ps]
        _lib.orc_cover_uncover.argtypes = [pp, ps]
        _lib.orc_tangent_window.argtypes = [pp, ps, _P(ctypes.c_double), _P(ctypes.c_double), ctypes.c_double,
                                            _P(ctypes.c_double), _P(ctypes.c_double), ctypes.c_int,
                                            _P(ctypes.c_double), _P(ctypes.c_double)]
    return _lib


def _ptr(a, t):
    return a.ctypes.data_as(ctypes.POINTER(t))


def velocities() -> np.ndarray:
    """the oracle's D3Q19 velocity table, [19][3]"""
    L = lib()
    return np.array([[L.orc_velocity(q, k) for k in range(3)] for q in range(19)], dtype=np.int64)


def equilibrium(q: int, rho: float, u) -> float:
    u = np.ascontiguousarray(u, dtype=np.float64)
    return lib().orc_equilibrium(q, rho, _ptr(u, ctypes.c_double))


def lambda_minus(tau: float) -> float:
    return lib().orc_lambda_minus(tau)


class Sim:
    """FP64 oracle simulation.  Arrays are NumPy, shaped [z][y][x] (PDFs [19][z][y][x])."""

    def __init__(self, wl=None, *, nx=None, ny=None, nz=None, tau=0.6, g=(0, 0, 0), bc=(0, 0, 0), sigma=0.0,
                 rho_g0=1.0, eps=0.0, near_tol=1e-4, n_substeps=10, sphere_mode=1, bubbles=(), spheres=(),
                 open_top=False, hydrostatic=False, max_bubbles=0, split_every=0, init=True):
        """bc per axis: 0 no-slip walls, 1 periodic, 2 free-slip walls; open_top: the +z face is
        open at the reference pressure; hydrostatic (open top only): start in hydrostatic
        equilibrium; max_bubbles: rows of the bubble table (room for the bubbles splitting
        makes); split_every > 0: bubbles split into their connected parts every split_every
        steps"""
        if wl is not None:
            nx, ny, nz, tau, g, bc = wl.nx, wl.ny, wl.nz, wl.tau, wl.g, wl.bc
            open_top, hydrostatic = wl.open_top, wl.hydrostatic
            max_bubbles, split_every = getattr(wl, "max_bubbles", 0), getattr(wl, "split_every", 0)
            sigma, rho_g0, eps, n_substeps, sphere_mode = wl.sigma, wl.rho_g0, wl.eps, wl.n_substeps, wl.sphere_mode
            bubbles = [(b.c[0], b.c[1], b.c[2], b.r) for b in wl.bubbles]
            spheres = [(s.x[0], s.x[1], s.x[2], s.r, s.rho, *s.u, *s.w) for s in wl.spheres]
        self.shape = (nz, ny, nx)
        self.N = nx * ny * nz
        p = _Params()
        p.nx, p.ny, p.nz = nx, ny, nz
        for k in range(3):
            p.bc[k] = 1 if int(bc[k]) == 1 else 0
            p.face[2 * k] = p.face[2 * k + 1] = FACE_SLIP if int(bc[k]) == 2 else FACE_WALL
            p.g[k] = float(g[k])
        if open_top:
            if int(bc[2]) == 1:
                raise ValueError("an open top needs a non-periodic z axis")
            p.face[5] = FACE_OPEN
        if hydrostatic:
            if not open_top:
                raise ValueError("a hydrostatic start needs the open top as its reference")
            p.hydrostatic = 1
        p.n_substeps, p.sphere_mode = int(n_substeps), int(sphere_mode)
        p.nbub, p.nsph = len(bubbles), len(spheres)
        p.max_bub, p.split_every = max(int(max_bubbles), len(bubbles)), int(split_every)
        p.tau, p.sigma, p.rho_g0, p.eps, p.near_tol = tau, sigma, rho_g0, eps, near_tol
        self.p = p
        N = self.N
        self.f = np.zeros((19,) + self.shape)
        self.ft = np.zeros((19,) + self.shape)
        self.flag = np.zeros(self.shape, np.uint8)
        self.mark = np.zeros(self.shape, np.uint8)
        self.m = np.zeros(self.shape)
        self.phi = np.zeros(self.shape)
        self.phit = np.zeros(self.shape)
        self.kappa = np.zeros(self.shape)
        self.owner = np.full(self.shape, -1, np.int32)
        self.nown = np.zeros(self.shape, np.int32)
        self.near = np.zeros(self.shape, np.int32)
        self.bub = np.zeros((max(1, len(bubbles), int(max_bubbles)), B_LEN))
        self.bub[:, B_ROOT] = np.arange(self.bub.shape[0])
        for b, (cx, cy, cz, r) in enumerate(bubbles):
            self.bub[b, B_C:B_C + 3] = (cx, cy, cz)
            self.bub[b, B_R] = r
        self.sph = np.zeros((max(1, len(spheres)), S_LEN))
        for a, sp in enumerate(spheres):
            x, y, z, r, rho = sp[:5]
            u = sp[5:8] if len(sp) >= 8 else (0, 0, 0)
            w = sp[8:11] if len(sp) >= 11 else (0, 0, 0)
            self.sph[a, S_X:S_X + 3] = (x, y, z)
            self.sph[a, S_U:S_U + 3] = u
            self.sph[a, S_W:S_W + 3] = w
            self.sph[a, S_R] = r
            self.sph[a, S_RHO] = rho
        self.scal = np.zeros(SC_LEN)
        self.scal[SC_NBUB] = len(bubbles)
        self._bind()
        if init:
            lib().orc_init(ctypes.byref(self.p), ctypes.byref(self.s))

    def _bind(self):
        s = _State()
        d, u8, i32 = ctypes.c_double, ctypes.c_uint8, ctypes.c_int32
        s.f, s.ft = _ptr(self.f, d), _ptr(self.ft, d)
        s.flag, s.mark = _ptr(self.flag, u8), _ptr(self.mark, u8)
        s.m, s.phi, s.phit, s.kappa = _ptr(self.m, d), _ptr(self.phi, d), _ptr(self.phit, d), _ptr(self.kappa, d)
        s.owner, s.nown, s.near = _ptr(self.owner, i32), _ptr(self.nown, i32), _ptr(self.near, i32)
        s.bub, s.sph, s.scal = _ptr(self.bub, d), _ptr(self.sph, d), _ptr(self.scal, d)
        self.s = s

    def step(self, n: int = 1) -> int:
        return lib().orc_step(ctypes.byref(self.p), ctypes.byref(self.s), int(n))

    def fields(self):
        """(rho [z][y][x], u [3][z][y][x]) of the active cells, 0 elsewhere"""
        rho = np.zeros(self.shape)
        u = np.zeros((3,) + self.shape)
        lib().orc_fields(ctypes.byref(self.p), ctypes.byref(self.s), _ptr(rho, ctypes.c_double), _ptr(u, ctypes.c_double))
        return rho, u

    def total_mass(self) -> float:
        return lib().orc_total_mass(ctypes.byref(self.p), ctypes.byref(self.s))

    def mass_budget(self):
        """(M, S_bb, S_cover, S_uncover, pool)"""
        return (self.total_mass(), self.scal[SC_SBB], self.scal[SC_SCOV], self.scal[SC_SUNC], self.scal[SC_POOL])

    def lubrication(self) -> np.ndarray:
        Fl = np.zeros((max(1, int(self.p.nsph)), 3))
        lib().orc_lubrication(ctypes.byref(self.p), ctypes.byref(self.s), _ptr(Fl, ctypes.c_double))
        return Fl[: self.p.nsph]

    def curvature(self):
        lib().orc_curvature(ctypes.byref(self.p), ctypes.byref(self.s))

    def bubble_model(self, split=False):
        """the bubble model on the current cells (volumes, gas densities, merging; with split,
        splitting too)"""
        f = lib().orc_bubble_model_split if split else lib().orc_bubble_model
        f(ctypes.byref(self.p), ctypes.byref(self.s))

    def conversions(self):
        """the cell conversions alone (step 2) on the current state, taken as the sweep's
        result: types, fill levels, masses and PDFs f*(t+1)"""
        lib().orc_conversions(ctypes.byref(self.p), ctypes.byref(self.s))

    def cover_uncover(self):
        """cells covered and uncovered by the spheres at their current centres (step 4), with
        the refill of uncovered cells"""
        lib().orc_cover_uncover(ctypes.byref(self.p), ctypes.byref(self.s))

    @property
    def n_bubbles(self) -> int:
        """bubble ids in use (those given at the start and those splitting made)"""
        return int(self.scal[SC_NBUB])

    def tangent_window(self, nsteps, dtau=0.0, dg=(0.0, 0.0, 0.0), jdir=(1.0, 0.0, 0.0)):
        """advance nsteps steps of the frozen liquid window with the derivative along
        (dtau, dg); returns (J, dJ), J = sum_t jdir . sum_P F_P(t).  The current state is
        taken as independent of the parameters."""
        df = np.zeros((19,) + self.shape)
        dft = np.zeros((19,) + self.shape)
        dgv = np.ascontiguousarray(dg, dtype=np.float64)
        jd = np.ascontiguousarray(jdir, dtype=np.float64)
        J = ctypes.c_double()
        dJ = ctypes.c_double()
        rc = lib().orc_tangent_window(ctypes.byref(self.p), ctypes.byref(self.s), _ptr(df, ctypes.c_double),
                                      _ptr(dft, ctypes.c_double), float(dtau), _ptr(dgv, ctypes.c_double),
                                      _ptr(jd, ctypes.c_double), int(nsteps), ctypes.byref(J), ctypes.byref(dJ))
        if rc != 0:
            raise ValueError("the tangent window needs a liquid-only state")
        return J.value, dJ.value

    def window_objective(self, nsteps, jdir=(1.0, 0.0, 0.0)):
        """J = sum over nsteps ordinary steps of jdir . sum_P F_P(t)"""
        J = 0.0
        jd = np.asarray(jdir, dtype=np.float64)
        for _ in range(nsteps):
            self.step(1)
            J += float(self.forces[0].sum(axis=0) @ jd)
        return J

    @property
    def forces(self):
        return self.sph[: self.p.nsph, S_F:S_F + 3].copy(), self.sph[: self.p.nsph, S_T:S_T + 3].copy()

    @property
    def positions(self):
        return self.sph[: self.p.nsph, S_X:S_X + 3].copy()

    @property
    def rho_gas(self):
        return self.bub[: self.n_bubbles, B_RHOG].copy()

    @property
    def volumes(self):
        return self.bub[: self.n_bubbles, B_V].copy()

    @property
    def roots(self):
        """root id of each bubble id (the smallest id of the merged bubble it belongs to)"""
        up = self.bub[: self.n_bubbles, B_ROOT].astype(np.int64)
        r = up.copy()
        for b in range(len(r)):
            while up[r[b]] != r[b]:
                r[b] = up[r[b]]
        return r

    def momentum(self, with_positions=False):
        """total first moment sum_x sum_q c_q f*_q over active cells; optionally also the
        angular moment sum_x x cross (sum_q c_q f*_q)"""
        c = velocities().astype(np.float64)
        act = (self.flag & (LIQ | IFACE)) != 0
        j = np.einsum("qk,qzyx->kzyx", c, self.f) * act
        P = j.reshape(3, -1).sum(axis=1)
        if not with_positions:
            return P
        z, y, x = np.meshgrid(*[np.arange(n, dtype=np.float64) for n in self.shape], indexing="ij")
        X = np.stack([x, y, z])
        L = np.cross(X.reshape(3, -1).T, j.reshape(3, -1).T).sum(axis=0)
        return P, L
