"""Python binding of the C ABI in include/lbm.h (ctypes; argument marshalling only).

PyTorch supplies the device memory (one arena tensor per simulation) and the stream
(``torch.cuda.current_stream()``); every step of the method runs in the library's CUDA
kernels.  There is no CPU path: without a GPU or without the built library, ``Sim`` raises.
"""
from __future__ import annotations

import ctypes
import os

import numpy as np

from . import build as _build
from . import workloads as _wl

_lib = None

LBM_OK, LBM_EINVAL, LBM_ESTATE, LBM_ECUDA, LBM_EUNSTABLE, LBM_EOVERFLOW, LBM_EMERGE, LBM_ESPLIT = 0, -1, -2, -3, -4, -5, -6, -7
CELL_LIQUID, CELL_INTERFACE, CELL_GAS, CELL_OBSTACLE = 1, 2, 4, 8
S_UNSTABLE, S_OVERFLOW, S_BUBBLE_GONE, S_BIN_OVERFLOW, S_FAST_SPHERE, S_MERGE, S_SPLIT = 1, 2, 4, 8, 32, 64, 128

# every entry point include/lbm.h declares
EXPORTS = ("lbm_arena_bytes", "lbm_init", "lbm_set_stream", "lbm_add_bubble", "lbm_add_sphere", "lbm_add_spheres", "lbm_step",
           "lbm_forces", "lbm_spheres", "lbm_lubrication", "lbm_bubbles", "lbm_bubble_roots", "lbm_bubble_splits", "lbm_fields", "lbm_export_state", "lbm_mass_budget",
           "lbm_status", "lbm_profile", "lbm_profile_read", "lbm_copy_bytes", "lbm_launch_count",
           "lbm_bubble_volumes_noalloc", "lbm_set_params", "lbm_import_state", "lbm_objective", "lbm_objective_read",
           "lbm_forward_frozen", "lbm_adjoint_step", "lbm_destroy", "lbm_strerror")


class Params(ctypes.Structure):
    _fields_ = [("nx", ctypes.c_int32), ("ny", ctypes.c_int32), ("nz", ctypes.c_int32), ("bc", ctypes.c_int32 * 3),
                ("storage", ctypes.c_int32), ("n_substeps", ctypes.c_int32), ("sphere_mode", ctypes.c_int32),
                ("max_bubbles", ctypes.c_int32), ("max_spheres", ctypes.c_int32), ("worklist_cap", ctypes.c_int32),
                ("tau", ctypes.c_double), ("g", ctypes.c_double * 3), ("sigma", ctypes.c_double),
                ("rho_gas0", ctypes.c_double), ("eps", ctypes.c_double), ("open_top", ctypes.c_int32),
                ("hydrostatic", ctypes.c_int32), ("split_every", ctypes.c_int32)]


class LBMError(RuntimeError):
    def __init__(self, fn, code):
        super().__init__("%s failed: %s (%d)" % (fn, load().lbm_strerror(code).decode(), code))
        self.code = code


def library_path() -> str:
    return _build.LIB


def load():
    """load the CUDA library; raises if it has not been built"""
    global _lib
    if _lib is not None:
        return _lib
    path = library_path()
    if not os.path.exists(path):
        raise RuntimeError("the CUDA library %s is not built (run __graft_entry__.build())" % path)
    L = ctypes.CDLL(path)
    vp, d, i32, sz = ctypes.c_void_p, ctypes.c_double, ctypes.c_int, ctypes.c_size_t
    pd = ctypes.POINTER(ctypes.c_double)
    L.lbm_arena_bytes.argtypes = [ctypes.POINTER(Params), ctypes.POINTER(sz)]
    L.lbm_init.argtypes = [ctypes.POINTER(Params), vp, sz, vp, ctypes.POINTER(vp)]
    L.lbm_set_stream.argtypes = [vp, vp]
    L.lbm_add_bubble.argtypes = [vp, pd, d, ctypes.POINTER(i32)]
    L.lbm_add_sphere.argtypes = [vp, pd, d, d, pd, pd, ctypes.POINTER(i32)]
    L.lbm_add_spheres.argtypes = [vp, i32, vp, vp, vp, vp, vp, ctypes.POINTER(i32)]
    L.lbm_step.argtypes = [vp, i32]
    L.lbm_forces.argtypes = [vp, pd, pd, i32]
    L.lbm_spheres.argtypes = [vp, pd, pd, pd, i32]
    L.lbm_lubrication.argtypes = [vp, pd, i32]
    L.lbm_bubbles.argtypes = [vp, pd, pd, pd, i32]
    L.lbm_bubble_roots.argtypes = [vp, ctypes.POINTER(i32), i32, ctypes.POINTER(i32)]
    L.lbm_bubble_splits.argtypes = [vp, ctypes.POINTER(i32), ctypes.POINTER(i32)]
    L.lbm_fields.argtypes = [vp, vp, vp, vp, vp]
    L.lbm_export_state.argtypes = [vp, vp, vp, vp, vp, vp, vp]
    L.lbm_mass_budget.argtypes = [vp, pd]
    L.lbm_status.argtypes = [vp, ctypes.POINTER(ctypes.c_uint32)]
    L.lbm_launch_count.argtypes = [vp, ctypes.POINTER(ctypes.c_uint64)]
    L.lbm_profile.argtypes = [vp, i32]
    L.lbm_copy_bytes.argtypes = [vp, ctypes.POINTER(ctypes.c_uint64), ctypes.POINTER(ctypes.c_uint64)]
    L.lbm_profile_read.argtypes = [vp, ctypes.POINTER(ctypes.c_double), ctypes.POINTER(ctypes.c_uint64)]
    L.lbm_bubble_volumes_noalloc.argtypes = [vp, vp, vp, sz, i32, vp, vp]
    L.lbm_set_params.argtypes = [vp, d, pd]
    L.lbm_import_state.argtypes = [vp, vp]
    L.lbm_objective.argtypes = [vp, pd]
    L.lbm_objective_read.argtypes = [vp, pd]
    L.lbm_forward_frozen.argtypes = [vp, vp, vp]
    L.lbm_adjoint_step.argtypes = [vp, vp, vp, vp, pd, i32, pd, pd]
    L.lbm_destroy.argtypes = [vp]
    L.lbm_strerror.argtypes = [i32]
    L.lbm_strerror.restype = ctypes.c_char_p
    _lib = L
    return L


def _check(fn, rc):
    if rc != LBM_OK:
        raise LBMError(fn, rc)


def _dp(a):
    return a.ctypes.data_as(ctypes.POINTER(ctypes.c_double))


def _v3(v):
    return np.ascontiguousarray(v, dtype=np.float64).reshape(3)


def make_params(wl: _wl.Workload, max_bubbles=None, max_spheres=None, worklist_cap=0) -> Params:
    p = Params()
    p.nx, p.ny, p.nz = wl.nx, wl.ny, wl.nz
    for k in range(3):
        p.bc[k] = int(wl.bc[k])
        p.g[k] = float(wl.g[k])
    p.storage = _wl.STORAGE[wl.storage]
    p.n_substeps = int(wl.n_substeps)
    p.sphere_mode = int(wl.sphere_mode)
    p.max_bubbles = int(max_bubbles or max(1, len(wl.bubbles), int(wl.max_bubbles)))
    p.max_spheres = int(max_spheres or max(1, len(wl.spheres)))
    p.worklist_cap = int(worklist_cap)
    p.tau, p.sigma, p.rho_gas0, p.eps = float(wl.tau), float(wl.sigma), float(wl.rho_g0), float(wl.eps)
    p.open_top = 1 if wl.open_top else 0
    p.hydrostatic = 1 if wl.hydrostatic else 0
    p.split_every = int(wl.split_every)
    return p


class Sim:
    """One simulation on the current CUDA device, fields in a torch-owned arena."""

    def __init__(self, wl: _wl.Workload, device=None, **kw):
        import torch
        if not torch.cuda.is_available():
            raise RuntimeError("Sim needs a CUDA device; there is no CPU fallback")
        self._torch = torch
        L = load()
        self.wl = wl
        self.device = torch.device(device) if device is not None else torch.device("cuda", torch.cuda.current_device())
        self.params = make_params(wl, **kw)
        nbytes = ctypes.c_size_t()
        _check("lbm_arena_bytes", L.lbm_arena_bytes(ctypes.byref(self.params), ctypes.byref(nbytes)))
        self.arena = torch.empty(nbytes.value, dtype=torch.uint8, device=self.device)
        self.ctx = ctypes.c_void_p()
        _check("lbm_init", L.lbm_init(ctypes.byref(self.params), ctypes.c_void_p(self.arena.data_ptr()), nbytes.value,
                                      ctypes.c_void_p(self._stream()), ctypes.byref(self.ctx)))
        self.shape = (wl.nz, wl.ny, wl.nx)
        self.N = wl.nx * wl.ny * wl.nz
        for b in wl.bubbles:
            _check("lbm_add_bubble", L.lbm_add_bubble(self.ctx, _dp(_v3(b.c)), float(b.r), None))
        if wl.spheres:   # one call for the whole table
            sp = wl.spheres
            x = np.ascontiguousarray([s.x for s in sp], dtype=np.float64)
            r = np.ascontiguousarray([s.r for s in sp], dtype=np.float64)
            rho = np.ascontiguousarray([s.rho for s in sp], dtype=np.float64)
            u = np.ascontiguousarray([s.u for s in sp], dtype=np.float64)
            w = np.ascontiguousarray([s.w for s in sp], dtype=np.float64)
            _check("lbm_add_spheres", L.lbm_add_spheres(self.ctx, len(sp), *[ctypes.c_void_p(a.ctypes.data) for a in (x, r, rho, u, w)],
                                                        None))
        self.nsph = len(wl.spheres)
        # bubble ids: the bubbles given, or with splitting every row of the table
        self.nbub = int(self.params.max_bubbles) if wl.split_every > 0 else len(wl.bubbles)
        self.steps_done = 0

    def _stream(self) -> int:
        return self._torch.cuda.current_stream(self.device).cuda_stream

    def _bind_stream(self):
        load().lbm_set_stream(self.ctx, ctypes.c_void_p(self._stream()))

    def step(self, n: int = 1):
        self._bind_stream()
        _check("lbm_step", load().lbm_step(self.ctx, int(n)))
        self.steps_done += int(n)

    def forces(self):
        """(F [n][3], T [n][3]) FP64 momentum-exchange force and torque of the last step"""
        self._bind_stream()
        F = np.zeros((max(1, self.nsph), 3))
        T = np.zeros((max(1, self.nsph), 3))
        _check("lbm_forces", load().lbm_forces(self.ctx, _dp(F), _dp(T), self.nsph))
        return F[: self.nsph], T[: self.nsph]

    def spheres(self):
        self._bind_stream()
        x, u, w = (np.zeros((max(1, self.nsph), 3)) for _ in range(3))
        _check("lbm_spheres", load().lbm_spheres(self.ctx, _dp(x), _dp(u), _dp(w), self.nsph))
        return x[: self.nsph], u[: self.nsph], w[: self.nsph]

    def lubrication(self):
        """Fl [n][3]: the lubrication force of the last sub-step of the last step"""
        self._bind_stream()
        Fl = np.zeros((max(1, self.nsph), 3))
        _check("lbm_lubrication", load().lbm_lubrication(self.ctx, _dp(Fl), self.nsph))
        return Fl[: self.nsph]

    def bubbles(self):
        self._bind_stream()
        V0, V, rg = (np.zeros(max(1, self.nbub)) for _ in range(3))
        _check("lbm_bubbles", load().lbm_bubbles(self.ctx, _dp(V0), _dp(V), _dp(rg), self.nbub))
        return V0[: self.nbub], V[: self.nbub], rg[: self.nbub]

    def bubble_splits(self):
        """(bubble ids in use: one past the highest id that carried cells, parts split off so far)"""
        self._bind_stream()
        n, ns = ctypes.c_int(0), ctypes.c_int(0)
        _check("lbm_bubble_splits", load().lbm_bubble_splits(self.ctx, ctypes.byref(n), ctypes.byref(ns)))
        return n.value, ns.value

    def bubble_roots(self):
        """(root id of every bubble id, number of merges so far)"""
        self._bind_stream()
        root = np.zeros(max(1, self.nbub), dtype=np.int32)
        nm = ctypes.c_int(0)
        _check("lbm_bubble_roots", load().lbm_bubble_roots(self.ctx, root.ctypes.data_as(ctypes.POINTER(ctypes.c_int)),
                                                           self.nbub, ctypes.byref(nm)))
        return root[: self.nbub].astype(np.int64), nm.value

    def fields(self):
        """dict of torch tensors on the device: rho [z,y,x], u [3,z,y,x], phi, flags"""
        t = self._torch
        out = {"rho": t.empty(self.shape, dtype=t.float32, device=self.device),
               "u": t.empty((3,) + self.shape, dtype=t.float32, device=self.device),
               "phi": t.empty(self.shape, dtype=t.float32, device=self.device),
               "flags": t.empty(self.shape, dtype=t.uint8, device=self.device)}
        self._bind_stream()
        _check("lbm_fields", load().lbm_fields(self.ctx, *[ctypes.c_void_p(out[k].data_ptr()) for k in ("rho", "u", "phi", "flags")]))
        return out

    def export_state(self):
        """dict of torch tensors on the device: f [19,z,y,x] (FP32 deviations f - w_q), flags,
        mass, phi, owner, kappa"""
        t = self._torch
        out = {"f": t.empty((19,) + self.shape, dtype=t.float32, device=self.device),
               "flags": t.empty(self.shape, dtype=t.uint8, device=self.device),
               "mass": t.empty(self.shape, dtype=t.float32, device=self.device),
               "phi": t.empty(self.shape, dtype=t.float32, device=self.device),
               "owner": t.empty(self.shape, dtype=t.int32, device=self.device),
               "kappa": t.empty(self.shape, dtype=t.float32, device=self.device)}
        self._bind_stream()
        _check("lbm_export_state", load().lbm_export_state(
            self.ctx, *[ctypes.c_void_p(out[k].data_ptr()) for k in ("f", "flags", "mass", "phi", "owner", "kappa")]))
        return out

    def mass_budget(self):
        """(M, S_bb, S_cover, S_uncover, pool), FP64"""
        self._bind_stream()
        out = np.zeros(5)
        _check("lbm_mass_budget", load().lbm_mass_budget(self.ctx, _dp(out)))
        return tuple(out)

    def status(self) -> int:
        self._bind_stream()
        s = ctypes.c_uint32()
        _check("lbm_status", load().lbm_status(self.ctx, ctypes.byref(s)))
        return s.value

    def profile(self, on: bool):
        _check("lbm_profile", load().lbm_profile(self.ctx, 1 if on else 0))

    def profile_read(self):
        """(bulk sweep milliseconds, rest-of-sweep milliseconds, number of steps) recorded
        since the last read"""
        ms = (ctypes.c_double * 2)()
        n = ctypes.c_uint64()
        _check("lbm_profile_read", load().lbm_profile_read(self.ctx, ms, ctypes.byref(n)))
        return ms[0], ms[1], n.value

    def copy_bytes(self):
        """(host->device, device->host) bytes the library has copied so far"""
        a, b = ctypes.c_uint64(), ctypes.c_uint64()
        _check("lbm_copy_bytes", load().lbm_copy_bytes(self.ctx, ctypes.byref(a), ctypes.byref(b)))
        return a.value, b.value

    def launches(self) -> int:
        n = ctypes.c_uint64()
        _check("lbm_launch_count", load().lbm_launch_count(self.ctx, ctypes.byref(n)))
        return n.value

    def set_params(self, tau, g):
        """relaxation time and body force of the steps that follow"""
        self._bind_stream()
        _check("lbm_set_params", load().lbm_set_params(self.ctx, float(tau), _dp(_v3(g))))
        self.params.tau = float(tau)
        for k in range(3):
            self.params.g[k] = float(g[k])

    def import_state(self, f):
        """replace the post-collision PDFs (FP32 deviations [19,z,y,x], device) of a window"""
        self._bind_stream()
        _check("lbm_import_state", load().lbm_import_state(self.ctx, ctypes.c_void_p(f.data_ptr())))

    def objective(self, jdir=None):
        """from now on accumulate jdir . sum_P F_P of every step on the device (None: stop)"""
        self._bind_stream()
        _check("lbm_objective", load().lbm_objective(self.ctx, _dp(_v3(jdir)) if jdir is not None else None))

    def objective_read(self) -> float:
        self._bind_stream()
        J = ctypes.c_double()
        _check("lbm_objective_read", load().lbm_objective_read(self.ctx, ctypes.byref(J)))
        return J.value

    def forward_frozen(self, f_in, f_out):
        """one step of the frozen liquid window on FP32 deviation tensors [19,z,y,x] (device)"""
        self._bind_stream()
        _check("lbm_forward_frozen", load().lbm_forward_frozen(self.ctx, ctypes.c_void_p(f_in.data_ptr()),
                                                               ctypes.c_void_p(f_out.data_ptr())))

    def adjoint_step(self, f_fwd, adj_in, adj_out, jdir, accumulate=True, read=False):
        """one reverse step (adj_out = dJ/df*(t) from f_fwd = f*(t), adj_in = dJ/df*(t+1));
        with read=True returns the accumulated (dJ/dg [3], dJ/dtau)"""
        self._bind_stream()
        jd = _v3(jdir)
        dg = np.zeros(3)
        dt = ctypes.c_double()
        _check("lbm_adjoint_step", load().lbm_adjoint_step(
            self.ctx, ctypes.c_void_p(f_fwd.data_ptr()), ctypes.c_void_p(adj_in.data_ptr()),
            ctypes.c_void_p(adj_out.data_ptr()), _dp(jd), 1 if accumulate else 0, _dp(dg) if read else None,
            ctypes.byref(dt) if read else None))
        return (dg, dt.value) if read else None

    def close(self):
        if getattr(self, "ctx", None) and self.ctx.value:
            load().lbm_destroy(self.ctx)
            self.ctx = ctypes.c_void_p()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass
