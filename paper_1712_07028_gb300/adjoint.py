"""Gradients of a frozen-flag liquid window through the hand-written adjoint (reverse mode)
of the stream-collide and bounce-back step.

The objective is J = sum over the window's steps t = 1..T of jdir . (sum over spheres of the
momentum-exchange force F_P(t)) (Eqs. netforce, momentum_transfer); the parameters are the
relaxation time tau (lambda_+ = -1/tau, lambda_- from the magic relation, Sec. 2.1) and the
body force g (Guo forcing).  The window is liquid only with fixed spheres and FP32 PDFs, so
no cell changes type and the step is a smooth map f*(t) -> f*(t+1).

Memory: the forward pass keeps a checkpoint of f* every K steps; the backward pass replays
each segment from its checkpoint with the frozen forward step (K states), then runs the
reverse steps of that segment, newest first.  Peak extra memory: (T/K + K + 2) states of
19 x N FP32.
"""
from __future__ import annotations

import numpy as np
import torch

from . import lbm as _lbm


def _state_like(sim):
    t = sim._torch
    return t.empty((19,) + sim.shape, dtype=t.float32, device=sim.device)


def forward_window(sim: _lbm.Sim, nsteps: int, jdir, every: int):
    """run nsteps ordinary steps from the current state; returns (J, checkpoints), the
    checkpoints being f* at steps 0, every, 2 every, ... (FP32 deviation tensors).  J is
    accumulated on the device (lbm_objective) and read once at the end."""
    if every < 1 or nsteps < 1:
        raise ValueError("nsteps and the checkpoint interval must be positive")
    sim.step(0)
    sim.objective(jdir)
    ckpts = []
    t = 0
    while t < nsteps:
        ckpts.append(sim.export_state()["f"])
        k = min(every, nsteps - t)
        sim.step(k)
        t += k
    J = sim.objective_read()
    sim.objective(None)
    return J, ckpts


def backward_window(sim: _lbm.Sim, nsteps: int, jdir, every: int, ckpts, adj_final=None):
    """reverse sweep over the window recorded by forward_window: returns
    (dJ/dtau, dJ/dg [3], dJ/df*(0) [19,z,y,x]); adj_final seeds dJ/df*(T) (zero if None)"""
    lam = _state_like(sim)
    lam_next = _state_like(sim)
    if adj_final is None:
        lam.zero_()
    else:
        lam.copy_(adj_final)
    lam_next.zero_()
    nseg = len(ckpts)
    seg_states = [_state_like(sim) for _ in range(max(0, min(every, nsteps) - 1))]
    first = True
    dg = np.zeros(3)
    dtau = 0.0
    for s in reversed(range(nseg)):
        t0 = s * every
        n = min(every, nsteps - t0)
        states = [ckpts[s]] + seg_states[: n - 1]
        for k in range(1, n):
            sim.forward_frozen(states[k - 1], states[k])
        for k in reversed(range(n)):
            last = s == 0 and k == 0
            out = sim.adjoint_step(states[k], lam, lam_next, jdir, accumulate=not first, read=last)
            first = False
            lam, lam_next = lam_next, lam
            if last:
                dg, dtau = out
    return dtau, dg, lam


def window_gradient(sim: _lbm.Sim, nsteps: int, jdir=(1.0, 0.0, 0.0), every: int = 50):
    """(J, dJ/dtau, dJ/dg) of the window of nsteps steps from the current state"""
    J, ck = forward_window(sim, nsteps, jdir, every)
    dtau, dg, _ = backward_window(sim, nsteps, jdir, every, ck)
    return J, dtau, dg


class LBMWindow(torch.autograd.Function):
    """J(tau, g, f0) of a frozen liquid window as a differentiable torch function.

    ``LBMWindow.apply(tau, g, f0, sim, nsteps, jdir, every)``: tau a 0-d and g a 3-vector
    float64 tensor, f0 the window's start state (FP32 deviations [19,z,y,x] on the device, as
    ``sim.export_state()["f"]`` gives it).  Every call sets the simulation's relaxation time and
    body force to (tau, g), imports f0 and runs the window, so J can be evaluated at any point
    (finite differences, optimisation loops).  Returns J as a 0-d float64 tensor; backward
    gives dJ/dtau, dJ/dg and dJ/df0 from the adjoint, with checkpoints every ``every`` steps."""

    @staticmethod
    def forward(ctx, tau, g, f0, sim, nsteps, jdir, every):
        tv, gv = float(tau), [float(v) for v in g]
        p = sim.params
        if tv != p.tau or any(gv[k] != p.g[k] for k in range(3)):
            sim.set_params(tv, gv)
        sim.step(0)
        sim.import_state(f0.detach())
        J, ck = forward_window(sim, int(nsteps), jdir, int(every))
        ctx.sim, ctx.nsteps, ctx.jdir, ctx.every, ctx.ckpts = sim, int(nsteps), jdir, int(every), ck
        ctx.params = (tv, gv)
        return torch.tensor(J, dtype=torch.float64)

    @staticmethod
    def backward(ctx, gJ):
        sim = ctx.sim
        tv, gv = ctx.params
        p = sim.params
        if tv != p.tau or any(gv[k] != p.g[k] for k in range(3)):   # another evaluation ran since
            sim.set_params(tv, gv)
        dtau, dg, lam = backward_window(sim, ctx.nsteps, ctx.jdir, ctx.every, ctx.ckpts)
        ctx.ckpts = None
        gf0 = (gJ.to(lam.dtype) * lam) if ctx.needs_input_grad[2] else None
        return gJ * dtau, gJ * torch.tensor(dg, dtype=torch.float64), gf0, None, None, None, None
