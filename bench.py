#!/usr/bin/env python
"""Throughput of the fused free-surface LBM step (MLUPS) on the 512x512x1024 bubble-particle
column, the largest single-GPU workload.

One step = the whole per-step hot path: sweep (stream, bounce-back, gas reconstruction,
mass exchange, TRT collision), cell conversions, bubble model, sphere update and
cover/uncover.  Headline workload: 512 x 512 x 1024 cells (268 M), walls, tau 0.6, gravity
1e-6 along -z, 32 gas bubbles r=24 and 100 000 free spheres r=4 of density 1.5 placed by
seeded rejection sampling, PDFs stored as FP16 deviations (two grids of 10.2 GB: inputs far
larger than L2).  Extra objects: the 256x256x512 column in FP32 and FP16 deviations (the
FP32-vs-FP16 configuration) and the 128^3 column.

Prints one JSON line (rank 0).  --impl reference times the FP64 CPU oracle instead (on a
bounded sub-box of the large columns).  Under torchrun every rank runs an independent
replica (the method needs no exchange between replicas; one GPU per domain).
"""
from __future__ import annotations

import argparse
import hashlib
import json
import os
import statistics
import subprocess
import sys
import tempfile
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "MLUPS and HBM-roofline fraction, FP32 / FP16-store vs FP64 oracle error"
FALLBACK_HBM_GBS = 6800.0

# dram bytes (read + write) per bulk-sweep launch, per workload and storage, from one ncu
# capture, with the hash of the sweep source it was taken on (null once the kernel changes)
NCU_TRAFFIC = {
    # one-pass capture of two launches on that column (mean)
    "column512x512x1024_32bubbles_100000spheres/f16dev": {"sha1": "c4593b323a98b5805bd80af15b7c6004e703ba0e",
                                                           "bytes_per_launch": 21821934208},
}


def _args():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=300)
    ap.add_argument("--warmup", type=int, default=5)
    ap.add_argument("--impl", default="gb300", choices=["gb300", "reference"])
    ap.add_argument("--workload", default="c4", choices=["c0", "c1", "c3", "c4"])
    ap.add_argument("--storage", default=None, choices=[None, "f32", "f16dev", "bf16dev"])
    ap.add_argument("--no-extras", action="store_true", help="only the timed region (for profilers)")
    ap.add_argument("--split-every", type=int, default=0,
                    help="bubbles split into their connected parts every so many steps (0: never)")
    ap.add_argument("--only", default=None, choices=[None, "adjoint"],
                    help="time only the differentiation path (the adjoint object of the full line)")
    return ap.parse_args()


_WL_CACHE = {}


def _workload(name, storage=None):
    """the named column (generated once per process; callers get their own copy)"""
    import dataclasses
    from paper_1712_07028_gb300 import workloads as W
    if name not in _WL_CACHE:
        _WL_CACHE[name] = {"c0": W.column_c0, "c1": W.column_c1, "c3": W.column_c3, "c4": W.column_c4}[name]()
    wl = dataclasses.replace(_WL_CACHE[name])
    if storage:
        wl.storage = storage
    return wl


def _cpu_sample(name):
    """the workload the CPU oracle steps for a column: the column itself up to ~2 M cells,
    else a 128 x 128 x 256 sub-box of it at the column's sphere and bubble densities"""
    from paper_1712_07028_gb300 import workloads as W
    wl = _workload(name)
    if wl.cells <= 2_200_000:
        return wl
    b = wl.bubbles[0].c
    size = (128, 128, 256)
    lo = tuple(int(min(max(0, round(b[k]) - size[k] // 2), (wl.nx, wl.ny, wl.nz)[k] - size[k])) for k in range(3))
    return W.sub_box(wl, lo, size)


def _job_ms(dist, ms, device):
    """the job's time: the maximum over ranks of each rank's timed region (milliseconds)"""
    if dist is None:
        return ms
    import torch
    t = torch.tensor([ms], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def _job_mlups(cells_per_rank, steps, ws, ms):
    """whole-job throughput: the cells all ranks updated over the job's time (weak scaling:
    every rank runs its own replica of the workload)"""
    return cells_per_rank * steps * ws / (ms * 1e-3) / 1e6


def _dist():
    ws = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return ws, rank, local


class Clocks:
    """nvidia-smi sampling of SM clock and throttle reasons during the timed region"""
    Q = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,clocks_event_reasons.hw_slowdown,"
         "clocks_event_reasons.hw_thermal_slowdown,clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_id):
        self.gpu_id = gpu_id
        self.proc = None
        self.path = None

    def start(self):
        fd, self.path = tempfile.mkstemp(suffix=".csv")
        os.close(fd)
        try:
            self.proc = subprocess.Popen(["nvidia-smi", "-i", str(self.gpu_id), "--query-gpu=" + self.Q,
                                          "--format=csv,noheader,nounits", "-lms", "50"],
                                         stdout=open(self.path, "w"), stderr=subprocess.DEVNULL)
            time.sleep(0.3)
        except OSError:
            self.proc = None

    def stop(self):
        if self.proc is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        time.sleep(0.1)
        self.proc.terminate()
        self.proc.wait()
        rows = [l.strip().split(", ") for l in open(self.path) if l.strip()]
        os.unlink(self.path)
        sm = [float(r[1]) for r in rows if len(r) >= 9 and r[1].replace(".", "").isdigit()]
        mx = [float(r[2]) for r in rows if len(r) >= 9 and r[2].replace(".", "").isdigit()]
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        reasons = sorted({names[k] for r in rows if len(r) >= 9 for k in range(4) if r[5 + k].strip() == "Active"})
        load = sorted(sm)[len(sm) // 2:] if sm else []
        return {"sm_mhz": statistics.median(load) if load else None, "sm_max_mhz": max(mx) if mx else None,
                "reasons": reasons, "samples": len(rows)}


def _gpu_index(torch, local):
    vis = os.environ.get("CUDA_VISIBLE_DEVICES")
    if vis:
        return vis.split(",")[local].strip()
    return local


def _peak_hbm():
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
            return float(json.load(f)["hbm_gbs"]), "measured"
    except (OSError, KeyError, ValueError):
        return FALLBACK_HBM_GBS, "fallback"


def _bulk_cells(torch, lbm, fl, bc):
    """liquid cells whose 18 D3Q19 neighbours all carry PDFs or lie beyond a wall: the cells
    the bulk sweep kernel streams (measurement only: the library keeps its own bit)"""
    act = (fl == lbm.CELL_LIQUID) | (fl == lbm.CELL_INTERFACE)
    ok = fl == lbm.CELL_LIQUID
    # one layer of padding: the periodic image on periodic axes, "carries PDFs" beyond a wall
    # (axes of fl are z, y, x)
    pad = act
    for ax, k in ((0, 2), (1, 1), (2, 0)):
        if bc[k]:
            pad = torch.cat([pad.narrow(ax, pad.shape[ax] - 1, 1), pad, pad.narrow(ax, 0, 1)], dim=ax)
        else:
            shape = list(pad.shape)
            shape[ax] = 1
            one = torch.ones(shape, dtype=torch.bool, device=fl.device)
            pad = torch.cat([one, pad, one], dim=ax)
    nz, ny, nx = act.shape
    for dz in (-1, 0, 1):
        for dy in (-1, 0, 1):
            for dx in (-1, 0, 1):
                if abs(dx) + abs(dy) + abs(dz) in (1, 2):
                    ok &= pad[1 + dz:1 + dz + nz, 1 + dy:1 + dy + ny, 1 + dx:1 + dx + nx]
    return int(ok.sum().item())


def _sweep_sha():
    h = hashlib.sha1()
    for n in ("lbm_sweep.cu", "lbm_internal.cuh"):
        h.update(open(os.path.join(ROOT, "paper_1712_07028_gb300", "csrc", n), "rb").read())
    return h.hexdigest()


def _cpu_baseline(name, budget_s=15.0):
    """the FP64 oracle as it stands, single thread, on a bounded sample of the workload: whole
    steps of the column (or of its sub-box) until about budget_s seconds have passed"""
    import oracle
    oracle.build()
    wl = _cpu_sample(name)
    t0 = time.perf_counter()
    o = oracle.Sim(wl)
    t1 = time.perf_counter()
    o.step(1)
    t2 = time.perf_counter()
    k = max(1, min(50, int(budget_s / max(t2 - t1, 1e-3))))
    o.step(k)
    t3 = time.perf_counter()
    full = _workload(name)
    what = ("the whole column" if wl.cells == full.cells else
            "a %dx%dx%d sub-box of the %dx%dx%d column (%d bubbles, %d spheres inside it, walls on its faces)"
            % (wl.nx, wl.ny, wl.nz, full.nx, full.ny, full.nz, len(wl.bubbles), len(wl.spheres)))
    return {"value": wl.cells * k / (t3 - t2) / 1e6, "unit": "MLUPS", "cores": 1, "kind": "oracle",
            "cpu": _cpu_model(), "nproc": os.cpu_count(),
            "sample": "FP64 oracle, single thread, on %s: init (%.1f s), 1 warm-up step, %d full steps timed (%.1f s)"
                      % (what, t1 - t0, k, t3 - t2)}


def _oracle_box_worker(args):
    """one single-threaded oracle process on a sub-box: (cells, steps, seconds)"""
    name, lo, size, budget_s = args
    import oracle
    from paper_1712_07028_gb300 import workloads as W
    wl = W.sub_box(_workload(name), lo, size)
    o = oracle.Sim(wl)
    o.step(1)
    t0 = time.perf_counter()
    k = 0
    while time.perf_counter() - t0 < budget_s:
        o.step(1)
        k += 1
    return wl.cells, k, time.perf_counter() - t0


def _cpu_baseline_all_cores(name, budget_s=12.0):
    """the FP64 oracle as it stands on every host core: one single-threaded process per core,
    each stepping its own sub-box of the column (weak scaling over the cores); aggregate MLUPS =
    all processes' cell updates over the slowest one's time"""
    import multiprocessing as mp
    from concurrent.futures import ProcessPoolExecutor
    import oracle
    oracle.build()
    full = _workload(name)
    n = os.cpu_count() or 1
    size = (min(full.nx, 128), min(full.ny, 128), min(full.nz, 128)) if full.cells > 2_200_000 else (full.nx, full.ny, full.nz)
    boxes = []
    for k in range(n):   # boxes spread along z (and x, y), within the column
        lo = tuple(int((k * 37 * (1 + a) + 11 * a) % max(1, (full.nx, full.ny, full.nz)[a] - size[a] + 1)) for a in range(3))
        boxes.append((name, lo, size, budget_s))
    t0 = time.perf_counter()
    with ProcessPoolExecutor(max_workers=n, mp_context=mp.get_context("spawn")) as ex:
        res = list(ex.map(_oracle_box_worker, boxes))
    wall = time.perf_counter() - t0
    updates = sum(c * k for c, k, _ in res)
    slowest = max(t for _, _, t in res)
    return {"value": updates / slowest / 1e6, "unit": "MLUPS", "cores": n, "kind": "oracle",
            "sample": "%d single-threaded FP64 oracle processes, one per core, each stepping a %dx%dx%d sub-box of the "
                      "column for ~%.0f s (%d to %d steps; %.0f s with start-up)"
                      % (n, size[0], size[1], size[2], budget_s, min(k for _, k, _ in res), max(k for _, k, _ in res), wall)}


def _cpu_model():
    """the host CPU's model name (lscpu, else /proc/cpuinfo)"""
    try:
        out = subprocess.run(["lscpu"], capture_output=True, text=True, timeout=10).stdout
        for line in out.splitlines():
            if line.strip().lower().startswith("model name"):
                return line.split(":", 1)[1].strip()
    except (OSError, subprocess.SubprocessError):
        pass
    try:
        for line in open("/proc/cpuinfo"):
            if line.lower().startswith(("model name", "cpu part", "hardware")):
                return line.split(":", 1)[1].strip()
    except OSError:
        pass
    import platform
    return platform.processor() or platform.machine()


def _oracle_error(torch, lbm, W):
    """error of the GPU path against the FP64 oracle on the 32^3 column after 200 steps, per
    PDF storage (the max over cells active in both, away from type mismatches)"""
    import numpy as np
    import oracle
    from tests import gpu_util as U
    oracle.build()
    base = W.column_c0()
    o = oracle.Sim(base)
    o.step(base.steps)
    out = {}
    for storage in ("f32", "f16dev", "bf16dev"):
        wl = W.column_c0()
        wl.storage = storage
        sim = lbm.Sim(wl)
        sim.step(wl.steps)
        st = U.gpu_state(sim)
        mism = st["flags"] != o.flag
        drho, du, _ = U.compare_fields(o, st, ~U.dilate(mism, 2))
        iface = (st["flags"] == oracle.IFACE) & (o.flag == oracle.IFACE) & ~U.dilate(mism, 2)
        dphi = float(np.abs(st["phi"] - o.phi)[iface].max()) if iface.any() else 0.0
        out[storage] = {"max_abs_drho": float(drho), "max_abs_du": float(du), "max_abs_dphi": dphi,
                        "type_mismatches": int(mism.sum())}
        sim.close()
    out["case"] = "32^3 column (bubble r=6, sphere r=3), 200 steps"
    return out


def _config_run(torch, lbm, name, storage, steps, warmup):
    """MLUPS of one column and PDF storage, the bulk sweep's roofline from CUDA events around
    its launches, and the whole step against the sweep's algorithmic bytes"""
    wl = _workload(name, storage)
    s_bytes = 4 if wl.storage == "f32" else 2
    sim = lbm.Sim(wl)
    sim.step(max(3, warmup))
    torch.cuda.synchronize()
    stream = torch.cuda.current_stream()
    e0 = torch.cuda.Event(enable_timing=True)
    e1 = torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    sim.step(steps)
    e1.record(stream)
    torch.cuda.synchronize()
    ms = e0.elapsed_time(e1) / steps
    sim.profile(True)
    sim.step(min(steps, 100))
    torch.cuda.synchronize()
    bulk_ms, rest_ms, nsw = sim.profile_read()
    sim.profile(False)
    fl = sim.fields()["flags"]
    n_act = int(((fl == lbm.CELL_LIQUID) | (fl == lbm.CELL_INTERFACE)).sum().item())
    n_bulk = _bulk_cells(torch, lbm, fl, wl.bc)
    del fl
    per_launch = n_bulk * (38 * s_bytes + 1) + (wl.cells - n_bulk)
    step_bytes = n_act * (38 * s_bytes + 1) + (wl.cells - n_act)
    avg_s = bulk_ms / max(1, nsw) * 1e-3
    peak, _ = _peak_hbm()
    st = sim.status()
    sim.close()
    torch.cuda.synchronize()
    return {"workload": wl.name, "storage": wl.storage, "value": wl.cells / (ms * 1e-3) / 1e6, "unit": "MLUPS",
            "ms_per_step": ms, "steps": steps, "bulk_kernel_ms": avg_s * 1e3,
            "bulk_kernel_achieved_gbs": per_launch / avg_s / 1e9, "bulk_kernel_frac": per_launch / avg_s / 1e9 / peak,
            "rest_of_sweep_ms": rest_ms / max(1, nsw), "active_cells": n_act, "bulk_cells": n_bulk,
            "step_sweep_bytes": step_bytes, "step_frac": step_bytes / (ms * 1e-3) / 1e9 / peak, "status": st}


def _split_run(torch, lbm, args):
    """step time of the 128^3 column with bubble splitting every step and every 10 steps
    (the six labelling launches run on those steps; on the others they return at once), against
    the same workload without splitting timed alongside"""
    import dataclasses
    out = {}
    for every in (0, 1, 10):
        wl = dataclasses.replace(_workload("c1"), split_every=every, max_bubbles=16 if every else 0)
        sim = lbm.Sim(wl)
        sim.step(max(3, args.warmup))
        torch.cuda.synchronize()
        stream = torch.cuda.current_stream()
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        n = min(args.steps, 2000)
        e0.record(stream)
        sim.step(n)
        e1.record(stream)
        torch.cuda.synchronize()
        ms = e0.elapsed_time(e1) / n
        out["every_%d" % every if every else "off"] = {"ms_per_step": ms, "status": sim.status(),
                                                       "splits": sim.bubble_splits()[1] if every else 0}
        sim.close()
    off = out["off"]["ms_per_step"]
    for k in ("every_1", "every_10"):
        out[k]["overhead_ms"] = out[k]["ms_per_step"] - off
    return out


def _adjoint_run(torch, lbm, W, window=True, graphs=True):
    """the differentiation path on the 96^3 periodic array of 27 fixed spheres: per-launch
    time and HBM roofline of the frozen replay step and of the reverse step, and the wall time
    of a 500-step window gradient (forward with checkpoints every 50, replay, reverse)"""
    from paper_1712_07028_gb300 import adjoint as A
    wl = W.periodic_array_c2()
    sim = lbm.Sim(wl)
    sim.step(0)
    st = sim.export_state()
    n_liq = int((st["flags"] == lbm.CELL_LIQUID).sum().item())
    # four states (268 MB, twice the L2) so that every call streams its operands from HBM
    fs = [st["f"]] + [torch.empty_like(st["f"]) for _ in range(3)]
    la, lb = torch.zeros_like(fs[0]), torch.zeros_like(fs[0])
    stream = torch.cuda.current_stream()
    e0 = torch.cuda.Event(enable_timing=True)
    e1 = torch.cuda.Event(enable_timing=True)
    k, reps = 50, 8

    def timed(fn):
        """seconds per call of fn (four of the timed steps): k calls captured in a
        CUDA graph (the library forks its second stream inside the capture), replayed after
        warm-up, so that host-side call overhead does not enter the kernel time"""
        for _ in range(5):
            fn()
        torch.cuda.synchronize()
        if not graphs:   # a few plain calls only (for a profiler's launch list)
            return float("nan")
        g = torch.cuda.CUDAGraph()
        with torch.cuda.graph(g):
            for _ in range(k):
                fn()
        g.replay()
        torch.cuda.synchronize()
        e0.record(stream)
        for _ in range(reps):
            g.replay()
        e1.record(stream)
        torch.cuda.synchronize()
        return e0.elapsed_time(e1) / (k * reps) * 1e-3

    def fwd():
        for j in range(4):
            sim.forward_frozen(fs[j], fs[(j + 1) % 4])

    def rev():
        for j in range(4):
            sim.adjoint_step(fs[3 - j], la if j % 2 == 0 else lb, lb if j % 2 == 0 else la, (1.0, 0.0, 0.0))

    t_f = timed(fwd) / 4
    t_r = timed(rev) / 4
    peak, kind = _peak_hbm()
    inactive = wl.cells - n_liq
    by_f = n_liq * (2 * 19 * 4 + 1) + inactive
    by_r = n_liq * (3 * 19 * 4 + 1) + inactive
    sim.close()
    out = {"workload": wl.name, "liquid_cells": n_liq,
           "replay_step": {"ms": t_f * 1e3, "bytes": by_f, "achieved": by_f / t_f / 1e9, "unit": "GB/s",
                           "frac": by_f / t_f / 1e9 / peak, "peak_source": kind},
           "reverse_step": {"ms": t_r * 1e3, "bytes": by_r, "achieved": by_r / t_r / 1e9, "unit": "GB/s",
                            "frac": by_r / t_r / 1e9 / peak, "peak_source": kind}}
    if not window:
        return out
    n, every = 500, 50
    sim = lbm.Sim(wl)
    sim.step(0)
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    J, dtau, dg = A.window_gradient(sim, n, (1.0, 0.0, 0.0), every)
    torch.cuda.synchronize()
    t_win = time.perf_counter() - t0
    sim.close()
    out["window"] = {"steps": n, "checkpoint_every": every, "seconds": t_win, "mlups": wl.cells * n / t_win / 1e6,
                     "includes": "forward steps with the objective accumulated on the device and checkpoints, replay, reverse",
                     "J": J, "dJ_dtau": dtau, "dJ_dg": list(dg)}
    return out


def run_reference(args):
    ws, rank, _ = _dist()
    if rank != 0:
        return 0
    import oracle
    oracle.build()
    full = _workload(args.workload, args.storage)
    wl = _cpu_sample(args.workload)
    # each timed step is one full oracle step of the sample (the column, or its sub-box at the
    # column's densities); the number of executed steps is capped so the run stays within
    # about a minute
    o = oracle.Sim(wl)
    t = time.perf_counter()
    o.step(1)
    t_step = time.perf_counter() - t
    warm = max(0, min(args.warmup, 2) - 1)
    o.step(warm)
    k = max(1, min(args.steps, int(60.0 / max(t_step, 1e-3))))
    t0 = time.perf_counter()
    o.step(k)
    dt = time.perf_counter() - t0
    v = wl.cells * k / dt / 1e6
    what = ("the whole column" if wl.cells == full.cells else "a %dx%dx%d sub-box of the column (%d bubbles, %d spheres)"
            % (wl.nx, wl.ny, wl.nz, len(wl.bubbles), len(wl.spheres)))
    line = {"metric": METRIC, "value": v, "unit": "MLUPS", "impl": "reference", "n_gpus": args.gpus,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": dt / k * 1e3 * full.cells / wl.cells,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
            "config": {"workload": full.name, "grid": [full.nx, full.ny, full.nz], "bubbles": len(full.bubbles),
                       "spheres": len(full.spheres), "storage": "f64 (oracle)", "parallelism": "replicas"},
            "cpu_baseline": {"value": v, "unit": "MLUPS", "cores": 1, "kind": "oracle", "cpu": _cpu_model(),
                             "nproc": os.cpu_count(),
                             "sample": "%d of %d requested steps of %s executed after %d warm-up (each a full FP64 "
                                       "oracle step of %d cells); ms_per_step scaled to the column's %d cells"
                                       % (k, args.steps, what, warm + 1, wl.cells, full.cells)},
            "e2e": {"value": v, "unit": "MLUPS", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line))
    return 0


def run_gpu(args):
    import torch
    ws, rank, local = _dist()
    torch.cuda.set_device(local)
    dist = None
    if ws > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl", device_id=torch.device("cuda", local))
    from paper_1712_07028_gb300 import lbm
    from paper_1712_07028_gb300 import workloads as W
    lbm.load()
    wl = _workload(args.workload, args.storage)
    if args.split_every > 0:
        wl.split_every, wl.max_bubbles = args.split_every, max(16, len(wl.bubbles))
    s_bytes = 4 if wl.storage == "f32" else 2

    def barrier():
        if dist is not None:
            dist.barrier()

    sim = lbm.Sim(wl)
    sim.step(max(3, args.warmup))
    torch.cuda.synchronize()
    barrier()
    clocks = Clocks(_gpu_index(torch, local))
    clocks.start()
    stream = torch.cuda.current_stream()
    e0 = torch.cuda.Event(enable_timing=True)
    e1 = torch.cuda.Event(enable_timing=True)
    n0 = sim.launches()
    torch.cuda.synchronize()
    barrier()
    e0.record(stream)
    sim.step(args.steps)
    e1.record(stream)
    torch.cuda.synchronize()
    barrier()
    clk = clocks.stop()
    launches = sim.launches() - n0
    ms = _job_ms(dist, e0.elapsed_time(e1), "cuda")
    st = sim.status()
    value = _job_mlups(wl.cells, args.steps, ws, ms)

    line = {"metric": METRIC, "value": value, "unit": "MLUPS", "n_gpus": ws, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": ms / args.steps, "higher_is_better": True, "scaling": "weak",
            "vs_baseline": None, "dtype": "f32" if wl.storage == "f32" else "f32 (" + wl.storage + " storage)",
            "data": "synthetic",
            "config": {"workload": wl.name, "grid": [wl.nx, wl.ny, wl.nz], "bubbles": len(wl.bubbles),
                       "spheres": len(wl.spheres), "storage": wl.storage, "tau": wl.tau, "g": list(wl.g),
                       "l2": "inputs larger than L2 (PDF grids %.0f MB each)" % (19 * wl.cells * s_bytes / 1e6),
                       "parallelism": "replicas" if ws > 1 else "single GPU"},
            "gpu_launches": launches, "clocks": clk, "status": st}

    if not args.no_extras:
        # roofline of the dominant kernel (the bulk sweep): CUDA events around each launch
        sim.profile(True)
        kp = min(args.steps, 100)
        sim.step(kp)
        torch.cuda.synchronize()
        bulk_ms, rest_ms, nsw = sim.profile_read()
        sim.profile(False)
        fl = sim.fields()["flags"]
        n_act = int(((fl == lbm.CELL_LIQUID) | (fl == lbm.CELL_INTERFACE)).sum().item())
        n_bulk = _bulk_cells(torch, lbm, fl, wl.bc)
        del fl
        per_launch = n_bulk * (38 * s_bytes + 1) + (wl.cells - n_bulk) * 1
        avg_s = bulk_ms / max(1, nsw) * 1e-3
        rest_s = rest_ms / max(1, nsw) * 1e-3
        peak, peak_kind = _peak_hbm()
        achieved = per_launch / avg_s / 1e9
        tr = NCU_TRAFFIC.get(wl.name + "/" + wl.storage)
        traffic = tr["bytes_per_launch"] if tr and tr["sha1"] == _sweep_sha() else None
        step_bytes = n_act * (38 * s_bytes + 1) + (wl.cells - n_act)
        line["roofline"] = {"bound": "hbm", "achieved": achieved, "peak": peak, "unit": "GB/s",
                            "frac": achieved / peak, "traffic": traffic, "peak_source": peak_kind,
                            "kernel": "sweep_bulk_kernel (concurrent with the previous step's end-of-step kernels)",
                            "algorithmic_bytes_per_launch": per_launch, "bulk_cells": n_bulk, "active_cells": n_act,
                            "avg_launch_ms": avg_s * 1e3, "launches_timed": nsw,
                            "rest_of_sweep_ms": rest_s * 1e3,
                            "step_sweep_bytes": step_bytes,
                            "step_frac": step_bytes / (ms / args.steps * 1e-3) / 1e9 / peak}
        sim.close()
        del sim
        torch.cuda.synchronize()

        # end to end through the public API from host inputs: context and tables from the host,
        # every step followed by the device->host read of the sphere forces (synchronising), the
        # fields copied to host at the end
        ke = min(args.steps, 1000) if wl.cells <= 2_200_000 else args.steps
        # page-locked host buffers for the final fields, allocated before the timed region (as a
        # caller that keeps them across runs would)
        shp = (wl.nz, wl.ny, wl.nx)
        host = {"rho": torch.empty(shp, dtype=torch.float32, pin_memory=True),
                "u": torch.empty((3,) + shp, dtype=torch.float32, pin_memory=True),
                "phi": torch.empty(shp, dtype=torch.float32, pin_memory=True),
                "flags": torch.empty(shp, dtype=torch.uint8, pin_memory=True)}
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        sim2 = lbm.Sim(wl)
        for _ in range(ke):
            sim2.step(1)
            sim2.forces()
        for k, v in sim2.fields().items():
            host[k].copy_(v, non_blocking=True)
        fields = host
        torch.cuda.synchronize()
        t1 = time.perf_counter()
        h2d, d2h = sim2.copy_bytes()
        d2h += sum(v.numel() * v.element_size() for v in fields.values())
        del fields, host
        line["e2e"] = {"value": wl.cells * ke * ws / (t1 - t0) / 1e6, "unit": "MLUPS",
                       "h2d_bytes_per_step": h2d / ke, "d2h_bytes_per_step": d2h / ke, "steps": ke,
                       "includes": "context + table upload + field init, per step lbm_step + lbm_forces "
                                   "(D2H of the sphere/bubble tables, sync), final fields D2H into page-locked "
                                   "host buffers allocated beforehand"}
        sim2.close()
        del sim2
        torch.cuda.synchronize()
        if rank == 0 and ws == 1:
            # the other columns: the 256x256x512 column in FP32 and FP16 deviations (the
            # FP32-vs-FP16 configuration) and the 128^3 column
            line["configs"] = {}
            for name, storage, k in (("c3", "f32", 300), ("c3", "f16dev", 300), ("c1", "f32", 2000),
                                     ("c1", "f16dev", 2000)):
                if name == args.workload and storage == wl.storage:
                    continue
                line["configs"]["%s_%s" % (_workload(name).name, storage)] = _config_run(torch, lbm, name, storage, k, 5)
            # bubble splitting (connected-component labelling) on the 128^3 column
            line["split"] = _split_run(torch, lbm, args)
            # the differentiation path (frozen liquid window) on its own workload
            line["adjoint"] = _adjoint_run(torch, lbm, W)
            # the CPU-baseline leg: the FP64 oracle timed on a bounded sample of the workload,
            # and the GPU path's error against it on the 32^3 column
            line["cpu_baseline"] = _cpu_baseline(args.workload)
            line["cpu_baseline"]["all_cores"] = _cpu_baseline_all_cores(args.workload)
            line["oracle_error"] = _oracle_error(torch, lbm, W)
    if rank == 0:
        print(json.dumps(line))
    if dist is not None:
        dist.barrier()
        dist.destroy_process_group()
    return 0


def main():
    args = _args()
    if args.impl == "reference":
        return run_reference(args)
    if args.only == "adjoint":
        import torch
        from paper_1712_07028_gb300 import lbm
        from paper_1712_07028_gb300 import workloads as W
        lbm.load()
        print(json.dumps(_adjoint_run(torch, lbm, W, window=not args.no_extras, graphs=not args.no_extras)))
        return 0
    return run_gpu(args)


if __name__ == "__main__":
    sys.exit(main())
