"""Seeded synthetic workloads: domain, bubbles and spheres of the bubble-particle columns.

This module only *places* things.  It holds none of the method's arithmetic, so both the
CUDA path and the CPU oracle may take their inputs from it.

Random numbers come from splitmix64 (Steele, Lea, Flood 2014) mapped to uniform doubles
by the top 53 bits.  Placement is rejection sampling, bubbles first, then spheres, with
every sampled centre rounded to integer cell coordinates (cells sit at integer
coordinates 0..n-1).  The shapes follow the paper's bubble-in-particle-bed runs
(Sec. 4: a spherical bubble rising through a random bed of resolved spheres of about five
cells per diameter) scaled to what one GPU holds.
"""
from __future__ import annotations

import dataclasses
import math
from typing import List, Tuple

_MASK = (1 << 64) - 1


class SplitMix64:
    """splitmix64 generator; ``uniform()`` returns a double in [0, 1)."""

    def __init__(self, seed: int):
        self.state = seed & _MASK

    def next_u64(self) -> int:
        self.state = (self.state + 0x9E3779B97F4A7C15) & _MASK
        z = self.state
        z = ((z ^ (z >> 30)) * 0xBF58476D1CE4E5B9) & _MASK
        z = ((z ^ (z >> 27)) * 0x94D049BB133111EB) & _MASK
        return z ^ (z >> 31)

    def uniform(self) -> float:
        return (self.next_u64() >> 11) * (1.0 / 9007199254740992.0)

    def uniform_in(self, lo: float, hi: float) -> float:
        return lo + (hi - lo) * self.uniform()


WALL, PERIODIC, FREESLIP = 0, 1, 2
STORAGE = {"f32": 0, "f16dev": 1, "bf16dev": 2}
SPHERES_FIXED, SPHERES_FREE, SPHERES_PRESCRIBED = 0, 1, 2


@dataclasses.dataclass
class Sphere:
    x: Tuple[float, float, float]
    r: float
    rho: float
    u: Tuple[float, float, float] = (0.0, 0.0, 0.0)
    w: Tuple[float, float, float] = (0.0, 0.0, 0.0)


@dataclasses.dataclass
class Bubble:
    c: Tuple[float, float, float]
    r: float


@dataclasses.dataclass
class Workload:
    name: str
    nx: int
    ny: int
    nz: int
    tau: float = 0.6
    g: Tuple[float, float, float] = (0.0, 0.0, 0.0)
    bc: Tuple[int, int, int] = (WALL, WALL, WALL)
    open_top: bool = False      # the +z face an open boundary at the reference pressure
    hydrostatic: bool = False   # (open top only) start in hydrostatic equilibrium
    split_every: int = 0        # > 0: bubbles split into their connected parts every so many steps
    max_bubbles: int = 0        # rows of the bubble table (0: the given bubbles); room for splits
    sigma: float = 0.0
    rho_g0: float = 1.0
    eps: float = 0.0
    n_substeps: int = 10
    sphere_mode: int = SPHERES_FREE
    storage: str = "f32"
    steps: int = 1
    bubbles: List[Bubble] = dataclasses.field(default_factory=list)
    spheres: List[Sphere] = dataclasses.field(default_factory=list)

    @property
    def cells(self) -> int:
        return self.nx * self.ny * self.nz

    def describe(self) -> dict:
        return {
            "workload": self.name,
            "grid": [self.nx, self.ny, self.nz],
            "tau": self.tau,
            "g": list(self.g),
            "bubbles": len(self.bubbles),
            "spheres": len(self.spheres),
            "storage": self.storage,
        }


class _Hash:
    """uniform-grid hash of sphere centres for the rejection test"""

    def __init__(self, h: float):
        self.h = h
        self.cells = {}

    def key(self, p):
        return tuple(int(math.floor(v / self.h)) for v in p)

    def near(self, p):
        k = self.key(p)
        for dz in (-1, 0, 1):
            for dy in (-1, 0, 1):
                for dx in (-1, 0, 1):
                    yield from self.cells.get((k[0] + dx, k[1] + dy, k[2] + dz), ())

    def add(self, p):
        self.cells.setdefault(self.key(p), []).append(p)


def _dist2(a, b):
    return (a[0] - b[0]) ** 2 + (a[1] - b[1]) ** 2 + (a[2] - b[2]) ** 2


def place_bubbles(rng: SplitMix64, n, r, dims, zrange, gap):
    """n bubbles of radius r, centres uniform in x,y in [r+2, n-3-r] and z in zrange,
    centre distance >= 2r + gap"""
    out = []
    for _ in range(200000):
        if len(out) == n:
            break
        c = (round(rng.uniform_in(r + 2, dims[0] - 3 - r)),
             round(rng.uniform_in(r + 2, dims[1] - 3 - r)),
             round(rng.uniform_in(zrange[0], zrange[1])))
        if all(_dist2(c, b.c) >= (2 * r + gap) ** 2 for b in out):
            out.append(Bubble(c=tuple(float(v) for v in c), r=float(r)))
    if len(out) != n:
        raise RuntimeError("bubble placement failed")
    return out


def place_spheres(rng: SplitMix64, n, R, rho, dims, bubbles, max_tries=None):
    """n spheres of radius R, centres uniform in [R+1, n-2-R] per axis; rejection keeps
    centre distances >= 2R+1 between spheres and >= r_b+R+2 to every bubble centre"""
    h = 2 * R + 1
    grid = _Hash(h)
    out = []
    tries = 0
    max_tries = max_tries or 200 * n + 1000
    while len(out) < n:
        tries += 1
        if tries > max_tries:
            raise RuntimeError("sphere placement failed after %d tries (%d placed)" % (tries, len(out)))
        c = (round(rng.uniform_in(R + 1, dims[0] - 2 - R)),
             round(rng.uniform_in(R + 1, dims[1] - 2 - R)),
             round(rng.uniform_in(R + 1, dims[2] - 2 - R)))
        if any(_dist2(c, b.c) < (b.r + R + 2) ** 2 for b in bubbles):
            continue
        if any(_dist2(c, o) < h * h for o in grid.near(c)):
            continue
        grid.add(c)
        out.append(Sphere(x=tuple(float(v) for v in c), r=float(R), rho=float(rho)))
    return out


def column_c0() -> Workload:
    """32^3, walls, tau 0.6, gravity 1e-5 along -z, one gas bubble r=6 at (16,16,10) and one
    sphere r=3 of density 2.0 at (16,16,22), 200 steps"""
    return Workload(name="column32_bubble_sphere", nx=32, ny=32, nz=32, tau=0.6, g=(0.0, 0.0, -1e-5),
                    steps=200, bubbles=[Bubble((16.0, 16.0, 10.0), 6.0)],
                    spheres=[Sphere((16.0, 16.0, 22.0), 3.0, 2.0)])


def column_c1() -> Workload:
    """128^3 FP32, walls, gravity 1e-6, one bubble r=16 at (64,64,32), 64 spheres r=4 of
    density 1.5, seed 1, 2000 steps"""
    dims = (128, 128, 128)
    rng = SplitMix64(1)
    bubbles = [Bubble((64.0, 64.0, 32.0), 16.0)]
    spheres = place_spheres(rng, 64, 4, 1.5, dims, bubbles)
    return Workload(name="column128_1bubble_64spheres", nx=128, ny=128, nz=128, tau=0.6, g=(0.0, 0.0, -1e-6),
                    steps=2000, bubbles=bubbles, spheres=spheres)


def periodic_array_c2() -> Workload:
    """96^3 periodic, liquid only, 27 static spheres r=4 on a jittered 32-lattice (seed 2),
    body force 1e-5 along +x, 500-step window"""
    rng = SplitMix64(2)
    spheres = []
    for k in range(3):
        for j in range(3):
            for i in range(3):
                c = tuple(float(round(16 + 32 * a + rng.uniform_in(-2.0, 2.0))) for a in (i, j, k))
                spheres.append(Sphere(c, 4.0, 1.5))
    return Workload(name="periodic96_27spheres", nx=96, ny=96, nz=96, tau=0.6, g=(1e-5, 0.0, 0.0),
                    bc=(PERIODIC, PERIODIC, PERIODIC), sphere_mode=SPHERES_FIXED, steps=500,
                    spheres=spheres)


def column_c3(storage="f32") -> Workload:
    """256x256x512, walls, gravity 1e-6, 8 bubbles r=16 in z in [40,256] (gap >= 8),
    20000 spheres r=4 of density 1.5, seed 3, 5000 steps"""
    dims = (256, 256, 512)
    rng = SplitMix64(3)
    bubbles = place_bubbles(rng, 8, 16, dims, (40, 256), 8)
    spheres = place_spheres(rng, 20000, 4, 1.5, dims, bubbles)
    return Workload(name="column256x256x512_8bubbles_20000spheres", nx=256, ny=256, nz=512, tau=0.6,
                    g=(0.0, 0.0, -1e-6), steps=5000, bubbles=bubbles, spheres=spheres, storage=storage)


def column_c4(storage="f16dev") -> Workload:
    """512x512x1024, FP16-deviation storage, gravity 1e-6, 32 bubbles r=24 in z in [56,512],
    100000 spheres r=4 of density 1.5, seed 4, 2000 steps"""
    dims = (512, 512, 1024)
    rng = SplitMix64(4)
    bubbles = place_bubbles(rng, 32, 24, dims, (56, 512), 8)
    spheres = place_spheres(rng, 100000, 4, 1.5, dims, bubbles)
    return Workload(name="column512x512x1024_32bubbles_100000spheres", nx=512, ny=512, nz=1024, tau=0.6,
                    g=(0.0, 0.0, -1e-6), steps=2000, bubbles=bubbles, spheres=spheres, storage=storage)


def liquid_box(n=32, bc=(WALL, WALL, WALL), g=(0.0, 0.0, 0.0), tau=0.6, name=None) -> Workload:
    """an all-liquid box, the simplest case of the sweep"""
    return Workload(name=name or "liquid%d" % n, nx=n, ny=n, nz=n, tau=tau, g=g, bc=bc)


# Sec. 3.2, Table 1: single rising bubbles in four shape regimes, parameterised by the liquid
# viscosity mu [Pa s], surface tension sigma [N/m] and gravity g [m/s^2] for a liquid of
# density 1000 kg/m^3, with dx = 1e-3 m and dt = 1e-4 s; the FSLBM's terminal Reynolds number
# Re_b* in the 40 x 40 x 100 column (free-slip sides, no-slip bottom, open top), and the
# figures' end times (steps)
RISING_BUBBLE_CASES = {
    "A": dict(mu=0.25, sigma=0.145, g=0.981, re_star=1.76, steps=20000, regime="spherical"),
    "B": dict(mu=0.42, sigma=0.145, g=9.81, re_star=4.43, steps=5000, regime="ellipsoidal"),
    "C": dict(mu=0.13211, sigma=0.014545, g=9.81, re_star=14.53, steps=4000, regime="skirted"),
    "D": dict(mu=0.75, sigma=0.014545, g=9.81, re_star=1.46, steps=8000, regime="dimpled"),
}
RISING_DX, RISING_DT, RISING_RHO = 1e-3, 1e-4, 1000.0


def rising_bubble_lattice(case: str):
    """(tau, g, sigma) in lattice units of a Table 1 case: nu = mu/rho dt/dx^2 and
    tau = 3 nu + 1/2 (Eq. latticeViscosity), g dt^2/dx, sigma/rho dt^2/dx^3"""
    c = RISING_BUBBLE_CASES[case]
    nu = c["mu"] / RISING_RHO * RISING_DT / RISING_DX ** 2
    return 3.0 * nu + 0.5, c["g"] * RISING_DT ** 2 / RISING_DX, c["sigma"] / RISING_RHO * RISING_DT ** 2 / RISING_DX ** 3


def rising_bubble(case: str, n=(40, 40, 100), r=6.0, zc=9.5, storage="f32") -> Workload:
    """Sec. 3.2 / Fig. bubbleSetup: a spherical bubble of radius r = 6 dx centred at
    (20, 20, 10) dx (cell centres at integer coordinates from 0: the point (19.5, 19.5, 9.5))
    in a quiescent liquid column, free-slip sides, no-slip bottom, open top; gravity along -z.
    The column starts in hydrostatic equilibrium and the gas at the pressure around it (at
    rest, as the paper's quiescent liquid)"""
    tau, g, sigma = rising_bubble_lattice(case)
    nx, ny, nz = n
    return Workload(name="rising_bubble_%s" % case, nx=nx, ny=ny, nz=nz, tau=tau, g=(0.0, 0.0, -g),
                    bc=(FREESLIP, FREESLIP, WALL), open_top=True, hydrostatic=True, sigma=sigma,
                    sphere_mode=SPHERES_FIXED,
                    steps=RISING_BUBBLE_CASES[case]["steps"], storage=storage,
                    bubbles=[Bubble((nx / 2 - 0.5, ny / 2 - 0.5, zc), r)])


# Sec. 4.1, Fig. bubbleParticle: a bubble of radius 0.01 m rising through a homogeneous bed of
# spheres of radius 8e-4 m (5 cells per diameter at dx = 8e-5 m, as the paper resolves them),
# solid density 3000 kg/m^3, sigma 0.145 N/m, g 0.981 m/s^2, liquid 1000 kg/m^3 and
# mu 0.25 kg/(m s); the paper's dimensionless terminal rise velocity u (rho/(sigma g))^(1/4)
# at bed solid fractions Phi = N V_P / (V - V_b)
BUBBLE_BED_VELOCITY = {0.0: 0.53687069058757, 0.01: 0.54376978332139, 0.03: 0.52166135018381,
                       0.05: 0.50675825176692, 0.075: 0.48794013951139, 0.1: 0.47890956185243}
BED = dict(R=0.01, R_P=8e-4, rho=1000.0, rho_s=3000.0, mu=0.25, sigma=0.145, g=0.981, dx=8e-5,
           n=(500, 500, 1300), c=(250, 250, 250))


def bubble_bed_lattice(scale: int, dt: float):
    """(dx, tau, g, sigma) in lattice units of the bed run coarsened `scale` times (dx grows,
    the bubble and the domain keep their sizes in metres), time step dt [s]"""
    dx = BED["dx"] * scale
    nu = BED["mu"] / BED["rho"] * dt / dx ** 2
    return dx, 3.0 * nu + 0.5, BED["g"] * dt ** 2 / dx, BED["sigma"] / BED["rho"] * dt ** 2 / dx ** 3


def bubble_in_bed(phi: float, scale: int = 5, dt: float = 1.36e-4, r_p_cells: float = 2.5, seed: int = 7,
                  storage: str = "f32") -> Workload:
    """Fig. bubbleParticle's run coarsened `scale` times: the domain (500 x 500 x 1300 cells at
    dx = 8e-5 m) and the bubble (radius 0.01 m at (250, 250, 250) dx) keep their sizes in metres;
    the particles keep the paper's resolution of 5 cells per diameter (radius r_p_cells), so
    their radius in metres grows with the scale.  N = Phi (V - V_b) / V_P spheres (the paper's
    Phi), placed uniformly at random (seeded, rejection as in the columns); free spheres of
    density 3, the column's boundaries and start those of the rising-bubble runs (free-slip
    sides, no-slip bottom, open top, hydrostatic start).  dt sets the lattice viscosity and
    the expected rise velocity (1.36e-4 s at scale 5: tau = 1.14, u ~ 0.02 cells per step)."""
    dx, tau, g, sigma = bubble_bed_lattice(scale, dt)
    nx, ny, nz = (v // scale for v in BED["n"])
    R = BED["R"] / dx
    c = tuple(float(v) / scale - 0.5 for v in BED["c"])
    bub = Bubble(c, R)
    V = nx * ny * nz - 4.0 / 3.0 * math.pi * R ** 3
    n = int(round(phi * V / (4.0 / 3.0 * math.pi * r_p_cells ** 3)))
    rng = SplitMix64(seed)
    sph = place_spheres(rng, n, r_p_cells, BED["rho_s"] / BED["rho"], (nx, ny, nz), [bub]) if n else []
    return Workload(name="bubble_bed_phi%g" % phi, nx=nx, ny=ny, nz=nz, tau=tau, g=(0.0, 0.0, -g),
                    bc=(FREESLIP, FREESLIP, WALL), open_top=True, hydrostatic=True, sigma=sigma,
                    sphere_mode=SPHERES_FREE, storage=storage, bubbles=[bub], spheres=sph)


def sub_box(wl: Workload, lo: Tuple[int, int, int], size: Tuple[int, int, int], name: str = None) -> Workload:
    """the part of a column inside the box [lo, lo + size) as a workload of its own (walls on
    every face): the spheres whose centres keep the placement margin R + 1 inside the box and
    the bubbles whose centres keep r + 2, shifted by -lo; the same densities of spheres and
    bubbles as the column, at a size a CPU can step (a bounded sample of a large column)"""
    def inside(c, m):
        return all(lo[k] + m <= c[k] <= lo[k] + size[k] - 1 - m for k in range(3))

    sph = [dataclasses.replace(s, x=tuple(s.x[k] - lo[k] for k in range(3))) for s in wl.spheres if inside(s.x, s.r + 1)]
    bub = [Bubble(tuple(b.c[k] - lo[k] for k in range(3)), b.r) for b in wl.bubbles if inside(b.c, b.r + 2)]
    return dataclasses.replace(wl, name=name or "%s_box%dx%dx%d" % (wl.name, *size), nx=size[0], ny=size[1], nz=size[2],
                               bc=(WALL, WALL, WALL), bubbles=bub, spheres=sph)

