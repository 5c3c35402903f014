"""Seeded synthetic inputs for the shallow-water time step.

This module is the only code shared by the FP64 CPU oracle and the CUDA
library, and it holds none of the scheme's arithmetic: it only produces input
data (terrain b, Manning n_M, initial depth and momentum, source lists and
hydrograph parameters).  Every random number comes from one counter-based
generator, SplitMix64 (S. Vigna's published finaliser), so a given
(seed, stream, index) triple maps to the same value on any machine.

The paper's own inputs (the Volga-Akhtuba digital elevation model, the
May 2011 hydrograph, the emergency-discharge scenario; Sec. 2.2 and Sec. 5)
are not available, so seeded stand-ins with the same shape are produced here:
fractal relief of 0-30 m (the depth range of Sec. 2.2), a carved river
channel, patchy Manning roughness and a Gaussian inflow hydrograph feeding a
strip of source cells (the sigma of Eq. 1).
"""
from __future__ import annotations

import dataclasses
import math
from typing import Optional

import numpy as np

_M64 = np.uint64(0xFFFFFFFFFFFFFFFF)
_GOLDEN = np.uint64(0x9E3779B97F4A7C15)
_MIX1 = np.uint64(0xBF58476D1CE4E5B9)
_MIX2 = np.uint64(0x94D049BB133111EB)

# Bed elevation given to cells that act as walls (closed gates).  The library
# adds a ring of such cells around every grid; the value only has to exceed
# any water level by far and stay finite in FP32.
WALL_BED = 1.0e30

# Terrain is quantised to multiples of 2**-10 m so that H = eta0 - b and
# H + b == eta0 hold exactly in FP32 and FP64 (lake-at-rest inputs).
BED_QUANTUM = 2.0 ** -10


def splitmix64(x: np.ndarray) -> np.ndarray:
    """SplitMix64 finaliser applied elementwise to uint64 counters."""
    z = (np.asarray(x, dtype=np.uint64) + _GOLDEN)
    z = (z ^ (z >> np.uint64(30))) * _MIX1
    z = (z ^ (z >> np.uint64(27))) * _MIX2
    return z ^ (z >> np.uint64(31))


def uniform(seed: int, stream: int, idx) -> np.ndarray:
    """Uniform doubles in [0, 1) for counters ``idx`` of (seed, stream)."""
    with np.errstate(over="ignore"):
        key = splitmix64(np.uint64(seed & 0xFFFFFFFF) << np.uint64(32)
                         | np.uint64(stream & 0xFFFFFFFF))
        z = splitmix64(key + np.asarray(idx, dtype=np.uint64))
    return (z >> np.uint64(11)).astype(np.float64) * (1.0 / 9007199254740992.0)


def diamond_square(k: int, seed: int, roughness: float = 0.5) -> np.ndarray:
    """Fractal height field on a (2**k + 1)^2 grid by the diamond-square
    midpoint-displacement method (Fournier, Fussell & Carpenter 1982).

    Each grid point receives exactly one random displacement, drawn from the
    counter equal to its linear index, so the field is reproducible and
    independent of evaluation order.  Amplitude shrinks by ``roughness`` per
    level.  Returns float64 array [y, x].
    """
    n = (1 << k) + 1
    z = np.zeros((n, n), dtype=np.float64)

    def rnd(yy, xx):
        return 2.0 * uniform(seed, 1, yy.astype(np.uint64) * np.uint64(n)
                             + xx.astype(np.uint64)) - 1.0

    c = np.array([0, n - 1])
    cy, cx = np.meshgrid(c, c, indexing="ij")
    z[np.ix_(c, c)] = rnd(cy, cx)
    s = n - 1
    amp = 1.0
    while s > 1:
        h = s // 2
        amp *= roughness
        # diamond step: square centres
        cen = 0.25 * (z[0:-1:s, 0:-1:s] + z[0:-1:s, s::s] + z[s::s, 0:-1:s] + z[s::s, s::s])
        ys = np.arange(h, n, s)
        yy, xx = np.meshgrid(ys, ys, indexing="ij")
        z[h::s, h::s] = cen + amp * rnd(yy, xx)
        # square step, lattice A: rows 0::s, columns h::s
        acc = z[0::s, 0:-1:s] + z[0::s, s::s]
        cnt = np.full(acc.shape, 2.0)
        acc[1:, :] += z[h::s, h::s]
        cnt[1:, :] += 1.0
        acc[:-1, :] += z[h::s, h::s]
        cnt[:-1, :] += 1.0
        yy, xx = np.meshgrid(np.arange(0, n, s), np.arange(h, n, s), indexing="ij")
        z[0::s, h::s] = acc / cnt + amp * rnd(yy, xx)
        # square step, lattice B: rows h::s, columns 0::s
        acc = z[0:-1:s, 0::s] + z[s::s, 0::s]
        cnt = np.full(acc.shape, 2.0)
        acc[:, 1:] += z[h::s, h::s]
        cnt[:, 1:] += 1.0
        acc[:, :-1] += z[h::s, h::s]
        cnt[:, :-1] += 1.0
        yy, xx = np.meshgrid(np.arange(h, n, s), np.arange(0, n, s), indexing="ij")
        z[h::s, 0::s] = acc / cnt + amp * rnd(yy, xx)
        s = h
    return z


def quantise_bed(b: np.ndarray) -> np.ndarray:
    return np.round(np.asarray(b, dtype=np.float64) / BED_QUANTUM) * BED_QUANTUM


@dataclasses.dataclass
class Hydrograph:
    """Inflow law q(t) [m/s]: kind 0 = Gaussian peak*exp(-(t-tp)^2/(2 s^2)),
    kind 1 = constant peak."""
    kind: int
    peak: float
    tp: float = 0.0
    s: float = 1.0

    def as_row(self):
        return [float(self.kind), float(self.peak), float(self.tp), float(self.s)]


@dataclasses.dataclass
class Sources:
    """Sparse source/drain cells (sigma and V of Eqs. 1-3).

    sigma at cell k is ``weight[k] * q_{hydro[k]}(t)``; ``vx, vy`` is the
    velocity V of the water entering there.  Cells must be distinct.
    """
    ix: np.ndarray
    iy: np.ndarray
    weight: np.ndarray
    vx: np.ndarray
    vy: np.ndarray
    hydro: np.ndarray
    hydrographs: list

    @staticmethod
    def empty() -> "Sources":
        z = np.zeros(0)
        zi = np.zeros(0, dtype=np.int32)
        return Sources(zi, zi, z, z, z, zi, [])

    def __len__(self):
        return int(len(self.ix))

    def hydro_table(self) -> np.ndarray:
        if not self.hydrographs:
            return np.zeros((0, 4))
        return np.array([h.as_row() for h in self.hydrographs], dtype=np.float64)


@dataclasses.dataclass
class Params:
    """Physical and numerical parameters of one grid (Eqs. 1-4, Fig. 2)."""
    nx: int
    ny: int
    dx: float
    g: float = 9.81
    cfl: float = 0.3
    eps: float = 1.0e-4
    dt_max: float = 1.0
    dt_fixed: float = 0.0
    nu: float = 0.0
    coriolis_f: float = 0.0
    wind_x: float = 0.0
    wind_y: float = 0.0
    c_a: float = 0.0
    rho_air_over_rho: float = 1.225e-3
    # distributed sources of Eq. 1 (m/s, uniform over the grid): rainfall,
    # evaporation, infiltration
    rain_rate: float = 0.0
    evap_rate: float = 0.0
    infil_rate: float = 0.0


@dataclasses.dataclass
class Problem:
    """One seeded scenario: parameters, statics, initial state, sources."""
    name: str
    params: Params
    b: np.ndarray          # [ny, nx] bed elevation (m)
    n_manning: np.ndarray  # [ny, nx] Manning coefficient
    H: np.ndarray          # [ny, nx] depth (m)
    Qx: np.ndarray         # [ny, nx] momentum H*Ux (m^2/s), the paper's HV
    Qy: np.ndarray
    sources: Sources
    solid: Optional[np.ndarray] = None  # [ny, nx] uint8, 1 = closed gate (wall)
    t0: float = 0.0

    def to_f32_values(self) -> "Problem":
        """Round every floating input to the nearest FP32 value (kept in
        float64 arrays) so an FP32 run and the FP64 oracle see equal inputs."""
        r = lambda a: np.asarray(a, dtype=np.float32).astype(np.float64)
        s = self.sources
        src = Sources(s.ix, s.iy, r(s.weight), r(s.vx), r(s.vy), s.hydro, s.hydrographs)
        return dataclasses.replace(self, b=r(self.b), n_manning=r(self.n_manning), H=r(self.H),
                                   Qx=r(self.Qx), Qy=r(self.Qy), sources=src)


# ---------------------------------------------------------------- terrains

def fractal_terrain(nx: int, ny: int, seed: int, relief: float = 30.0,
                    roughness: float = 0.5) -> np.ndarray:
    """Seeded diamond-square relief cropped to [ny, nx], scaled to [0, relief]."""
    k = 1
    while (1 << k) + 1 < max(nx, ny):
        k += 1
    z = diamond_square(k, seed, roughness)[:ny, :nx]
    lo, hi = float(z.min()), float(z.max())
    b = relief * (z - lo) / (hi - lo if hi > lo else 1.0)
    return b


def channel_centre_y(x: np.ndarray, length_y: float, length_x: float) -> np.ndarray:
    """Sinuous centreline y_c(x) = Ly/2 + (Ly/8) sin(2 pi x / (Lx/2))."""
    return 0.5 * length_y + 0.125 * length_y * np.sin(2.0 * np.pi * x / (0.5 * length_x))


def carve_channel(b: np.ndarray, dx: float, width: float = 40.0, depth_below: float = 2.0,
                  slope: float = 1.0e-4) -> np.ndarray:
    """Carve a sinuous channel of the given width into ``b``.

    The channel bed lies ``depth_below`` under the lowest terrain point and
    falls by ``slope`` per metre in +x (water enters at the left edge)."""
    ny, nx = b.shape
    b = b.copy()
    xc = (np.arange(nx) + 0.5) * dx
    yc = channel_centre_y(xc, ny * dx, nx * dx)
    yy = (np.arange(ny) + 0.5) * dx
    bmin = float(b.min())
    bed = bmin - depth_below - slope * xc
    mask = np.abs(yy[:, None] - yc[None, :]) <= 0.5 * width
    b[mask] = np.broadcast_to(bed[None, :], b.shape)[mask]
    return b


def manning_patches(nx: int, ny: int, seed: int, patch: int = 64,
                    lo: float = 0.02, hi: float = 0.05) -> np.ndarray:
    """Manning n uniform in [lo, hi] per patch x patch block of cells."""
    px = (nx + patch - 1) // patch
    py = (ny + patch - 1) // patch
    vals = lo + (hi - lo) * uniform(seed, 2, np.arange(px * py)).reshape(py, px)
    return np.repeat(np.repeat(vals, patch, axis=0), patch, axis=1)[:ny, :nx].copy()


def source_strip(nx: int, ny: int, dx: float, ncells: int = 100, col: int = 2,
                 hydro: Optional[Hydrograph] = None) -> Sources:
    """A column strip of ``ncells`` source cells at x index ``col`` centred on
    the channel; the hydrograph value is shared equally (weight 1/ncells)."""
    ncells = min(ncells, ny)
    yc = float(channel_centre_y(np.array([(col + 0.5) * dx]), ny * dx, nx * dx)[0])
    jc = int(yc // dx)
    j0 = min(max(jc - ncells // 2, 0), ny - ncells)
    iy = np.arange(j0, j0 + ncells, dtype=np.int32)
    ix = np.full(ncells, col, dtype=np.int32)
    w = np.full(ncells, 1.0 / ncells)
    z = np.zeros(ncells)
    if hydro is None:
        hydro = Hydrograph(0, 5.0, 60.0, 20.0)
    return Sources(ix, iy, w, z.copy(), z.copy(), np.zeros(ncells, dtype=np.int32), [hydro])


# ---------------------------------------------------------------- problems

def dam_break(n: int = 256, dx: float = 1.0, h_left: float = 2.0, h_right: float = 1.0,
              x0: Optional[float] = None, ny: Optional[int] = None, cfl: float = 0.3) -> Problem:
    """1-D dam break along x on a flat frictionless bed with walls:
    H = h_left for cell centres x < x0, else h_right; U = 0."""
    ny = n if ny is None else ny
    x0 = 0.5 * n * dx if x0 is None else x0
    xc = (np.arange(n) + 0.5) * dx
    H = np.where(xc < x0, h_left, h_right)[None, :].repeat(ny, axis=0).astype(np.float64)
    z = np.zeros((ny, n))
    p = Params(nx=n, ny=ny, dx=dx, cfl=cfl, dt_max=10.0)
    return Problem("dam_break", p, z.copy(), z.copy(), H, z.copy(), z.copy(), Sources.empty())


def lake_at_rest(n: int, dx: float, seed: int, eta0: float = 10.0, relief: float = 30.0,
                 nu: float = 1.0, coriolis_f: float = 1.08382e-4) -> Problem:
    """Still water at level eta0 over fractal terrain with dry islands."""
    b = quantise_bed(fractal_terrain(n, n, seed, relief))
    H = np.maximum(0.0, eta0 - b)
    z = np.zeros_like(b)
    nm = manning_patches(n, n, seed + 1)
    p = Params(nx=n, ny=n, dx=dx, nu=nu, coriolis_f=coriolis_f)
    return Problem("lake_at_rest", p, b, nm, H, z.copy(), z.copy(), Sources.empty())


def thacker_bowl(n: int, half_width: float = 2.0, a: float = 1.0, h0: float = 0.1,
                 amp: float = 0.5, g: float = 9.81) -> Problem:
    """Planar free surface oscillating in a paraboloid bowl b = h0 r^2/a^2,
    initial data at t = 0: eta = h0 + (2 A h0/a^2) x, U = (0, A omega)."""
    dx = 2.0 * half_width / n
    xc = -half_width + (np.arange(n) + 0.5) * dx
    X, Y = np.meshgrid(xc, xc, indexing="xy")
    b = h0 * (X * X + Y * Y) / (a * a)
    omega = math.sqrt(2.0 * g * h0) / a
    eta = h0 + 2.0 * amp * h0 / (a * a) * X
    H = np.maximum(0.0, eta - b)
    Qx = np.zeros_like(H)
    Qy = H * (amp * omega)
    z = np.zeros_like(H)
    p = Params(nx=n, ny=n, dx=dx, g=g, dt_max=1.0, eps=1.0e-6)
    return Problem("thacker", p, b, z, H, Qx, Qy, Sources.empty())


def floodplain(n: int, dx: float, terrain_seed: int, manning_seed: int,
               hydro: Optional[Hydrograph] = None, ny: Optional[int] = None,
               nsrc: int = 100) -> Problem:
    """Fractal floodplain with a carved 40 m channel, patchy Manning n,
    viscosity 1 m^2/s, Coriolis at 48 N, 10 m/s east wind (C_a = 1.3e-3),
    a 100-cell source strip fed by a Gaussian hydrograph, dry start."""
    ny = n if ny is None else ny
    b = fractal_terrain(n, ny, terrain_seed)
    b = quantise_bed(carve_channel(b, dx))
    nm = manning_patches(n, ny, manning_seed)
    z = np.zeros((ny, n))
    src = source_strip(n, ny, dx, ncells=nsrc, hydro=hydro)
    f48 = 2.0 * 7.2921159e-5 * math.sin(math.radians(48.0))
    p = Params(nx=n, ny=ny, dx=dx, nu=1.0, coriolis_f=f48, wind_x=10.0, wind_y=0.0,
               c_a=1.3e-3, rho_air_over_rho=1.225e-3, cfl=0.3, eps=1.0e-4, dt_max=1.0)
    return Problem("floodplain", p, b, nm, z.copy(), z.copy(), z.copy(), src)


def random_wet_dry(nx: int, ny: int, seed: int, dx: float = 10.0, wet_frac: float = 0.6,
                   with_sources: bool = True, drain: float = -0.01) -> Problem:
    """Small random state with a wet/dry mix for stage-wise parity: fractal
    bed, random depth where wet, random velocities, all physics terms on.
    About 30% of the source cells are drains of rate ``drain`` (m/s) times a
    weight in [0.5, 1.5]; a strong rate makes drains that empty their cell."""
    b = quantise_bed(fractal_terrain(nx, ny, seed, relief=3.0))
    u = uniform(seed, 3, np.arange(nx * ny * 4)).reshape(4, ny, nx)
    wet = u[0] < wet_frac
    H = np.where(wet, 0.05 + 2.0 * u[1], 0.0)
    # a few thin films at or just above the dry threshold
    film = (u[0] > 0.97)
    H = np.where(film, 1.0e-4 * (0.5 + u[1]), H)
    Qx = np.where(H > 1.0e-4, H * (2.0 * u[2] - 1.0), 0.0)
    Qy = np.where(H > 1.0e-4, H * (2.0 * u[3] - 1.0), 0.0)
    nm = 0.02 + 0.03 * uniform(seed, 4, np.arange(nx * ny)).reshape(ny, nx)
    f48 = 2.0 * 7.2921159e-5 * math.sin(math.radians(48.0))
    p = Params(nx=nx, ny=ny, dx=dx, nu=1.0, coriolis_f=f48, wind_x=10.0, wind_y=-3.0,
               c_a=1.3e-3, cfl=0.3, eps=1.0e-4, dt_max=1.0)
    if with_sources:
        ns = max(1, (nx * ny) // 200)
        cells = np.unique((uniform(seed, 5, np.arange(ns)) * nx * ny).astype(np.int64))
        ns = len(cells)
        ix = (cells % nx).astype(np.int32)
        iy = (cells // nx).astype(np.int32)
        wts = 0.5 + uniform(seed, 6, np.arange(ns))
        hyd = [Hydrograph(0, 0.02, 0.0, 50.0), Hydrograph(1, drain)]
        hid = (uniform(seed, 7, np.arange(ns)) < 0.3).astype(np.int32)
        vx = np.where(hid == 0, 2.0 * uniform(seed, 8, np.arange(ns)) - 1.0, 0.0)
        vy = np.where(hid == 0, 2.0 * uniform(seed, 9, np.arange(ns)) - 1.0, 0.0)
        src = Sources(ix, iy, wts, vx, vy, hid, hyd)
    else:
        src = Sources.empty()
    return Problem("random_wet_dry", p, b, nm, H, Qx, Qy, src)


def with_gates(prob: Problem, seed: int, ngates: int) -> Problem:
    """Close ``ngates`` seeded cells on the channel centreline (walls)."""
    p = prob.params
    solid = np.zeros((p.ny, p.nx), dtype=np.uint8)
    if ngates > 0:
        xs = (0.1 + 0.8 * uniform(seed, 10, np.arange(ngates))) * p.nx
        ix = xs.astype(np.int64)
        yc = channel_centre_y((ix + 0.5) * p.dx, p.ny * p.dx, p.nx * p.dx)
        iy = np.clip((yc // p.dx).astype(np.int64), 0, p.ny - 1)
        solid[iy, ix] = 1
    return dataclasses.replace(prob, solid=solid)


@dataclasses.dataclass
class GateSchedule:
    """Gate cells of one scenario: initial state and one toggle step each."""
    ix: np.ndarray
    iy: np.ndarray
    closed0: np.ndarray   # uint8, state at step 0
    toggle_step: np.ndarray  # int64, step before which the gate flips


def ensemble(n: int, seed_base: int = 10000, nmin: int = 512, nmax: int = 2048, dx: float = 10.0,
             toggle_steps: int = 2000, max_gates: int = 8, indices=None):
    """Seeded flood-scenario ensemble: scenario s has a square grid with N
    uniform in [nmin, nmax], its own fractal terrain (seed seed_base + s)
    with the carved channel, a 100-cell inflow strip fed by a Gaussian
    hydrograph with peak time uniform in [1, 6] h, peak uniform in
    [1, 10] m/s*cells and width t_p / 3, and 0..max_gates gate cells on the
    channel with a seeded initial state and one seeded toggle step in
    [0, toggle_steps).  Scenario s depends on s alone: `indices` (default
    all of range(n)) picks which scenarios to build.  Returns (problems,
    gate schedules)."""
    probs, gates = [], []
    for s in (range(n) if indices is None else indices):
        if not 0 <= s < n:
            raise ValueError(f"scenario {s} outside an ensemble of {n}")
        u = uniform(seed_base, 20, np.arange(4) + 4 * s)
        N = int(nmin + int(u[0] * (nmax - nmin + 1)))
        tp = 3600.0 * (1.0 + 5.0 * u[1])
        peak = 1.0 + 9.0 * u[2]
        p = floodplain(N, dx, seed_base + s, seed_base + 5000 + s, hydro=Hydrograph(0, peak, tp, tp / 3.0),
                       nsrc=min(100, N))
        ng = int(u[3] * (max_gates + 1))
        g = uniform(seed_base + s, 21, np.arange(3 * max(ng, 1)))
        xs = (0.2 + 0.7 * g[:ng]) * N
        ix = xs.astype(np.int64)
        yc = channel_centre_y((ix + 0.5) * dx, N * dx, N * dx)
        iy = np.clip((yc // dx).astype(np.int64), 0, N - 1)
        cells, keep = set(), []
        for m in range(ng):
            key = (int(iy[m]), int(ix[m]))
            if key not in cells:
                cells.add(key)
                keep.append(m)
        keep = np.array(keep, dtype=np.int64)
        sched = GateSchedule(ix[keep].astype(np.int32) if ng else np.zeros(0, np.int32),
                             iy[keep].astype(np.int32) if ng else np.zeros(0, np.int32),
                             (g[ng:2 * ng][keep] < 0.5).astype(np.uint8) if ng else np.zeros(0, np.uint8),
                             (g[2 * ng:3 * ng][keep] * toggle_steps).astype(np.int64) if ng else np.zeros(0, np.int64))
        solid = np.zeros((N, N), dtype=np.uint8)
        if ng:
            solid[sched.iy, sched.ix] = sched.closed0
        probs.append(dataclasses.replace(p, name=f"scenario{s}", solid=solid))
        gates.append(sched)
    return probs, gates


# Named workloads of the benchmark suite, by what they are.
def workload(name: str) -> Problem:
    if name == "dambreak-256sq-dx1m":
        return dam_break(256, 1.0)
    if name == "floodplain-2048sq-dx10m":
        return floodplain(2048, 10.0, 2017, 2018)
    if name == "floodplain-4096sq-dx5m":
        return floodplain(4096, 5.0, 2021, 2022)
    if name == "floodplain-16384sq-dx2m":
        return floodplain(16384, 2.0, 2019, 2020)
    raise KeyError(name)
