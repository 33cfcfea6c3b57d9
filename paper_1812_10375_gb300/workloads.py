"""Seeded synthetic workloads shaped like the cases of Hu & Liu (arXiv 1812.10375).

This module builds initial fields, geometry descriptions and nucleation-site
lists.  It holds none of the model's arithmetic: the coexistence densities,
the critical temperature and every other property of the equation of state are
passed in by the caller, so the GPU library and the FP64 reference can be fed
identical inputs.

Cases (lattice units; temperatures are given as multiples of Tc):

* ``flat_interface``: 1D conduction across a flat liquid-vapour interface
  (Section 3.2, transposed): 4 x 200, solid Dirichlet rows 0 and 199 at
  T = 1 and T = 0, liquid slab in the middle half with tanh interfaces of width 5,
  EOS temperature fixed at 0.86 Tc, no gravity, no wetting force.
* ``film``: film evaporation on a heated wall (Section 3.3): 200 x 100, 20 solid
  rows, a 30-row liquid film above them, vapour above the film, open top at
  rho_v, bottom row at Ts + 0.05 Tc, gravity 3e-5.
* ``pool``: pool boiling (Section 4.2): 400 x 400, 25 heater rows at
  Ts + 0.1 Tc, saturated liquid at Ts, 5 seeded nucleation sites of width 10
  with minima cycling over (0, -0.3, -0.6), convective top, gravity 3e-5.
* ``sweep``: 32 square domains with sides drawn from {256, ..., 512}, superheats
  evenly spaced over 0.02-0.30 Tc, 3-9 nucleation sites each.
"""
from __future__ import annotations

from dataclasses import dataclass, field

import numpy as np

BASE_SEED = 1812
SITE_WIDTH = 10.0
SITE_MINIMA = (0.0, -0.3, -0.6)
TS_OVER_TC = 0.86
GRAVITY = 3e-5


@dataclass
class Case:
    """Geometry, boundary kinds and initial fields of one domain."""

    name: str
    nx: int
    ny: int
    wall_rows: int
    top_bc: str                      # "wall" | "const_rho" | "convective"
    T_bottom_over_Tc: float | None   # None: absolute value in T_bottom_abs
    T_top_over_Tc: float | None
    eos_T_fixed: bool
    g_y: float
    Gw0: float
    sites: list = field(default_factory=list)  # (x_centre, width, g_min)
    T_bottom_abs: float | None = None
    T_top_abs: float | None = None
    steps: int = 1000

    def T_bottom(self, Tc: float) -> float:
        return self.T_bottom_abs if self.T_bottom_abs is not None else self.T_bottom_over_Tc * Tc

    def T_top(self, Tc: float) -> float:
        if self.T_top_abs is not None:
            return self.T_top_abs
        return 0.0 if self.T_top_over_Tc is None else self.T_top_over_Tc * Tc


def _grid(ny: int, nx: int):
    y = np.arange(ny, dtype=np.float64)[:, None] * np.ones((1, nx))
    x = np.ones((ny, 1)) * np.arange(nx, dtype=np.float64)[None, :]
    return y, x


def tanh_slab(ny: int, nx: int, rho_l: float, rho_v: float, y1: float, y2: float, width: float = 5.0):
    """Liquid between y1 and y2, vapour elsewhere, tanh interfaces of the given width."""
    y, _ = _grid(ny, nx)
    return rho_v + 0.5 * (rho_l - rho_v) * (np.tanh(2.0 * (y - y1) / width) - np.tanh(2.0 * (y - y2) / width))


def tanh_film(ny: int, nx: int, rho_l: float, rho_v: float, y_top: float, width: float = 5.0):
    """Liquid below y_top, vapour above."""
    y, _ = _grid(ny, nx)
    return 0.5 * (rho_l + rho_v) - 0.5 * (rho_l - rho_v) * np.tanh(2.0 * (y - y_top) / width)


def droplet(ny: int, nx: int, rho_l: float, rho_v: float, xc: float, yc: float, radius: float,
            width: float = 5.0):
    """A liquid disc in vapour."""
    y, x = _grid(ny, nx)
    r = np.sqrt((x - xc) ** 2 + (y - yc) ** 2)
    return rho_v + 0.5 * (rho_l - rho_v) * (1.0 - np.tanh(2.0 * (r - radius) / width))


def layered_T(ny: int, nx: int, wall_rows: int, T_wall: float, T_fluid: float):
    """Solid rows at the wall temperature, fluid at another."""
    y, _ = _grid(ny, nx)
    return np.where(y < wall_rows, T_wall, T_fluid)


def draw_sites(rng: np.random.Generator, nx: int, n_sites: int, width: float = SITE_WIDTH,
               minima=SITE_MINIMA):
    """n_sites non-overlapping site centres (integer columns), minima cycled."""
    spacing = width + 2.0
    if n_sites * spacing > nx:
        raise ValueError("too many sites for this width")
    centres: list[int] = []
    tries = misses = 0
    while len(centres) < n_sites:
        tries += 1
        if tries > 1000000:
            raise RuntimeError("could not place sites")
        if misses > 2000:  # earlier sites leave no gap wide enough: start over
            centres, misses = [], 0
        c = int(rng.integers(0, nx))
        if all(min(abs(c - o), nx - abs(c - o)) >= spacing for o in centres):
            centres.append(c)
            misses = 0
        else:
            misses += 1
    centres.sort()
    return [(float(c), float(width), float(minima[j % len(minima)])) for j, c in enumerate(centres)]


def flat_interface(steps: int = 2000) -> Case:
    return Case("flat_interface", nx=4, ny=200, wall_rows=1, top_bc="wall",
                T_bottom_over_Tc=None, T_top_over_Tc=None, T_bottom_abs=1.0, T_top_abs=0.0,
                eos_T_fixed=True, g_y=0.0, Gw0=0.0, steps=steps)


def film(steps: int = 20000, nx: int = 200, ny: int = 100) -> Case:
    return Case("film", nx=nx, ny=ny, wall_rows=20, top_bc="const_rho",
                T_bottom_over_Tc=TS_OVER_TC + 0.05, T_top_over_Tc=None,
                eos_T_fixed=False, g_y=-GRAVITY, Gw0=0.3, steps=steps)


def pool(steps: int = 60000, nx: int = 400, ny: int = 400, superheat: float = 0.1, n_sites: int = 5,
         seed: int = BASE_SEED, heater_rows: int = 25) -> Case:
    rng = np.random.default_rng(seed)
    sites = draw_sites(rng, nx, n_sites)
    return Case(f"pool_{nx}x{ny}", nx=nx, ny=ny, wall_rows=heater_rows, top_bc="convective",
                T_bottom_over_Tc=TS_OVER_TC + superheat, T_top_over_Tc=None,
                eos_T_fixed=False, g_y=-GRAVITY, Gw0=0.3, sites=sites, steps=steps)


def sweep(n_domains: int = 32, seed: int = BASE_SEED, sides=(256, 320, 384, 448, 512),
          superheat_range=(0.02, 0.30), sites_range=(3, 9), steps: int = 40000) -> list[Case]:
    """The boiling-curve sweep: square domains of seeded sides and evenly spaced superheats."""
    rng = np.random.default_rng(seed)
    dts = np.linspace(superheat_range[0], superheat_range[1], n_domains)
    out = []
    for d in range(n_domains):
        side = int(rng.choice(np.asarray(sides)))
        n_sites = int(rng.integers(sites_range[0], sites_range[1] + 1))
        sites = draw_sites(rng, side, n_sites)
        out.append(Case(f"sweep{d:02d}_{side}", nx=side, ny=side, wall_rows=25, top_bc="convective",
                        T_bottom_over_Tc=TS_OVER_TC + float(dts[d]), T_top_over_Tc=None,
                        eos_T_fixed=False, g_y=-GRAVITY, Gw0=0.3, sites=sites, steps=steps))
    return out


def initial_fields(case: Case, rho_l: float, rho_v: float, Tc: float):
    """(rho0, T0) float64 arrays of shape (ny, nx) for a case."""
    ny, nx = case.ny, case.nx
    Ts = TS_OVER_TC * Tc
    if case.name == "flat_interface":
        rho = tanh_slab(ny, nx, rho_l, rho_v, ny / 4.0, 3.0 * ny / 4.0)
        T = np.full((ny, nx), 0.5 * (case.T_bottom(Tc) + case.T_top(Tc)))
    elif case.name == "film":
        rho = tanh_film(ny, nx, rho_l, rho_v, case.wall_rows + 30.0)
        T = layered_T(ny, nx, case.wall_rows, case.T_bottom(Tc), Ts)
    else:  # pool and sweep: saturated liquid at Ts above the heater
        rho = np.full((ny, nx), rho_l)
        T = layered_T(ny, nx, case.wall_rows, case.T_bottom(Tc), Ts)
    return rho, T
