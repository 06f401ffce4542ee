"""Seeded synthetic workloads for the 2D electrostatic trench PIC.

This module is shared by the CUDA path's tests and benchmark and by the
CPU oracle.  It holds the workload recipes (grid sizes, geometry numbers,
species parameters) and the seeded particle generators, and nothing of the
method's arithmetic: no weighting, no field, no push, no Poisson solve.

Units are the paper's normalised ones (Sec. II): lengths in Debye lengths,
times in inverse plasma periods, velocities in electron thermal speeds,
potentials in T_e/e.  x is the direction normal to the plates, y runs along
them.  Grids are row-major [i_x][j_y] with y fastest.

Initial state (Sec. III-A): positions uniform inside each plasma cell
(``ppc`` particles per cell per species, the trench interior included),
velocities Gaussian in each component with the species thermal speed
(Eq. (6)); v_i = v_e (m_e tau / m_i)^(1/2).
"""
from __future__ import annotations

import dataclasses
from dataclasses import dataclass, field
from typing import List, Tuple

import numpy as np

E_SPECIES, I_SPECIES = 0, 1


@dataclass
class Workload:
    """One simulation's parameters, in normalised units."""

    name: str
    nx: int                      # cells along x (normal to the plates)
    ny: int                      # cells along y (along the plates)
    periodic_x: bool = False
    periodic_y: bool = True
    dt: float = 0.1
    phi_top: float = 0.0         # Dirichlet value of the x = 0 plate
    phi_electrode: float = 0.0   # Dirichlet value of the x = nx plate and of the electrode slab
    trench_depth: int = 0        # electrode slab thickness in cells (cells i >= nx - depth)
    trench_y0: int = 0           # first open (plasma) column of the trench
    trench_width: int = 0        # open columns; 0 = flat slab (or no slab when depth = 0)
    mass_ratio: float = 1836.0   # m_i / m_e
    tau: float = 0.1             # T_i / T_e
    ppc: int = 50                # particles per plasma cell per species
    seed: int = 1
    nsteps: int = 500
    surface_charge: bool = False  # bottom-face hits feed back into rho
    poisson_rtol: float = 1e-6
    sort_every: int = 8
    # RF bias of the electrode (Sec. III-B): its Dirichlet value at time t is
    # phi_electrode + phi_rf_amp * sin(omega_rf * t)
    phi_rf_amp: float = 0.0
    omega_rf: float = 0.0
    # ion recycling (Sec. III-A, III-C): an absorbed ion is re-loaded as a
    # thermal ion at a uniform position in the source rows [source_x0,
    # source_x1) of cells (all y); source_x1 = 0 means nx - trench_depth
    recycle: bool = False
    source_x0: int = 0
    source_x1: int = 0
    recycle_seed: int = 0

    # ---- species constants (paper Sec. II: alpha_e = -1, alpha_i = (m_e/m_i)(q_i/e)) ----
    @property
    def charge(self) -> Tuple[float, float]:
        return (-1.0, 1.0)

    @property
    def alpha(self) -> Tuple[float, float]:
        return (-1.0, 1.0 / self.mass_ratio)

    @property
    def vth(self) -> Tuple[float, float]:
        return (1.0, float(np.sqrt(self.tau / self.mass_ratio)))

    def replace(self, **kw) -> "Workload":
        return dataclasses.replace(self, **kw)


def plasma_cells(w: Workload) -> np.ndarray:
    """Boolean [nx, ny] map of the cells particles are loaded into.

    The electrode slab occupies cells i >= nx - trench_depth; the trench
    columns [trench_y0, trench_y0 + trench_width) are cut through it.
    """
    m = np.ones((w.nx, w.ny), dtype=bool)
    if w.trench_depth > 0:
        m[w.nx - w.trench_depth:, :] = False
        if w.trench_width > 0:
            m[w.nx - w.trench_depth:, w.trench_y0:w.trench_y0 + w.trench_width] = True
    return m


# ---------------------------------------------------------------------------
# Workload recipes
# ---------------------------------------------------------------------------

def periodic_square_64(**kw) -> Workload:
    """64x64 doubly periodic box, 50 ppc/species, dt = 0.1, 500 steps."""
    return Workload(name="periodic_square_64x64_ppc50", nx=64, ny=64,
                    periodic_x=True, periodic_y=True, ppc=50, seed=1,
                    nsteps=500).replace(**kw)


def bounded_square_256(**kw) -> Workload:
    """256x256 box, all four walls grounded and absorbing, 100 ppc/species."""
    return Workload(name="bounded_square_256x256_ppc100", nx=256, ny=256,
                    periodic_x=False, periodic_y=False, ppc=100, seed=2,
                    nsteps=2000).replace(**kw)


def trench_512x1024(**kw) -> Workload:
    """512 (y, periodic) x 1024 (x) cells between a grounded plate at x = 0
    and an electrode at -20 T_e/e; a 10-wide, 200-deep trench cut into the
    electrode, centred in y; 100 ppc/species; bottom hits charge the trench
    bottom."""
    return Workload(name="trench_512x1024_w10_d200_ppc100", nx=1024, ny=512,
                    periodic_x=False, periodic_y=True, phi_top=0.0,
                    phi_electrode=-20.0, trench_depth=200, trench_y0=251,
                    trench_width=10, ppc=100, seed=3, nsteps=5000,
                    surface_charge=True).replace(**kw)


def small_trench(nx=64, ny=32, depth=16, width=6, ppc=8, seed=5, **kw) -> Workload:
    """A reduced trench geometry with the same structure as the 512x1024 one."""
    y0 = (ny - width) // 2
    return Workload(name=f"trench_{ny}x{nx}_w{width}_d{depth}_ppc{ppc}", nx=nx, ny=ny,
                    periodic_x=False, periodic_y=True, phi_top=0.0,
                    phi_electrode=-20.0, trench_depth=depth, trench_y0=y0,
                    trench_width=width, ppc=ppc, seed=seed, nsteps=100,
                    surface_charge=True).replace(**kw)


_ENSEMBLE_GRIDS = [(128, 256), (256, 256), (256, 512), (512, 512)]  # (W = y cells, H = x cells)


def ensemble_member(k: int, **kw) -> Workload:
    """Member k (0..47) of the trench-width sweep: width 1 + round(39k/47),
    grid cycling through 128x256 ... 512x512, depth ~0.195 H, 64 ppc."""
    wy, hx = _ENSEMBLE_GRIDS[k % 4]
    width = 1 + int(round(39 * k / 47))
    depth = int(round(0.195 * hx))
    y0 = (wy - width) // 2
    return Workload(name=f"ensemble{k}_{wy}x{hx}_w{width}", nx=hx, ny=wy,
                    periodic_x=False, periodic_y=True, phi_electrode=-20.0,
                    trench_depth=depth, trench_y0=y0, trench_width=width,
                    ppc=64, seed=1000 + k, nsteps=2000,
                    surface_charge=True).replace(**kw)


def paper_trench(width: int = 15, seed: int = 1, **kw) -> Workload:
    """The paper's own trench runs (Sec. III-C): a 60 x 30 periodic bulk above
    a 20-deep electrode (80 x-cells, 30 y-cells), trench of width 15 at
    5 <= y <= 20 (Fig. 5) or of width 4 at 10 <= y <= 14 (Fig. 6); grounded
    plate at x = 0, RF electrode Phi = 5 sin(0.01 t) (Sec. III-B);
    m_i / m_e = 3672, T_i = T_e (Sec. III); 100 ppc/species; ions recycled
    into the bulk rows 0 <= x < 60 (Sec. III-A, III-C); dt = 0.1 up to
    t = 1000."""
    y0 = {15: 5, 4: 10}.get(width, (30 - width) // 2)
    return Workload(name=f"paper_trench_80x30_w{width}", nx=80, ny=30, periodic_x=False,
                    periodic_y=True, phi_top=0.0, phi_electrode=0.0, phi_rf_amp=5.0,
                    omega_rf=0.01, trench_depth=20, trench_y0=y0, trench_width=width,
                    mass_ratio=3672.0, tau=1.0, ppc=100, seed=seed, nsteps=10000,
                    recycle=True, source_x0=0, source_x1=60, recycle_seed=seed,
                    surface_charge=False).replace(**kw)


def paper_buildup_density(w: Workload, value: float = 5.0) -> np.ndarray:
    """The fixed test-ion density of the paper's charge build-up run (Sec.
    III-D): n_i = 5 on the node row x = nx - 1 (x = 79) across the trench
    bottom, y = y0 .. y0 + width (5 <= y <= 20 for the width-15 trench)."""
    nyn = w.ny if w.periodic_y else w.ny + 1
    rho = np.zeros((w.nx + 1, nyn))
    rho[w.nx - 1, w.trench_y0:w.trench_y0 + w.trench_width + 1] = value
    return rho


# ---------------------------------------------------------------------------
# Particle generators
# ---------------------------------------------------------------------------

@dataclass
class Particles:
    x: np.ndarray
    y: np.ndarray
    vx: np.ndarray
    vy: np.ndarray
    ids: np.ndarray

    def __len__(self) -> int:
        return int(self.x.shape[0])

    def subset(self, sel) -> "Particles":
        return Particles(self.x[sel], self.y[sel], self.vx[sel], self.vy[sel], self.ids[sel])


def maxwellian_load(w: Workload, species: int, ppc: int | None = None,
                    seed: int | None = None) -> Particles:
    """ppc particles per plasma cell, uniform inside the cell, Gaussian
    velocities with standard deviation vth[species] per component."""
    ppc = w.ppc if ppc is None else ppc
    seed = w.seed if seed is None else seed
    rng = np.random.default_rng([seed, species])
    ci, cj = np.nonzero(plasma_cells(w))
    n = ci.size * ppc
    x = np.repeat(ci.astype(np.float64), ppc)
    x += rng.random(n)
    y = np.repeat(cj.astype(np.float64), ppc)
    y += rng.random(n)
    s = w.vth[species]
    vx = rng.standard_normal(n) * s
    vy = rng.standard_normal(n) * s
    return Particles(x, y, vx, vy, np.arange(n, dtype=np.uint32))


def keep_off_faces(p: Particles, w: Workload, margin: float = 1e-4) -> Particles:
    """Nudge positions at least ``margin`` away from every cell face (used by
    parity tests that need each face crossing decided far from a tie)."""
    def nudge(a):
        f = a - np.floor(a)
        lo = f < margin
        hi = f > 1.0 - margin
        a = a.copy()
        a[lo] += margin - f[lo]
        a[hi] -= f[hi] - (1.0 - margin)
        return a
    return Particles(nudge(p.x), nudge(p.y), p.vx, p.vy, p.ids)


def random_state(w: Workload, species: int, n: int, seed: int,
                 vscale: float = 1.0) -> Particles:
    """n particles uniform over the plasma cells (random cell, random
    offset), Gaussian velocities scaled by vscale * vth[species]."""
    rng = np.random.default_rng([seed, 77, species])
    ci, cj = np.nonzero(plasma_cells(w))
    pick = rng.integers(0, ci.size, size=n)
    x = ci[pick] + rng.random(n)
    y = cj[pick] + rng.random(n)
    s = w.vth[species] * vscale
    return Particles(x, y, rng.standard_normal(n) * s, rng.standard_normal(n) * s,
                     np.arange(n, dtype=np.uint32))


def random_rho(w: Workload, seed: int, scale: float = 1.0) -> np.ndarray:
    """A seeded node-centred density field (for Poisson tests)."""
    nxn = w.nx if w.periodic_x else w.nx + 1
    nyn = w.ny if w.periodic_y else w.ny + 1
    rng = np.random.default_rng([seed, 99])
    return rng.standard_normal((nxn, nyn)) * scale
