"""Geometry of the simulation box (oracle; test infrastructure).

Paper: Sec. III-A (grounded square, Phi = 0 on all four walls), Sec. III-B
(y periodic, Dirichlet plates at x = 0 and x = x_max), Sec. III-C (a trench
cut into the biased plate; trench bottom at x = x_max, side walls at the
trench's y edges).

Sec. III-B also drives the electrode with an RF bias, Phi = Phi_0
sin(omega_RF t).  Here the electrode's Dirichlet value at time t is
phi_electrode + phi_rf_amp * sin(omega_rf * t) (phi_electrode = 0 gives the
paper's pure RF bias); every node held at the electrode potential follows it.

Readings taken where the paper is silent:
  * Nodes sit at integer coordinates.  A bounded direction with N cells has
    N + 1 nodes (both end rows Dirichlet); a periodic one has N nodes.
  * The electrode is a conductor slab of cells i >= nx - depth, with the
    trench columns [y0, y0 + width) open down to x = nx.
  * Every node that touches a conductor cell is a Dirichlet node held at the
    electrode potential.  Precedence of values where categories meet:
    conductor / x = nx row (electrode) > x = 0 row (top plate) > y walls of
    a bounded-y box (grounded, 0).
"""
from __future__ import annotations

import numpy as np


class Geometry:
    def __init__(self, nx, ny, periodic_x, periodic_y, phi_top=0.0, phi_electrode=0.0,
                 trench_depth=0, trench_y0=0, trench_width=0, phi_rf_amp=0.0, omega_rf=0.0):
        self.nx, self.ny = int(nx), int(ny)
        self.px, self.py = bool(periodic_x), bool(periodic_y)
        self.nxn = self.nx if self.px else self.nx + 1
        self.nyn = self.ny if self.py else self.ny + 1

        cond = np.zeros((self.nx, self.ny), dtype=bool)
        if trench_depth > 0:
            cond[self.nx - trench_depth:, :] = True
            if trench_width > 0:
                cond[self.nx - trench_depth:, trench_y0:trench_y0 + trench_width] = False
        self.conductor = cond

        D = np.zeros((self.nxn, self.nyn), dtype=bool)
        g = np.zeros((self.nxn, self.nyn), dtype=np.float64)
        elec = np.zeros((self.nxn, self.nyn), dtype=bool)   # held at the electrode value
        if not self.py:                      # grounded side walls
            D[:, 0] = D[:, -1] = True
            g[:, 0] = g[:, -1] = 0.0
        if not self.px:
            D[0, :] = True
            g[0, :] = phi_top
            D[-1, :] = True
            g[-1, :] = phi_electrode
            elec[-1, :] = True
        # nodes touching a conductor cell
        ci, cj = np.nonzero(cond)
        for di in (0, 1):
            for dj in (0, 1):
                ni = ci + di
                nj = cj + dj
                if self.px:
                    ni = ni % self.nxn
                if self.py:
                    nj = nj % self.nyn
                D[ni, nj] = True
                g[ni, nj] = phi_electrode
                elec[ni, nj] = True
        self.dirichlet = D
        self.electrode = elec
        self.g_static = np.where(D, g, 0.0)
        self.g = self.g_static.copy()
        self.phi_rf_amp = float(phi_rf_amp)
        self.omega_rf = float(omega_rf)

    # -- time-dependent Dirichlet values (RF bias, Sec. III-B) -------------
    def rf_offset(self, t):
        """The electrode's RF part at time t: phi_rf_amp * sin(omega_rf * t)."""
        return self.phi_rf_amp * np.sin(self.omega_rf * t)

    def set_time(self, t):
        """Dirichlet values at time t: the static ones plus the RF part on
        every node held at the electrode potential."""
        self.g = self.g_static + self.rf_offset(t) * self.electrode

    # -- cells ------------------------------------------------------------
    def cell_is_plasma(self, i, j):
        """Vectorised: True where cell (i, j) lies in the domain (after the
        periodic wrap) and is not a conductor."""
        i = np.asarray(i)
        j = np.asarray(j)
        if self.px:
            i = np.mod(i, self.nx)
        if self.py:
            j = np.mod(j, self.ny)
        inside = (i >= 0) & (i < self.nx) & (j >= 0) & (j < self.ny)
        ii = np.clip(i, 0, self.nx - 1)
        jj = np.clip(j, 0, self.ny - 1)
        return inside & ~self.conductor[ii, jj]

    @property
    def free(self):
        return ~self.dirichlet


def from_workload(w) -> Geometry:
    return Geometry(w.nx, w.ny, w.periodic_x, w.periodic_y, w.phi_top, w.phi_electrode,
                    w.trench_depth, w.trench_y0, w.trench_width,
                    getattr(w, "phi_rf_amp", 0.0), getattr(w, "omega_rf", 0.0))
