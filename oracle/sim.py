"""The per-timestep loop and its diagnostics (oracle; test infrastructure).

One step n -> n+1 (Sec. II, leapfrog; the printed order "(1),(2), then (5),
then (3),(4)" is read as the standard leapfrog cycle of ref. [bir86]):

  1. gather E^n at x^n and kick: v^{n+1/2} = v^{n-1/2} + alpha_j E^n dt  (Eqs. 1-2)
  2. drift: x^{n+1} = x^n + v^{n+1/2} dt                                  (Eqs. 3-4)
  3. absorb particles that reach a wall or a conductor; tally the hits
     per wall and, on the x = nx plate, per bottom cell (Sec. III-A, III-C)
  4. deposit rho^{n+1} = sum_s q_s n_s + rho_ext + bottom surface charge   (Eq. 5, Sec. III-D)
  5. solve Eq. (5) for Phi^{n+1} and form E^{n+1} = -grad Phi^{n+1}       (Sec. II)

Velocities live at half steps.  A species loaded with velocities at t = 0
is started with the half back-kick v^{-1/2} = v^0 - (1/2) alpha_j E^0 dt.

RF bias (Sec. III-B): the solve at time level n uses the electrode value at
t = n dt (geometry.Geometry.set_time).

Ion recycling (Sec. III-A: a lost ion is replaced by a thermal ion in the
bulk plasma, as ionisation of the neutral gas; Sec. III-C: with the trench,
ionisation only in the bulk region above the electrode).  Reading taken:
every ion absorbed during step n (tallied and recorded as usual) re-enters,
with its id, in the same step at a uniform position in the source rows
[source_x0, source_x1) of cells (all y) with a Maxwellian velocity of the
ion thermal speed, taken as its v^{n+1/2}; it joins the deposit of
rho^{n+1}.  The draws are Philox4x32-10 (oracle.rng) keyed by the seed, with
counter (id, n, 1, k):
  k = 0: words r0..r3 -> cell row  source_x0 + floor(r0 L / 2^32)  (L rows),
         cell column floor(r1 ny / 2^32), offsets top24(r2), top24(r3) / 2^24;
  k = 1: Box-Muller on u1 = (top24(q0) + 1) / 2^24, u2 = top24(q1) / 2^24.
Positions are then exact dyadic numbers, the same on any machine.

Diagnostics of the step just taken (time level n):
  KE_s = 1/2 m_s w_s sum_p v^{n-1/2} . v^{n+1/2}  (m_s = q_s / alpha_s, w_s = 1/ppc_s)
  FE   = 1/2 sum_nodes |E^n|^2
  P_s  = m_s w_s sum_p v^{n+1/2}
"""
from __future__ import annotations

import numpy as np

from . import deposit, field, poisson, push, rng
from .geometry import from_workload

RECYCLE_TAG = 1


class Sim:
    def __init__(self, w, surface_charge=None):
        self.w = w
        self.geom = from_workload(w)
        self.surface_charge = w.surface_charge if surface_charge is None else surface_charge
        self.q = np.array(w.charge)
        self.alpha = np.array(w.alpha)
        self.mass = self.q / self.alpha
        self.weight = np.array([1.0 / w.ppc, 1.0 / w.ppc])
        empty = np.zeros(0)
        self.p = [dict(x=empty, y=empty, vx=empty, vy=empty, ids=np.zeros(0, np.uint32))
                  for _ in range(2)]
        self.rho_ext = np.zeros((self.geom.nxn, self.geom.nyn))
        self.counts = np.zeros((2, push.N_WALLS), dtype=np.int64)
        self.bottom = np.zeros((2, w.ny), dtype=np.int64)
        self.hits = []
        self.nstep = 0
        self.dirty = True
        self.halfkick = [False, False]
        self.phi = np.zeros((self.geom.nxn, self.geom.nyn))
        self.Ex = np.zeros_like(self.phi)
        self.Ey = np.zeros_like(self.phi)
        self.ke = np.zeros(2)
        self.fe = 0.0
        self.rho = np.zeros_like(self.phi)

    # ------------------------------------------------------------------
    def load(self, s, x, y, vx, vy, ids=None, v_at_t0=False):
        n = len(x)
        self.p[s] = dict(x=np.asarray(x, np.float64).copy(), y=np.asarray(y, np.float64).copy(),
                         vx=np.asarray(vx, np.float64).copy(), vy=np.asarray(vy, np.float64).copy(),
                         ids=(np.arange(n, dtype=np.uint32) if ids is None
                              else np.asarray(ids, np.uint32).copy()))
        self.halfkick[s] = bool(v_at_t0)
        self.dirty = True

    def load_particles(self, s, parts, v_at_t0=False):
        self.load(s, parts.x, parts.y, parts.vx, parts.vy, parts.ids, v_at_t0)

    def set_rho_ext(self, rho_ext):
        self.rho_ext = np.asarray(rho_ext, np.float64).copy()
        self.dirty = True

    # ------------------------------------------------------------------
    def species_density(self, s):
        ps = self.p[s]
        return deposit.cic_density(self.geom, ps["x"], ps["y"], self.weight[s])

    def charge_density(self):
        rho = self.rho_ext.copy()
        for s in range(2):
            rho += self.q[s] * self.species_density(s)
        if self.surface_charge and not self.geom.px:
            sigma = (self.q[:, None] * self.weight[:, None] * self.bottom).sum(axis=0)
            rho += deposit.surface_charge_density(self.geom, sigma)
        return rho

    def solve_fields(self):
        self.geom.set_time(self.nstep * self.w.dt)
        self.rho = self.charge_density()
        self.phi = poisson.solve_direct(self.geom, self.rho)
        self.Ex, self.Ey = field.efield(self.geom, self.phi)

    def prepare(self):
        if not self.dirty:
            return
        self.solve_fields()
        for s in range(2):
            if self.halfkick[s]:
                ps = self.p[s]
                ex, ey = push.gather(self.geom, self.Ex, self.Ey, ps["x"], ps["y"])
                ps["vx"] = ps["vx"] - 0.5 * self.alpha[s] * ex * self.w.dt
                ps["vy"] = ps["vy"] - 0.5 * self.alpha[s] * ey * self.w.dt
                self.halfkick[s] = False
        self.dirty = False

    # ------------------------------------------------------------------
    def push_species(self, s):
        """Steps 1-3 for species s; returns the hit records of this step."""
        ps = self.p[s]
        x1, y1, vx1, vy1, alive, wall, wcell = push.leapfrog(
            self.geom, self.alpha[s], self.w.dt, ps["x"], ps["y"], ps["vx"], ps["vy"],
            self.Ex, self.Ey)
        self.ke[s] = 0.5 * self.mass[s] * self.weight[s] * float(
            np.sum(ps["vx"] * vx1 + ps["vy"] * vy1))
        dead = ~alive
        np.add.at(self.counts[s], wall[dead], 1)
        xm = dead & (wall == push.WALL_XMAX)
        np.add.at(self.bottom[s], wcell[xm], 1)
        rec = dict(ids=ps["ids"][dead], species=np.full(int(dead.sum()), s), wall=wall[dead],
                   cell=wcell[dead], step=np.full(int(dead.sum()), self.nstep),
                   vx=vx1[dead], vy=vy1[dead])
        new = dict(x=x1[alive], y=y1[alive], vx=vx1[alive], vy=vy1[alive], ids=ps["ids"][alive])
        if s == 1 and getattr(self.w, "recycle", False) and dead.any():
            r = self.recycled(ps["ids"][dead], self.nstep)
            for k in new:
                new[k] = np.concatenate([new[k], r[k]])
        self.p[s] = new
        return rec

    def source_rows(self):
        x0 = int(getattr(self.w, "source_x0", 0))
        x1 = int(getattr(self.w, "source_x1", 0)) or self.w.nx - self.w.trench_depth
        return x0, x1

    def recycled(self, ids, step):
        """The thermal ions that replace the absorbed ions `ids` during step
        `step` (see the module docstring)."""
        ids = np.asarray(ids, np.uint64)
        key = rng.seed_key(getattr(self.w, "recycle_seed", 0))
        ctr = np.zeros((ids.size, 4), np.uint64)
        ctr[:, 0] = ids
        ctr[:, 1] = np.uint64(step)
        ctr[:, 2] = RECYCLE_TAG
        r = rng.philox4x32_10(ctr, key)
        ctr[:, 3] = 1
        q = rng.philox4x32_10(ctr, key)
        x0, x1 = self.source_rows()
        i = x0 + rng.below(r[:, 0], x1 - x0)
        j = rng.below(r[:, 1], self.w.ny)
        z0, z1 = rng.box_muller(rng.unit24_open(q[:, 0]), rng.unit24(q[:, 1]))
        vth = self.w.vth[1]
        return dict(x=i + rng.unit24(r[:, 2]), y=j + rng.unit24(r[:, 3]), vx=vth * z0, vy=vth * z1,
                    ids=ids.astype(np.uint32))

    def step(self, n=1):
        for _ in range(n):
            self.prepare()
            self.fe = field.field_energy(self.Ex, self.Ey)
            for s in range(2):
                self.hits.append(self.push_species(s))
            self.nstep += 1
            self.solve_fields()

    # ------------------------------------------------------------------
    def momentum(self):
        out = np.zeros((2, 2))
        for s in range(2):
            ps = self.p[s]
            out[s, 0] = self.mass[s] * self.weight[s] * ps["vx"].sum()
            out[s, 1] = self.mass[s] * self.weight[s] * ps["vy"].sum()
        return out

    def live(self):
        return np.array([self.p[0]["x"].size, self.p[1]["x"].size], dtype=np.int64)

    def hit_table(self):
        keys = ("ids", "species", "wall", "cell", "step", "vx", "vy")
        if not self.hits:
            return {k: np.zeros(0) for k in keys}
        return {k: np.concatenate([h[k] for h in self.hits]) for k in keys}
