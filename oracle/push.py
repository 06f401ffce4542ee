"""Gather, leapfrog push and absorption (oracle; test infrastructure).

Equations of motion, Eqs. (1)-(4) of Sec. II, in normalised units:
dv/dt = alpha_j E(x, y), dx/dt = v, with alpha_e = -1 and
alpha_i = (m_e/m_i)(q_i/e).  They are advanced by the leapfrog method
(Sec. II, refs. [bir86, rut83]) with velocities at half steps:

    v^{n+1/2} = v^{n-1/2} + alpha_j E^n(x^n) dt
    x^{n+1}   = x^n + v^{n+1/2} dt

E^n(x^n) is gathered from the nodes with the cloud-in-cell weights used by
the deposit (the paper does not state its weighting; bilinear is the
reading taken).

Absorption (Sec. III-A: particles reaching a wall are lost; Sec. III-C:
tallies of ions reaching the trench bottom and side walls).  The move is
taken as the straight segment x^n -> x^{n+1}.  Its cell faces are visited
in order of the segment parameter at which they are crossed; on an exact
tie the x face is taken first.  A particle whose position lies exactly on a
face belongs to the higher cell, so a move that ends exactly on x = nx is a
hit.  The first face whose far cell is a conductor or outside a bounded
direction absorbs the particle; that face names the wall:

    0 x = 0 plate        1 x = nx plate (trench bottom inside the trench)
    2 y = 0 wall          3 y = ny wall                (bounded y only)
    4 conductor entered moving +x (electrode top)
    5 conductor entered moving -x
    6 conductor entered moving +y (trench wall at the trench's upper y)
    7 conductor entered moving -y (trench wall at the trench's lower y)

and the cell index along the face (y index for x faces, x index for y
faces) is recorded with it.

Pinned by (tests/test_oracle_push.py): leapfrog in a uniform field is exact
for constant acceleration (closed form); cold plasma oscillation frequency
(2/dt) asin(omega_p dt / 2); hand-worked face classifications.
"""
from __future__ import annotations

import numpy as np

WALL_XMIN, WALL_XMAX, WALL_YMIN, WALL_YMAX = 0, 1, 2, 3
WALL_COND_PX, WALL_COND_MX, WALL_COND_PY, WALL_COND_MY = 4, 5, 6, 7
N_WALLS = 8


def gather(geom, Ex, Ey, x, y):
    """CIC interpolation of the node field to absolute positions (x, y)."""
    i = np.floor(x).astype(np.int64)
    j = np.floor(y).astype(np.int64)
    fx = x - i
    fy = y - j
    ex = np.zeros_like(x)
    ey = np.zeros_like(y)
    for di, wx in ((0, 1.0 - fx), (1, fx)):
        for dj, wy in ((0, 1.0 - fy), (1, fy)):
            ni = i + di
            nj = j + dj
            if geom.px:
                ni = ni % geom.nxn
            if geom.py:
                nj = nj % geom.nyn
            wgt = wx * wy
            ex += wgt * Ex[ni, nj]
            ey += wgt * Ey[ni, nj]
    return ex, ey


def classify(geom, x0, y0, x1, y1, max_crossings=64):
    """Walk the segment (x0, y0) -> (x1, y1) cell by cell.

    Returns (alive, wall, wall_cell) arrays; wall = -1 for live particles.
    The start cells must be plasma cells.
    """
    ci = np.floor(x0).astype(np.int64)
    cj = np.floor(y0).astype(np.int64)
    ti = np.floor(x1).astype(np.int64)
    tj = np.floor(y1).astype(np.int64)
    dx = x1 - x0
    dy = y1 - y0
    sx = np.where(ti > ci, 1, -1)
    sy = np.where(tj > cj, 1, -1)
    n = x0.size
    alive = np.ones(n, dtype=bool)
    wall = -np.ones(n, dtype=np.int64)
    wcell = -np.ones(n, dtype=np.int64)
    active = (ci != ti) | (cj != tj)
    for _ in range(max_crossings):
        if not active.any():
            break
        a = np.nonzero(active)[0]
        needx = ci[a] != ti[a]
        needy = cj[a] != tj[a]
        facex = np.where(sx[a] > 0, ci[a] + 1, ci[a]).astype(np.float64)
        facey = np.where(sy[a] > 0, cj[a] + 1, cj[a]).astype(np.float64)
        # x face first when t_x <= t_y, i.e. |facex-x0|*|dy| <= |facey-y0|*|dx|
        xfirst = np.abs(facex - x0[a]) * np.abs(dy[a]) <= np.abs(facey - y0[a]) * np.abs(dx[a])
        takex = needx & (~needy | xfirst)
        ci[a] += np.where(takex, sx[a], 0)
        cj[a] += np.where(takex, 0, sy[a])
        ok = geom.cell_is_plasma(ci[a], cj[a])
        hit = a[~ok]
        if hit.size:
            tx = takex[~ok]
            hi, hj = ci[hit], cj[hit]
            w = np.empty(hit.size, dtype=np.int64)
            c = np.empty(hit.size, dtype=np.int64)
            up_x = sx[hit] > 0
            up_y = sy[hit] > 0
            hj_w = hj % geom.ny if geom.py else hj
            hi_w = hi % geom.nx if geom.px else hi
            bx = not geom.px
            by = not geom.py
            out_xmax = (hi >= geom.nx) & bx
            out_xmin = (hi < 0) & bx
            out_ymax = (hj >= geom.ny) & by
            out_ymin = (hj < 0) & by
            # x faces
            m = tx & up_x
            w[m] = np.where(out_xmax[m], WALL_XMAX, WALL_COND_PX)
            m = tx & ~up_x
            w[m] = np.where(out_xmin[m], WALL_XMIN, WALL_COND_MX)
            c[tx] = hj_w[tx]
            # y faces
            m = ~tx & up_y
            w[m] = np.where(out_ymax[m], WALL_YMAX, WALL_COND_PY)
            m = ~tx & ~up_y
            w[m] = np.where(out_ymin[m], WALL_YMIN, WALL_COND_MY)
            c[~tx] = hi_w[~tx]
            alive[hit] = False
            wall[hit] = w
            wcell[hit] = c
        active[a] = ok & ((ci[a] != ti[a]) | (cj[a] != tj[a]))
    if active.any():
        raise RuntimeError("segment crossed more faces than max_crossings")
    return alive, wall, wcell


def wrap_positions(geom, x, y):
    if geom.px:
        x = np.mod(x, geom.nx)
        x = np.where(x >= geom.nx, x - geom.nx, x)
    if geom.py:
        y = np.mod(y, geom.ny)
        y = np.where(y >= geom.ny, y - geom.ny, y)
    return x, y


def leapfrog(geom, alpha, dt, x, y, vx, vy, Ex, Ey):
    """One leapfrog step of Eqs. (1)-(4) for one species with absorption.

    Returns (x1, y1, vx1, vy1, alive, wall, wall_cell); positions of live
    particles are wrapped into the periodic box.
    """
    ex, ey = gather(geom, Ex, Ey, x, y)
    vx1 = vx + alpha * ex * dt
    vy1 = vy + alpha * ey * dt
    x1 = x + vx1 * dt
    y1 = y + vy1 * dt
    alive, wall, wcell = classify(geom, x, y, x1, y1)
    x1, y1 = wrap_positions(geom, x1, y1)
    return x1, y1, vx1, vy1, alive, wall, wcell
