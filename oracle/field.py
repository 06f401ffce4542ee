"""Electric field at the nodes, E = -grad(Phi) (oracle; test infrastructure).

Sec. II: E_x = -d Phi/dx, E_y = -d Phi/dy, with central differences inside
and a two-point ("Euler") difference at the boundaries.  Sec. III-A: the
field component along a conducting surface is zero.

Reading taken for nodes on internal conductor surfaces (electrode top,
trench walls, trench mouth corners): a mesh edge between two neighbouring
nodes is OPEN when at least one of the two cells on either side of it is a
plasma cell.  E along a direction at a node is minus the mean of the
potential differences over the open edges of that node in that direction:
two open edges give the central difference, one gives the two-point
one-sided difference, none gives 0.  Along a conductor surface both nodes
of an edge hold the same Dirichlet value, so the tangential component is 0
as Sec. III-A requires.

Pinned by (tests/test_oracle_field.py): a linear potential gives its exact
uniform field at every node used by a particle; a quadratic potential gives
the exact derivative at interior nodes; the tangential field on the
grounded walls and trench walls is zero.
"""
from __future__ import annotations

import numpy as np


def _edge_open_x(geom):
    """open_x[i, j]: the edge from node (i, j) to node (i+1, j) is open."""
    nxe = geom.nxn if geom.px else geom.nxn - 1
    i = np.arange(nxe)[:, None]
    j = np.arange(geom.nyn)[None, :]
    # cells beside the x-edge at y = j: (i, j-1) and (i, j)
    a = geom.cell_is_plasma(np.broadcast_to(i, (nxe, geom.nyn)), np.broadcast_to(j - 1, (nxe, geom.nyn)))
    b = geom.cell_is_plasma(np.broadcast_to(i, (nxe, geom.nyn)), np.broadcast_to(j, (nxe, geom.nyn)))
    return a | b


def _edge_open_y(geom):
    """open_y[i, j]: the edge from node (i, j) to node (i, j+1) is open."""
    nye = geom.nyn if geom.py else geom.nyn - 1
    i = np.arange(geom.nxn)[:, None]
    j = np.arange(nye)[None, :]
    a = geom.cell_is_plasma(np.broadcast_to(i - 1, (geom.nxn, nye)), np.broadcast_to(j, (geom.nxn, nye)))
    b = geom.cell_is_plasma(np.broadcast_to(i, (geom.nxn, nye)), np.broadcast_to(j, (geom.nxn, nye)))
    return a | b


def efield(geom, phi):
    """(Ex, Ey) on the full node grid from phi on the full node grid."""
    phi = np.asarray(phi, dtype=np.float64)
    ox = _edge_open_x(geom)
    oy = _edge_open_y(geom)
    # potential differences along open edges
    if geom.px:
        dx = np.roll(phi, -1, axis=0) - phi
    else:
        dx = phi[1:, :] - phi[:-1, :]
    if geom.py:
        dy = np.roll(phi, -1, axis=1) - phi
    else:
        dy = phi[:, 1:] - phi[:, :-1]
    dx = np.where(ox, dx, 0.0)
    dy = np.where(oy, dy, 0.0)
    ox = ox.astype(np.float64)
    oy = oy.astype(np.float64)

    # per node: edge below (i-1 -> i) and edge above (i -> i+1)
    sx = np.zeros_like(phi)
    cx = np.zeros_like(phi)
    if geom.px:
        sx += dx + np.roll(dx, 1, axis=0)
        cx += ox + np.roll(ox, 1, axis=0)
    else:
        sx[:-1, :] += dx
        cx[:-1, :] += ox
        sx[1:, :] += dx
        cx[1:, :] += ox
    sy = np.zeros_like(phi)
    cy = np.zeros_like(phi)
    if geom.py:
        sy += dy + np.roll(dy, 1, axis=1)
        cy += oy + np.roll(oy, 1, axis=1)
    else:
        sy[:, :-1] += dy
        cy[:, :-1] += oy
        sy[:, 1:] += dy
        cy[:, 1:] += oy
    Ex = np.where(cx > 0, -sx / np.maximum(cx, 1.0), 0.0)
    Ey = np.where(cy > 0, -sy / np.maximum(cy, 1.0), 0.0)
    return Ex, Ey


def field_energy(Ex, Ey):
    """Electrostatic energy 1/2 sum_nodes |E|^2 (unit cell area)."""
    return 0.5 * float(np.sum(Ex * Ex) + np.sum(Ey * Ey))
