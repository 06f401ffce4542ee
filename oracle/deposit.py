"""Charge assignment (oracle; test infrastructure).

The paper does not say how particles are weighted to the grid.  The reading
taken is cloud-in-cell (bilinear area weighting, Birdsall & Langdon, the
paper's ref. [bir86]): a particle at (i + fx, j + fy) gives (1-fx)(1-fy),
fx(1-fy), (1-fx)fy and fx*fy of its weight to the nodes (i, j), (i+1, j),
(i, j+1), (i+1, j+1).  With unit mesh spacing the node density is the sum
of those shares times the particle weight 1/ppc (densities in units of n_0,
Eq. (5)).

Pinned by: the sum of the node density equals the total particle weight
(charge conservation) and the hand-computed shares of single particles
(tests/test_oracle_deposit.py).
"""
from __future__ import annotations

import numpy as np


def cic_density(geom, x, y, weight):
    """Node density [nxn, nyn] from particles at absolute (x, y), each of
    the given weight (scalar or array).  Periodic directions wrap."""
    x = np.asarray(x, dtype=np.float64)
    y = np.asarray(y, dtype=np.float64)
    wgt = np.broadcast_to(np.asarray(weight, dtype=np.float64), x.shape)
    i = np.floor(x).astype(np.int64)
    j = np.floor(y).astype(np.int64)
    fx = x - i
    fy = y - j
    rho = np.zeros((geom.nxn, geom.nyn), dtype=np.float64)
    for di, wx in ((0, 1.0 - fx), (1, fx)):
        for dj, wy in ((0, 1.0 - fy), (1, fy)):
            ni = i + di
            nj = j + dj
            if geom.px:
                ni = ni % geom.nxn
            if geom.py:
                nj = nj % geom.nyn
            np.add.at(rho, (ni, nj), wgt * wx * wy)
    return rho


def surface_charge_density(geom, sigma_bottom):
    """Node density of the charge collected on the x = nx face.

    sigma_bottom[k] is the net collected charge (in particle weights times
    species charge) on the face of bottom cell k, y in [k, k+1].  The paper
    places its prescribed build-up charge one node row above the trench
    bottom (Sec. III-D: x = 79 with the bottom at x = 80); the reading taken
    here puts half of face k's charge on node (nx-1, k) and half on
    (nx-1, k+1).  Nodes that are Dirichlet ignore it.
    """
    rho = np.zeros((geom.nxn, geom.nyn), dtype=np.float64)
    if geom.px:
        return rho
    k = np.arange(geom.ny)
    half = 0.5 * np.asarray(sigma_bottom, dtype=np.float64)
    np.add.at(rho, (np.full_like(k, geom.nx - 1), k), half)
    kp = k + 1
    if geom.py:
        kp = kp % geom.nyn
    np.add.at(rho, (np.full_like(k, geom.nx - 1), kp), half)
    return rho
