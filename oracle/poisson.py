"""The normalised Poisson equation, Eq. (5) of Sec. II (oracle; test
infrastructure).

Eq. (5) reads (d2/dx2 + d2/dy2) Phi = n_e - (q_i/e) n_i.  With unit mesh
spacing and the 5-point Laplacian Delta_h, the discrete system on the free
(non-Dirichlet) nodes is

    A phi = b,   A = -Delta_h,   b = rho + (sum of Dirichlet neighbour values),

with rho = (q_i/e) n_i - n_e the net charge density (rho = sum_s q_s n_s
with q_e = -1).  Dirichlet nodes (conductors, the plates) hold their values
(Sec. II: homogeneous Dirichlet on one electrode, a set bias on the other;
Sec. III-A: grounded walls).  A periodic direction wraps (Sec. III-B).  A
doubly periodic box has no Dirichlet node; A is then singular and the
reading taken is: remove the mean of rho and fix phi by zero mean.

Solvers
  solve_direct  sparse LU of A (scipy), factorised once per geometry
  solve_dft     exact separable DFT solve for the doubly periodic box
                (eigenvalues 4 - 2cos(2 pi k/Nx) - 2cos(2 pi l/Ny))
  gauss_seidel  lexicographic Gauss-Seidel, the paper's solver (Sec. II)
  jacobi        Jacobi, the paper's other solver (Sec. II)

Pinned by (tests/test_oracle_poisson.py): the DFT and the direct solve agree
on a periodic box; the linear potential between biased plates is
reproduced exactly; a continuous manufactured solution converges at second
order; Gauss-Seidel and Jacobi agree with the direct solve on a trench.
"""
from __future__ import annotations

import numpy as np
import scipy.sparse as sp
import scipy.sparse.linalg as spla


def _neighbours(geom, i, j):
    """The four neighbour node indices of nodes (i, j), wrapped where
    periodic.  Only used for free nodes, which are interior in any bounded
    direction."""
    out = []
    for di, dj in ((-1, 0), (1, 0), (0, -1), (0, 1)):
        ni = i + di
        nj = j + dj
        if geom.px:
            ni = ni % geom.nxn
        if geom.py:
            nj = nj % geom.nyn
        out.append((ni, nj))
    return out


def system(geom):
    """(A, free_i, free_j, lift): A over the free nodes in row-major order
    and the Dirichlet lift vector of the geometry's current Dirichlet
    values.  A and the neighbour indices are cached on the geometry; the
    lift is formed from geom.g on every call (it changes with an RF bias)."""
    cache = getattr(geom, "_poisson_system", None)
    if cache is None:
        free = geom.free
        fi, fj = np.nonzero(free)
        nf = fi.size
        index = -np.ones((geom.nxn, geom.nyn), dtype=np.int64)
        index[fi, fj] = np.arange(nf)
        rows = [np.arange(nf)]
        cols = [np.arange(nf)]
        vals = [np.full(nf, 4.0)]
        dir_nbrs = []
        for ni, nj in _neighbours(geom, fi, fj):
            m = index[ni, nj]
            isfree = m >= 0
            rows.append(np.arange(nf)[isfree])
            cols.append(m[isfree])
            vals.append(-np.ones(int(isfree.sum())))
            dir_nbrs.append((np.nonzero(~isfree)[0], ni[~isfree], nj[~isfree]))
        A = sp.csc_matrix((np.concatenate(vals), (np.concatenate(rows), np.concatenate(cols))),
                          shape=(nf, nf))
        cache = (A, fi, fj, dir_nbrs)
        geom._poisson_system = cache
    A, fi, fj, dir_nbrs = cache
    lift = np.zeros(fi.size)
    for k, ni, nj in dir_nbrs:
        lift[k] += geom.g[ni, nj]
    return A, fi, fj, lift


def rhs(geom, rho):
    """b on the free nodes: rho plus the Dirichlet lift."""
    A, fi, fj, lift = system(geom)
    return np.asarray(rho, dtype=np.float64)[fi, fj] + lift


def is_singular(geom):
    return not geom.dirichlet.any()


def apply_A(geom, phi):
    """(A phi) on the free nodes, phi given on the full node grid (its
    Dirichlet entries are taken from phi itself)."""
    A, fi, fj, lift = system(geom)
    out = 4.0 * phi[fi, fj]
    for ni, nj in _neighbours(geom, fi, fj):
        out -= phi[ni, nj]
    return out


def residual_rel(geom, phi, rho):
    """||b - A phi||_2 / ||b||_2 over the free nodes, phi on the full grid
    with Dirichlet nodes at their values (b includes the lift)."""
    A, fi, fj, lift = system(geom)
    b = np.asarray(rho, dtype=np.float64)[fi, fj]
    if is_singular(geom):
        b = b - b.mean()
    r = b - apply_A(geom, phi)
    # apply_A took the Dirichlet neighbours from phi, so b here has no lift
    nb = np.linalg.norm(b + lift)
    return float(np.linalg.norm(r) / nb) if nb > 0 else float(np.linalg.norm(r))


def full_grid(geom, phi_free):
    A, fi, fj, lift = system(geom)
    phi = geom.g.copy()
    phi[fi, fj] = phi_free
    return phi


def solve_direct(geom, rho):
    """Sparse LU solve of A phi = b; phi returned on the full node grid."""
    if is_singular(geom):
        return solve_dft(geom, rho)
    A, fi, fj, lift = system(geom)
    lu = getattr(geom, "_poisson_lu", None)
    if lu is None:
        lu = spla.splu(A, permc_spec="COLAMD")
        geom._poisson_lu = lu
    return full_grid(geom, lu.solve(rhs(geom, rho)))


def solve_dft(geom, rho):
    """Exact solve on the doubly periodic box: phi_hat = rho_hat / lambda,
    lambda(k, l) = 4 - 2 cos(2 pi k / Nx) - 2 cos(2 pi l / Ny); the (0, 0)
    mode (the mean) is set to zero."""
    assert geom.px and geom.py
    r = np.asarray(rho, dtype=np.float64)
    rh = np.fft.fft2(r - r.mean())
    kx = np.arange(geom.nxn)[:, None]
    ky = np.arange(geom.nyn)[None, :]
    lam = 4.0 - 2.0 * np.cos(2 * np.pi * kx / geom.nxn) - 2.0 * np.cos(2 * np.pi * ky / geom.nyn)
    lam[0, 0] = 1.0
    ph = rh / lam
    ph[0, 0] = 0.0
    return np.real(np.fft.ifft2(ph))


def gauss_seidel(geom, rho, tol=1e-12, max_sweeps=200000, phi0=None):
    """Lexicographic Gauss-Seidel on the free nodes (the paper's solver,
    Sec. II): phi_n <- (b_n + sum of free neighbour phi) / 4, swept in
    row-major order until the relative residual is below tol."""
    A, fi, fj, lift = system(geom)
    b = rhs(geom, rho)
    if is_singular(geom):
        b = b - b.mean()
    nf = fi.size
    index = -np.ones((geom.nxn, geom.nyn), dtype=np.int64)
    index[fi, fj] = np.arange(nf)
    nb = [index[ni, nj] for ni, nj in _neighbours(geom, fi, fj)]
    nbr = np.stack(nb, axis=1)            # [nf, 4], -1 = Dirichlet
    u = np.zeros(nf) if phi0 is None else np.asarray(phi0, dtype=np.float64)[fi, fj].copy()
    nrm = np.linalg.norm(b)
    nbr_l = nbr.tolist()
    b_l = b.tolist()
    for sweep in range(max_sweeps):
        ul = u.tolist()
        for n in range(nf):
            s = b_l[n]
            for m in nbr_l[n]:
                if m >= 0:
                    s += ul[m]
            ul[n] = 0.25 * s
        u = np.asarray(ul)
        if sweep % 20 == 19:
            r = b - A @ u
            if np.linalg.norm(r) <= tol * nrm:
                break
    if is_singular(geom):
        u = u - u.mean()
    return full_grid(geom, u)


def jacobi(geom, rho, tol=1e-10, max_sweeps=2000000):
    """Jacobi iteration on the free nodes (the paper's other solver)."""
    A, fi, fj, lift = system(geom)
    b = rhs(geom, rho)
    if is_singular(geom):
        b = b - b.mean()
    nf = fi.size
    offd = A - sp.diags(A.diagonal())
    u = np.zeros(nf)
    nrm = np.linalg.norm(b)
    for sweep in range(max_sweeps):
        u = (b - offd @ u) / 4.0
        if sweep % 50 == 49 and np.linalg.norm(b - A @ u) <= tol * nrm:
            break
    if is_singular(geom):
        u = u - u.mean()
    return full_grid(geom, u)
