"""Shared helpers of the GPU parity tests: run the CUDA path (through the
C ABI) and the FP64 oracle from identical seeded states and compare."""
import numpy as np

import synth
from oracle import push as opush
from oracle.sim import Sim as OracleSim

# Tolerances of the parity protocol (floating point, GPU FP32 vs FP64 oracle)
RHO_TOL = 1e-5      # of max |rho|
FIELD_TOL = 1e-5    # of max |E| (both solves to rel. residual 1e-10)
POS_TOL = 1e-5      # cells
VEL_TOL = 1e-5      # of max(|v|, v_th)


def gpu_sim(w, capacity=None, **kw):
    import paper_1610_03918_gb300 as pg
    return pg.Sim(w, capacity=capacity, **kw)


def oracle_sim(w):
    return OracleSim(w)


def load_both(gs, os_, species, p, v_at_t0=False):
    gs.load_particles(species, p, v_at_t0=v_at_t0)
    os_.load_particles(species, p, v_at_t0=v_at_t0)


def by_id(state):
    """GPU state [5, n] (x, y, vx, vy, id) sorted by id."""
    order = np.argsort(state[4], kind="stable")
    return state[:, order]


def oracle_state(os_, s):
    ps = os_.p[s]
    order = np.argsort(ps["ids"], kind="stable")
    return np.stack([ps["x"][order], ps["y"][order], ps["vx"][order], ps["vy"][order],
                     ps["ids"][order].astype(np.float64)])


def periodic_diff(a, b, period):
    d = a - b
    if period:
        d = d - period * np.round(d / period)
    return d


def compare_states(gstate, ostate, w, s):
    g = by_id(gstate)
    o = ostate
    assert g.shape == o.shape, (g.shape, o.shape)
    assert np.array_equal(g[4], o[4]), "live particle ids differ"
    dx = periodic_diff(g[0], o[0], w.nx if w.periodic_x else 0)
    dy = periodic_diff(g[1], o[1], w.ny if w.periodic_y else 0)
    assert np.abs(dx).max(initial=0) <= POS_TOL, np.abs(dx).max()
    assert np.abs(dy).max(initial=0) <= POS_TOL, np.abs(dy).max()
    vs = np.maximum(np.maximum(np.abs(o[2]), np.abs(o[3])), w.vth[s])
    assert (np.abs(g[2] - o[2]) <= VEL_TOL * vs).all(), np.abs(g[2] - o[2]).max()
    assert (np.abs(g[3] - o[3]) <= VEL_TOL * vs).all(), np.abs(g[3] - o[3]).max()


def vacuum_field(w):
    """E of the empty box (Dirichlet values only) by the oracle."""
    from oracle import field, poisson
    from oracle.geometry import from_workload
    geom = from_workload(w)
    phi = poisson.solve_direct(geom, np.zeros((geom.nxn, geom.nyn)))
    return field.efield(geom, phi)


def off_face_state(w, species, n, seed, vscale, E, margin=1e-4):
    """A random state whose one-step moves under the node field E (oracle
    push) end at least ``margin`` from every cell face and are at least
    ``margin`` away from a tie between an x and a y face crossing, so that
    the FP32 and FP64 walks classify every particle alike."""
    from oracle.geometry import from_workload
    geom = from_workload(w)
    p = synth.random_state(w, species, n, seed, vscale=vscale)
    p = synth.keep_off_faces(p, w, margin=1e-3)
    ex, ey = opush.gather(geom, E[0], E[1], p.x, p.y)
    a = w.alpha[species]
    vx1 = p.vx + a * ex * w.dt
    vy1 = p.vy + a * ey * w.dt
    x1 = p.x + vx1 * w.dt
    y1 = p.y + vy1 * w.dt
    fx = x1 - np.floor(x1)
    fy = y1 - np.floor(y1)
    ok = (np.minimum(fx, 1 - fx) > margin) & (np.minimum(fy, 1 - fy) > margin)
    i0, j0 = np.floor(p.x), np.floor(p.y)
    facex = np.where(vx1 > 0, i0 + 1, i0)
    facey = np.where(vy1 > 0, j0 + 1, j0)
    dx, dy = np.abs(vx1 * w.dt), np.abs(vy1 * w.dt)
    tx = np.abs(facex - p.x) / np.maximum(dx, 1e-30)
    ty = np.abs(facey - p.y) / np.maximum(dy, 1e-30)
    ok &= np.abs(tx - ty) > margin
    return p.subset(np.nonzero(ok)[0])


def face_distance(x):
    f = x - np.floor(x)
    return np.minimum(f, 1.0 - f)


def compare_states_grazing(gstate, ostate, w, s, graze=1e-5):
    """compare_states, except that particles alive on one side only must
    have ended within ``graze`` of a cell face (FP32 and FP64 may then
    decide the crossing differently)."""
    g = by_id(gstate)
    o = ostate
    gi = g[4].astype(np.int64)
    oi = o[4].astype(np.int64)
    common, ig, io = np.intersect1d(gi, oi, assume_unique=True, return_indices=True)
    only_g = np.setdiff1d(np.arange(gi.size), ig)
    only_o = np.setdiff1d(np.arange(oi.size), io)
    for arr, idx in ((g, only_g), (o, only_o)):
        if idx.size:
            d = np.minimum(face_distance(arr[0, idx]), face_distance(arr[1, idx]))
            assert (d <= graze).all(), ("non-grazing aliveness mismatch", d.max())
    compare_states(g[:, ig], o[:, io], w, s)
    return common.size, only_g.size + only_o.size
