"""Shared helpers of the GPU parity tests: run the CUDA path (through the
C ABI) and the FP64 oracle from identical seeded states and compare."""
import numpy as np

import synth
from oracle import push as opush
from oracle.geometry import from_workload
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


def gpu_drift_end(w, before, vx1, vy1):
    """The GPU's own x^{n+1} before any wrap or absorption: its drift adds
    v^{n+1/2} dt to the in-cell offset in FP32 (product and sum each rounded
    to nearest), and the end cell is the floor of that sum.  `before` is an
    exported state [5, n]; its positions are i + f with f the exact FP32
    offset, so the offsets are recovered exactly."""
    f32 = np.float32
    i = np.floor(before[0])
    j = np.floor(before[1])
    fx = (before[0] - i).astype(f32)
    fy = (before[1] - j).astype(f32)
    dt = f32(w.dt)
    nfx = fx + np.asarray(vx1, f32) * dt
    nfy = fy + np.asarray(vy1, f32) * dt
    return i + nfx.astype(np.float64), j + nfy.astype(np.float64)


def _near_tie(x0, y0, x1, y1, tol=1e-6, maxc=4):
    """True where the segment crosses an x face and a y face at segment
    parameters closer than tol (the crossing order is then decided by
    rounding, FP32 on the GPU against exact FP64 in the oracle)."""
    dx, dy = x1 - x0, y1 - y0
    ci, cj = np.floor(x0), np.floor(y0)
    ti, tj = np.floor(x1), np.floor(y1)
    nx_c = np.abs(ti - ci).astype(np.int64)
    ny_c = np.abs(tj - cj).astype(np.int64)
    tie = (nx_c > maxc) | (ny_c > maxc)
    both = (nx_c > 0) & (ny_c > 0) & ~tie
    if not both.any():
        return tie
    sx = np.where(dx > 0, 1.0, -1.0)
    sy = np.where(dy > 0, 1.0, -1.0)
    fx0 = np.where(dx > 0, ci + 1, ci)
    fy0 = np.where(dy > 0, cj + 1, cj)
    best = np.full(x0.size, np.inf)
    for a in range(maxc):
        tx = np.abs(fx0 + a * sx - x0) / np.maximum(np.abs(dx), 1e-300)
        for b in range(maxc):
            ty = np.abs(fy0 + b * sy - y0) / np.maximum(np.abs(dy), 1e-300)
            ok = both & (a < nx_c) & (b < ny_c)
            best = np.where(ok, np.minimum(best, np.abs(tx - ty)), best)
    return tie | (best <= tol)


def check_gpu_classification(w, before, after, hits, step, walls_delta, bottom_delta):
    """Protocol part (ii): the oracle's face classifier run on the GPU's own
    x^n and x^{n+1} (grazing particles included) must reproduce, bit for
    bit, which particles the GPU absorbed, their walls and wall cells, and
    the per-wall and per-bottom-cell tallies of the step.  v^{n+1/2} comes
    from the GPU: the post-step state for live particles, the hit record for
    absorbed ones.  Live end positions must equal the GPU's drift to FP32
    rounding.  Returns the number of particles whose x/y crossing order was
    a near tie (exempt; expected 0 on these sizes)."""
    geom = from_workload(w)
    hs = hits[hits["step"] == step]
    ties = 0
    walls = np.zeros((2, opush.N_WALLS), np.int64)
    bottom = np.zeros((2, w.ny), np.int64)
    for s in (0, 1):
        b = by_id(before[s])
        a = by_id(after[s])
        hsel = hs[hs["species"] == s]
        ids_b = b[4].astype(np.int64)
        ids_a = a[4].astype(np.int64)
        if s == 1 and getattr(w, "recycle", False) and hsel.size:
            # every ion absorbed this step re-enters with its id: its position
            # must be the oracle's draw bit for bit, its velocity within the
            # push tolerance (FP32 Box-Muller against FP64)
            reborn = np.isin(ids_a, hsel["id"].astype(np.int64))
            r = OracleSim(w).recycled(np.sort(hsel["id"]), step)
            ar = a[:, reborn]
            assert np.array_equal(ar[4].astype(np.int64), r["ids"].astype(np.int64))
            assert np.array_equal(ar[0], r["x"]) and np.array_equal(ar[1], r["y"])
            assert np.abs(ar[2] - r["vx"]).max() <= VEL_TOL * w.vth[1]
            assert np.abs(ar[3] - r["vy"]).max() <= VEL_TOL * w.vth[1]
            a = a[:, ~reborn]
            ids_a = ids_a[~reborn]
        pos_a = np.searchsorted(ids_b, ids_a)
        assert np.array_equal(ids_b[np.minimum(pos_a, ids_b.size - 1)], ids_a)
        pos_h = np.searchsorted(ids_b, hsel["id"].astype(np.int64))
        assert np.array_equal(ids_b[np.minimum(pos_h, ids_b.size - 1)], hsel["id"].astype(np.int64))
        vx1 = np.full(ids_b.size, np.nan)
        vy1 = np.full(ids_b.size, np.nan)
        vx1[pos_a], vy1[pos_a] = a[2], a[3]
        vx1[pos_h], vy1[pos_h] = hsel["vx"], hsel["vy"]
        assert np.isfinite(vx1).all(), "a particle neither live nor recorded as a hit"
        x1, y1 = gpu_drift_end(w, b, vx1, vy1)
        alive, wall, wcell = opush.classify(geom, b[0], b[1], x1, y1)
        g_alive = np.zeros(ids_b.size, bool)
        g_alive[pos_a] = True
        g_wall = np.full(ids_b.size, -1, np.int64)
        g_cell = np.full(ids_b.size, -1, np.int64)
        g_wall[pos_h] = hsel["wall"]
        g_cell[pos_h] = hsel["cell"]
        mism = (alive != g_alive) | (wall != g_wall) | (~alive & (wcell != g_cell))
        tie = _near_tie(b[0], b[1], x1, y1)
        assert not (mism & ~tie).any(), ("classification differs", int((mism & ~tie).sum()))
        ties += int(tie.sum())
        # the stored end positions are the drift's, wrapped where periodic
        xw = np.mod(x1[pos_a], w.nx) if w.periodic_x else x1[pos_a]
        yw = np.mod(y1[pos_a], w.ny) if w.periodic_y else y1[pos_a]
        ex = periodic_diff(a[0], xw, w.nx if w.periodic_x else 0)
        ey = periodic_diff(a[1], yw, w.ny if w.periodic_y else 0)
        assert np.abs(ex).max(initial=0) <= 2.0 ** -22 and np.abs(ey).max(initial=0) <= 2.0 ** -22
        np.add.at(walls[s], g_wall[~g_alive], 1)
        xm = ~g_alive & (g_wall == opush.WALL_XMAX)
        np.add.at(bottom[s], g_cell[xm], 1)
    if walls_delta is not None:
        assert np.array_equal(walls, walls_delta)
    if bottom_delta is not None:
        assert np.array_equal(bottom, bottom_delta)
    return ties


def check_rho_of_gpu_state(w, gs, after):
    """The GPU's rho^{n+1} against the oracle's FP64 deposit of the GPU's own
    post-step state plus the surface charge of its bottom counts, at the
    deposit tolerance (no allowance for grazing particles: both sides
    deposit the same particles)."""
    ref = OracleSim(w)
    for s in (0, 1):
        a = after[s]
        ref.load(s, a[0], a[1], a[2], a[3], a[4].astype(np.uint32))
    ref.bottom[:] = gs.surface()
    ro = ref.charge_density()
    rg = gs.rho()
    assert np.abs(rg - ro).max() <= RHO_TOL * np.abs(ro).max(), np.abs(rg - ro).max() / np.abs(ro).max()


def parity_pre(w, gs, step=0):
    """First half of one step of the step-by-step protocol for a GPU run
    `gs` (a Sim view): the oracle restarts from the GPU's state (its bottom
    charge and tallies included) and both fields of that state agree."""
    before = [gs.state(0), gs.state(1)]
    walls0 = gs.counts()[0]
    bottom0 = gs.surface()
    os_ = OracleSim(w)
    for s in (0, 1):
        st = before[s]
        os_.load(s, st[0], st[1], st[2], st[3], st[4].astype(np.uint32))
    os_.bottom[:] = bottom0
    os_.counts[:] = walls0
    os_.nstep = step            # the time level (RF bias) and the draws' step index
    os_.prepare()
    Exg, Eyg = gs.efield()
    emax = max(np.abs(os_.Ex).max(), np.abs(os_.Ey).max())
    assert np.abs(Exg - os_.Ex).max() <= FIELD_TOL * emax
    assert np.abs(Eyg - os_.Ey).max() <= FIELD_TOL * emax
    return dict(before=before, walls0=walls0, bottom0=bottom0, os=os_)


def parity_post(w, gs, pre, step):
    """Second half, after the GPU took its step: the oracle takes its own;
    states agree (grazing particles excepted), the GPU's classification is
    reproduced bit for bit by the oracle's classifier on the GPU's own
    positions, and the GPU's rho is the oracle deposit of the GPU's state.
    Returns (near-tie crossings exempted, the oracle run)."""
    os_ = pre["os"]
    os_.step(1)
    after = [gs.state(0), gs.state(1)]
    for s in (0, 1):
        compare_states_grazing(after[s], oracle_state(os_, s), w, s)
    ties = check_gpu_classification(w, pre["before"], after, gs.hits(), step,
                                    gs.counts()[0] - pre["walls0"], gs.surface() - pre["bottom0"])
    check_rho_of_gpu_state(w, gs, after)
    return ties, os_


def step_parity_once(w, gs, advance, step):
    """One step of the step-by-step protocol: parity_pre, advance(), parity_post."""
    pre = parity_pre(w, gs, step)
    advance()
    return parity_post(w, gs, pre, step)
