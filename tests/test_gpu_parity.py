"""CUDA path (through the C ABI) against the FP64 oracle on identical seeded
states: deposit, Poisson solve, field, push, absorption tallies, surface
charge, per-step parity and edge cases.  Needs a GB300."""
import numpy as np
import pytest

import synth
from oracle import field as ofield
from oracle import poisson as opoisson
from oracle.geometry import from_workload

from gpu_helpers import (FIELD_TOL, RHO_TOL, compare_states, gpu_sim, load_both, off_face_state,
                         oracle_sim, oracle_state, step_parity_once, vacuum_field)

pytestmark = pytest.mark.gpu

# workloads small enough for the oracle, spanning several 16x16 tiles with
# ragged tails
SMALL = {
    "trench": synth.small_trench(nx=72, ny=40, depth=20, width=6, ppc=12, seed=11),
    "bounded": synth.bounded_square_256(nx=45, ny=38, ppc=10, seed=12),
    "periodic": synth.periodic_square_64(nx=48, ny=34, ppc=10, seed=13),
}


# boxes periodic in y with a power-of-two ny and bounded in x: the direct
# (FFT / tridiagonal / interface) inner Poisson solve applies
DIRECT = {
    "trench64": synth.small_trench(nx=72, ny=64, depth=20, width=6, ppc=12, seed=31),
    "trench32_wide": synth.small_trench(nx=40, ny=32, depth=10, width=11, ppc=12, seed=32),
    "plates": synth.small_trench(nx=48, ny=64, depth=0, width=0, ppc=10, seed=33),
    "slit": synth.small_trench(nx=48, ny=64, depth=12, width=1, ppc=10, seed=34),
}
ALL = {**SMALL, **DIRECT}


@pytest.fixture(scope="module", autouse=True)
def _built():
    import __graft_entry__
    __graft_entry__.build()


def _loaded(w, rtol=1e-10, **kw):
    w = w.replace(poisson_rtol=rtol)
    gs = gpu_sim(w, **kw)
    os_ = oracle_sim(w)
    for s in (0, 1):
        load_both(gs, os_, s, synth.maxwellian_load(w, s))
    return w, gs, os_


@pytest.mark.parametrize("name", list(SMALL))
def test_deposit_matches_oracle(name):
    w, gs, os_ = _loaded(SMALL[name])
    gs.step(0)
    rg = gs.rho()
    ro = os_.charge_density()
    scale = np.abs(ro).max()
    assert np.abs(rg - ro).max() <= RHO_TOL * scale, np.abs(rg - ro).max() / scale
    # charge conservation: the fixed-point deposit is exact per particle
    assert rg.sum() == pytest.approx(ro.sum(), abs=1e-9 * np.abs(ro).sum())


def test_deposit_particles_on_grid_lines():
    # Particles exactly on the horizontal grid lines of every other cell row:
    # the node row above each line gets shares 0 from the fixed-point rounding
    # and -1 where the three rounded shares overshoot, and nothing else, so
    # the chunk sums of those nodes are negative.  The exact CIC density is 0
    # there; a sum decoded as unsigned would be off by 2^32 units.
    w = synth.periodic_square_64(nx=48, ny=34, ppc=100, seed=17)
    rng = np.random.default_rng(17)
    ci, cj = np.meshgrid(np.arange(48), np.arange(0, 34, 2), indexing="ij")
    ci, cj = np.repeat(ci.ravel(), 100), np.repeat(cj.ravel(), 100)
    n = ci.size
    p = synth.Particles(ci + rng.random(n), cj.astype(np.float64), np.zeros(n), np.zeros(n),
                        np.arange(n, dtype=np.uint32))
    gs = gpu_sim(w)
    os_ = oracle_sim(w)
    for s in (0, 1):
        q = p if s == 0 else p.subset(slice(0, n, 3))
        load_both(gs, os_, s, q)
    gs.step(0)
    rg, ro = gs.rho(), os_.charge_density()
    assert np.all(ro[:, 1::2] == 0.0)
    assert np.abs(rg - ro).max() <= RHO_TOL * np.abs(ro).max()
    assert rg.sum() == pytest.approx(ro.sum(), abs=1e-9 * np.abs(ro).sum())


@pytest.mark.parametrize("name", list(ALL))
def test_poisson_and_field_match_oracle(name):
    import paper_1610_03918_gb300 as pg
    w = ALL[name].replace(poisson_rtol=1e-10)
    gs = gpu_sim(w)
    assert gs.solver() == (pg.POISSON_AUTO if name in DIRECT else pg.POISSON_MULTIGRID)
    geom = from_workload(w)
    rho = synth.random_rho(w, seed=21, scale=0.3)
    gs.set_rho_ext(rho)
    gs.step(0)
    it, outer, rel, ms, rel0 = gs.poisson_stats()
    assert rel <= 1e-10
    phi_g = gs.phi()
    phi_o = opoisson.solve_direct(geom, rho)
    # the oracle's own FP64 residual of the GPU potential certifies it
    assert opoisson.residual_rel(geom, phi_g, rho) <= 2e-10
    assert np.abs(phi_g - phi_o).max() <= 1e-6 * np.abs(phi_o).max()
    Exg, Eyg = gs.efield()
    Exo, Eyo = ofield.efield(geom, phi_o)
    emax = max(np.abs(Exo).max(), np.abs(Eyo).max())
    assert np.abs(Exg - Exo).max() <= FIELD_TOL * emax
    assert np.abs(Eyg - Eyo).max() <= FIELD_TOL * emax


def test_poisson_trench_bias_vacuum():
    # the biased electrode with the trench and no charge: a pure Laplace solve
    w = synth.small_trench(nx=96, ny=64, depth=40, width=10).replace(poisson_rtol=1e-10)
    gs = gpu_sim(w)
    gs.step(0)
    geom = from_workload(w)
    phi_o = opoisson.solve_direct(geom, np.zeros((geom.nxn, geom.nyn)))
    assert np.abs(gs.phi() - phi_o).max() <= 1e-6 * 20.0


def test_direct_and_multigrid_solves_agree():
    import paper_1610_03918_gb300 as pg
    w = DIRECT["trench64"].replace(poisson_rtol=1e-10)
    rho = synth.random_rho(w, seed=23, scale=0.3)
    out = []
    for method in (pg.POISSON_AUTO, pg.POISSON_MULTIGRID):
        gs = gpu_sim(w, poisson_method=method)
        assert gs.solver() == method
        gs.set_rho_ext(rho)
        gs.step(0)
        out.append((gs.phi(), gs.poisson_stats()))
    (pd, sd), (pm, sm) = out
    assert np.abs(pd - pm).max() <= 1e-8 * np.abs(pm).max()
    # the direct inner solve needs a refinement pass or two, not an iteration count
    assert sd[0] <= 3


def test_tuned_sort_interval_changes_no_result():
    # sort_every = 0: the library times the particle kernel after a sort and
    # picks the interval; the physics must be bitwise that of a fixed interval
    # (exact deposit, order-independent push, fixed-order reductions)
    w = DIRECT["trench64"]
    runs = []
    for se in (0, 8):
        gs = gpu_sim(w.replace(sort_every=se))
        for s in (0, 1):
            gs.load_particles(s, synth.maxwellian_load(w, s), v_at_t0=True)
        gs.step(60)
        runs.append(gs)
    tuned, fixed = runs
    S, was_tuned = tuned.sort_interval()
    assert was_tuned and 4 <= S <= 48, S
    assert fixed.sort_interval() == (8, False)
    by_id = lambda st: st[:, np.argsort(st[4], kind="stable")]
    for s in (0, 1):
        assert np.array_equal(by_id(tuned.state(s)), by_id(fixed.state(s)))
    assert np.array_equal(tuned.rho(), fixed.rho())
    assert np.array_equal(tuned.phi(), fixed.phi())
    assert np.array_equal(tuned.counts()[0], fixed.counts()[0])


@pytest.mark.parametrize("name", ["trench64", "trench"])
def test_phase_timing_changes_no_result(name):
    # timed graph steps carry event nodes between the phases and record them
    # into a pool of slots read back later; the physics is the same bitwise,
    # and the counts of steps and launches agree with the untimed run's
    w = ALL[name].replace(sort_every=8)
    runs = []
    for timing in (True, False):
        gs = gpu_sim(w, timing=timing)
        for s in (0, 1):
            gs.load_particles(s, synth.maxwellian_load(w, s), v_at_t0=True)
        gs.step(1)
        gs.timing()
        gs.step(70)                 # more steps than the pool's 64 slots
        gs.set_timing(not timing)   # both graph kinds within one run
        gs.step(5)
        runs.append((gs, gs.timing()))
    (a, ta), (b, tb) = runs
    by_id = lambda st: st[:, np.argsort(st[4], kind="stable")]
    for s in (0, 1):
        assert np.array_equal(by_id(a.state(s)), by_id(b.state(s)))
    assert np.array_equal(a.phi(), b.phi())
    assert np.array_equal(a.efield()[0], b.efield()[0])
    assert ta["steps"] == tb["steps"] == 75
    assert ta["launches"] == tb["launches"] > 75 * 4
    assert ta["ms_particles"] > 0 and ta["ms_poisson"] > 0 and tb["ms_particles"] > 0


@pytest.mark.parametrize("name", ["trench64", "trench"])
def test_warm_start_modes_reach_the_same_fields(name):
    import paper_1610_03918_gb300 as pg
    # zero, previous, extrapolated and lift (the empty-box potential)
    # initial guesses (in the captured step graph the first two differ in
    # their kernels: with the direct solve and the previous potential the
    # first residual pass also forms rho)
    w = ALL[name].replace(poisson_rtol=1e-10, sort_every=8)
    phis = []
    for ws in (0, 1, 2, 4):
        gs = gpu_sim(w, warm_start=ws)
        for s in (0, 1):
            gs.load_particles(s, synth.maxwellian_load(w, s), v_at_t0=True)
        gs.step(3)
        it, outer, rel, ms, rel0 = gs.poisson_stats()
        assert rel <= 1e-10 and outer >= 1, (ws, rel, outer)
        # from the zero guess the initial residual is b itself (the multigrid
        # solve checks the guess; the direct one checks after its first correction)
        if ws == 0 and gs.solver() == pg.POISSON_MULTIGRID:
            assert abs(rel0 - 1.0) <= 1e-5, rel0
        assert rel0 >= rel
        assert gs.status() == 0
        phis.append(gs.phi())
    for p in phis[1:]:
        assert np.abs(p - phis[0]).max() <= 1e-6 * np.abs(phis[0]).max()


def test_load_from_pinned_host_memory_matches_pageable():
    # pinned arrays are read by the conversion kernel in place, pageable ones
    # go through the staging copies: the loaded state is the same
    torch = pytest.importorskip("torch")
    w = SMALL["trench"]
    p = synth.maxwellian_load(w, 0)
    a, b = gpu_sim(w), gpu_sim(w)
    a.load_particles(0, p)
    pin = [torch.from_numpy(np.ascontiguousarray(v, dtype=np.float64)).pin_memory()
           for v in (p.x, p.y, p.vx, p.vy)]
    ids = torch.from_numpy(np.ascontiguousarray(p.ids, dtype=np.uint32).view(np.int32)).pin_memory()
    b.load(0, *[t.numpy() for t in pin], ids.numpy().view(np.uint32))
    by_id = lambda st: st[:, np.argsort(st[4], kind="stable")]   # export order is arbitrary
    assert np.array_equal(by_id(a.state(0)), by_id(b.state(0)))


def test_direct_solver_applies_only_to_its_geometry():
    import paper_1610_03918_gb300 as pg
    for w in (synth.small_trench(nx=40, ny=40),            # ny not a power of two
              synth.bounded_square_256(nx=32, ny=32),      # y bounded
              synth.periodic_square_64(nx=32, ny=32)):     # x periodic
        assert gpu_sim(w).solver() == pg.POISSON_MULTIGRID, w.name


@pytest.mark.parametrize("name,graphs", [(n, True) for n in SMALL] + [("trench", False)] +
                         [("trench64", True), ("trench64", False)])
def test_step_by_step_parity(name, graphs):
    """Each step starts the oracle from the GPU's state (its own fields
    recomputed from it).  After the step: states agree (moves ending within
    1e-5 of a face may be decided differently by FP32 and FP64), the oracle's
    classifier on the GPU's own positions reproduces the GPU's absorptions,
    walls, wall cells and tallies bit for bit, and the GPU's rho is the
    oracle deposit of the GPU's state within 1e-5 of max |rho|.  graphs=False
    drives the same kernels from the host loop instead of the captured step
    graph."""
    w, gs, os_ = _loaded(ALL[name], graphs=graphs)
    gs.step(0)
    ties = 0
    for k in range(4):
        t, os_ = step_parity_once(w, gs, lambda: gs.step(1), k)
        ties += t
        e = gs.energy()
        assert e[0] == pytest.approx(os_.ke[0], rel=1e-5)
        assert e[1] == pytest.approx(os_.ke[1], rel=1e-5)
        assert e[2] == pytest.approx(os_.fe, rel=1e-5)
    assert ties <= 2, ties


def test_absorption_tallies_bit_exact():
    # negligible particle weight: the field is the vacuum field of the biased
    # electrode, so the off-face margins hold for both sides
    w = synth.small_trench(nx=72, ny=40, depth=24, width=8, ppc=10 ** 7, seed=5).replace(
        poisson_rtol=1e-10)
    E = vacuum_field(w)
    gs = gpu_sim(w, capacity=200000)
    os_ = oracle_sim(w)
    pe = off_face_state(w, 0, 120000, seed=1, vscale=6.0, E=E)
    pi = off_face_state(w, 1, 120000, seed=2, vscale=400.0, E=E)
    load_both(gs, os_, 0, pe)
    load_both(gs, os_, 1, pi)
    gs.step(1)
    os_.step(1)
    walls, live = gs.counts()
    assert np.array_equal(walls, os_.counts)
    assert np.array_equal(live, os_.live())
    assert walls.sum() > 1000 and walls[1, 1] > 10 and walls[0, 6] > 0 and walls[0, 7] > 0
    assert np.array_equal(gs.surface(), os_.bottom)
    hg = gs.hits()
    ho = os_.hit_table()
    kg = sorted(zip(hg["species"].tolist(), hg["id"].tolist(), hg["wall"].tolist(), hg["cell"].tolist()))
    ko = sorted(zip(ho["species"].tolist(), ho["ids"].tolist(), ho["wall"].tolist(), ho["cell"].tolist()))
    assert kg == ko
    for s in (0, 1):
        compare_states(gs.state(s), oracle_state(os_, s), w, s)


def test_surface_charge_feeds_rho():
    w = synth.small_trench(nx=48, ny=32, depth=16, width=6, ppc=4).replace(poisson_rtol=1e-10)
    gs = gpu_sim(w)
    os_ = oracle_sim(w)
    y0 = w.trench_y0
    # ions moving straight into the bottom of the trench
    x = np.full(6, 47.95)
    y = y0 + 0.5 + np.arange(6, dtype=np.float64)
    load_both(gs, os_, 1, synth.Particles(x, y, np.full(6, 1.0), np.zeros(6), np.arange(6, dtype=np.uint32)))
    gs.step(1)
    os_.step(1)
    assert np.array_equal(gs.surface(), os_.bottom)
    assert gs.surface()[1, y0:y0 + 6].tolist() == [1] * 6
    np.testing.assert_allclose(gs.rho(), os_.rho, atol=1e-12)


def test_v_at_t0_half_kick_closed_form():
    w = synth.Workload(name="plates", nx=40, ny=16, periodic_y=True, phi_top=0.0,
                       phi_electrode=-20.0, ppc=10 ** 9, poisson_rtol=1e-10)
    gs = gpu_sim(w, capacity=16)
    x0, y0, v0x, v0y = 20.3, 3.6, 0.05, -0.02
    gs.load(1, [x0], [y0], [v0x], [v0y], v_at_t0=True)
    gs.step(50)
    t = 50 * w.dt
    a = w.alpha[1] * 0.5
    st = gs.state(1)
    assert st[0, 0] == pytest.approx(x0 + v0x * t + 0.5 * a * t * t, abs=2e-5)
    assert st[1, 0] == pytest.approx(y0 + v0y * t, abs=2e-5)


def test_edge_cases():
    import paper_1610_03918_gb300 as pg
    w = SMALL["trench"].replace(poisson_rtol=1e-10)
    gs = gpu_sim(w, capacity=1000)
    # empty species and an empty step
    gs.step(2)
    assert gs.counts()[1].tolist() == [0, 0]
    # particles exactly on faces and nodes, one per tile corner
    x = np.array([0.0, 16.0, 31.0, 47.0, 51.0])
    y = np.array([0.0, 16.0, 17.0, 32.0, 39.0])
    os_ = oracle_sim(w)
    p = synth.Particles(x, y, np.zeros(5), np.zeros(5), np.arange(5, dtype=np.uint32))
    load_both(gs, os_, 0, p)
    gs.step(0)
    os_.prepare()
    np.testing.assert_allclose(gs.rho(), os_.charge_density(), atol=1e-6)
    # over capacity
    big = np.zeros(1001)
    assert pg.pic_load(gs.ctx, 0, big, big, big, big) == pg.PIC_EOVERFLOW
    # a particle inside the conductor is dropped and flagged
    st = pg.pic_load(gs.ctx, 1, np.array([70.5, 3.5]), np.array([2.5, 3.5]), np.zeros(2), np.zeros(2))
    assert st == pg.PIC_OK
    gs.step(0)
    assert gs.counts()[1].tolist()[1] == 1
    assert gs.status() & pg.PIC_ST_RANGE
    assert gs.status() == 0


def test_hit_buffer_full_keeps_tallies_exact():
    import paper_1610_03918_gb300 as pg
    w = synth.small_trench(nx=48, ny=32, depth=16, width=6, ppc=10 ** 7).replace(poisson_rtol=1e-8)
    gs = gpu_sim(w, capacity=50000, hit_capacity=10)
    os_ = oracle_sim(w)
    E = vacuum_field(w)
    pe = off_face_state(w, 0, 40000, seed=3, vscale=8.0, E=E)
    load_both(gs, os_, 0, pe)
    gs.step(1)
    os_.step(1)
    walls, _ = gs.counts()
    assert np.array_equal(walls, os_.counts)
    assert len(gs.hits()) == 10
    assert gs.status() & pg.PIC_ST_FULL


def test_periodic_box_conservation():
    w = synth.periodic_square_64(ppc=20, poisson_rtol=1e-8)
    gs = gpu_sim(w)
    for s in (0, 1):
        gs.load_particles(s, synth.maxwellian_load(w, s), v_at_t0=True)
    gs.step(1)
    m0 = gs.momentum().sum(axis=0)
    e0 = gs.energy()
    tot0 = e0[0] + e0[1] + e0[2]
    gs.step(199)
    m1 = gs.momentum().sum(axis=0)
    e1 = gs.energy()
    tot1 = e1[0] + e1[1] + e1[2]
    # thermal momentum scale: sqrt(N) * m w v_th for electrons
    n = 64 * 64 * 20
    pscale = np.sqrt(n) / 20
    assert np.abs(m1 - m0).max() <= 1e-3 * pscale
    assert abs(tot1 - tot0) <= 0.01 * tot0


def test_walk_limit_drops_and_flags_the_particle():
    # A move across more cell faces than the walk limit (16) is dropped
    # untallied and flagged (PIC_ST_CFL); a long move within the limit (12
    # faces, out of the tile's shared-memory window) lands where the oracle's
    # segment walk puts it.
    import paper_1610_03918_gb300 as pg
    w = synth.periodic_square_64(ppc=1, poisson_rtol=1e-10)
    gs = gpu_sim(w, capacity=64)
    os_ = oracle_sim(w)
    x = np.array([10.5, 20.25, 30.5, 40.5])
    y = np.array([10.5, 20.75, 40.5, 50.5])
    vx = np.array([12.0, 10.0, 0.1, -0.2]) / w.dt
    vy = np.array([0.0, 10.0, 0.0, 0.3]) / w.dt
    p = synth.Particles(x, y, vx, vy, np.arange(4, dtype=np.uint32))
    load_both(gs, os_, 0, p)
    gs.step(1)
    os_.step(1)
    assert gs.status() & pg.PIC_ST_CFL
    assert gs.status() == 0          # reading cleared it
    walls, live = gs.counts()
    assert live.tolist() == [3, 0]
    assert walls.sum() == 0
    o = oracle_state(os_, 0)
    keep = o[4] != 1
    compare_states(gs.state(0), o[:, keep], w, 0)


@pytest.mark.parametrize("graphs", [False, True])
def test_unreachable_tolerance_is_reported(graphs):
    # rtol below what the double-float residual can show: the solve of the
    # loaded state stops after its pass cap and pic_step reports it
    # (PIC_ENOCONV, the fields stay marked for another solve); the field it
    # leaves is still the oracle's to the field tolerance.
    import paper_1610_03918_gb300 as pg
    w = SMALL["trench"].replace(poisson_rtol=1e-30)
    gs = gpu_sim(w, graphs=graphs)
    os_ = oracle_sim(w.replace(poisson_rtol=1e-12))
    for s in (0, 1):
        load_both(gs, os_, s, synth.maxwellian_load(w, s), v_at_t0=True)
    assert pg.pic_step(gs.ctx, 0) == pg.PIC_ENOCONV
    assert pg.pic_step(gs.ctx, 1) == pg.PIC_ENOCONV   # no step before a solve succeeds
    gs.status()
    assert gs.counts()[1].sum() == sum(len(synth.maxwellian_load(w, s)) for s in (0, 1))
    os_.prepare()
    E = np.stack(gs.efield())
    Eo = np.stack([os_.Ex, os_.Ey])
    assert np.abs(E - Eo).max() <= FIELD_TOL * np.abs(Eo).max()
