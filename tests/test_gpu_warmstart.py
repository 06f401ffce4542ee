"""The learned warm start end to end on a reduced trench: pairs dumped by the
GPU code itself, the U-Net trained by the library's kernels, and the solve
started from the network's guess.  The solve always reaches its tolerance;
the test measures what the trained network gains over the zero start.  The
warm start serves the iterative inner solver (multigrid PCG); the direct one
reaches the tolerance in one pass from any start, so it is not used here."""
import numpy as np
import pytest

import synth

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def trained():
    import torch
    import __graft_entry__
    __graft_entry__.build()
    import paper_1610_03918_gb300 as pg
    from paper_1610_03918_gb300 import warmstart as ws
    w = synth.small_trench(nx=64, ny=32, depth=16, width=6, ppc=30, seed=21)
    sim = pg.Sim(w, warm_start=1, poisson_method=pg.POISSON_MULTIGRID)
    for s in (0, 1):
        sim.load_particles(s, synth.maxwellian_load(w, s), v_at_t0=True)
    sim.step(20)
    pairs = ws.dump_pairs(sim, steps=400, every=2)
    net = pg.Unet(1, ws.padded_rows(sim.nxn), sim.nyn)
    net.init(seed=0)
    ws.train(net, pairs, epochs=6, lr=1e-3)
    # held-out states: another seed of the same geometry
    w2 = w.replace(seed=99)
    ev = pg.Sim(w2, warm_start=1, poisson_method=pg.POISSON_MULTIGRID)
    for s in (0, 1):
        ev.load_particles(s, synth.maxwellian_load(w2, s), v_at_t0=True)
    ev.step(30)
    yield pg, ws, net, ev, w2
    net.close()


def test_learned_warm_start_reaches_tolerance_in_fewer_iterations(trained):
    pg, ws, net, ev, w = trained
    lw = ws.LearnedWarmStart(net)
    it_zero, it_learned = [], []
    for k in range(8):
        ev.step(3)
        z = ev.poisson(0)
        assert z[2] <= w.poisson_rtol
        l, ms = lw.solve(ev)
        assert l[2] <= w.poisson_rtol
        it_zero.append(z[0])
        it_learned.append(l[0])
    assert np.mean(it_learned) <= 0.85 * np.mean(it_zero), (it_zero, it_learned)


def test_guess_variants_all_converge(trained):
    pg, ws, net, ev, w = trained
    for g in (0, 1, 2):
        st = ev.poisson(g)
        assert st[2] <= w.poisson_rtol and st[0] >= 0


def test_he_initialisation_moments():
    # every weight tensor of the library's initialiser has mean 0 and the
    # He standard deviation sqrt(gain / fan_in) (gain 2 before a ReLU, 1 for
    # the linear head); biases are zero; a seed fixes the draws
    import paper_1610_03918_gb300 as pg
    from oracle.unet import layer_shapes     # the parameter layout only
    net = pg.Unet(1, 32, 32)
    net.init(seed=11)
    p = net.get_params()
    net.init(seed=11)
    assert np.array_equal(p, net.get_params())
    net.init(seed=12)
    assert not np.array_equal(p, net.get_params())
    k = 0
    for name, shp in layer_shapes():
        n = int(np.prod(shp))
        v = p[k:k + n].astype(np.float64)
        k += n
        if name.endswith(".b"):
            assert np.all(v == 0), name
            continue
        if name.startswith("up"):
            fan, gain = shp[2], 2.0
        elif name == "head.W":
            fan, gain = shp[0], 1.0
        else:
            fan, gain = 9 * shp[3], 2.0
        std = np.sqrt(gain / fan)
        assert abs(v.mean()) <= 5 * std / np.sqrt(n), name
        # sample standard deviation within 5 of its own standard errors (or 30% for tiny layers)
        assert abs(v.std() / std - 1) <= max(5 / np.sqrt(2 * n), 0.3), (name, v.std(), std)
    assert k == p.size
    net.close()


def test_learned_target_kernel(trained):
    # (phi - phi_L) / s formed by the library, against the same arithmetic on
    # the potentials it exports
    pg, ws, net, ev, w = trained
    hpad = ws.padded_rows(ev.nxn)
    x, s = ev.learned_input(hpad)
    t = ev.learned_target(hpad, s).cpu().numpy()
    ref = (ev.phi() - ev.phi_vacuum()) / s
    assert np.abs(t[: ev.nxn] - ref).max() <= 1e-6 * max(np.abs(ref).max(), 1.0)
    assert np.all(t[ev.nxn:] == 0)


@pytest.mark.parametrize("graphs", [True, False])
def test_learned_start_inside_the_step(trained, graphs, tmp_path):
    # warm_start 3: the network's guess is formed on the device inside every
    # step (captured in the step graph); each solve still meets its
    # tolerance and the run tracks one started from the previous potential
    pg, ws, net, ev, w = trained
    path = str(tmp_path / "net.f32")
    net.save(path)
    runs = []
    for mode in ("file", "previous"):
        kw = dict(warm_start=3, unet_weights=path) if mode == "file" else dict(warm_start=1)
        sim = pg.Sim(w, poisson_method=pg.POISSON_MULTIGRID, graphs=graphs, **kw)
        for s in (0, 1):
            sim.load_particles(s, synth.maxwellian_load(w, s), v_at_t0=True)
        sim.step(5)
        assert sim.poisson_stats()[2] <= w.poisson_rtol and sim.status() == 0
        runs.append(sim)
    a, b = runs
    assert np.abs(a.phi() - b.phi()).max() <= 1e-4 * np.abs(b.phi()).max()
    # switching a running context to the learned guess re-captures its graphs
    b.set_learned_start(net)
    b.step(3)
    assert b.poisson_stats()[2] <= w.poisson_rtol and b.status() == 0
