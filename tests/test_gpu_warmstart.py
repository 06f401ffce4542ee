"""The learned warm start end to end on a reduced trench: pairs dumped by the
GPU code itself, the U-Net trained by the library's kernels, and the solve
started from the network's guess.  The solve always reaches its tolerance;
the test measures what the trained network gains over the zero start.  The
warm start serves the iterative inner solver (multigrid PCG); the direct one
reaches the tolerance in one pass from any start, so it is not used here."""
import numpy as np
import pytest

import synth
from oracle import unet as ounet

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
    net.set_params(ounet.flat(ounet.init_params(0)).astype(np.float32))
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
