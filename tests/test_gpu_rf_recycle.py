"""RF bias of the electrode (Sec. III-B) and ion recycling (Sec. III-A,
III-C) on the CUDA path, against closed forms and the FP64 oracle.  Needs a
GB300."""
import numpy as np
import pytest

import synth
from oracle import poisson as opoisson
from oracle.geometry import from_workload

from gpu_helpers import gpu_sim, step_parity_once

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _built():
    import __graft_entry__
    __graft_entry__.build()


def test_rf_bias_between_plates_follows_the_closed_form():
    # no charge, no trench: phi(x, t_n) is linear between the plates at every
    # time level, with the electrode at phi_e + A sin(w n dt)
    w = synth.Workload(name="rf_plates", nx=48, ny=32, periodic_y=True, phi_top=1.5,
                       phi_electrode=-2.0, phi_rf_amp=5.0, omega_rf=0.7, ppc=1,
                       poisson_rtol=1e-10)
    for graphs in (True, False):
        gs = gpu_sim(w, capacity=16, graphs=graphs)
        gs.step(0)
        x = np.arange(w.nx + 1, dtype=np.float64)[:, None]
        for n in range(6):
            if n:
                gs.step(1)
            pe = w.phi_electrode + w.phi_rf_amp * np.sin(w.omega_rf * n * w.dt)
            ref = np.broadcast_to(w.phi_top + (pe - w.phi_top) * x / w.nx, (w.nx + 1, w.ny))
            assert np.abs(gs.phi() - ref).max() <= 1e-6 * 7.0, (graphs, n)
        gs.close()


@pytest.mark.parametrize("method", ["auto", "multigrid"])
def test_rf_bias_trench_vacuum_matches_oracle(method):
    import paper_1610_03918_gb300 as pg
    w = synth.small_trench(nx=72, ny=64, depth=20, width=6).replace(
        phi_rf_amp=5.0, omega_rf=0.3, poisson_rtol=1e-10)
    gs = gpu_sim(w, capacity=16, poisson_method=pg.POISSON_AUTO if method == "auto"
                 else pg.POISSON_MULTIGRID)
    gs.step(4)
    geom = from_workload(w)
    geom.set_time(4 * w.dt)
    phi_o = opoisson.solve_direct(geom, np.zeros((geom.nxn, geom.nyn)))
    assert np.abs(gs.phi() - phi_o).max() <= 1e-6 * 25.0
    assert opoisson.residual_rel(geom, gs.phi(), np.zeros_like(phi_o)) <= 2e-10


@pytest.mark.parametrize("graphs", [True, False])
def test_step_parity_with_rf_bias_and_recycling(graphs):
    # a reduced trench with the electrode RF-biased and ions recycled; fast
    # ions are added so that many are absorbed (and re-enter) every step.  The
    # step protocol checks the re-entered ions' positions bit for bit against
    # the oracle's Philox draws, and their velocities to the push tolerance.
    w = synth.small_trench(nx=72, ny=40, depth=20, width=6, ppc=8, seed=61).replace(
        phi_rf_amp=5.0, omega_rf=0.2, recycle=True, recycle_seed=2 ** 40 + 17,
        source_x0=3, source_x1=45, poisson_rtol=1e-10, sort_every=2)
    ions = synth.maxwellian_load(w, 1)
    fast = synth.random_state(w, 1, 4000, seed=62, vscale=1200.0)
    fast.ids = fast.ids + np.uint32(len(ions))
    ions = synth.Particles(*(np.concatenate([getattr(ions, k), getattr(fast, k)])
                             for k in ("x", "y", "vx", "vy", "ids")))
    gs = gpu_sim(w, capacity=len(ions) + 16, graphs=graphs)
    gs.load_particles(0, synth.maxwellian_load(w, 0))
    gs.load_particles(1, ions)
    gs.step(0)
    n0 = gs.counts()[1]
    ties = 0
    for k in range(4):
        t, os_ = step_parity_once(w, gs, lambda: gs.step(1), k)
        ties += t
    walls, live = gs.counts()
    assert walls[1].sum() > 100           # ions were absorbed and re-entered
    assert live[1] == n0[1]               # ... so the ion count is unchanged
    assert live[0] + walls[0].sum() == n0[0]
    assert ties <= 2
