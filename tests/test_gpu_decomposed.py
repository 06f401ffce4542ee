"""A run split by particles (pic_step_particles / exchange / pic_step_fields)
on one GPU: R ranks held by this process, their exchange buffers summed by
pic_exchange_sum (the single-device stand-in for the all-reduce; the ranks'
kernels never wait on one another), against one context holding every
particle.  rho, phi, E, the union of the particle states, the summed tallies
and bottom counts and the union of hit records must be equal bit for bit.
Needs a GB300."""
import numpy as np
import pytest

import synth

from gpu_helpers import by_id, gpu_sim

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _built():
    import __graft_entry__
    __graft_entry__.build()


def _hits_sorted(h):
    return h[np.lexsort((h["id"], h["species"], h["step"]))]


@pytest.mark.parametrize("ranks,graphs", [(2, True), (3, True), (2, False)])
def test_split_run_equals_single_run(ranks, graphs):
    import paper_1610_03918_gb300 as pg
    from paper_1610_03918_gb300 import distributed as pd
    # RF bias, ion recycling and surface charge on: every exchanged part matters
    w = synth.small_trench(nx=72, ny=64, depth=20, width=6, ppc=10, seed=81).replace(
        phi_rf_amp=5.0, omega_rf=0.2, recycle=True, recycle_seed=3, sort_every=4)
    loads = [synth.maxwellian_load(w, s) for s in (0, 1)]
    cap = max(len(p) for p in loads) + 64
    one = gpu_sim(w, capacity=cap, graphs=graphs)
    for s in (0, 1):
        one.load_particles(s, loads[s], v_at_t0=True)
    parts = [gpu_sim(w, capacity=cap, graphs=graphs, decomposed=True) for _ in range(ranks)]
    for r, sim in enumerate(parts):
        for s in (0, 1):
            sim.load_particles(s, pd.shard(loads[s], r, ranks), v_at_t0=True)
    nsteps = 9
    one.step(0)
    for k in range(nsteps + 1):          # the first pair brings the fields up to date
        for sim in parts:
            sim.step_particles()
        pg.exchange_sum(parts)
        for sim in parts:
            sim.step_fields()
    one.step(nsteps)
    for sim in parts:
        assert np.array_equal(sim.rho(), one.rho())
        assert np.array_equal(sim.phi(), one.phi())
        ex, ey = sim.efield()
        assert np.array_equal(ex, one.efield()[0]) and np.array_equal(ey, one.efield()[1])
    for s in (0, 1):
        union = np.concatenate([p.state(s) for p in parts], axis=1)
        assert np.array_equal(by_id(union), by_id(one.state(s))), s
    walls = sum(p.counts()[0] for p in parts)
    assert np.array_equal(walls, one.counts()[0])
    assert walls[1].sum() > 0
    assert np.array_equal(sum(p.surface() for p in parts), one.surface())
    hits = np.concatenate([p.hits() for p in parts])
    assert np.array_equal(_hits_sorted(hits), _hits_sorted(one.hits()))
    ke = sum(p.energy()[:2] for p in parts)
    np.testing.assert_allclose(ke, one.energy()[:2], rtol=1e-6)
    assert parts[0].energy()[2] == one.energy()[2]


def test_phases_out_of_order_are_refused():
    import paper_1610_03918_gb300 as pg
    w = synth.small_trench(nx=48, ny=32, depth=12, width=6, ppc=4).replace(sort_every=4)
    sim = gpu_sim(w, decomposed=True)
    with pytest.raises(pg.PicError) as e:
        sim.step_fields()
    assert e.value.code == pg.PIC_ESTATE
    with pytest.raises(pg.PicError) as e:
        sim.step(1)
    assert e.value.code == pg.PIC_ESTATE
    sim.step_particles()
    with pytest.raises(pg.PicError) as e:
        sim.step_particles()
    assert e.value.code == pg.PIC_ESTATE


def test_distributed_driver_over_nccl_single_rank():
    # distributed.DistributedSim through a real NCCL process group (one rank on
    # this GPU): the all-reduce of the exchange buffer on the context's stream
    # is then the identity, and the run equals an undecomposed one bit for bit
    import socket
    import torch
    import torch.distributed as dist
    import paper_1610_03918_gb300 as pg
    from paper_1610_03918_gb300 import distributed as pd
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        port = s.getsockname()[1]
    dist.init_process_group("nccl", init_method=f"tcp://127.0.0.1:{port}", rank=0, world_size=1)
    try:
        w = synth.small_trench(nx=72, ny=64, depth=20, width=6, ppc=8, seed=82).replace(
            recycle=True, recycle_seed=4, sort_every=4)
        loads = [synth.maxwellian_load(w, s) for s in (0, 1)]
        cap = max(len(p) for p in loads) + 64
        one = gpu_sim(w, capacity=cap)
        rank = gpu_sim(w, capacity=cap, decomposed=True)
        for s in (0, 1):
            one.load_particles(s, loads[s], v_at_t0=True)
            rank.load_particles(s, pd.shard(loads[s], 0, 1), v_at_t0=True)
        one.step(7)
        drv = pd.DistributedSim(rank)
        drv.step(8)                      # the first step brings the fields up to date
        torch.cuda.synchronize()
        assert np.array_equal(rank.rho(), one.rho()) and np.array_equal(rank.phi(), one.phi())
        for s in (0, 1):
            assert np.array_equal(by_id(rank.state(s)), by_id(one.state(s)))
        walls, live = drv.counts()
        assert np.array_equal(walls, one.counts()[0]) and np.array_equal(live, one.counts()[1])
        np.testing.assert_allclose(drv.energy()[:2], one.energy()[:2], rtol=1e-6)
    finally:
        dist.destroy_process_group()
