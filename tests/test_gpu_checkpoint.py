"""Checkpoint and restart (pic_save / pic_restore): 2N uninterrupted steps
equal N steps, a checkpoint restored into a new context, and N more steps,
bit for bit (particles, rho, phi, E, tallies, bottom counts, hit records).
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


def _loaded(w, **kw):
    gs = gpu_sim(w, capacity=int(synth.plasma_cells(w).sum()) * w.ppc + 64, **kw)
    for s in (0, 1):
        gs.load_particles(s, synth.maxwellian_load(w, s), v_at_t0=True)
    return gs


@pytest.mark.parametrize("graphs,warm_start", [(True, 1), (True, 2), (False, 0)])
def test_restart_continues_bit_for_bit(graphs, warm_start):
    # RF bias, ion recycling and surface charge on, so every part of the
    # state matters; the sort interval does not divide N, so the checkpoint
    # falls between sorts
    w = synth.small_trench(nx=72, ny=64, depth=20, width=6, ppc=10, seed=71).replace(
        phi_rf_amp=5.0, omega_rf=0.2, recycle=True, recycle_seed=9, sort_every=5)
    N = 7
    a = _loaded(w, graphs=graphs, warm_start=warm_start)
    a.step(2 * N)
    b = _loaded(w, graphs=graphs, warm_start=warm_start)
    b.step(N)
    blob = b.save()
    b.close()
    c = gpu_sim(w, capacity=int(synth.plasma_cells(w).sum()) * w.ppc + 64, graphs=graphs,
                warm_start=warm_start)
    c.restore(blob)
    c.step(N)
    for s in (0, 1):
        assert np.array_equal(by_id(a.state(s)), by_id(c.state(s))), s
    for f in ("rho", "phi"):
        assert np.array_equal(getattr(a, f)(), getattr(c, f)()), f
    assert np.array_equal(a.efield()[0], c.efield()[0])
    assert np.array_equal(a.efield()[1], c.efield()[1])
    assert np.array_equal(a.counts()[0], c.counts()[0])
    assert np.array_equal(a.surface(), c.surface())
    ha, hc = _hits_sorted(a.hits()), _hits_sorted(c.hits())
    assert ha.size > 0 and np.array_equal(ha, hc)
    np.testing.assert_allclose(a.energy(), c.energy(), rtol=1e-6)
    assert a.counts()[0][1].sum() > 0          # ions were absorbed (and recycled)
    # a checkpoint of the restarted run is the uninterrupted run's checkpoint,
    # up to the order of the particles
    assert len(a.save()) == len(c.save())


def test_restore_rejects_another_geometry():
    import paper_1610_03918_gb300 as pg
    w = synth.small_trench(nx=48, ny=32, depth=12, width=6, ppc=4)
    a = _loaded(w)
    a.step(2)
    blob = a.save()
    other = gpu_sim(w.replace(nx=50), capacity=100000)
    with pytest.raises(pg.PicError) as e:
        other.restore(blob)
    assert e.value.code == pg.PIC_EINVAL
    small = gpu_sim(w, capacity=10)
    with pytest.raises(pg.PicError) as e:
        small.restore(blob)
    assert e.value.code == pg.PIC_EOVERFLOW
    with pytest.raises(pg.PicError):
        a.restore(blob[:-8])                   # truncated
