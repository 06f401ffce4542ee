"""The particle store's tile variants and their autotuner (pic_autotune):
every variant gives the same run bit for bit (the deposit is exact, the
window and global paths round alike), the tuner keeps the fastest variant
measured on the live run, and its cache file serves the next context of the
same GPU, grid and loading without timing anything.  Needs a GB300."""
import json

import numpy as np
import pytest

import synth

from gpu_helpers import by_id, gpu_sim

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _built():
    import __graft_entry__
    __graft_entry__.build()


W = synth.small_trench(nx=96, ny=64, depth=24, width=6, ppc=12, seed=91).replace(sort_every=5)


def _run(variant=0, steps=0, **kw):
    gs = gpu_sim(W, tile_variant=variant, **kw)
    for s in (0, 1):
        gs.load_particles(s, synth.maxwellian_load(W, s), v_at_t0=True)
    gs.step(steps)
    return gs


def _same(a, b):
    for s in (0, 1):
        assert np.array_equal(by_id(a.state(s)), by_id(b.state(s))), s
    assert np.array_equal(a.rho(), b.rho())
    assert np.array_equal(a.phi(), b.phi())
    assert np.array_equal(a.counts()[0], b.counts()[0])
    assert np.array_equal(a.surface(), b.surface())


def test_every_tile_variant_gives_the_same_run():
    runs = [_run(v, 13) for v in range(4)]
    shapes = [r.tile() for r in runs]
    assert [s[:3] for s in shapes] == [(0, 16, 16), (1, 32, 16), (2, 16, 32), (3, 32, 32)]
    for r in runs[1:]:
        _same(runs[0], r)


def test_autotune_picks_and_caches_a_variant(tmp_path):
    cache = str(tmp_path / "tiles.json")
    steps = 4
    a = _run()
    v = a.autotune(steps, cache)
    assert a.tile()[0] == v
    entries = json.load(open(cache))
    assert len(entries) == 1 and entries[0]["tile_variant"] == v
    assert len(entries[0]["particle_ms"]) == 4 and min(entries[0]["particle_ms"]) > 0
    # the tuning steps advanced the run: 1 step per variant to sort into its
    # tiles plus the timed steps; a fixed-variant run of as many steps matches
    taken = 4 * (1 + steps)
    a.step(3)
    b = _run(0, taken + 3)
    _same(a, b)
    # a second context reads the cache: same choice, no steps taken
    c = _run()
    c.step(0)
    assert c.autotune(steps, cache) == v
    c.step(taken + 3)
    _same(b, c)
    assert len(json.load(open(cache))) == 1


def test_bad_variant_is_rejected():
    import paper_1610_03918_gb300 as pg
    with pytest.raises(pg.PicError) as e:
        gpu_sim(W, tile_variant=4)
    assert e.value.code == pg.PIC_EINVAL
