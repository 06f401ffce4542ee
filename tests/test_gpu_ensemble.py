"""The ensemble (pic_batch_*): members of different grid sizes and trench
widths advanced together by one graph launch per step must reproduce, bit
for bit, the same runs advanced alone (the deposit is integer, reductions
run in a fixed order, members share no buffers).  Each solo run is in turn
checked against the oracle by the parity tests."""
import numpy as np
import pytest

import synth

from gpu_helpers import parity_post, parity_pre

pytestmark = pytest.mark.gpu


def _members():
    # the trench-width sweep recipe at reduced particle count, plus two odd sizes
    ws = [synth.ensemble_member(k, ppc=3) for k in (0, 13, 30, 47)]
    ws.append(synth.small_trench(nx=72, ny=40, depth=20, width=6, ppc=6, seed=41))
    ws.append(synth.bounded_square_256(nx=45, ny=38, ppc=5, seed=42, sort_every=8))
    return [w.replace(sort_every=8, poisson_rtol=1e-8) for w in ws]


def _by_id(st):
    return st[:, np.argsort(st[4], kind="stable")]


@pytest.fixture(scope="module")
def lib():
    import __graft_entry__
    __graft_entry__.build()
    import paper_1610_03918_gb300 as pg
    return pg


def test_batch_matches_solo_runs_bitwise(lib):
    pg = lib
    ws = _members()
    loads = [[synth.maxwellian_load(w, s) for s in (0, 1)] for w in ws]
    caps = [max(len(p[0]), len(p[1])) for p in loads]
    batch = pg.Batch(ws, capacities=caps)
    for m, p in zip(batch.members, loads):
        for s in (0, 1):
            m.load_particles(s, p[s], v_at_t0=True)
    batch.step(11)                      # crosses the sort at step 8
    for k, w in enumerate(ws):
        solo = pg.Sim(w, capacity=caps[k])
        for s in (0, 1):
            solo.load_particles(s, loads[k][s], v_at_t0=True)
        solo.step(11)
        m = batch.members[k]
        for s in (0, 1):
            assert np.array_equal(_by_id(m.state(s)), _by_id(solo.state(s))), (k, s)
        assert np.array_equal(m.rho(), solo.rho())
        assert np.array_equal(m.phi(), solo.phi())
        assert np.array_equal(m.counts()[0], solo.counts()[0])
        assert np.array_equal(m.surface(), solo.surface())
        e_b, e_s = m.energy(), solo.energy()
        np.testing.assert_allclose(e_b, e_s, rtol=1e-6)
        solo.close()
    t = batch.timing()
    batch.close()
    assert t["steps"] == 0 or t["ms"] >= 0


def test_batch_members_match_oracle_per_step(lib):
    # members of different grid sizes and trench widths, each checked
    # against the FP64 oracle step by step by the parity protocol (the
    # oracle restarts from the member's state before every step)
    pg = lib
    ws = [synth.small_trench(nx=72, ny=40, depth=20, width=6, ppc=8, seed=51),
          synth.small_trench(nx=48, ny=64, depth=12, width=3, ppc=8, seed=52),
          synth.bounded_square_256(nx=37, ny=30, ppc=6, seed=53)]
    ws = [w.replace(sort_every=2, poisson_rtol=1e-10) for w in ws]
    loads = [[synth.maxwellian_load(w, s) for s in (0, 1)] for w in ws]
    batch = pg.Batch(ws, capacities=[max(len(p[0]), len(p[1])) for p in loads])
    for m, p in zip(batch.members, loads):
        for s in (0, 1):
            m.load_particles(s, p[s], v_at_t0=True)
    batch.step(0)
    ties = 0
    for k in range(3):                 # crosses a sort (every 2 steps)
        pres = [parity_pre(w, m, k) for w, m in zip(ws, batch.members)]
        batch.step(1)
        for w, m, pre in zip(ws, batch.members, pres):
            t, os_ = parity_post(w, m, pre, k)
            ties += t
            e = m.energy()
            assert e[0] == pytest.approx(os_.ke[0], rel=1e-5)
            assert e[2] == pytest.approx(os_.fe, rel=1e-5)
    assert ties <= 2
    batch.close()


def test_solo_runs_are_bitwise_reproducible(lib):
    # the particle order after a sort varies from run to run; results must not
    pg = lib
    w = synth.ensemble_member(0, ppc=3).replace(sort_every=4, poisson_rtol=1e-8)
    loads = [synth.maxwellian_load(w, s) for s in (0, 1)]
    outs = []
    for _ in range(2):
        sm = pg.Sim(w, capacity=max(len(p) for p in loads))
        for s in (0, 1):
            sm.load_particles(s, loads[s], v_at_t0=True)
        sm.step(10)
        outs.append(([_by_id(sm.state(s)) for s in (0, 1)], sm.rho(), sm.phi()))
        sm.close()
    for s in (0, 1):
        assert np.array_equal(outs[0][0][s], outs[1][0][s])
    assert np.array_equal(outs[0][1], outs[1][1])
    assert np.array_equal(outs[0][2], outs[1][2])


def test_batch_rejects_mixed_sort_schedules(lib):
    pg = lib
    ws = [synth.small_trench(sort_every=8), synth.small_trench(sort_every=4)]
    with pytest.raises(pg.PicError):
        pg.Batch(ws)
