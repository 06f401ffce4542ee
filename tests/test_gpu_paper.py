"""The paper's own trench runs (Sec. III-C, III-D; 80 x 30 cells, widths 15
and 4, the fixed n_i = 5 build-up above the bottom, RF electrode, m_i/m_e =
3672, T_i = T_e, ions recycled, t <= 1000) on the CUDA path: the paper's
qualitative findings about the ions reaching the trench bottom and
sidewalls hold.  Needs a GB300."""
import numpy as np
import pytest

import synth

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def tallies():
    import __graft_entry__
    __graft_entry__.build()
    import bench
    import paper_1610_03918_gb300 as pg
    cases = list(bench.PAPER_TALLIES)
    ws, tags = [], []
    for case in cases:
        for seed in (1, 2):
            ws.append(synth.paper_trench(4 if case == "w4" else 15, seed=seed, sort_every=8))
            tags.append(case)
    batch = pg.Batch(ws, capacities=[int(synth.plasma_cells(w).sum()) * w.ppc + 64 for w in ws],
                     hit_capacity=16)
    for m, w, tag in zip(batch.members, ws, tags):
        for s in (0, 1):
            m.load_particles(s, synth.maxwellian_load(w, s), v_at_t0=True)
        if tag == "w15_buildup":
            m.set_rho_ext(synth.paper_buildup_density(w))
    marks, done = {}, 0
    for at in (6000, 7000, 10000):
        batch.step(at - done)
        done = at
        marks[at] = [m.counts()[0][1].copy() for m in batch.members]
    for m in batch.members:
        assert m.status() & ~pg.PIC_ST_FULL == 0    # only the (tiny) hit buffer filled
    out = {}
    for case in cases:
        start = bench.PAPER_TALLIES[case][2]
        d = sum(marks[10000][k] - marks[start][k] for k, t in enumerate(tags) if t == case)
        window = (1000 - start * 0.1)
        out[case] = dict(bottom=d[pg.WALL_XMAX] / window,
                         side=(d[pg.WALL_COND_PY] + d[pg.WALL_COND_MY]) / window)
    batch.close()
    return out


def test_narrow_trench_is_more_anisotropic(tallies):
    # Sec. III-C: the ratio sidewalls / bottom is smaller for the 4-wide trench
    r15 = tallies["w15"]["side"] / tallies["w15"]["bottom"]
    r4 = tallies["w4"]["side"] / tallies["w4"]["bottom"]
    assert tallies["w4"]["bottom"] > 0 and r4 < 0.85 * r15, (r4, r15)


def test_charge_build_up_repels_ions_from_the_bottom(tallies):
    # Sec. III-D: the fixed positive charge above the bottom sends fewer ions to
    # the bottom per unit time and raises the sidewall / bottom ratio
    a, b = tallies["w15"], tallies["w15_buildup"]
    assert b["bottom"] < 0.6 * a["bottom"], (b, a)
    assert b["side"] / b["bottom"] > 1.5 * a["side"] / a["bottom"]
