"""Pins of the oracle's RF bias (Sec. III-B), ion recycling (Sec. III-A,
III-C) and its counter-based generator, against closed forms, published
known-answer vectors and sampling statistics."""
import numpy as np
import pytest

import synth
from oracle import poisson, rng
from oracle.geometry import Geometry, from_workload
from oracle.sim import Sim

pytestmark = pytest.mark.filterwarnings("ignore::RuntimeWarning")


def test_philox_known_answer_vectors():
    # Philox4x32-10 against the vectors published with the generator
    import os
    path = os.path.join(os.path.dirname(__file__), "golden", "philox4x32_10_kat.txt")
    n = 0
    for line in open(path):
        if line.startswith("#") or not line.strip():
            continue
        v = [int(t, 16) for t in line.split()]
        out = rng.philox4x32_10(np.array(v[:4]), np.array(v[4:6]))
        assert [int(x) for x in out] == v[6:]
        n += 1
    assert n == 3


def test_philox_is_counter_based():
    # a draw depends only on its counter and key: a batch equals its rows one by one
    ctr = np.array([[k, 7, 1, 0] for k in range(5)], np.uint64)
    key = rng.seed_key(2 ** 40 + 3)
    batch = rng.philox4x32_10(ctr, key)
    for k in range(5):
        assert np.array_equal(batch[k], rng.philox4x32_10(ctr[k], key))
    assert len({tuple(r) for r in batch.tolist()}) == 5


def test_rf_bias_between_plates_is_linear_at_every_step():
    # no charge, no trench: the discrete Laplacian of a linear profile is zero,
    # so phi(x, t_n) = phi_top + (phi_e + A sin(w n dt) - phi_top) x / nx exactly
    w = synth.Workload(name="rf_plates", nx=24, ny=8, periodic_y=True, phi_top=1.5,
                       phi_electrode=-2.0, phi_rf_amp=5.0, omega_rf=0.7, ppc=1)
    s = Sim(w)
    x = np.arange(w.nx + 1, dtype=np.float64)[:, None]
    for n in range(6):
        if n == 0:
            s.prepare()
        else:
            s.step(1)
        pe = w.phi_electrode + w.phi_rf_amp * np.sin(w.omega_rf * n * w.dt)
        ref = w.phi_top + (pe - w.phi_top) * x / w.nx
        np.testing.assert_allclose(s.phi, np.broadcast_to(ref, s.phi.shape), atol=1e-12)


def test_rf_bias_on_the_trench_is_a_superposition():
    # with no charge the potential is linear in the Dirichlet data: phi(t) =
    # phi_static + A sin(w t) u, u the potential of electrode 1 / top plate 0;
    # every node held at the electrode potential (trench walls and bottom
    # included) follows the bias
    w = synth.small_trench(nx=40, ny=24, depth=12, width=6).replace(phi_rf_amp=5.0, omega_rf=0.3)
    geom = from_workload(w)
    zero = np.zeros((geom.nxn, geom.nyn))
    static = poisson.solve_direct(from_workload(w.replace(phi_rf_amp=0.0)), zero)
    unit = poisson.solve_direct(from_workload(w.replace(phi_top=0.0, phi_electrode=1.0,
                                                        phi_rf_amp=0.0)), zero)
    s = Sim(w)
    s.prepare()
    s.step(3)
    t = 3 * w.dt
    amp = w.phi_rf_amp * np.sin(w.omega_rf * t)
    np.testing.assert_allclose(s.phi, static + amp * unit, atol=1e-11)
    assert np.allclose(s.phi[geom.electrode], w.phi_electrode + amp, atol=1e-14)
    assert geom.electrode[-1].all() and geom.electrode[w.nx - w.trench_depth, 0]


def test_recycled_ions_are_uniform_and_thermal():
    w = synth.small_trench(nx=64, ny=32, depth=16, width=6).replace(recycle=True, recycle_seed=99)
    assert Sim(w).source_rows() == (0, 48)       # default: the bulk above the electrode
    w = w.replace(source_x0=4, source_x1=40)
    s = Sim(w)
    n = 200_000
    r = s.recycled(np.arange(n, dtype=np.uint32), step=17)
    x0, x1 = s.source_rows()
    assert (x0, x1) == (4, 40)
    # positions: uniform over the source rows and all columns
    assert r["x"].min() >= x0 and r["x"].max() < x1 and r["y"].min() >= 0 and r["y"].max() < w.ny
    L = x1 - x0
    assert abs(r["x"].mean() - 0.5 * (x0 + x1)) <= 4 * L / np.sqrt(12 * n)
    assert abs(r["y"].mean() - 0.5 * w.ny) <= 4 * w.ny / np.sqrt(12 * n)
    assert abs(r["x"].var() - L * L / 12) <= 0.02 * L * L / 12
    # every row and column is drawn about equally often
    rows = np.bincount(np.floor(r["x"]).astype(int) - x0, minlength=L)
    assert rows.min() > 0.85 * n / L and rows.max() < 1.15 * n / L
    # offsets are exact multiples of 2^-24
    f = (r["x"] - np.floor(r["x"])) * 2 ** 24
    assert np.array_equal(f, np.round(f))
    # velocities: Maxwellian of the ion thermal speed in each component (Eq. 6)
    vth = w.vth[1]
    for v in (r["vx"], r["vy"]):
        assert abs(v.mean()) <= 4 * vth / np.sqrt(n)
        assert abs(v.var() / vth ** 2 - 1) <= 4 * np.sqrt(2 / n)
        # fourth moment of a Gaussian: 3 sigma^4
        assert abs(np.mean(v ** 4) / vth ** 4 - 3) <= 0.1
    assert abs(np.corrcoef(r["vx"], r["vy"])[0, 1]) <= 4 / np.sqrt(n)
    # a pure function of (seed, step, id)
    again = s.recycled(np.arange(10, dtype=np.uint32), step=17)
    assert np.array_equal(again["x"], r["x"][:10]) and np.array_equal(again["vy"], r["vy"][:10])
    other = s.recycled(np.arange(10, dtype=np.uint32), step=18)
    assert not np.array_equal(other["x"], r["x"][:10])


def test_recycling_keeps_the_ion_count_and_ids():
    # ions launched into the trench bottom are tallied and re-enter in the bulk
    w = synth.small_trench(nx=48, ny=32, depth=16, width=6, ppc=4).replace(recycle=True,
                                                                           recycle_seed=5)
    s = Sim(w)
    y0 = w.trench_y0
    x = np.concatenate([np.full(6, 47.95), np.full(4, 10.5)])
    y = np.concatenate([y0 + 0.5 + np.arange(6.0), np.full(4, 3.5)])
    s.load(1, x, y, np.concatenate([np.full(6, 1.0), np.zeros(4)]), np.zeros(10),
           np.arange(10, dtype=np.uint32))
    s.step(1)
    assert s.counts[1, 1] == 6 and s.bottom[1].sum() == 6
    assert s.live()[1] == 10
    ids = np.sort(s.p[1]["ids"])
    assert np.array_equal(ids, np.arange(10))
    back = np.isin(s.p[1]["ids"], np.arange(6))
    assert (s.p[1]["x"][back] < w.nx - w.trench_depth).all()
    ref = s.recycled(np.arange(6, dtype=np.uint32), step=0)
    order = np.argsort(s.p[1]["ids"][back])
    assert np.array_equal(s.p[1]["x"][back][order], ref["x"])
    # electrons are not recycled
    w2 = w.replace()
    s2 = Sim(w2)
    s2.load(0, np.full(3, 47.95), y0 + 0.5 + np.arange(3.0), np.full(3, 1.0), np.zeros(3))
    s2.step(1)
    assert s2.live()[0] == 0
