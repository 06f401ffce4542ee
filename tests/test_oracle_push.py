"""Pins of the oracle's leapfrog push, absorption and time loop (CPU):
closed-form uniform-field motion, hand-worked face classifications, the
cold plasma oscillation frequency, momentum conservation and energy drift
in a periodic box."""
import numpy as np
import pytest
import scipy.optimize as so

import synth
from oracle import push
from oracle.geometry import Geometry, from_workload
from oracle.sim import Sim


# ---------------------------------------------------------------- Eqs. (1)-(4)
@pytest.mark.parametrize("alpha", [-1.0, 1.0 / 1836.0])
def test_uniform_field_leapfrog_is_exact(alpha):
    geom = Geometry(200, 200, False, False)
    E0 = np.array([0.37, -0.21])
    Ex = np.full((201, 201), E0[0])
    Ey = np.full((201, 201), E0[1])
    dt = 0.1
    x0 = np.array([100.3]); y0 = np.array([99.7])
    v0 = np.array([0.4, -0.25])
    # v^{-1/2} from v^0 by the half back-kick
    x, y = x0.copy(), y0.copy()
    vx = v0[0] - 0.5 * alpha * E0[0] * dt + np.zeros(1)
    vy = v0[1] - 0.5 * alpha * E0[1] * dt + np.zeros(1)
    for n in range(1, 61):
        x, y, vx, vy, alive, wall, wc = push.leapfrog(geom, alpha, dt, x, y, vx, vy, Ex, Ey)
        assert alive.all()
        t = n * dt
        assert x[0] == pytest.approx(x0[0] + v0[0] * t + 0.5 * alpha * E0[0] * t * t, abs=1e-12)
        assert y[0] == pytest.approx(y0[0] + v0[1] * t + 0.5 * alpha * E0[1] * t * t, abs=1e-12)
        # v^{n+1/2} = v^0 + alpha E (n + 1/2) dt
        assert vx[0] == pytest.approx(v0[0] + alpha * E0[0] * (n - 0.5) * dt, abs=1e-13)


# ---------------------------------------------------------------- absorption
def _cls(geom, p0, p1):
    a, w, c = push.classify(geom, np.array([p0[0]]), np.array([p0[1]]),
                            np.array([p1[0]]), np.array([p1[1]]))
    return bool(a[0]), int(w[0]), int(c[0])


def test_classification_by_hand_trench():
    # 64 (x) x 32 (y) cells, electrode x >= 48, trench y in [13, 19)
    geom = from_workload(synth.small_trench())
    assert _cls(geom, (47.5, 5.5), (48.5, 5.5)) == (False, push.WALL_COND_PX, 5)
    assert _cls(geom, (55.5, 13.2), (55.5, 12.7)) == (False, push.WALL_COND_MY, 55)
    assert _cls(geom, (55.5, 18.7), (55.5, 19.1)) == (False, push.WALL_COND_PY, 55)
    assert _cls(geom, (63.5, 15.5), (64.1, 15.5)) == (False, push.WALL_XMAX, 15)
    assert _cls(geom, (0.3, 5.5), (-0.2, 5.5)) == (False, push.WALL_XMIN, 5)
    # ending exactly on x = nx is a hit; ending exactly on a lower face is not
    assert _cls(geom, (63.5, 15.5), (64.0, 15.5)) == (False, push.WALL_XMAX, 15)
    assert _cls(geom, (10.5, 5.5), (10.0, 5.5))[0] is True
    # exact tie at the trench mouth corner: the x face is taken first
    assert _cls(geom, (47.5, 12.5), (48.125, 13.125)) == (False, push.WALL_COND_PX, 12)
    # into the trench mouth without touching a corner
    assert _cls(geom, (47.5, 13.5), (48.5, 13.5))[0] is True
    # periodic y re-entry
    assert _cls(geom, (10.5, 31.8), (10.5, 32.3))[0] is True


def test_classification_bounded_box():
    geom = Geometry(16, 12, False, False)
    assert _cls(geom, (5.5, 0.2), (5.5, -0.3)) == (False, push.WALL_YMIN, 5)
    assert _cls(geom, (5.5, 11.9), (5.5, 12.0)) == (False, push.WALL_YMAX, 5)
    assert _cls(geom, (15.9, 11.9), (16.2, 12.05)) == (False, push.WALL_XMAX, 11)


def test_sim_tallies_and_surface_charge():
    w = synth.small_trench(nx=24, ny=16, depth=8, width=4, ppc=4)
    s = Sim(w)
    # one ion heading straight into the trench bottom, one electron into the top plate
    s.load(1, [23.9], [7.5], [2.0], [0.0])
    s.load(0, [0.05], [3.5], [-1.0], [0.0])
    s.step(1)
    assert s.counts[1, push.WALL_XMAX] == 1 and s.bottom[1, 7] == 1
    assert s.counts[0, push.WALL_XMIN] == 1
    assert s.live().sum() == 0
    rho = s.charge_density()
    assert rho[23, 7] == pytest.approx(0.5 / 4) and rho[23, 8] == pytest.approx(0.5 / 4)
    ht = s.hit_table()
    assert sorted(ht["wall"].tolist()) == [push.WALL_XMIN, push.WALL_XMAX]


# ---------------------------------------------------------------- time loop
def test_cold_plasma_oscillation_frequency():
    # Cold electrons on a lattice with a small sinusoidal displacement in x,
    # immobile ions.  Leapfrog gives sin(omega dt / 2) = omega_p dt / 2.
    w = synth.Workload(name="cold", nx=64, ny=4, periodic_x=True, periodic_y=True,
                       ppc=4, mass_ratio=1e15, tau=0.0)
    nxp = 4
    x0 = (np.arange(64 * nxp) + 0.5) / nxp
    X0, Y0 = np.meshgrid(x0, np.arange(4) + 0.5, indexing="ij")
    X0, Y0 = X0.ravel(), Y0.ravel()
    k = 2 * np.pi / 64
    amp = 0.01
    s = Sim(w)
    s.load(0, X0 + amp * np.sin(k * X0), Y0, np.zeros_like(X0), np.zeros_like(X0), v_at_t0=True)
    s.load(1, X0, Y0, np.zeros_like(X0), np.zeros_like(X0))
    sig = []
    for n in range(300):
        d = s.p[0]["x"] - X0
        d = d - 64 * np.round(d / 64)
        sig.append(np.sum(d * np.sin(k * X0)))
        s.step(1)
    sig = np.array(sig)
    t = np.arange(300) * w.dt

    def model(p):
        return p[0] * np.cos(p[1] * t + p[2]) - sig
    fit = so.least_squares(model, [sig[0], 1.0, 0.0])
    omega = fit.x[1]
    expected = (2.0 / w.dt) * np.arcsin(1.0 * w.dt / 2.0)
    assert omega == pytest.approx(expected, rel=5e-3)
    assert np.abs(model(fit.x)).max() < 0.05 * np.abs(sig).max()


def test_periodic_momentum_conserved():
    w = synth.periodic_square_64(nx=16, ny=16, ppc=8, mass_ratio=20.0, tau=1.0)
    s = Sim(w)
    for sp in (0, 1):
        s.load_particles(sp, synth.maxwellian_load(w, sp), v_at_t0=True)
    s.prepare()
    p0 = s.momentum().sum(axis=0)
    scale = sum(s.mass[sp] * s.weight[sp] * np.abs(s.p[sp]["vx"]).sum() for sp in (0, 1))
    s.step(40)
    p1 = s.momentum().sum(axis=0)
    assert np.all(np.abs(p1 - p0) <= 1e-12 * scale), (p1 - p0, scale)


@pytest.mark.slow
def test_periodic_energy_drift_small():
    w = synth.periodic_square_64(nx=32, ny=32, ppc=20)
    s = Sim(w)
    for sp in (0, 1):
        s.load_particles(sp, synth.maxwellian_load(w, sp), v_at_t0=True)
    tot = []
    for n in range(200):
        s.step(1)
        tot.append(s.ke.sum() + s.fe)
    tot = np.array(tot)
    assert np.abs(tot - tot[0]).max() <= 0.01 * tot[0]


def test_loading_moments():
    w = synth.small_trench(ppc=20)
    for sp in (0, 1):
        p = synth.maxwellian_load(w, sp)
        n = len(p)
        vt = w.vth[sp]
        for v in (p.vx, p.vy):
            assert abs(v.mean()) < 4 * vt / np.sqrt(n)
            assert abs(v.var() / vt ** 2 - 1) < 4 * np.sqrt(2.0 / n)
        cells = synth.plasma_cells(w)
        assert n == cells.sum() * w.ppc
        assert cells[np.floor(p.x).astype(int), np.floor(p.y).astype(int)].all()


def test_sim_halfkick_between_biased_plates():
    # Vacuum field between the plates: E_x = -(dPhi/dx) = 20/40 = 0.5.  A
    # particle of negligible weight started with v at t = 0 follows the
    # constant-acceleration closed form.
    w = synth.Workload(name="plates", nx=40, ny=8, periodic_y=True, phi_top=0.0,
                       phi_electrode=-20.0, ppc=10 ** 9)
    s = Sim(w)
    x0, y0, v0x, v0y = 20.3, 3.6, 0.05, -0.02
    s.load(1, [x0], [y0], [v0x], [v0y], v_at_t0=True)
    s.step(50)
    t = 50 * w.dt
    a = w.alpha[1] * 0.5
    assert s.p[1]["x"][0] == pytest.approx(x0 + v0x * t + 0.5 * a * t * t, abs=1e-9)
    assert s.p[1]["y"][0] == pytest.approx(y0 + v0y * t, abs=1e-9)
    # field energy of the uniform vacuum field: 1/2 * 41 * 8 nodes * 0.5^2
    assert s.fe == pytest.approx(0.5 * 41 * 8 * 0.25, rel=1e-9)


def test_sim_kinetic_energy_and_momentum_free_particles():
    # a single particle sitting on a node of a periodic box feels no self-force
    w = synth.periodic_square_64(nx=8, ny=8, ppc=4)
    for sp, v, m in ((0, (0.3, -0.4), 1.0), (1, (0.01, 0.02), 1836.0)):
        s = Sim(w)
        s.load(sp, [3.0], [5.0], [v[0]], [v[1]])
        s.step(1)
        assert s.ke[sp] == pytest.approx(0.5 * m * 0.25 * (v[0] ** 2 + v[1] ** 2), rel=1e-12)
        assert s.momentum()[sp] == pytest.approx([m * 0.25 * v[0], m * 0.25 * v[1]], rel=1e-12)
