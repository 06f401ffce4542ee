"""Pins of the oracle's units, deposit, field and Poisson solvers against the
paper's printed numbers, closed forms and independent solvers (CPU)."""
import math
import os

import numpy as np
import pytest

import synth
from oracle import deposit, field, poisson, units
from oracle.geometry import Geometry, from_workload

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


def _golden(name):
    out = {}
    for line in open(os.path.join(GOLDEN, name)):
        line = line.strip()
        if line and not line.startswith("#"):
            k, v = line.split()
            out[k] = float(v)
    return out


# ---------------------------------------------------------------- units (Sec. III)
def test_unit_example_matches_paper():
    g = _golden("units_example.txt")
    n0_m3 = g["n0_cm3"] * 1e6
    lam_cm = units.debye_length_m(g["te_ev"], n0_m3) * 100.0
    om = units.plasma_frequency(n0_m3)
    orf = units.normalised_frequency(g["f_rf_hz"], n0_m3)
    # The printed values sit within 0.7% of the definitions of Sec. II (the
    # definitions give 1.560e-2 cm and 8.499e9 1/s; the printed pair keeps
    # lambda_e * omega_e = v_e within 0.4%), so the pin allows 1%: a dropped
    # 2 pi, a wrong mass or a missing square root misses it by far more.
    assert lam_cm == pytest.approx(g["lambda_e_cm"], rel=1e-2)
    assert om == pytest.approx(g["omega_e_per_s"], rel=1e-2)
    assert orf == pytest.approx(g["omega_rf_normalised"], rel=1e-2)


# ---------------------------------------------------------------- deposit
def test_cic_single_particle_by_hand():
    geom = Geometry(8, 8, False, False)
    rho = deposit.cic_density(geom, [2.25], [3.5], 1.0)
    exp = np.zeros_like(rho)
    exp[2, 3] = 0.75 * 0.5
    exp[3, 3] = 0.25 * 0.5
    exp[2, 4] = 0.75 * 0.5
    exp[3, 4] = 0.25 * 0.5
    np.testing.assert_allclose(rho, exp, atol=1e-15)


def test_cic_periodic_wrap_by_hand():
    geom = Geometry(8, 8, True, True)
    rho = deposit.cic_density(geom, [7.5], [7.75], 2.0)
    assert rho[7, 7] == pytest.approx(2 * 0.5 * 0.25)
    assert rho[0, 7] == pytest.approx(2 * 0.5 * 0.25)
    assert rho[7, 0] == pytest.approx(2 * 0.5 * 0.75)
    assert rho[0, 0] == pytest.approx(2 * 0.5 * 0.75)


@pytest.mark.parametrize("wl", [synth.periodic_square_64(), synth.small_trench(),
                                synth.bounded_square_256(nx=32, ny=24)])
def test_cic_conserves_charge(wl):
    geom = from_workload(wl)
    p = synth.random_state(wl, 0, 5000, seed=3)
    rho = deposit.cic_density(geom, p.x, p.y, 0.01)
    assert rho.sum() == pytest.approx(50.0, rel=1e-13)


def test_surface_charge_split_conserves():
    wl = synth.small_trench()
    geom = from_workload(wl)
    sigma = np.zeros(wl.ny)
    sigma[wl.trench_y0 + 2] = 3.0
    rho = deposit.surface_charge_density(geom, sigma)
    assert rho[wl.nx - 1, wl.trench_y0 + 2] == 1.5
    assert rho[wl.nx - 1, wl.trench_y0 + 3] == 1.5
    assert rho.sum() == 3.0


# ---------------------------------------------------------------- Poisson (Eq. 5)
def test_dft_matches_min_norm_dense_solve():
    geom = Geometry(8, 6, True, True)
    rng = np.random.default_rng(1)
    rho = rng.standard_normal((8, 6))
    A, fi, fj, lift = poisson.system(geom)
    b = rho[fi, fj] - rho.mean()
    x = np.linalg.lstsq(A.toarray(), b, rcond=None)[0]   # min-norm = zero-mean
    phi = poisson.solve_dft(geom, rho)
    np.testing.assert_allclose(phi[fi, fj], x, atol=1e-12)
    assert abs(phi.mean()) < 1e-13


def test_linear_potential_between_biased_plates():
    w = synth.Workload(name="plates", nx=40, ny=8, periodic_y=True, phi_top=0.0,
                       phi_electrode=-20.0)
    geom = from_workload(w)
    phi = poisson.solve_direct(geom, np.zeros((41, 8)))
    exp = -20.0 * np.arange(41)[:, None] / 40.0 * np.ones((1, 8))
    np.testing.assert_allclose(phi, exp, atol=1e-11)


def test_manufactured_solution_second_order():
    errs = []
    for n in (16, 32, 64):
        geom = Geometry(n, n, False, False)
        x = np.arange(n + 1)[:, None]
        y = np.arange(n + 1)[None, :]
        k = math.pi / n
        exact = np.sin(k * x) * np.sin(2 * k * y)
        rho = (k * k + 4 * k * k) * exact
        phi = poisson.solve_direct(geom, rho)
        errs.append(np.abs(phi - exact).max())
    r1, r2 = errs[0] / errs[1], errs[1] / errs[2]
    assert 3.6 < r1 < 4.4 and 3.8 < r2 < 4.2, errs


def test_trench_direct_matches_gauss_seidel_and_jacobi():
    w = synth.small_trench(nx=24, ny=16, depth=8, width=4)
    geom = from_workload(w)
    rho = synth.random_rho(w, seed=4, scale=0.5)
    ref = poisson.solve_direct(geom, rho)
    gs = poisson.gauss_seidel(geom, rho, tol=1e-12)
    ja = poisson.jacobi(geom, rho, tol=1e-11)
    np.testing.assert_allclose(gs, ref, atol=1e-9 * np.abs(ref).max())
    np.testing.assert_allclose(ja, ref, atol=1e-8 * np.abs(ref).max())
    assert poisson.residual_rel(geom, ref, rho) < 1e-13


def test_periodic_dft_matches_gauss_seidel():
    geom = Geometry(12, 10, True, True)
    rho = np.random.default_rng(7).standard_normal((12, 10))
    ref = poisson.solve_dft(geom, rho)
    gs = poisson.gauss_seidel(geom, rho, tol=1e-12)
    np.testing.assert_allclose(gs, ref, atol=1e-9 * np.abs(ref).max())


def test_dirichlet_nodes_of_trench():
    w = synth.small_trench(nx=24, ny=16, depth=8, width=4)   # trench y in [6, 10), x >= 16
    geom = from_workload(w)
    D, g = geom.dirichlet, geom.g
    assert D[0].all() and (g[0] == 0).all()
    assert D[24].all() and (g[24] == -20).all()
    assert D[16, 0] and g[16, 0] == -20          # electrode top surface
    assert not D[15, 0]                          # plasma above the electrode
    assert D[20, 6] and D[20, 10]                # trench side walls
    assert not D[20, 7] and not D[20, 9]         # trench interior
    assert not D[16, 8]                          # trench mouth centre
    assert D[16, 6] and D[16, 10]                # trench mouth corners


# ---------------------------------------------------------------- field (Sec. II)
def test_field_linear_potential_exact_everywhere():
    geom = Geometry(10, 7, False, False)
    x = np.arange(11)[:, None] * np.ones((1, 8))
    y = np.ones((11, 1)) * np.arange(8)[None, :]
    Ex, Ey = field.efield(geom, 0.3 * x - 1.7 * y + 2.0)
    np.testing.assert_allclose(Ex, -0.3, atol=1e-13)
    np.testing.assert_allclose(Ey, 1.7, atol=1e-13)


def test_field_quadratic_central_exact_inside():
    geom = Geometry(10, 6, False, True)
    x = np.arange(11)[:, None] * np.ones((1, 6))
    Ex, Ey = field.efield(geom, x * x)
    np.testing.assert_allclose(Ex[1:-1], -2 * x[1:-1], atol=1e-12)
    # two-point one-sided at the plates
    assert Ex[0, 0] == pytest.approx(-(1 - 0))
    assert Ex[10, 0] == pytest.approx(-(100 - 81))
    np.testing.assert_allclose(Ey, 0.0, atol=1e-13)


def test_field_tangential_zero_on_conductors():
    w = synth.small_trench(nx=24, ny=16, depth=8, width=4)
    geom = from_workload(w)
    rho = synth.random_rho(w, seed=9)
    phi = poisson.solve_direct(geom, rho)
    Ex, Ey = field.efield(geom, phi)
    np.testing.assert_allclose(Ey[0], 0.0, atol=1e-12)           # top plate
    np.testing.assert_allclose(Ex[17:24, 6], 0.0, atol=1e-12)    # lower trench wall
    np.testing.assert_allclose(Ex[17:24, 10], 0.0, atol=1e-12)   # upper trench wall
    np.testing.assert_allclose(Ey[16, :6], 0.0, atol=1e-12)      # electrode top
    # one-sided normal field on the electrode top, from the plasma side
    assert Ex[16, 2] == pytest.approx(-(phi[16, 2] - phi[15, 2]))
    # inside the conductor the field vanishes
    assert Ex[20, 2] == 0 and Ey[20, 2] == 0
    # one-sided normal field on a trench wall, from the trench side
    assert Ey[20, 6] == pytest.approx(-(phi[20, 7] - phi[20, 6]))
