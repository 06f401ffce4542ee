"""Normalisation of Sec. II and the unit example of Sec. III (oracle; test
infrastructure).

Sec. II: lambda_e = (eps0 T_e / (n_0 e^2))^(1/2), omega_e = (n_0 e^2 /
(eps0 m_e))^(1/2); lengths in lambda_e, times in 1/omega_e, potentials in
T_e/e, velocities in v_e = lambda_e omega_e.  Sec. III: with T_e = 10 eV
and n_0 = 2.27e10 cm^-3, lambda_e = 1.55e-2 cm and omega_e = 8.52e9 s^-1,
and the 13.56 MHz RF frequency becomes 0.01 in normalised units.

Pinned by tests/golden/units_example.txt (the paper's printed numbers).
"""
from __future__ import annotations

import math

# CODATA 2018 exact / recommended SI values
E_CHARGE = 1.602176634e-19        # C
EPS0 = 8.8541878128e-12           # F/m
M_E = 9.1093837015e-31            # kg


def debye_length_m(te_ev: float, n0_m3: float) -> float:
    return math.sqrt(EPS0 * te_ev * E_CHARGE / (n0_m3 * E_CHARGE ** 2))


def plasma_frequency(n0_m3: float) -> float:
    return math.sqrt(n0_m3 * E_CHARGE ** 2 / (EPS0 * M_E))


def normalised_frequency(f_hz: float, n0_m3: float) -> float:
    return 2.0 * math.pi * f_hz / plasma_frequency(n0_m3)
