"""Closed-form calculators of Sec. 5 (test infrastructure; part of the oracle).

- B-spline Fourier shape factor chi_r(k) and finite-grid plasma frequency,
  Eq. shape-factor-results;
- cold relativistic two-stream growth rate Gamma_TS, Eqs. rel-ts-cont, gamma-ts;
- cold relativistic Weibel growth rate Gamma_W, Eq. weibel-dispersion-updated
  and the A, C expressions below it.
"""
from __future__ import annotations

import math


def gamma_of_velocity(v0: float, kappa: float = 1.0) -> float:
    """Lorentz factor of a speed v0, Eq. rel-particle-def."""
    return 1.0 / math.sqrt(1.0 - v0 * v0 / (kappa * kappa))


def sinc(z: float) -> float:
    return 1.0 if z == 0.0 else math.sin(z) / z


def chi(k: float, dx: float, r: int = 2) -> float:
    """chi_r(k) = sinc(k dx / 2)^(r+1)."""
    return sinc(0.5 * k * dx) ** (r + 1)


def omega_ph2(k: float, dx: float, r: int = 2, sigma1: float = 1.0, rho0: float = 1.0) -> float:
    """omega_{p,h}^2 = sigma1 rho0 |chi_r(k)|^2."""
    return sigma1 * rho0 * chi(k, dx, r) ** 2


def two_stream_rate(k: float, v0: float, dx: float, r: int = 2, kappa: float = 1.0,
                    sigma1: float = 1.0, rho0: float = 1.0) -> float:
    """Gamma_TS = [sqrt(a^2 + 4ab) - a - b]^(1/2), a = w^2/(2 g0^3), b = k^2 v0^2."""
    g0 = gamma_of_velocity(v0, kappa)
    a = omega_ph2(k, dx, r, sigma1, rho0) / (2.0 * g0 ** 3)
    b = k * k * v0 * v0
    return math.sqrt(math.sqrt(a * a + 4.0 * a * b) - a - b)


def weibel_coeffs(k: float, v0: float, dx: float, r: int = 2, kappa: float = 1.0,
                  sigma1: float = 1.0, rho0: float = 1.0):
    """A = kappa^2 k^2 + w^2/g0^3 and C = k^2 w^2 v0^2 / g0."""
    g0 = gamma_of_velocity(v0, kappa)
    w2 = omega_ph2(k, dx, r, sigma1, rho0)
    A = kappa * kappa * k * k + w2 / g0 ** 3
    Cc = k * k * w2 * v0 * v0 / g0
    return A, Cc


def weibel_rate(k: float, v0: float, dx: float, r: int = 2, kappa: float = 1.0,
                sigma1: float = 1.0, rho0: float = 1.0) -> float:
    """Gamma_W^2 = (-A + sqrt(A^2 + 4C)) / 2."""
    A, Cc = weibel_coeffs(k, v0, dx, r, kappa, sigma1, rho0)
    return math.sqrt(0.5 * (-A + math.sqrt(A * A + 4.0 * Cc)))
