"""Closed-form and asymptotic solutions used to pin the oracle (Sec. 3).

Test infrastructure (see ``oracle/__init__``).

* Hertz / JKR for a paraboloid on a homogeneous half-space: Eqs. (22)/(23) at
  epsilon = 0 (the a << h series reduces to them).  The displacement-controlled
  jump-off point (minimum of d(a)) and the force-controlled pull-off (minimum of
  F(a)) follow from the same two expressions.
* Flat punch on a homogeneous half-space: stiffness 2 a E* (the classical
  Boussinesq result; Eq. 4 is its Fourier form).
* Thin layer on a rigid base (a >> h): Eqs. (14)-(21).
* Thick layer (a << h) on a rigid base: Eqs. (22)-(25), with a_m from Eq. (24)
  by adaptive quadrature of Eq. (25).
* Adhesion parameter, Eq. (26).
"""
import numpy as np
from scipy import integrate

from .kernel import e_star, e_tilde, lam_rigid


def hertz(a, R, Es):
    """Paraboloid, no adhesion: F = 4 E* a^3/(3R), d = a^2/R."""
    return 4.0 * Es * a ** 3 / (3.0 * R), a * a / R


def hertz_pressure(r, a, R, Es):
    """Hertz pressure p0 sqrt(1 - r^2/a^2), p0 = 2 E* a/(pi R)."""
    p0 = 2.0 * Es * a / (np.pi * R)
    return np.where(r < a, p0 * np.sqrt(np.maximum(1.0 - (r / a) ** 2, 0.0)), 0.0)


def jkr(a, R, Es, dgamma):
    """Eqs. (22)/(23) at epsilon = 0: F = 4E*a^3/(3R) - sqrt(8 pi dgamma E* a^3),
    d = a^2/R - sqrt(2 pi a dgamma / E*)."""
    F = 4.0 * Es * a ** 3 / (3.0 * R) - np.sqrt(8.0 * np.pi * dgamma * Es * a ** 3)
    d = a * a / R - np.sqrt(2.0 * np.pi * a * dgamma / Es)
    return F, d


def jkr_jump_off(R, Es, dgamma):
    """Minimum of d(a) (displacement control): a^3 = pi R^2 dgamma/(8 E*),
    F = -(5/6) pi R dgamma.  Returns (a, F, d)."""
    a = (np.pi * R * R * dgamma / (8.0 * Es)) ** (1.0 / 3.0)
    F, d = jkr(a, R, Es, dgamma)
    return a, F, d


def jkr_pull_off_force(R, dgamma):
    """Minimum of F(a) (force control): F = -(3/2) pi R dgamma."""
    return -1.5 * np.pi * R * dgamma


def flat_punch_stiffness(a, Es):
    """Rigid flat cylindrical punch on a homogeneous half-space: F/d = 2 a E*."""
    return 2.0 * a * Es


def thin_layer_stiffness(a, h, E1, nu1):
    """Eq. (14): k = pi a^2 E~1 / h, E~1 from Eq. (15)."""
    return np.pi * a * a * e_tilde(E1, nu1) / h


def thin_layer_flat_punch_critical(a, h, E1, nu1, dgamma):
    """Eq. (16): d_c = -sqrt(2 dgamma h/E~1), F_c = -pi a^2 sqrt(2 E~1 dgamma/h)."""
    Et = e_tilde(E1, nu1)
    return -np.sqrt(2.0 * dgamma * h / Et), -np.pi * a * a * np.sqrt(2.0 * Et * dgamma / h)


def thin_layer_sphere(a, R, h, E1, nu1, dgamma):
    """Eqs. (17)/(18): F(a), d(a) for a paraboloid on a thin layer, rigid base."""
    Et = e_tilde(E1, nu1)
    s = np.sqrt(2.0 * h * dgamma / Et)
    F = np.pi * Et * a * a / h * (a * a / (4.0 * R) - s)
    d = a * a / (2.0 * R) - s
    return F, d


def thin_layer_sphere_critical(R, h, E1, nu1, dgamma):
    """Eq. (19): (d_crit, a_crit, F_crit)."""
    Et = e_tilde(E1, nu1)
    return (-np.sqrt(2.0 * h * dgamma / Et), (8.0 * R * R * h * dgamma / Et) ** 0.25,
            -2.0 * np.pi * R * dgamma)


def thin_layer_dimensionless(at):
    """Eqs. (20)/(21): F~ = a~^4 - 2 a~^2, d~ = a~^2 - 1."""
    return at ** 4 - 2.0 * at ** 2, at ** 2 - 1.0


def a_coefficient(m, nu):
    """Eq. (24): a_m = (-1)^m / (2^{2m} (m!)^2) * int_0^inf Lambda(u) u^{2m} du."""
    val, _ = integrate.quad(lambda u: lam_rigid(u, nu) * u ** (2 * m), 0.0, np.inf,
                            epsabs=1e-14, epsrel=1e-13, limit=400)
    fact = float(np.prod(np.arange(1, m + 1))) if m > 0 else 1.0
    return (-1.0) ** m / (2.0 ** (2 * m) * fact * fact) * val


def thick_layer_sphere(a, R, h, E1, nu1, dgamma, a0=None, a1=None):
    """Eqs. (22)/(23): F(a), d(a) to order epsilon^4, epsilon = a/h, rigid base."""
    if a0 is None:
        a0 = a_coefficient(0, nu1)
    if a1 is None:
        a1 = a_coefficient(1, nu1)
    Es = e_star(E1, nu1)
    eps = a / h
    pi = np.pi
    root = np.sqrt(2.0 * pi * Es * a * dgamma)
    F = (4.0 * Es * a ** 3 / (3.0 * R)) * (1.0 - eps ** 3 * 8.0 * a1 / (3.0 * pi)) * (
        1.0 - 3.0 * R * root / (2.0 * Es * a * a))
    d = (a * a / R) * (1.0 - eps * 4.0 * a0 / (3.0 * pi) - eps ** 3 * 16.0 * a1 / (5.0 * pi)
                       + eps ** 4 * 32.0 * a0 * a1 / (9.0 * pi * pi)
                       - R * root / (Es * a * a) * (1.0 - eps * 2.0 * a0 / pi
                                                    - eps ** 3 * 16.0 * a1 / (3.0 * pi)
                                                    + eps ** 4 * 16.0 * a0 * a1 / (3.0 * pi * pi)))
    return F, d


def adhesion_parameter(dgamma, R, E1, nu1, h):
    """Eq. (26): alpha = sqrt(2 dgamma R^2 / (E1* h^3))."""
    return np.sqrt(2.0 * dgamma * R * R / (e_star(E1, nu1) * h ** 3))
