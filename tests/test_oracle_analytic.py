"""Cross-checks of the closed forms of Sec. 3 against each other and against Eq. (13).

Each formula in oracle/analytic.py is typed once; these tests derive it a second
way (Eq. 13 from a stiffness law, a limit of another equation, a minimum found
numerically), so a typo in any one of them fails here."""
import numpy as np
import pytest
from scipy.optimize import minimize_scalar

from oracle import analytic, kernel


def eq13_dc(dk_da, a, dgamma):
    """Eq. (13) solved for the critical separation: dk/da d_c^2/2 = 2 pi a dgamma."""
    return -np.sqrt(4 * np.pi * a * dgamma / dk_da)


def test_eq16_from_eq13_and_eq14():
    a, h, E1, nu1, dg = 3.0, 0.1, 2.0, 0.3, 0.05
    Et = kernel.e_tilde(E1, nu1)
    dk_da = 2 * np.pi * a * Et / h                      # derivative of Eq. (14)
    dc, Fc = analytic.thin_layer_flat_punch_critical(a, h, E1, nu1, dg)
    assert dc == pytest.approx(eq13_dc(dk_da, a, dg), rel=1e-14)
    assert Fc == pytest.approx(analytic.thin_layer_stiffness(a, h, E1, nu1) * dc, rel=1e-14)


def test_jkr_adhesive_term_from_eq13_and_flat_punch():
    a, R, E, nu, dg = 0.3, 1.0, 1.0, 0.3, 0.01
    Es = kernel.e_star(E, nu)
    dc = eq13_dc(2 * Es, a, dg)                          # k(a) = 2 a E*
    F, d = analytic.jkr(a, R, Es, dg)
    assert d - a * a / R == pytest.approx(dc, rel=1e-14)
    assert F - analytic.hertz(a, R, Es)[0] == pytest.approx(2 * a * Es * dc, rel=1e-14)


def test_jkr_minima():
    R, Es, dg = 1.0, 1.3, 0.02
    resF = minimize_scalar(lambda a: analytic.jkr(a, R, Es, dg)[0], bounds=(1e-4, 1), method="bounded",
                           options=dict(xatol=1e-12))
    assert resF.fun == pytest.approx(analytic.jkr_pull_off_force(R, dg), rel=1e-9)
    resd = minimize_scalar(lambda a: analytic.jkr(a, R, Es, dg)[1], bounds=(1e-4, 1), method="bounded",
                           options=dict(xatol=1e-12))
    a, F, d = analytic.jkr_jump_off(R, Es, dg)
    assert resd.x == pytest.approx(a, rel=1e-5)
    assert F == pytest.approx(-5.0 / 6.0 * np.pi * R * dg, rel=1e-12)


def test_thin_layer_dimensionless_eqs_17_to_21():
    R, h, E1, nu1, dg = 2.0, 0.01, 1.0, 0.3, 1e-4
    d_crit, a_crit, F_crit = analytic.thin_layer_sphere_critical(R, h, E1, nu1, dg)
    for at in [0.3, 0.9, 1.0, 1.7]:
        F, d = analytic.thin_layer_sphere(at * a_crit, R, h, E1, nu1, dg)
        Ft, dt = analytic.thin_layer_dimensionless(at)
        assert F / abs(F_crit) == pytest.approx(Ft, rel=1e-12, abs=1e-14)
        assert d / abs(d_crit) == pytest.approx(dt, rel=1e-12, abs=1e-14)
    # F_crit is the minimum of Eq. (17); d_crit is d(a -> 0) of Eq. (18)
    res = minimize_scalar(lambda a: analytic.thin_layer_sphere(a, R, h, E1, nu1, dg)[0],
                          bounds=(1e-6, 5 * a_crit), method="bounded", options=dict(xatol=1e-14))
    assert res.fun == pytest.approx(F_crit, rel=1e-9)
    assert analytic.thin_layer_sphere(1e-12, R, h, E1, nu1, dg)[1] == pytest.approx(d_crit, rel=1e-9)


def test_thick_layer_series_limits():
    R, E1, nu1, dg, a = 1.0, 1.0, 0.3, 0.01, 0.2
    Es = kernel.e_star(E1, nu1)
    F, d = analytic.thick_layer_sphere(a, R, 1e12, E1, nu1, dg)        # epsilon -> 0: JKR
    Fj, dj = analytic.jkr(a, R, Es, dg)
    assert F == pytest.approx(Fj, rel=1e-10) and d == pytest.approx(dj, rel=1e-10)
    F, d = analytic.thick_layer_sphere(a, R, 1e12, E1, nu1, 0.0)       # and no adhesion: Hertz
    Fh, dh = analytic.hertz(a, R, Es)
    assert F == pytest.approx(Fh, rel=1e-10) and d == pytest.approx(dh, rel=1e-10)


def test_eq24_coefficients_from_rigid_base_kernel():
    """a0 = int Lambda is the k -> 0 limit of the rigid-base kernel's deficit:
    K(0+) = h/E~1 = 2/E1* * lim (1 - Lambda(kh))/k, and the same integral appears as
    the first moment of (1 - k E1* K/2).  Cross-check a0 with a trapezoid sum of
    Eq. (25) evaluated through the layered kernel of Eq. (9) (E2 = inf)."""
    nu1, E1, h = 0.3, 1.0, 1.0
    u = np.linspace(1e-9, 40.0, 400001)
    lam_via_eq9 = 1.0 - kernel.khat_layered(u / h, h, E1, nu1, np.inf, 0.3) * kernel.e_star(E1, nu1) * (u / h) / 2.0
    a0_trap = np.trapezoid(lam_via_eq9, u)
    a1_trap = -0.25 * np.trapezoid(lam_via_eq9 * u * u, u)
    assert analytic.a_coefficient(0, nu1) == pytest.approx(a0_trap, rel=1e-7)
    assert analytic.a_coefficient(1, nu1) == pytest.approx(a1_trap, rel=1e-7)


def test_adhesion_parameter_fig5():
    """Eq. (26) with the Fig. 5 parameters: alpha = 0.1 ... 15 maps to R."""
    E1, nu1, h, dg = 1e9, 0.3, 2e-3, 100.0
    for alpha in [0.1, 0.2, 0.5, 15]:
        R = alpha * np.sqrt(kernel.e_star(E1, nu1) * h ** 3 / (2 * dg))
        assert analytic.adhesion_parameter(dg, R, E1, nu1, h) == pytest.approx(alpha, rel=1e-14)
