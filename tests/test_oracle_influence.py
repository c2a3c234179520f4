"""Pins of the oracle's non-periodic operator (Love's square-cell influence
coefficients of a homogeneous half-space, convolved over the open plane)."""
import numpy as np
import pytest
from scipy import integrate

from oracle import analytic, contact, influence, kernel
from paper_1807_01885_gb300 import inputs


def test_centre_value_is_loves():
    """Displacement at the centre of a uniformly loaded square: 4 ln(1 + sqrt 2)
    delta / (pi E*) per unit pressure (Love)."""
    delta, E, nu = 0.3, 2.0, 0.3
    G = influence.influence_love(4, delta, E, nu)
    assert G[3, 3] == pytest.approx(4 * np.log(1 + np.sqrt(2)) * delta / (np.pi * kernel.e_star(E, nu)),
                                    rel=1e-14)


@pytest.mark.parametrize("x,y", [(0.0, 0.0), (1.0, 0.0), (1.0, 1.0), (2.0, -1.0), (0.3, 0.7), (5.0, 3.0)])
def test_closed_form_against_quadrature(x, y):
    """The closed form against adaptive quadrature of the defining double integral of
    1/r over the cell (the singular centre case split into four corner squares)."""
    delta = 1.0
    h = delta / 2
    f = lambda eta, xi: 1.0 / np.hypot(x - xi, y - eta)
    if abs(x) < h and abs(y) < h:
        q = 0.0
        for x0, x1 in ((-h, x), (x, h)):
            for y0, y1 in ((-h, y), (y, h)):
                q += integrate.dblquad(f, x0, x1, y0, y1, epsabs=1e-12, epsrel=1e-11)[0]
    else:
        q = integrate.dblquad(f, -h, h, -h, h, epsabs=1e-12, epsrel=1e-11)[0]
    assert influence.cell_integral(x, y, delta) == pytest.approx(q, rel=1e-9)


def test_far_field_is_point_load():
    """Far from the cell the influence is Boussinesq's P / (pi E* r), P = delta^2,
    with a relative correction of order (delta / r)^2 (the cell's second moment)."""
    N, delta, E, nu = 64, 0.5, 1.0, 0.25
    G = influence.influence_love(N, delta, E, nu)
    for i, j in ((0, 40), (30, 30), (-50, 10)):
        r = np.hypot(i, j) * delta
        pt = delta ** 2 / (np.pi * kernel.e_star(E, nu) * r)
        assert G[i + N - 1, j + N - 1] / pt - 1 == pytest.approx(0.0, abs=(delta / r) ** 2 / 10)


def test_symmetry_positivity_and_fft_form():
    N, delta = 8, 1.0
    G = influence.influence_love(N, delta, 1.0, 0.3)
    assert np.allclose(G, G[::-1, :]) and np.allclose(G, G[:, ::-1]) and np.allclose(G, G.T)
    rng = np.random.default_rng(1)
    p, q = rng.standard_normal((N, N)), rng.standard_normal((N, N))
    up, uq = influence.matvec_dense_np(G, p), influence.matvec_dense_np(G, q)
    assert np.sum(q * up) == pytest.approx(np.sum(p * uq), rel=1e-12)
    # the matrix of the operator on the window is positive definite
    Kmat = np.array([influence.matvec_dense_np(G, e.reshape(N, N)).ravel() for e in np.eye(N * N)])
    assert np.linalg.eigvalsh(0.5 * (Kmat + Kmat.T))[0] > 0
    np.testing.assert_allclose(influence.matvec_fft_np(G, p), up, rtol=0, atol=1e-13 * np.abs(up).max())


def test_hertz_with_the_open_plane_operator():
    """Sphere on a homogeneous half-space under force control with the non-periodic
    operator: contact radius (from the contact area) and peak pressure approach Hertz
    (a^3 = 3FR/4E*, p0 = 3F/(2 pi a^2), d = a^2/R) within the grid's discretisation
    error (0.5 % at a 16-cell radius); the periodic operator gives the pressure but
    the depth only up to its k = 0 datum."""
    N, R, E, nu = 64, 1.0, 1.0, 0.3
    Es = kernel.e_star(E, nu)
    a_H = 16.0 / N                       # Hertz radius of 16 cells at delta = 1/N
    delta = 1.0 / N
    F = 4 * Es * a_H ** 3 / (3 * R)
    G = influence.influence_love(N, delta, E, nu)
    f = inputs.sphere_height(N, delta, R)
    s = contact.solve_nonadhesive(lambda p: influence.matvec_fft_np(G, p), f, delta, "force", F, tol=1e-12)
    a_eq = np.sqrt(s["n_contact"] * delta ** 2 / np.pi)
    assert a_eq / a_H == pytest.approx(1.0, abs=0.01)
    p0 = 3 * F / (2 * np.pi * a_H ** 2)
    assert s["p"].max() / p0 == pytest.approx(1.0, abs=0.005)
    d_H = a_H ** 2 / R
    assert s["d"] / d_H == pytest.approx(1.0, abs=0.005)
    # the periodic product of Eq. (11) gives the same pressure but its depth only up
    # to the k = 0 datum: 20 % low here
    from oracle import operator
    Kg = operator.khat_grid(N, delta, np.inf, E, nu, E, nu)
    sp = contact.solve_nonadhesive(lambda p: operator.matvec_fft(Kg, p), f, delta, "force", F, tol=1e-12)
    assert sp["p"].max() / p0 == pytest.approx(1.0, abs=0.04)
    assert sp["d"] / d_H < 0.85


def test_spectrum_fits_a_folded_real_table():
    """The transform of the wrap-around coefficient array is real, even in each wave
    index and symmetric between them, so the (N+1) x (N+1) quarter of it determines
    the whole: the layout of the periodic product's compliance table."""
    N, delta = 16, 1.0
    G = influence.influence_love(N, delta, 1.0, 0.3)
    M = 2 * N
    W = np.zeros((M, M))
    idx = np.arange(-(N - 1), N) % M
    W[np.ix_(idx, idx)] = G
    S = np.fft.fft2(W)
    assert np.abs(S.imag).max() < 1e-12 * np.abs(S.real).max()
    R = S.real
    i = np.arange(M)
    assert np.allclose(R, R[(-i) % M, :]) and np.allclose(R, R[:, (-i) % M]) and np.allclose(R, R.T)
    Q = R[:N + 1, :N + 1]
    fold = lambda k: np.minimum(k, M - k)
    assert np.allclose(R, Q[fold(i)[:, None], fold(i)[None, :]])


@pytest.mark.parametrize("N", [32, 64])
def test_flat_punch_stiffness_on_the_open_plane(N):
    """Rigid flat punch of radius a = N/4 cells on a homogeneous half-space: the open
    plane operator gives Boussinesq's F/d = 2 a E* (within 0.5 %), where the periodic
    product of the same window is 43 % stiffer (its images and k = 0 datum)."""
    delta, a, E, nu = 1.0, N / 4, 1.0, 0.3
    f = inputs.flat_punch_height(N, delta, a)
    G = influence.influence_love(N, delta, E, nu)
    d = 1e-3 * a
    s = contact.solve_nonadhesive(lambda p: influence.matvec_fft_np(G, p), f, delta, "depth", d, tol=1e-12)
    k_B = analytic.flat_punch_stiffness(a, kernel.e_star(E, nu))
    assert s["force"] / d / k_B == pytest.approx(1.0, abs=0.005)
