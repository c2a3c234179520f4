"""Pins of the oracle's transforms and of the discrete operator of Eqs. (1), (2), (11)."""
import numpy as np
import pytest

from oracle import dft, kernel, operator


@pytest.mark.parametrize("M", [2, 4, 8, 32, 128])
def test_radix2_fft_matches_definition(M):
    rng = np.random.default_rng(M)
    x = rng.standard_normal((3, M)) + 1j * rng.standard_normal((3, M))
    np.testing.assert_allclose(dft.fft(x), dft.dft(x), atol=1e-12 * M)
    np.testing.assert_allclose(dft.fft(x, inverse=True), dft.dft(x, inverse=True), atol=1e-12 * M)
    # Parseval and round trip
    X = dft.fft(x)
    np.testing.assert_allclose(np.sum(abs(X) ** 2, -1), M * np.sum(abs(x) ** 2, -1), rtol=1e-12)
    np.testing.assert_allclose(dft.fft(X, inverse=True) / M, x, atol=1e-13)


def test_fft_of_delta_and_exponential():
    M = 16
    e = np.zeros(M); e[3] = 1.0
    np.testing.assert_allclose(dft.fft(e), np.exp(-2j * np.pi * 3 * np.arange(M) / M), atol=1e-14)
    x = np.exp(2j * np.pi * 5 * np.arange(M) / M)
    X = dft.fft(x)
    ref = np.zeros(M, complex); ref[5] = M
    np.testing.assert_allclose(X, ref, atol=1e-12)


def test_identity_kernel_gives_identity_operator():
    N = 8
    p = np.random.default_rng(0).standard_normal((N, N))
    ones = np.ones((2 * N, 2 * N))
    np.testing.assert_allclose(operator.matvec_fft(ones, p), p, atol=1e-13)
    np.testing.assert_allclose(operator.matvec_dense(ones, p), p, atol=1e-13)


@pytest.mark.parametrize("N", [4, 8, 16])
@pytest.mark.parametrize("dc_mode", [0, 1])
def test_dense_sum_equals_fft_form(N, dc_mode):
    Kg = operator.khat_grid(N, 0.1, 0.35, 3.0, 0.3, 1.0, 0.45, dc_mode=dc_mode)
    rng = np.random.default_rng(N)
    p = rng.standard_normal((N, N))
    a = operator.matvec_dense(Kg, p)
    b = operator.matvec_fft(Kg, p)
    np.testing.assert_allclose(a, b, atol=1e-13 * abs(a).max())


def test_symmetric_positive():
    N = 8
    Kg = operator.khat_grid(N, 0.2, 0.5, 0.3, 0.3, 1.0, 0.3)
    Km = operator.dense_matrix(Kg)
    np.testing.assert_allclose(Km, Km.T, atol=1e-14 * abs(Km).max())
    assert np.linalg.eigvalsh(Km).min() > 0


def test_wavenumber_grid():
    N, d = 4, 0.25
    k = operator.wavenumbers(N, d)
    M = 2 * N
    assert k[0, 0] == 0.0
    assert k[0, 1] == pytest.approx(2 * np.pi / (M * d))
    assert k[0, M - 1] == pytest.approx(2 * np.pi / (M * d))       # wrap-around
    assert k[N, N] == pytest.approx(np.sqrt(2) * np.pi / d)         # Nyquist corner


def test_uniform_circular_load():
    """Homogeneous half-space under a uniform pressure P on a disc of radius b
    (classical Boussinesq integral): u(0) = 2 P b / E*, and for r > b
    u(r) = 4 P r / (pi E*) [E(m) - (1 - m) K(m)], m = (b/r)^2.  The DC rule and the
    periodic images add a near-constant offset, so u(0) - u(r) is compared."""
    from scipy.special import ellipe, ellipk
    N, delta, E, nu, P = 64, 1.0, 2.0, 0.3, 1.0
    Kg = operator.khat_grid(N, delta, np.inf, E, nu, E, nu)
    c0 = N // 2
    y, x = np.mgrid[0:N, 0:N]
    r = np.hypot(x - c0, y - c0)
    b = 8
    p = np.where(r <= b, P, 0.0)
    b_eff = np.sqrt(p.sum() / np.pi)           # disc of the same area as the cells
    u = operator.matvec_fft(Kg, p)
    Es = kernel.e_star(E, nu)
    for k in (2, 3):
        r0 = k * b
        m = (b_eff / r0) ** 2
        u_r0 = 4 * P * r0 / (np.pi * Es) * (ellipe(m) - (1 - m) * ellipk(m))
        ref = 2 * P * b_eff / Es - u_r0
        assert u[c0, c0] - u[c0, c0 + r0] == pytest.approx(ref, rel=1e-2)


STACKS = {
    "layered": (0.35, 3.0, 0.3, 1.0, 0.45),
    "rigid_base": (0.35, 1.0, 0.3, np.inf, 0.3),
    "homogeneous": (np.inf, 2.0, 0.3, 2.0, 0.3),
}


@pytest.mark.parametrize("N", [4, 8, 16])
@pytest.mark.parametrize("dc_mode", [0, 1])
@pytest.mark.parametrize("stack", sorted(STACKS))
def test_influence_at_equals_inverse_dft(N, dc_mode, stack):
    """``influence_at`` (one offset at a time, the reference of the full-size GPU
    impulse test) against the naive 2-D inverse DFT of the same sampled compliance
    (``influence``) at every offset (dy, dx) in (-N, N)^2, wrapped onto the 2N period,
    and against the columns of the dense matrix of Eq. (1) (the response at every
    window cell to a unit pressure on one cell).  A wrong wrap of negative offsets, a
    wrong 1/M^2 factor or a wrong wave-number grid fails here."""
    delta = 0.1
    h, E1, nu1, E2, nu2 = STACKS[stack]
    M = 2 * N
    Kg = operator.khat_grid(N, delta, h, E1, nu1, E2, nu2, dc_mode=dc_mode)
    G = operator.influence(Kg)
    offs = [(dy, dx) for dy in range(-(N - 1), N) for dx in range(-(N - 1), N)]
    got = operator.influence_at(N, delta, h, E1, nu1, E2, nu2, offs, dc_mode=dc_mode)
    ref = np.array([G[dy % M, dx % M] for dy, dx in offs])
    scale = abs(ref).max()
    np.testing.assert_allclose(got, ref, rtol=0, atol=1e-13 * scale)
    # columns of the dense matrix: K[(r, c), (s, t)] = G(r - s, c - t)
    Km = operator.dense_matrix(Kg)
    for s, t in [(0, 0), (N - 1, 0), (N // 2, N - 1), (1, 2)]:
        col = Km[:, s * N + t].reshape(N, N)
        o = [(r - s, c - t) for r in range(N) for c in range(N)]
        vals = operator.influence_at(N, delta, h, E1, nu1, E2, nu2, o, dc_mode=dc_mode).reshape(N, N)
        np.testing.assert_allclose(vals, col, rtol=0, atol=1e-13 * scale)
