"""Pins of the oracle warm-start network: truncated transforms against numpy's FFT,
the adjoints by the inner-product identity, and every gradient by central finite
differences of the loss."""
import numpy as np
import pytest

from oracle import fno


def test_truncated_dft_matches_numpy_fft():
    rng = np.random.default_rng(0)
    N, m = 16, 3
    v = rng.standard_normal((2, 3, N, N))
    Xh = fno.dft_trunc(v, m)
    F = np.fft.fft2(v)
    kx, ky = fno.mode_indices(N, m)
    np.testing.assert_allclose(Xh, F[..., kx[:, None], ky[None, :]], atol=1e-11)
    Y = rng.standard_normal((2, 3, 2 * m, m)) + 1j * rng.standard_normal((2, 3, 2 * m, m))
    Z = np.zeros((2, 3, N, N), complex)
    c = np.where(ky == 0, 1.0, 2.0)
    Z[..., kx[:, None], ky[None, :]] = Y * c
    np.testing.assert_allclose(fno.idft_trunc(Y, N), np.real(np.fft.ifft2(Z)), atol=1e-12)


def test_adjoints():
    rng = np.random.default_rng(1)
    N, m = 12, 3
    v = rng.standard_normal((N, N))
    G = rng.standard_normal((2 * m, m)) + 1j * rng.standard_normal((2 * m, m))
    lhs = np.sum(np.real(np.conj(G) * fno.dft_trunc(v, m)))
    rhs = np.sum(v * fno.dft_trunc_adjoint(G, N))
    assert lhs == pytest.approx(rhs, rel=1e-12)
    g = rng.standard_normal((N, N))
    Y = rng.standard_normal((2 * m, m)) + 1j * rng.standard_normal((2 * m, m))
    lhs = np.sum(g * fno.idft_trunc(Y, N))
    rhs = np.sum(np.real(np.conj(fno.idft_trunc_adjoint(g, m)) * Y))
    assert lhs == pytest.approx(rhs, rel=1e-12)


def test_gelu_derivative():
    z = np.linspace(-4, 4, 33)
    e = 1e-6
    np.testing.assert_allclose(fno.gelu_grad(z), (fno.gelu(z + e) - fno.gelu(z - e)) / (2 * e), atol=1e-8)


def test_gradients_by_finite_differences():
    rng = np.random.default_rng(2)
    B, C, N, W, m, L, H = 2, 3, 8, 4, 2, 2, 5
    P = fno.init_params(rng, C, W, m, L, H)
    for k in P:
        P[k] = P[k] + 0.1 * rng.standard_normal(P[k].shape)     # non-zero biases too
    x = rng.standard_normal((B, C, N, N))
    t = rng.standard_normal((B, N, N))
    out, cache = fno.forward(P, x, m)
    G = fno.backward(P, cache, out, t, m)
    eps = 1e-6
    for key in P:
        flat = P[key].reshape(-1)
        idx = rng.choice(flat.size, size=min(6, flat.size), replace=False)
        for i in idx:
            old = flat[i]
            flat[i] = old + eps
            lp = fno.loss(fno.forward(P, x, m)[0], t)
            flat[i] = old - eps
            lm = fno.loss(fno.forward(P, x, m)[0], t)
            flat[i] = old
            fd = (lp - lm) / (2 * eps)
            an = G[key].reshape(-1)[i]
            assert an == pytest.approx(fd, rel=1e-5, abs=1e-9), (key, i, an, fd)


def test_gelu_is_z_times_normal_cdf():
    """gelu(z) = z Phi(z), Phi the standard normal distribution function (scipy's).
    The oracle's 1 + erf form cancels in the far negative tail, so the bound there is
    absolute (1e-15, against values of order 1e-9 at z = -6)."""
    stats = pytest.importorskip("scipy.stats")
    z = np.linspace(-6, 6, 49)
    np.testing.assert_allclose(fno.gelu(z), z * stats.norm.cdf(z), rtol=1e-14, atol=1e-15)
