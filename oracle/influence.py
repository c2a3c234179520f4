"""Non-periodic surface operator of a homogeneous half-space (test infrastructure).

Test infrastructure (see ``oracle/__init__``); no CUDA counterpart yet.  The
periodic product of Eq. (11) samples K^ on the 2N period and needs a convention
for the k = 0 term.  The non-periodic alternative takes the surface displacement
of a uniformly loaded square cell in real space and convolves it with the cell
pressures over the open plane (zero-padded, so the circular convolution on the
2N period is the exact linear one):

  u(x_r) = sum_s G(x_r - x_s) p_s,
  G(x, y) = 1/(pi E*) * integral over the cell |xi|, |eta| <= delta/2 of
            d xi d eta / sqrt((x - xi)^2 + (y - eta)^2),

the Boussinesq point-load solution u = P / (pi E* r) (Eq. 4 transformed back to
real space) integrated over the cell.  The double integral has a closed form (Love):
with F(s, t) = s asinh(t/|s|) + t asinh(s/|t|),

  integral = F(x+h, y+h) - F(x+h, y-h) - F(x-h, y+h) + F(x-h, y-h),  h = delta/2,

(the s ln|s| and t ln|t| parts of the antiderivative cancel between the corners).

* ``cell_integral``     the double integral above, closed form.
* ``influence_love``    G on the offsets -(N-1)..N-1 in both directions.
* ``matvec_dense_np``   u = G * p by the direct double sum.
* ``matvec_fft_np``     the same by zero-padded FFTs (the oracle's own radix-2 FFT).

Pinned by tests/test_oracle_influence.py: Love's centre value 4 ln(1 + sqrt 2) delta
/ (pi E*), numerical quadrature of the defining integral, the far field P/(pi E* r),
symmetry and positivity, dense = FFT, and Hertz contact.
"""
import numpy as np

from . import dft as _dft
from . import kernel as _kernel


def _F(s, t):
    s = np.asarray(s, dtype=np.float64)
    t = np.asarray(t, dtype=np.float64)
    with np.errstate(divide="ignore", invalid="ignore"):
        a = np.where(s != 0.0, s * np.arcsinh(t / np.abs(s)), 0.0)
        b = np.where(t != 0.0, t * np.arcsinh(s / np.abs(t)), 0.0)
    return a + b


def cell_integral(x, y, delta):
    """Integral of 1/r over the square cell of side delta centred at the origin, seen
    from the surface point (x, y)."""
    h = 0.5 * delta
    return _F(x + h, y + h) - _F(x + h, y - h) - _F(x - h, y + h) + _F(x - h, y - h)


def influence_love(N, delta, E, nu):
    """G[i + N - 1, j + N - 1] = displacement at offset (row i, column j) cells per unit
    pressure on one cell, i, j in -(N-1)..N-1."""
    off = np.arange(-(N - 1), N) * delta
    X, Y = np.meshgrid(off, off, indexing="xy")
    return cell_integral(X, Y, delta) / (np.pi * _kernel.e_star(E, nu))


def matvec_dense_np(G, p):
    """u_r = sum_s G(r - s) p_s over the N x N window (direct O(N^4) sum)."""
    N = p.shape[0]
    u = np.zeros((N, N))
    for r in range(N):
        for c in range(N):
            # G index of offset (r - s, c - t) is (r - s + N - 1, c - t + N - 1)
            u[r, c] = np.sum(G[r + N - 1 - np.arange(N)][:, c + N - 1 - np.arange(N)] * p)
    return u


def matvec_fft_np(G, p):
    """The same product by FFT: G in wrap-around order on the 2N period (offset N
    unused, zero), p zero-padded; the circular convolution equals the linear one on
    the window."""
    N = p.shape[0]
    M = 2 * N
    W = np.zeros((M, M))
    idx = np.arange(-(N - 1), N) % M
    W[np.ix_(idx, idx)] = G
    pad = np.zeros((M, M))
    pad[:N, :N] = p
    U = _dft.ifft2(_dft.fft2(W) * _dft.fft2(pad))
    return U.real[:N, :N].copy()
