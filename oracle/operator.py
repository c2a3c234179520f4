"""The discrete surface operator u = K p of Eq. (1), evaluated as in Eq. (11).

Test infrastructure (see ``oracle/__init__``).  Plain FP64 numpy.

Discretisation (Sec. 2, Fig. 2): an N x N window of square cells of side delta,
row-major, row index r along y and column index c along x; the pressure is
uniform per cell.  Reading of Eq. (11) used here (the paper states the periodic
form only): the window is embedded in an M x M period with M = 2N (zero pressure outside the
window), the compliance of Eq. (9) is sampled on that period's wave-number grid
k = 2 pi (i~, j~)/(M delta) with i~ = i for i <= N and i - M otherwise, the k = 0
term takes the finite part of ``kernel.khat_dc`` (or 0 with dc_mode=1, the literal
"no DC component" rule), and u is read back on the window.

* ``khat_grid``     the sampled compliance on the full M x M grid.
* ``khat_grid_layers``  the same for a stack of layers on a substrate
                    (``kernel.khat_multilayer`` at every distinct |k|).
* ``influence``     G(x) = (1/M^2) sum_k K(k) e^{i k.x}, by the naive 2-D inverse DFT.
* ``dense_matrix``  the N^2 x N^2 matrix K of Eq. (1): K[r, s] = G(x_r - x_s).
* ``matvec_dense``  Eq. (1) as a dense product (O(N^4); tiny N only).
* ``matvec_fft``    Eq. (2)/(11) with the oracle's own radix-2 FFT.
"""
import numpy as np

from . import dft as _dft
from . import kernel as _kernel


def wavenumbers(N, delta):
    """|k| on the 2N x 2N grid (Eq. 11: k = sqrt(kx^2 + ky^2)), shape (M, M)."""
    M = 2 * N
    i = np.arange(M)
    it = np.where(i <= N, i, i - M).astype(np.float64)
    kx = 2.0 * np.pi * it / (M * delta)
    return np.sqrt(kx[:, None] ** 2 + kx[None, :] ** 2)


def khat_grid(N, delta, h, E1, nu1, E2, nu2, dc_mode=0):
    """Eq. (9) sampled on the padded grid, with the DC rule described above."""
    k = wavenumbers(N, delta)
    K = np.zeros_like(k)
    nz = k > 0
    if np.isinf(h):
        K[nz] = _kernel.khat_homogeneous(k[nz], E1, nu1)
    else:
        K[nz] = _kernel.khat_layered(k[nz], h, E1, nu1, E2, nu2)
    if dc_mode == 0 and np.isfinite(h):
        K[0, 0] = _kernel.khat_dc(h, E1, nu1, E2, nu2)
    else:
        K[0, 0] = 0.0
    return K


def khat_grid_layers(N, delta, layers, E_sub, nu_sub, dc_mode=0, dc_value=None):
    """Compliance of a stack of bonded layers (``layers``: (h, E, nu) from the surface
    down) on a substrate (E_sub = inf: rigid base) sampled on the padded grid, with the
    same k = 0 reading as ``khat_grid``: the finite part (``kernel.khat_multilayer_dc``,
    or ``dc_value`` when the caller has it already) or 0 (dc_mode=1).  Each distinct
    |k| is evaluated once (K depends on i^2 + j^2 only)."""
    M = 2 * N
    i = np.arange(M)
    it = np.where(i <= N, i, i - M)
    sq = it[:, None] ** 2 + it[None, :] ** 2
    K = np.zeros((M, M))
    for s2 in np.unique(sq):
        if s2 == 0:
            continue
        k = 2.0 * np.pi * np.sqrt(float(s2)) / (M * delta)
        K[sq == s2] = _kernel.khat_multilayer(k, layers, E_sub, nu_sub)
    if dc_mode == 0:
        K[0, 0] = dc_value if dc_value is not None else _kernel.khat_multilayer_dc(layers, E_sub, nu_sub)
    return K


def influence(Kgrid):
    """G on the M x M period by the naive inverse DFT (a double sum written as
    two DFT-matrix products), including the 1/M^2 factor."""
    M = Kgrid.shape[0]
    n = np.arange(M)
    W = np.exp(2j * np.pi * np.outer(n, n) / M)
    G = W @ Kgrid @ W.T / (M * M)
    return G.real


def dense_matrix(Kgrid):
    """Eq. (1): the N^2 x N^2 matrix, K[(r,c), (s,t)] = G(r - s, c - t) (mod M)."""
    M = Kgrid.shape[0]
    N = M // 2
    G = influence(Kgrid)
    r = np.arange(N)
    dr = (r[:, None] - r[None, :]) % M
    # index [(r, c), (s, t)] -> G[dr[r, s], dr[c, t]]
    Kmat = G[dr[:, None, :, None], dr[None, :, None, :]]
    return Kmat.reshape(N * N, N * N)


def matvec_dense(Kgrid, p):
    """u = K p by the dense O(N^4) product of Eq. (1)."""
    N = p.shape[0]
    return (dense_matrix(Kgrid) @ p.reshape(-1)).reshape(N, N)


def matvec_fft(Kgrid, p):
    """u = IFFT[K(k) FFT(p)] on the 2N period, cropped to the window (Eq. 11)."""
    N = p.shape[0]
    M = 2 * N
    pad = np.zeros((M, M), dtype=np.float64)
    pad[:N, :N] = p
    U = _dft.ifft2(Kgrid * _dft.fft2(pad))
    return U.real[:N, :N].copy()


def influence_at(N, delta, h, E1, nu1, E2, nu2, offsets, dc_mode=0):
    """G at given integer cell offsets (dy, dx) by the direct sum over all M^2 wave
    numbers, G(x) = (1/M^2) sum_k K(k) cos(k.x) (K is even, so the sine part
    cancels).  One output at a time: usable at N = 2048."""
    M = 2 * N
    Kg = khat_grid(N, delta, h, E1, nu1, E2, nu2, dc_mode)
    i = np.arange(M)
    out = []
    for dy, dx in offsets:
        cy = np.cos(2.0 * np.pi * i * dy / M)
        cx = np.cos(2.0 * np.pi * i * dx / M)
        sy = np.sin(2.0 * np.pi * i * dy / M)
        sx = np.sin(2.0 * np.pi * i * dx / M)
        # cos(a + b) = cos a cos b - sin a sin b, summed as two rank-one contractions
        out.append((cy @ Kg @ cx - sy @ Kg @ sx) / (M * M))
    return np.array(out)
