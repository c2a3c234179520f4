"""Discrete Fourier transforms written out from their definition (no library FFT).

Test infrastructure (see ``oracle/__init__``).  Eq. (2) and Eq. (11) of the paper
use FFT/IFFT without fixing a convention; the reading used throughout is the
unnormalised forward transform X[k] = sum_n x[n] e^{-2 pi i k n / M} and the inverse
with the factor 1/M (1/M^2 in two dimensions).

* ``dft``      O(M^2) sum, straight from the definition (tiny sizes).
* ``fft``      textbook iterative radix-2 Cooley-Tukey: bit-reversal permutation,
               then log2(M) butterfly stages; vectorised over leading axes.
* ``fft2`` / ``ifft2``  rows then columns with ``fft``.

Pinned by tests against ``dft`` on random inputs, Parseval, the transform of a
delta and of a pure exponential, and linearity.
"""
import numpy as np


def dft(x, inverse=False):
    """Plain O(M^2) DFT along the last axis (unnormalised in both directions)."""
    x = np.asarray(x, dtype=np.complex128)
    M = x.shape[-1]
    n = np.arange(M)
    sign = 1.0 if inverse else -1.0
    W = np.exp(sign * 2j * np.pi * np.outer(n, n) / M)
    return x @ W.T


def _bit_reverse(M):
    bits = M.bit_length() - 1
    idx = np.arange(M)
    rev = np.zeros(M, dtype=np.int64)
    for b in range(bits):
        rev |= ((idx >> b) & 1) << (bits - 1 - b)
    return rev


def fft(x, inverse=False):
    """Iterative radix-2 FFT along the last axis; length must be a power of two.

    Unnormalised in both directions (the inverse omits 1/M).
    """
    x = np.asarray(x, dtype=np.complex128)
    M = x.shape[-1]
    if M & (M - 1):
        raise ValueError("radix-2 FFT needs a power-of-two length")
    lead = x.shape[:-1]
    a = x[..., _bit_reverse(M)].copy()
    sign = 1.0 if inverse else -1.0
    size = 2
    while size <= M:
        half = size // 2
        w = np.exp(sign * 2j * np.pi * np.arange(half) / size)
        a = a.reshape(lead + (M // size, size))
        even = a[..., :half].copy()
        odd = a[..., half:] * w
        a[..., :half] = even + odd
        a[..., half:] = even - odd
        a = a.reshape(lead + (M,))
        size *= 2
    return a


def fft2(x):
    """2-D forward transform: ``fft`` over the last axis, then the one before it."""
    y = fft(x)
    return np.swapaxes(fft(np.swapaxes(y, -1, -2)), -1, -2)


def ifft2(X):
    """2-D inverse transform including the 1/(M0 M1) factor."""
    y = fft(X, inverse=True)
    y = np.swapaxes(fft(np.swapaxes(y, -1, -2), inverse=True), -1, -2)
    return y / (X.shape[-1] * X.shape[-2])
