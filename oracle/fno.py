"""FP64 Fourier-neural-operator forward and backward (reference for the warm-start network).

Test infrastructure (see ``oracle/__init__``).  The paper has no learned component;
this network seeds the contact solve with a predicted pressure field.  The layer
definitions below are the ones the CUDA kernels implement:

  lift       v0 = P x + p               (pointwise, C_IN -> W channels)
  layer l    z = S_l(v) + W_l v + b_l,  v' = gelu(z)   (no gelu after the last layer)
  spectral   S(v) = idft(R * dft(v)) on the retained modes kx in {0..m-1, N-m..N-1},
             ky in {0..m-1}:
               dft(v)[kx, ky]  = sum_{x,y} v[x, y] e^{-2 pi i (kx x + ky y)/N}
               (R * V)[o]      = sum_i R[i, o] V[i]          (complex, per mode)
               idft(Y)[x, y]   = (1/N^2) sum_{kx,ky} c_ky Re(Y[kx, ky] e^{+2 pi i (kx x + ky y)/N}),
                                 c_0 = 1, c_ky = 2 otherwise (the half-spectrum convention)
  project    h = gelu(Q1 v + q1),  out = Q2 h + q2
  gelu(z)    = z Phi(z) (exact, with the error function)
  loss       mean((out - target)^2)

Arrays are channels-first: x [B, C, N, N].  Parameters are a dict of float64 arrays;
complex spectral weights are stored as separate real and imaginary parts
R_re, R_im [L, W_in, W_out, 2m, m].  Pinned by central finite differences of the loss
and by numpy's FFT for the truncated transforms (tests/test_oracle_fno.py).
"""
import math

import numpy as np

SQRT2 = math.sqrt(2.0)


def mode_indices(N, m):
    kx = np.concatenate([np.arange(m), np.arange(N - m, N)])
    ky = np.arange(m)
    return kx, ky


def dft_trunc(v, m):
    """[..., N, N] real -> [..., 2m, m] complex, retained modes of the 2-D DFT."""
    N = v.shape[-1]
    kx, ky = mode_indices(N, m)
    n = np.arange(N)
    Ex = np.exp(-2j * np.pi * np.outer(kx, n) / N)      # [2m, N]
    Ey = np.exp(-2j * np.pi * np.outer(n, ky) / N)      # [N, m]
    return np.einsum("ax,...xy,yb->...ab", Ex, v, Ey)


def idft_trunc(Y, N):
    """[..., 2m, m] complex -> [..., N, N] real (half-spectrum weights c_ky)."""
    m = Y.shape[-1]
    kx, ky = mode_indices(N, m)
    n = np.arange(N)
    c = np.where(ky == 0, 1.0, 2.0)
    Ex = np.exp(2j * np.pi * np.outer(n, kx) / N)       # [N, 2m]
    Ey = np.exp(2j * np.pi * np.outer(ky, n) / N)       # [m, N]
    return np.real(np.einsum("xa,...ab,b,by->...xy", Ex, Y, c, Ey)) / (N * N)


def dft_trunc_adjoint(G, N):
    """Adjoint of dft_trunc: d/dv of sum Re(conj(G) dft(v)) = Re(sum G e^{+i theta})."""
    m = G.shape[-1]
    kx, ky = mode_indices(N, m)
    n = np.arange(N)
    Ex = np.exp(2j * np.pi * np.outer(n, kx) / N)
    Ey = np.exp(2j * np.pi * np.outer(ky, n) / N)
    return np.real(np.einsum("xa,...ab,by->...xy", Ex, G, Ey))


def idft_trunc_adjoint(g, m):
    """Adjoint of idft_trunc: dL/dY = (c_ky / N^2) sum_{x,y} g e^{-i theta}."""
    N = g.shape[-1]
    kx, ky = mode_indices(N, m)
    c = np.where(ky == 0, 1.0, 2.0)
    return dft_trunc(g, m) * c / (N * N)


def gelu(z):
    from scipy.special import erf
    return 0.5 * z * (1.0 + erf(z / SQRT2))


def gelu_grad(z):
    from scipy.special import erf
    return 0.5 * (1.0 + erf(z / SQRT2)) + z * np.exp(-0.5 * z * z) / math.sqrt(2.0 * math.pi)


def pointwise(Wt, b, x):
    """[O, C] weights, [O] bias, x [B, C, N, N] -> [B, O, N, N]."""
    return np.einsum("oc,bcxy->boxy", Wt, x) + b[None, :, None, None]


def init_params(rng, c_in, width, m, layers, hidden):
    """Random initial weights (scaled so activations stay O(1))."""
    P = {}
    P["P_w"] = rng.standard_normal((width, c_in)) / math.sqrt(c_in)
    P["P_b"] = np.zeros(width)
    scale = 1.0 / (width * width)
    P["R_re"] = scale * rng.random((layers, width, width, 2 * m, m))
    P["R_im"] = scale * rng.random((layers, width, width, 2 * m, m))
    P["W_w"] = rng.standard_normal((layers, width, width)) / math.sqrt(width)
    P["W_b"] = np.zeros((layers, width))
    P["Q1_w"] = rng.standard_normal((hidden, width)) / math.sqrt(width)
    P["Q1_b"] = np.zeros(hidden)
    P["Q2_w"] = rng.standard_normal((1, hidden)) / math.sqrt(hidden)
    P["Q2_b"] = np.zeros(1)
    return P


def forward(P, x, m):
    """Returns (out [B, N, N], cache for backward)."""
    N = x.shape[-1]
    L = P["R_re"].shape[0]
    cache = {"x": x}
    v = pointwise(P["P_w"], P["P_b"], x)
    cache["v"] = [v]
    cache["z"] = []
    cache["Xh"] = []
    for l in range(L):
        Xh = dft_trunc(v, m)                                             # [B, W, 2m, m]
        R = P["R_re"][l] + 1j * P["R_im"][l]                             # [Wi, Wo, 2m, m]
        Yh = np.einsum("niac,ioac->noac", Xh, R)
        z = idft_trunc(Yh, N) + pointwise(P["W_w"][l], P["W_b"][l], v)
        cache["Xh"].append(Xh)
        cache["z"].append(z)
        v = gelu(z) if l < L - 1 else z
        cache["v"].append(v)
    a = pointwise(P["Q1_w"], P["Q1_b"], v)
    h = gelu(a)
    out = pointwise(P["Q2_w"], P["Q2_b"], h)[:, 0]
    cache["a"] = a
    cache["h"] = h
    return out, cache


def loss(out, target):
    return float(np.mean((out - target) ** 2))


def backward(P, cache, out, target, m):
    """Gradients of loss(out, target) with respect to every parameter."""
    x = cache["x"]
    N = x.shape[-1]
    L = P["R_re"].shape[0]
    G = {k: np.zeros_like(v) for k, v in P.items()}
    d_out = 2.0 * (out - target) / out.size                               # [B, N, N]
    d_out4 = d_out[:, None]
    h, a = cache["h"], cache["a"]
    G["Q2_w"] = np.einsum("boxy,bcxy->oc", d_out4, h)
    G["Q2_b"] = d_out4.sum(axis=(0, 2, 3))
    d_h = np.einsum("oc,boxy->bcxy", P["Q2_w"], d_out4)
    d_a = d_h * gelu_grad(a)
    v = cache["v"][L]
    G["Q1_w"] = np.einsum("boxy,bcxy->oc", d_a, v)
    G["Q1_b"] = d_a.sum(axis=(0, 2, 3))
    d_v = np.einsum("oc,boxy->bcxy", P["Q1_w"], d_a)
    for l in range(L - 1, -1, -1):
        z = cache["z"][l]
        d_z = d_v * gelu_grad(z) if l < L - 1 else d_v
        v_in = cache["v"][l]
        Xh = cache["Xh"][l]
        # pointwise branch
        G["W_w"][l] = np.einsum("boxy,bcxy->oc", d_z, v_in)
        G["W_b"][l] = d_z.sum(axis=(0, 2, 3))
        d_vin = np.einsum("oc,boxy->bcxy", P["W_w"][l], d_z)
        # spectral branch: z += idft(sum_i R[i,o] Xh[i])
        d_Yh = idft_trunc_adjoint(d_z, m)                                 # [B, Wo, 2m, m]
        R = P["R_re"][l] + 1j * P["R_im"][l]
        d_R = np.einsum("niac,noac->ioac", np.conj(Xh), d_Yh)
        G["R_re"][l] = d_R.real
        G["R_im"][l] = d_R.imag
        d_Xh = np.einsum("ioac,noac->niac", np.conj(R), d_Yh)
        d_vin = d_vin + dft_trunc_adjoint(d_Xh, N)
        d_v = d_vin
    G["P_w"] = np.einsum("boxy,bcxy->oc", d_v, x)
    G["P_b"] = d_v.sum(axis=(0, 2, 3))
    return G
