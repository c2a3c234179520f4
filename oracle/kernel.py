"""Surface compliance of an elastic layer on an elastic half-space, in Fourier space.

Test infrastructure (see ``oracle/__init__``).  Plain FP64 numpy.

* ``khat_homogeneous``   Eq. (4): u_z/p0 = 2/(E* |k|), E* = E/(1 - nu^2).
* ``coefficients``       Eq. (10): the constants A, B, C, D, written literally.
* ``coefficients_normalised``  the same four constants divided by the common
  factor (E2(1+nu1) + E1(1+nu2))^2, which cancels in Eq. (9); finite for E2 = inf.
* ``khat_layered``       Eq. (9)/(11): the factor multiplying FFT(p).
* ``khat_dc``            the k -> 0 finite part used for the zero wave number (the
  paper's Eq. (11) is defined for k != 0 only, so the value at k = 0 is a reading:
  the finite part lim_{k->0} [K^(k) - 2/(E2* k)]).
* ``lam_rigid``          Eq. (25): Lambda(u), L = 4 nu - 3.
* ``khat_multilayer``     the same transfer-matrix solve for a stack of layers on a
  substrate (the multi-layer generalisation of Eqs. 9/10); ``khat_multilayer_mp``
  the same in mpmath arithmetic, and ``khat_multilayer_dc`` its k -> 0 finite part
  by Richardson extrapolation in that arithmetic.
* ``khat_transfer_matrix``  an independent derivation: Eq. (5) written as a
  first-order system in (u_k, u_z, sigma_kz, sigma_zz), propagated through the layer
  by a matrix exponential, with the decaying invariant subspace of the half-space
  and boundary conditions (a)-(d) of Sec. 2.  It shares nothing with Eq. (9) and
  is only used to pin it.

Sign convention (Sec. 2, condition (c)): sigma_zz(z=0) = -p0, z points into the
body, u_z > 0 is a displacement into the body, so the compliance is positive.
"""
import numpy as np
import scipy.linalg


def e_star(E, nu):
    """Reduced modulus E* = E / (1 - nu^2) (Sec. 2, after Eq. 4)."""
    return E / (1.0 - nu * nu)


def e_tilde(E, nu):
    """Thin-layer modulus of Eq. (15): E(1-nu)/((1+nu)(1-2nu))."""
    return E * (1.0 - nu) / ((1.0 + nu) * (1.0 - 2.0 * nu))


def khat_homogeneous(k, E, nu):
    """Eq. (4): surface compliance of a homogeneous half-space, 2/(E* k)."""
    return 2.0 / (e_star(E, nu) * np.asarray(k, dtype=np.float64))


def coefficients(E1, nu1, E2, nu2):
    """Eq. (10), typed in literally (finite E2 only)."""
    A = (E2 * (3 - 4 * nu1) * (1 + nu1) - E1 * (3 - 4 * nu2) * (1 + nu2)) * (
        E1 * (1 + nu2) - E2 * (1 + nu1))
    B = 4 * (E2 * (1 + nu1) + E1 * (3 - 4 * nu2) * (1 + nu2)) * (
        E1 * (1 + nu2) - E2 * (1 + nu1))
    C = (E1 ** 2 * (4 * nu2 - 3) * (nu2 + 1) ** 2
         - 2 * E1 * E2 * (nu1 + 1) * (2 * nu1 - 1) * (nu2 + 1) * (2 * nu2 - 1)
         + E2 ** 2 * (8 * nu1 ** 2 - 12 * nu1 + 5) * (nu1 + 1) ** 2)
    D = (E2 * (1 + nu1) + E1 * (3 - 4 * nu2) * (1 + nu2)) * (
        E2 * (3 - 4 * nu1) * (1 + nu1) + E1 * (1 + nu2))
    return A, B, C, D


def coefficients_normalised(E1, nu1, E2, nu2):
    """Eq. (10) divided by (E2(1+nu1) + E1(1+nu2))^2.

    With a = E2(1+nu1), b = E1(1+nu2) every constant of Eq. (10) is a quadratic
    form in (a, b); dividing by (a+b)^2 leaves forms in alpha = a/(a+b) and
    beta = b/(a+b).  E2 = inf gives alpha = 1, beta = 0, i.e. A = L, B = -4,
    C = (L^2+1)/2, D = -L with L = 4 nu1 - 3 (the rigid-base case of Eq. 25).
    """
    if np.isinf(E2):
        alpha, beta = 1.0, 0.0
    else:
        a = E2 * (1 + nu1)
        b = E1 * (1 + nu2)
        alpha, beta = a / (a + b), b / (a + b)
    A = ((3 - 4 * nu1) * alpha - (3 - 4 * nu2) * beta) * (beta - alpha)
    B = 4 * (alpha + (3 - 4 * nu2) * beta) * (beta - alpha)
    C = ((4 * nu2 - 3) * beta ** 2
         - 2 * (2 * nu1 - 1) * (2 * nu2 - 1) * alpha * beta
         + (8 * nu1 ** 2 - 12 * nu1 + 5) * alpha ** 2)
    D = (alpha + (3 - 4 * nu2) * beta) * ((3 - 4 * nu1) * alpha + beta)
    return A, B, C, D


def khat_layered(k, h, E1, nu1, E2, nu2):
    """Eq. (9) / (11): u_z(k)/p0 for the coated half-space, k > 0 (array ok).

    Written as in the paper: 2(1-nu1^2)/E1 * (A e^{-4kh} + B kh e^{-2kh} + D) /
    (k (-A e^{-4kh} - B k^2h^2 e^{-2kh} + 2C e^{-2kh} + D)), with the constants of
    Eq. (10) in their normalised form (the common factor cancels).
    """
    k = np.asarray(k, dtype=np.float64)
    A, B, C, D = coefficients_normalised(E1, nu1, E2, nu2)
    x = k * h
    e2 = np.exp(-2.0 * x)
    e4 = np.exp(-4.0 * x)
    num = A * e4 + B * x * e2 + D
    den = -A * e4 - B * x * x * e2 + 2.0 * C * e2 + D
    return 2.0 * (1.0 - nu1 * nu1) / E1 * num / (k * den)


def khat_dc(h, E1, nu1, E2, nu2):
    """Finite part of Eq. (9) at k = 0: lim_{k->0} [K(k) - 2/(E2* k)].

    Eq. (9) is k K(k) = c F(kh) with F(x) = N(x)/Den(x) and c = 2(1-nu1^2)/E1.
    F(0) c = 2/E2* (the substrate alone governs long waves), so the finite part is
    c h F'(0), with N'(0) = B - 4A and Den'(0) = 4A - 4C (the x^2 term has zero
    slope).  For E2 = inf this is h/E~1 (Eqs. 14/15); for E1 = E2 it is 0.
    """
    A, B, C, D = coefficients_normalised(E1, nu1, E2, nu2)
    n0 = A + D
    d0 = -A + 2.0 * C + D
    dn = B - 4.0 * A
    dd = 4.0 * A - 4.0 * C
    c = 2.0 * (1.0 - nu1 * nu1) / E1
    return c * h * (dn * d0 - n0 * dd) / (d0 * d0)


def lam_rigid(u, nu):
    """Eq. (25): Lambda(u) with L = 4 nu - 3."""
    u = np.asarray(u, dtype=np.float64)
    L = 4.0 * nu - 3.0
    num = 2.0 * L * np.exp(-4.0 * u) - (L * L + 1.0 + 4.0 * u + 4.0 * u * u) * np.exp(-2.0 * u)
    den = L - (L * L + 1.0 + 4.0 * u * u) * np.exp(-2.0 * u) + L * np.exp(-4.0 * u)
    return num / den


def _lame(E, nu):
    lam = E * nu / ((1.0 + nu) * (1.0 - 2.0 * nu))
    mu = E / (2.0 * (1.0 + nu))
    return lam, mu


def _navier_matrix(k, E, nu):
    """Eq. (5) for u = (u_k(z), u_z(z)) e^{ikx} as s' = A s, s = (u_k, u_z, s_kz, s_zz).

    Hooke's law: s_kz = mu (u_k' + i k u_z), s_zz = lam i k u_k + (lam+2mu) u_z',
    s_kk = (lam+2mu) i k u_k + lam u_z'.  Equilibrium: i k s_kk + s_kz' = 0 and
    i k s_kz + s_zz' = 0.  Solving these for the z-derivatives gives A.
    """
    lam, mu = _lame(E, nu)
    ik = 1j * k
    M = np.zeros((4, 4), dtype=np.complex128)
    # u_k' = s_kz/mu - ik u_z
    M[0, 1] = -ik
    M[0, 2] = 1.0 / mu
    # u_z' = (s_zz - lam ik u_k)/(lam+2mu)
    M[1, 0] = -lam * ik / (lam + 2 * mu)
    M[1, 3] = 1.0 / (lam + 2 * mu)
    # s_kz' = -ik s_kk = -ik[(lam+2mu) ik u_k + lam u_z']
    M[2, :] = -ik * lam * M[1, :]
    M[2, 0] += k * k * (lam + 2 * mu)
    # s_zz' = -ik s_kz
    M[3, 2] = -ik
    return M


def khat_transfer_matrix(k, h, E1, nu1, E2, nu2):
    """Independent pin of Eq. (9): u_z(0)/p0 from Eq. (5) and conditions (a)-(d).

    (d) the half-space state at z = h lies in the decaying invariant subspace of its
    system matrix (ordered Schur form, left half-plane); (a) displacements and
    tractions are continuous at z = h; the layer carries the state from z = h to
    z = 0 by expm(-A1 h); (b) s_kz(0) = 0; (c) s_zz(0) = -p0 with p0 = 1.
    Scalar k > 0 and finite E2 only; moderate k h (the exponential grows like e^{kh}).
    """
    A1 = _navier_matrix(k, E1, nu1)
    A2 = _navier_matrix(k, E2, nu2)
    T, Z, sdim = scipy.linalg.schur(A2, output="complex", sort="lhp")
    assert sdim == 2, "half-space must have a two-dimensional decaying subspace"
    Q = Z[:, :2]                        # state at z = h = Q c
    P = scipy.linalg.expm(-A1 * h)      # state at z = 0 = P Q c
    S0 = P @ Q
    rhs = np.array([0.0, -1.0], dtype=np.complex128)   # (b) s_kz = 0, (c) s_zz = -1
    c = np.linalg.solve(S0[2:4, :], rhs)
    uz0 = (S0 @ c)[1]
    return float(uz0.real)


def khat_multilayer(k, layers, E_sub, nu_sub):
    """Surface compliance u_z(0)/p0 of a stack of bonded layers on a substrate, by the
    same transfer-matrix solve of Eq. (5) as ``khat_transfer_matrix`` (the multi-layer
    generalisation of Eqs. 9/10, which the paper gives for one layer).

    ``layers`` lists (thickness, E, nu) from the surface down.  At the bottom of the
    stack the state lies in the decaying invariant subspace of the substrate's system
    matrix (finite E_sub), or has zero displacements (E_sub = inf: a rigid base, the
    tractions free); every layer carries the state from its bottom to its top by
    expm(-A h), which keeps displacements and tractions continuous at each interface
    (condition (a) at every interface); at z = 0 s_kz = 0 and s_zz = -1 (conditions
    (b), (c)).  Scalar k > 0; moderate k times the total thickness.
    """
    if np.isinf(E_sub):
        Q = np.zeros((4, 2), dtype=np.complex128)
        Q[2, 0] = 1.0
        Q[3, 1] = 1.0
    else:
        A = _navier_matrix(k, E_sub, nu_sub)
        T, Z, sdim = scipy.linalg.schur(A, output="complex", sort="lhp")
        assert sdim == 2, "substrate must have a two-dimensional decaying subspace"
        Q = Z[:, :2]
    S = Q
    for h, E, nu in reversed(list(layers)):
        if h > 0.0:
            S = scipy.linalg.expm(-_navier_matrix(k, E, nu) * h) @ S
    c = np.linalg.solve(S[2:4, :], np.array([0.0, -1.0], dtype=np.complex128))
    return float((S @ c)[1].real)


def _navier_matrix_mp(k, E, nu):
    """``_navier_matrix`` in mpmath arithmetic (same first-order system of Eq. 5)."""
    import mpmath as mp
    E, nu, k = mp.mpf(E), mp.mpf(nu), mp.mpf(k)
    lam = E * nu / ((1 + nu) * (1 - 2 * nu))
    mu = E / (2 * (1 + nu))
    ik = mp.mpc(0, 1) * k
    M = mp.zeros(4, 4)
    M[0, 1] = -ik
    M[0, 2] = 1 / mu
    M[1, 0] = -lam * ik / (lam + 2 * mu)
    M[1, 3] = 1 / (lam + 2 * mu)
    for j in range(4):
        M[2, j] = -ik * lam * M[1, j]
    M[2, 0] += k * k * (lam + 2 * mu)
    M[3, 2] = -ik
    return M


def khat_multilayer_mp(k, layers, E_sub, nu_sub, dps=50):
    """``khat_multilayer`` evaluated in mpmath with ``dps`` digits, for the long-wave
    limit below.  The substrate's decaying subspace is found without a Schur form:
    its system matrix A has the eigenvalues +k and -k, each twice (one Jordan block
    each), so (A - k I)^2 vanishes on the growing pair and maps the whole space onto
    the decaying pair; two fixed generic combinations of its columns span it."""
    import mpmath as mp
    with mp.workdps(dps):
        k = mp.mpf(k)
        if np.isinf(E_sub):
            S = mp.zeros(4, 2)
            S[2, 0] = 1
            S[3, 1] = 1
        else:
            A = _navier_matrix_mp(k, E_sub, nu_sub)
            B = A - k * mp.eye(4)
            R = mp.matrix([[1, 0.37], [0.29, 1], [-0.53, 0.61], [0.71, -0.43]])
            S = (B * B) * R
        for h, E, nu in reversed(list(layers)):
            if h > 0.0:
                S = mp.expm(-_navier_matrix_mp(k, E, nu) * mp.mpf(h)) * S
        T = mp.matrix([[S[2, 0], S[2, 1]], [S[3, 0], S[3, 1]]])
        c = mp.lu_solve(T, mp.matrix([0, -1]))
        uz = S[1, 0] * c[0] + S[1, 1] * c[1]
        return mp.re(uz)


def khat_multilayer_dc(layers, E_sub, nu_sub, levels=5, dps=50):
    """Finite part lim_{k->0} [K(k) - 2/(E_sub* k)] of the stack's compliance (the
    same k = 0 reading as ``khat_dc``; 2/(E_sub* k) is absent for a rigid base).
    phi(k) = k K(k) = phi(0) + phi'(0) k + ..., and the finite part is phi'(0),
    taken by Richardson extrapolation of (phi(k) - phi(0))/k over k = k0/2^i with
    k0 times the stack's thickness 1e-6, in ``dps``-digit arithmetic so that the
    difference keeps its digits."""
    import mpmath as mp
    H = sum(h for h, _, _ in layers)
    with mp.workdps(dps):
        phi0 = mp.mpf(0) if np.isinf(E_sub) else 2 * (1 - mp.mpf(nu_sub) ** 2) / mp.mpf(E_sub)
        k0 = mp.mpf("1e-6") / mp.mpf(H)
        T = []
        for i in range(levels):
            kk = k0 / 2 ** i
            T.append([(kk * khat_multilayer_mp(kk, layers, E_sub, nu_sub, dps) - phi0) / kk])
        for j in range(1, levels):
            for i in range(j, levels):
                T[i].append((2 ** j * T[i][j - 1] - T[i - 1][j - 1]) / (2 ** j - 1))
        return float(T[-1][-1])
