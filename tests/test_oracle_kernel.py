"""Pins of the oracle's Fourier-space compliance (Eqs. 4, 9, 10, 14, 15, 25).

None of these retypes Eq. (9): each compares it with something fixed independently
(Eq. 4, the h -> 0 / h -> inf limits, the rigid-base form of Eq. 25, Eq. 15, an
independent transfer-matrix solve of Eq. 5 with conditions (a)-(d), Richardson
extrapolation of the DC limit).
"""
import numpy as np
import pytest

from oracle import kernel as K
from oracle import kernel

PARAMS = [  # (h, E1, nu1, E2, nu2)
    (1.0, 4.0, 0.3, 1.0, 0.3),
    (0.5, 0.2, 0.3, 1.0, 0.45),
    (2.0, 1.0, 0.25, 7.0, 0.4),
    (0.3, 3.0, 0.49, 0.05, 0.2),
    (0.01, 20.0, 0.2, 1.0, 0.49),
]


@pytest.mark.parametrize("E,nu", [(1.0, 0.3), (210e9, 0.29), (3.0, 0.45)])
@pytest.mark.parametrize("h", [1e-3, 0.5, 7.0])
def test_homogeneous_reduces_to_eq4(E, nu, h):
    k = np.geomspace(1e-3, 1e3, 41) / h
    a = K.khat_layered(k, h, E, nu, E, nu)
    b = K.khat_homogeneous(k, E, nu)
    np.testing.assert_allclose(a, b, rtol=1e-13)
    A, B, C, D = K.coefficients_normalised(E, nu, E, nu)
    assert abs(A) < 1e-15 and abs(B) < 1e-15 and abs(C) < 1e-15 and D > 0


@pytest.mark.parametrize("p", PARAMS)
def test_limits_h_to_zero_and_infinity(p):
    _, E1, nu1, E2, nu2 = p
    k = np.geomspace(1e-2, 1e2, 9)
    np.testing.assert_allclose(K.khat_layered(k, 1e-12, E1, nu1, E2, nu2),
                               K.khat_homogeneous(k, E2, nu2), rtol=1e-7)
    np.testing.assert_allclose(K.khat_layered(k, 1e4, E1, nu1, E2, nu2),
                               K.khat_homogeneous(k, E1, nu1), rtol=1e-14)


@pytest.mark.parametrize("nu1", [0.2, 0.3, 0.45])
def test_rigid_base_matches_eq25(nu1):
    h, E1 = 0.7, 3.0
    k = np.geomspace(1e-2, 30.0, 50) / h
    a = K.khat_layered(k, h, E1, nu1, np.inf, 0.3)
    b = 2.0 * (1.0 - K.lam_rigid(k * h, nu1)) / (K.e_star(E1, nu1) * k)
    np.testing.assert_allclose(a, b, rtol=1e-10)
    # E2 = e^100 (the paper's stand-in for a rigid base) agrees with E2 = inf
    np.testing.assert_allclose(K.khat_layered(k, h, E1, nu1, np.exp(100.0), 0.3), a, rtol=1e-13)


def test_normalised_equals_literal_eq10():
    for h, E1, nu1, E2, nu2 in PARAMS:
        A, B, C, D = K.coefficients(E1, nu1, E2, nu2)
        s = (E2 * (1 + nu1) + E1 * (1 + nu2)) ** 2
        np.testing.assert_allclose(np.array([A, B, C, D]) / s,
                                   K.coefficients_normalised(E1, nu1, E2, nu2), rtol=1e-13, atol=1e-15)


@pytest.mark.parametrize("p", PARAMS)
def test_independent_transfer_matrix(p):
    h, E1, nu1, E2, nu2 = p
    for k in [0.05 / h, 0.3 / h, 1.0 / h, 3.0 / h]:
        a = K.khat_layered(k, h, E1, nu1, E2, nu2)
        b = K.khat_transfer_matrix(k, h, E1, nu1, E2, nu2)
        assert abs(a - b) <= 1e-11 * abs(b), (k, a, b)


def test_dc_finite_part():
    # rigid base: K(0+) = h / E~1 (Eqs. 14, 15)
    for nu1 in [0.2, 0.3, 0.45]:
        assert K.khat_dc(0.37, 2.0, nu1, np.inf, 0.3) == pytest.approx(0.37 / K.e_tilde(2.0, nu1), rel=1e-14)
        ks = np.array([1e-4, 1e-5])
        np.testing.assert_allclose(K.khat_layered(ks, 0.37, 2.0, nu1, np.inf, 0.3),
                                   0.37 / K.e_tilde(2.0, nu1), rtol=1e-3)
    # homogeneous: the finite part vanishes (the paper's literal rule)
    assert abs(K.khat_dc(1.0, 1.0, 0.3, 1.0, 0.3)) < 1e-15
    # finite E2: Richardson extrapolation of K(k) - 2/(E2* k) as k -> 0
    for h, E1, nu1, E2, nu2 in PARAMS:
        k = np.array([4e-5, 2e-5, 1e-5]) / h
        v = K.khat_layered(k, h, E1, nu1, E2, nu2) - K.khat_homogeneous(k, E2, nu2)
        r1 = 2 * v[1] - v[0]
        r2 = 2 * v[2] - v[1]
        extrap = (4 * r2 - r1) / 3
        c0 = K.khat_dc(h, E1, nu1, E2, nu2)
        assert abs(extrap - c0) <= 1e-5 * max(abs(c0), h / E1), (extrap, c0)


def test_positive_operator_scan():
    rng = np.random.default_rng(5)
    for _ in range(200):
        h = 10 ** rng.uniform(-3, 3)
        E1 = 10 ** rng.uniform(np.log10(0.05), np.log10(20))
        nu1, nu2 = rng.uniform(0.2, 0.49, 2)
        k = np.geomspace(1e-3, 1e3, 61) / h
        v = K.khat_layered(k, h, E1, nu1, 1.0, nu2)
        assert np.all(v > 0) and np.all(np.isfinite(v))


# ---- multi-layer stacks (the transfer-matrix generalisation of Eqs. 9/10) --------

@pytest.mark.parametrize("kh", [0.05, 0.7, 3.0])
def test_multilayer_one_layer_is_eq9(kh):
    h, E1, nu1, E2, nu2 = 0.2, 3.0, 0.3, 1.0, 0.45
    k = kh / h
    ref = K.khat_layered(np.array([k]), h, E1, nu1, E2, nu2)[0]
    assert K.khat_multilayer(k, [(h, E1, nu1)], E2, nu2) == pytest.approx(ref, rel=1e-11)


@pytest.mark.parametrize("kh", [0.1, 1.0, 4.0])
def test_multilayer_rigid_base_is_eq25(kh):
    """One layer on a rigid base: 2 (1 - Lambda(kh)) / (E1* k), Lambda of Eq. (25)."""
    h, E1, nu1 = 0.3, 2.0, 0.35
    k = kh / h
    ref = 2.0 * (1.0 - K.lam_rigid(kh, nu1)) / (K.e_star(E1, nu1) * k)
    assert K.khat_multilayer(k, [(h, E1, nu1)], np.inf, 0.3) == pytest.approx(ref, rel=1e-10)


def test_multilayer_split_layer_and_homogeneous_stack():
    k = 2.5
    one = K.khat_multilayer(k, [(0.5, 3.0, 0.3)], 1.0, 0.4)
    split = K.khat_multilayer(k, [(0.2, 3.0, 0.3), (0.3, 3.0, 0.3), (0.0, 9.0, 0.2)], 1.0, 0.4)
    assert split == pytest.approx(one, rel=1e-12)
    same = K.khat_multilayer(k, [(0.1, 2.0, 0.3), (0.4, 2.0, 0.3)], 2.0, 0.3)
    assert same == pytest.approx(K.khat_homogeneous(k, 2.0, 0.3), rel=1e-12)


def test_multilayer_limits_and_ordering():
    """High wave numbers see only the top layer (2/(E_top* k)); low ones the substrate
    (2/(E_sub* k)); a stiff top layer over a soft one is stiffer than the reverse."""
    layers = [(0.05, 5.0, 0.3), (0.1, 0.5, 0.25)]
    k_hi = 40.0 / 0.05
    assert K.khat_multilayer(k_hi, layers, 1.0, 0.3) == pytest.approx(
        K.khat_homogeneous(k_hi, 5.0, 0.3), rel=1e-9)
    k_lo = 1e-4
    assert K.khat_multilayer(k_lo, layers, 1.0, 0.3) == pytest.approx(
        K.khat_homogeneous(k_lo, 1.0, 0.3), rel=1e-3)
    k = 10.0
    stiff_top = K.khat_multilayer(k, layers, 1.0, 0.3)
    soft_top = K.khat_multilayer(k, layers[::-1], 1.0, 0.3)
    assert stiff_top < soft_top


@pytest.mark.parametrize("stack", [(0.35, 3.0, 0.3, 1.0, 0.45), (0.8, 0.2, 0.45, 1.0, 0.3), (0.35, 1.0, 0.3, np.inf, 0.3)])
def test_multilayer_dc_one_layer_is_eq9_finite_part(stack):
    """The stack's long-wave finite part (Richardson extrapolation in mpmath) reduces,
    for one layer, to the closed-form finite part of Eq. (9)."""
    h, E1, nu1, E2, nu2 = stack
    assert kernel.khat_multilayer_dc([(h, E1, nu1)], E2, nu2) == pytest.approx(
        kernel.khat_dc(h, E1, nu1, E2, nu2), rel=1e-12, abs=1e-15)


def test_multilayer_dc_rigid_base_is_uniaxial_compression():
    """On a rigid base a uniform pressure compresses each layer in uniaxial strain
    (no lateral expansion over an infinite wavelength): K(0) = sum h_j / E~_j, the
    thin-layer modulus of Eq. (15) per layer."""
    layers = [(0.1, 0.8, 0.25), (0.15, 4.0, 0.35), (0.3, 1.5, 0.3)]
    ref = sum(h / kernel.e_tilde(E, nu) for h, E, nu in layers)
    assert kernel.khat_multilayer_dc(layers, np.inf, 0.3) == pytest.approx(ref, rel=1e-13)


def test_multilayer_dc_split_and_substrate_layer():
    """Splitting a layer in two of the same material, or adding a layer of the
    substrate's own material below the stack, leaves the finite part unchanged."""
    base = kernel.khat_multilayer_dc([(0.2, 3.0, 0.3), (0.5, 0.5, 0.4)], 1.0, 0.45)
    split = kernel.khat_multilayer_dc([(0.2, 3.0, 0.3), (0.2, 0.5, 0.4), (0.3, 0.5, 0.4)], 1.0, 0.45)
    below = kernel.khat_multilayer_dc([(0.2, 3.0, 0.3), (0.5, 0.5, 0.4), (0.4, 1.0, 0.45)], 1.0, 0.45)
    assert split == pytest.approx(base, rel=1e-12)
    assert below == pytest.approx(base, rel=1e-12)
    # a stack of the substrate's material is the homogeneous half-space: finite part 0
    assert abs(kernel.khat_multilayer_dc([(0.3, 1.0, 0.45)], 1.0, 0.45)) < 1e-13


def test_multilayer_mp_matches_double():
    layers = [(0.2, 3.0, 0.3), (0.5, 0.5, 0.4)]
    for k in (0.05, 0.7, 9.0):
        for Es in (1.0, np.inf):
            assert float(kernel.khat_multilayer_mp(k, layers, Es, 0.45)) == pytest.approx(
                kernel.khat_multilayer(k, layers, Es, 0.45), rel=1e-12)


def test_multilayer_grid_one_layer_equals_eq9_grid():
    from oracle import operator
    N, d = 8, 0.1
    a = operator.khat_grid_layers(N, d, [(0.35, 3.0, 0.3)], 1.0, 0.45)
    b = operator.khat_grid(N, d, 0.35, 3.0, 0.3, 1.0, 0.45)
    np.testing.assert_allclose(a, b, rtol=1e-12)


def test_multilayer_golden_file_is_current():
    """tests/golden/multilayer_dc.json (read by the GPU tests, whose box has no mpmath)
    holds what the oracle computes now."""
    import json
    import os
    import sys
    here = os.path.join(os.path.dirname(os.path.abspath(__file__)), "golden")
    sys.path.insert(0, here)
    import make_multilayer_dc
    stored = json.load(open(os.path.join(here, "multilayer_dc.json")))
    for name, (layers, Es, nus) in make_multilayer_dc.STACKS.items():
        assert stored[name]["dc"] == pytest.approx(kernel.khat_multilayer_dc(layers, Es, nus), rel=1e-13), name
