"""GPU parity of the open-plane (non-periodic) operator of a homogeneous half-space
(op_kind BEM_OP_OPEN) against the oracle's Love-cell convolution
(``oracle/influence.py``), through the C ABI: the compliance table (the transform
of the wrap-around coefficient array), the product in both precisions, and the
contact pins the oracle is held to (Hertz, Boussinesq's flat punch), which the
periodic product of Eq. (11) misses by its images and its k = 0 datum."""
import numpy as np
import pytest
import torch

from oracle import analytic, contact, dft, influence, kernel
from paper_1807_01885_gb300 import bem, inputs

pytestmark = pytest.mark.gpu


def rel(a, b):
    return np.linalg.norm(a - b) / max(np.linalg.norm(b), 1e-300)


def open_kernel(N, delta, E, nu, precision="fp64", h=np.inf, E2=None, nu2=None):
    return bem.Kernel(N, delta, h, E, nu, E if E2 is None else E2, nu if nu2 is None else nu2, precision=precision,
                      op_kind=bem.BEM_OP_OPEN)


def wrap(G, N):
    M = 2 * N
    W = np.zeros((M, M))
    idx = np.arange(-(N - 1), N) % M
    W[np.ix_(idx, idx)] = G
    return W


@pytest.mark.parametrize("N", [4, 16, 64])
def test_open_table_is_the_transform_of_the_cell_coefficients(cuda, N):
    delta, E, nu = 0.5, 2.0, 0.3
    G = influence.influence_love(N, delta, E, nu)
    S = dft.fft2(wrap(G, N))
    ref = S.real[: N + 1, : N + 1]
    with open_kernel(N, delta, E, nu) as k:
        got = k.table().cpu().numpy()
    np.testing.assert_allclose(got, ref, rtol=0, atol=1e-12 * np.abs(ref).max())


@pytest.mark.parametrize("N", [4, 8, 16, 64, 256])
def test_open_product_parity(cuda, N):
    delta, E, nu = 1.0 / N, 1.0, 0.25
    G = influence.influence_love(N, delta, E, nu)
    p = np.random.default_rng(N).standard_normal((N, N))
    ref = influence.matvec_dense_np(G, p) if N <= 16 else influence.matvec_fft_np(G, p)
    with open_kernel(N, delta, E, nu) as k:
        u = k.matvec(torch.tensor(p, device=cuda)).cpu().numpy()
    # The closed form of the cell coefficients is a sum of four terms of size about
    # L log(L/delta) whose result falls like delta^2 / r: at the far offsets both sides
    # (CUDA's and numpy's asinh) lose ~log10((L/delta)^2) digits to that cancellation,
    # which leaves ~1e-12 on the product at N = 256 besides the FFT's rounding.
    assert rel(u, ref) < 5e-12
    with open_kernel(N, delta, E, nu, "fp32") as k:
        u32 = k.matvec(torch.tensor(p, device=cuda, dtype=torch.float32)).double().cpu().numpy()
    assert rel(u32, ref) < 2e-6


def test_open_homogeneous_forms_agree(cuda):
    """h = INFINITY with (E1, nu1), h = 0 with (E2, nu2) and a coating of the
    substrate's own material give the same operator."""
    N, delta, E, nu = 16, 0.1, 3.0, 0.35
    tabs = []
    for h, E1, nu1, E2, nu2 in [(np.inf, E, nu, 1.0, 0.2), (0.0, 1.0, 0.2, E, nu), (0.4, E, nu, E, nu)]:
        with bem.Kernel(N, delta, h, E1, nu1, E2, nu2, op_kind=bem.BEM_OP_OPEN) as k:
            tabs.append(k.table().cpu().numpy())
    np.testing.assert_array_equal(tabs[0], tabs[1])
    np.testing.assert_array_equal(tabs[0], tabs[2])


def test_open_rejects_a_coating(cuda):
    with pytest.raises(bem.BemError) as e:
        bem.Kernel(16, 0.1, 0.3, 4.0, 0.3, 1.0, 0.3, op_kind=bem.BEM_OP_OPEN)
    assert e.value.status == bem.BEM_EUNSUPPORTED
    with pytest.raises(bem.BemError) as e:
        bem.Kernel(16, 0.1, layers=[(0.3, 4.0, 0.3)], E2=1.0, nu2=0.3, op_kind=bem.BEM_OP_OPEN)
    assert e.value.status == bem.BEM_EUNSUPPORTED


@pytest.mark.parametrize("precision,tol_p,tol_f", [("fp64", 1e-10, 1e-10), ("fp32", 2e-4, 1e-5)])
def test_open_hertz(cuda, precision, tol_p, tol_f):
    """Sphere under force control (N = 64, Hertz radius 16 cells): pressure and depth
    equal the oracle's open-plane solve, and radius, peak pressure and depth approach
    Hertz (a^3 = 3FR/4E*, p0 = 3F/(2 pi a^2), d = a^2/R) within the grid's 0.5 %; the
    periodic operator's depth is 20 % low here (the oracle pin)."""
    N, R, E, nu = 64, 1.0, 1.0, 0.3
    Es = kernel.e_star(E, nu)
    a_H, delta = 16.0 / N, 1.0 / N
    F = 4 * Es * a_H ** 3 / (3 * R)
    f = inputs.sphere_height(N, delta, R)
    G = influence.influence_love(N, delta, E, nu)
    ref = contact.solve_nonadhesive(lambda p: influence.matvec_fft_np(G, p), f, delta, "force", F, tol=1e-13)
    dt = torch.float64 if precision == "fp64" else torch.float32
    with open_kernel(N, delta, E, nu, precision) as k:
        p, res = k.solve(torch.tensor(f, device=cuda, dtype=dt), "force", F,
                         tol=1e-13 if precision == "fp64" else 1e-8)
    assert res["status"] == 0
    p = p.double().cpu().numpy()
    assert rel(p, ref["p"]) < tol_p
    assert res["depth"] == pytest.approx(ref["d"], rel=tol_f)
    d_H = a_H ** 2 / R
    assert res["depth"] / d_H == pytest.approx(1.0, abs=0.005)
    assert res["a_eq"] / a_H == pytest.approx(1.0, abs=0.01)
    assert p.max() / (3 * F / (2 * np.pi * a_H ** 2)) == pytest.approx(1.0, abs=0.005)


@pytest.mark.parametrize("N", [64, 256])
def test_open_flat_punch_stiffness(cuda, N):
    """Rigid flat punch of radius N/4 cells: F/d = 2 a E* (Boussinesq) within 0.5 %,
    in both precisions; the periodic product of the same window is 43 % stiffer."""
    delta, a, E, nu = 1.0, N / 4, 1.0, 0.3
    f = inputs.flat_punch_height(N, delta, a)
    d = 1e-3 * a
    k_B = analytic.flat_punch_stiffness(a, kernel.e_star(E, nu))
    for precision, dt in (("fp64", torch.float64), ("fp32", torch.float32)):
        with open_kernel(N, delta, E, nu, precision) as k:
            _, res = k.solve(torch.tensor(f, device=cuda, dtype=dt), "depth", d,
                             tol=1e-12 if precision == "fp64" else 1e-8)
        assert res["status"] == 0
        assert res["force"] / d / k_B == pytest.approx(1.0, abs=0.005), precision
