"""The flat-punch stiffness sweep on the GPU: a rigid cylindrical punch of radius a on
a coating (L = 4a, N = 256, a = 64 cells, nu1 = 0.3, nu2 = 0.45), h/a in
{0.1, 0.3, 1, 3, 10} x E1/E2 in {0.1, 0.5, 2, 10}, under depth control, in FP64 and
FP32, with the literal k = 0 rule (dc_mode 1; the finite part makes the stiff thick
coating indefinite on the punch, see the indefinite-operator test).

Checks: the FP32 stiffness equals the FP64 one to the force tolerance of the float
path; two cells equal the oracle's solve; every normalised stiffness lies between
the substrate's and the coating's Boussinesq values 2aE2* and 2aE1* (classical flat
punch, Eq. 4 in real space), moves monotonically towards the coating's as h/a grows
and reaches it within 1 % at h/a = 10 (Eq. 14 context, Sec. 3)."""
import numpy as np
import pytest
import torch

from oracle import analytic, contact, kernel, operator
from paper_1807_01885_gb300 import bem, inputs

pytestmark = pytest.mark.gpu

N, DELTA, A = 256, 1.0, 64.0
E2, NU1, NU2 = 1.0, 0.3, 0.45
D = 1e-3 * A
HOA = (0.1, 0.3, 1.0, 3.0, 10.0)
RATIOS = (0.1, 0.5, 2.0, 10.0)


def gpu_stiffness(f_dev, h, E1, nu1, Es, nus, precision):
    with bem.Kernel(N, DELTA, h, E1, nu1, Es, nus, precision=precision, dc_mode=bem.BEM_DC_ZERO) as k:
        _, res = k.solve(f_dev, "depth", D, tol=1e-12 if precision == "fp64" else 1e-8)
    assert res["status"] == 0, res
    return res["force"] / D, res


@pytest.fixture(scope="module")
def sweep(cuda):
    f = inputs.flat_punch_height(N, DELTA, A)
    out = {}
    for precision, dt in (("fp64", torch.float64), ("fp32", torch.float32)):
        fd = torch.tensor(f, device=cuda, dtype=dt)
        k_hom, _ = gpu_stiffness(fd, np.inf, 1.0, 0.3, 1.0, 0.3, precision)
        out[(precision, "hom")] = k_hom
        for r in RATIOS:
            for hoa in HOA:
                out[(precision, r, hoa)] = gpu_stiffness(fd, hoa * A, r * E2, NU1, E2, NU2, precision)[0]
    return f, out


def test_fp32_stiffness_equals_fp64(sweep):
    _, s = sweep
    assert s[("fp32", "hom")] == pytest.approx(s[("fp64", "hom")], rel=1e-5)
    for r in RATIOS:
        for hoa in HOA:
            assert s[("fp32", r, hoa)] == pytest.approx(s[("fp64", r, hoa)], rel=1e-5), (r, hoa)


@pytest.mark.parametrize("r,hoa", [(10.0, 3.0), (0.1, 0.3)])
def test_sweep_cells_equal_oracle(sweep, r, hoa):
    f, s = sweep
    Kg = operator.khat_grid(N, DELTA, hoa * A, r * E2, NU1, E2, NU2, dc_mode=1)
    ref = contact.solve_nonadhesive(lambda p: operator.matvec_fft(Kg, p), f, DELTA, "depth", D, tol=1e-12)
    assert s[("fp64", r, hoa)] == pytest.approx(ref["force"] / D, rel=1e-10)


def test_sweep_bracketed_and_monotone(sweep):
    _, s = sweep
    k_hom = s[("fp64", "hom")] / analytic.flat_punch_stiffness(A, kernel.e_star(1.0, 0.3))
    # the period's images and the zero-mean datum stiffen every punch on this grid alike
    assert 1.2 < k_hom < 1.6
    for precision in ("fp64", "fp32"):
        for r in RATIOS:
            lo, hi = sorted([1.0, kernel.e_star(r, NU1) / kernel.e_star(E2, NU2)])
            ks = [s[(precision, r, hoa)] / (k_hom * analytic.flat_punch_stiffness(A, kernel.e_star(E2, NU2)))
                  for hoa in HOA]
            assert all(lo * (1 - 1e-5) <= k <= hi * (1 + 1e-5) for k in ks), (precision, r, ks)
            steps = np.diff(ks)
            assert np.all(steps > 0) if r > 1 else np.all(steps < 0), (precision, r, ks)
            coat = kernel.e_star(r, NU1) / kernel.e_star(E2, NU2)
            assert ks[-1] == pytest.approx(coat, rel=0.01), (precision, r, ks)
