"""GPU parity of the coating-stack operator (bem_make_kernel_layers, the multi-layer
generalisation of Eqs. 9/10) against the oracle's transfer-matrix compliance
(``oracle.kernel.khat_multilayer``), through the C ABI: the table, the product in
both precisions and a contact solve.  The k = 0 finite parts come from
tests/golden/multilayer_dc.json (written by the oracle; the GPU machine has no mpmath)."""
import json
import math
import os

import numpy as np
import pytest
import torch

from oracle import contact, kernel, operator
from paper_1807_01885_gb300 import bem, inputs

pytestmark = pytest.mark.gpu

GOLDEN = json.load(open(os.path.join(os.path.dirname(os.path.abspath(__file__)), "golden", "multilayer_dc.json")))


def stack(name):
    g = GOLDEN[name]
    Es = math.inf if g["E_sub"] == "inf" else float(g["E_sub"])
    return [tuple(x) for x in g["layers"]], Es, float(g["nu_sub"]), float(g["dc"])


def rel(a, b):
    return np.linalg.norm(a - b) / max(np.linalg.norm(b), 1e-300)


@pytest.mark.parametrize("name", ["two_on_substrate", "three_on_rigid", "stiff_over_soft"])
@pytest.mark.parametrize("dc_mode", [0, 1])
def test_stack_table_parity(cuda, name, dc_mode):
    """Every entry of the (N+1)^2 table at N = 32 (k times the stack's thickness up
    to about 30) against the oracle's transfer-matrix solve, and the k = 0 entry
    against the oracle's long-wave finite part."""
    layers, Es, nus, dc = stack(name)
    N, delta = 32, 0.1
    with bem.Kernel(N, delta, layers=layers, E2=Es, nu2=nus, dc_mode=dc_mode) as k:
        got = k.table().cpu().numpy()
    ref = operator.khat_grid_layers(N, delta, layers, Es, nus, dc_mode=dc_mode, dc_value=dc)[: N + 1, : N + 1]
    np.testing.assert_allclose(got, ref, rtol=1e-12, atol=0)


def test_one_layer_stack_equals_single_coating(cuda):
    """A stack of one layer is the operator of Eq. (9): same table (to rounding) at
    N = 512, including the closed-form finite part, in both DC modes."""
    N, delta = 512, 1.0 / 512
    for dc_mode in (0, 1):
        for h, E1, nu1, E2, nu2 in [(0.05, 4.0, 0.3, 1.0, 0.45), (0.02, 0.5, 0.25, math.inf, 0.3)]:
            with bem.Kernel(N, delta, h, E1, nu1, E2, nu2, dc_mode=dc_mode) as k:
                a = k.table().cpu().numpy()
            with bem.Kernel(N, delta, layers=[(h, E1, nu1)], E2=E2, nu2=nu2, dc_mode=dc_mode) as k:
                b = k.table().cpu().numpy()
            # k != 0: the same formula evaluated two ways, to rounding
            a0, b0 = a[0, 0], b[0, 0]
            a[0, 0] = b[0, 0] = 1.0
            np.testing.assert_allclose(b, a, rtol=1e-13, atol=0)
            # k = 0: the closed-form finite part of Eq. (9) against the dual-number
            # derivative through the stack's solve (cancellation leaves ~1e-13)
            assert b0 == pytest.approx(a0, rel=1e-12, abs=1e-15 * abs(a).max())


def test_stack_table_large_grid_samples(cuda):
    """N = 1024 with a thick stack (k times the thickness up to about 4000, where the
    oracle's exponentials would overflow): sampled entries with k H <= 30 against the
    oracle, and the high-k entries against the top layer's homogeneous compliance
    2/(E1* k) (Eq. 4), which the stack reaches once the other layers are far below."""
    layers, Es, nus, dc = stack("two_on_substrate")
    N = 1024
    delta = 0.7 / 64
    with bem.Kernel(N, delta, layers=layers, E2=Es, nu2=nus) as k:
        got = k.table().cpu().numpy()
    assert got[0, 0] == pytest.approx(dc, rel=1e-12)
    H = sum(h for h, _, _ in layers)
    kstep = 2 * np.pi / (2 * N * delta)
    rng = np.random.default_rng(3)
    for _ in range(60):
        i, j = rng.integers(0, 60, size=2)
        if i == 0 and j == 0:
            continue
        kk = kstep * np.hypot(i, j)
        assert kk * H < 31
        assert got[i, j] == pytest.approx(kernel.khat_multilayer(kk, layers, Es, nus), rel=1e-12)
    E1, nu1 = layers[0][1], layers[0][2]
    for i, j in [(N, N), (N, 300), (700, 700)]:
        kk = kstep * np.hypot(i, j)
        assert got[i, j] == pytest.approx(kernel.khat_homogeneous(kk, E1, nu1), rel=1e-12)
    assert np.all(np.isfinite(got)) and np.all(got[1:, 1:] > 0)


@pytest.mark.parametrize("name", ["two_on_substrate", "three_on_rigid"])
def test_stack_matvec_parity(cuda, name):
    layers, Es, nus, dc = stack(name)
    N, delta = 32, 0.1
    Kg = operator.khat_grid_layers(N, delta, layers, Es, nus, dc_value=dc)
    pr = np.random.default_rng(5).standard_normal((N, N))
    ref = operator.matvec_fft(Kg, pr)
    with bem.Kernel(N, delta, layers=layers, E2=Es, nu2=nus) as k:
        u = k.matvec(torch.tensor(pr, device=cuda)).cpu().numpy()
    assert rel(u, ref) < 1e-12
    with bem.Kernel(N, delta, layers=layers, E2=Es, nu2=nus, precision="fp32") as k:
        u32 = k.matvec(torch.tensor(pr, device=cuda, dtype=torch.float32)).double().cpu().numpy()
    assert rel(u32, ref) < 2e-6


@pytest.mark.parametrize("precision,tol_p,tol_f", [("fp64", 1e-10, 1e-10), ("fp32", 2e-4, 1e-5)])
def test_stack_sphere_solve_parity(cuda, precision, tol_p, tol_f):
    """A sphere pressed into the three-layer coating on a rigid base (force control):
    pressure and force against the oracle's constrained CG on the same operator."""
    layers, Es, nus, dc = stack("three_on_rigid")
    N, R = 32, 1.0
    delta = 0.04
    F = 0.02
    f = inputs.sphere_height(N, delta, R)
    Kg = operator.khat_grid_layers(N, delta, layers, Es, nus, dc_value=dc)
    ref = contact.solve_nonadhesive(lambda p: operator.matvec_fft(Kg, p), f, delta, "force", F, tol=1e-13)
    dt = torch.float64 if precision == "fp64" else torch.float32
    with bem.Kernel(N, delta, layers=layers, E2=Es, nu2=nus, precision=precision) as k:
        p, res = k.solve(torch.tensor(f, device=cuda, dtype=dt), "force", F,
                         tol=1e-13 if precision == "fp64" else 1e-8)
    assert res["status"] == 0
    assert 10 < ref["n_contact"] < N * N // 2
    assert rel(p.double().cpu().numpy(), ref["p"]) < tol_p
    assert abs(res["force"] / ref["force"] - 1) < tol_f
