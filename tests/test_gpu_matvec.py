"""GPU parity of the compliance table (Eqs. 9/10) and of u = K p (Eqs. 1, 11)
against the oracle, through the C ABI."""
import numpy as np
import pytest
import torch

from oracle import operator
from paper_1807_01885_gb300 import bem

pytestmark = pytest.mark.gpu

PARAMS = [  # (h, E1, nu1, E2, nu2, dc_mode) -- delta scaled per case
    (0.5, 4.0, 0.3, 1.0, 0.3, 0),
    (0.1, 0.2, 0.3, 1.0, 0.45, 0),
    (2.0, 1.0, 0.25, np.inf, 0.3, 0),
    (np.inf, 1.0, 0.3, 1.0, 0.3, 0),
    (0.3, 3.0, 0.49, 0.05, 0.2, 1),
]


def _kernel(N, delta, p, precision="fp64"):
    h, E1, nu1, E2, nu2, dc = p
    return bem.Kernel(N, delta, h, E1, nu1, E2, nu2, precision=precision, dc_mode=dc)


@pytest.mark.parametrize("p", PARAMS)
@pytest.mark.parametrize("N", [4, 64, 512])
def test_table_parity(cuda, p, N):
    delta = 1.0 / N
    with _kernel(N, delta, p) as k:
        got = k.table().cpu().numpy()
    ref = operator.khat_grid(N, delta, *p[:5], dc_mode=p[5])[: N + 1, : N + 1]
    np.testing.assert_allclose(got, ref, rtol=1e-13, atol=0)


@pytest.mark.parametrize("p", PARAMS)
@pytest.mark.parametrize("N", [4, 8, 16, 32, 64, 256])
def test_matvec_fp64_parity(cuda, p, N):
    delta = 1.0 / N
    rng = np.random.default_rng(N)
    pr = rng.standard_normal((N, N))
    Kg = operator.khat_grid(N, delta, *p[:5], dc_mode=p[5])
    ref = operator.matvec_dense(Kg, pr) if N <= 16 else operator.matvec_fft(Kg, pr)
    with _kernel(N, delta, p) as k:
        u = k.matvec(torch.tensor(pr, device=cuda)).cpu().numpy()
    assert np.linalg.norm(u - ref) / np.linalg.norm(ref) < 1e-12


@pytest.mark.parametrize("p", PARAMS[:3])
@pytest.mark.parametrize("N", [8, 64, 512])
def test_matvec_fp32_parity(cuda, p, N):
    delta = 1.0 / N
    rng = np.random.default_rng(N + 1)
    pr = rng.standard_normal((N, N))
    ref = operator.matvec_fft(operator.khat_grid(N, delta, *p[:5], dc_mode=p[5]), pr)
    with _kernel(N, delta, p, "fp32") as k:
        u = k.matvec(torch.tensor(pr, device=cuda, dtype=torch.float32)).double().cpu().numpy()
    # float FFT error grows like log2(2N) * eps32
    assert np.linalg.norm(u - ref) / np.linalg.norm(ref) < 2e-6


def test_matvec_host_arguments(cuda):
    N, p = 32, PARAMS[0]
    pr = np.random.default_rng(7).standard_normal((N, N))
    with _kernel(N, 1.0 / N, p) as k:
        u_host = k.matvec(pr.copy())
        u_dev = k.matvec(torch.tensor(pr, device=cuda)).cpu().numpy()
    np.testing.assert_array_equal(u_host, u_dev)


@pytest.mark.parametrize("precision,tol", [("fp64", 1e-11), ("fp32", 3e-5)])
def test_matvec_full_size_impulse_samples(cuda, precision, tol):
    """N = 2048 (the benchmark size): the response to a unit pressure in one cell is
    the influence function G(r - s); sampled outputs are compared with the
    oracle's direct sum over all (2N)^2 wave numbers, one output at a time."""
    N, delta = 2048, 1.0 / 2048
    h, E1, nu1, E2, nu2 = 8 * delta, 0.5, 0.3, 1.0, 0.45
    s = (1000, 1100)
    with bem.Kernel(N, delta, h, E1, nu1, E2, nu2, precision=precision) as k:
        e = torch.zeros((N, N), dtype=k.torch_dtype, device=cuda)
        e[s] = 1.0
        u = k.matvec(e).double().cpu().numpy()
    rng = np.random.default_rng(3)
    cells = [(1000, 1100), (1001, 1100), (1000, 1105), (0, 0), (2047, 2047), (1500, 20)]
    cells += [tuple(x) for x in rng.integers(0, N, (6, 2))]
    offs = [(r - s[0], c - s[1]) for r, c in cells]
    G = operator.influence_at(N, delta, h, E1, nu1, E2, nu2, offs)
    got = np.array([u[r, c] for r, c in cells])
    scale = abs(G).max()
    np.testing.assert_allclose(got, G, rtol=0, atol=tol * scale)


def test_matvec_properties_full_size(cuda):
    """N = 2048, FP64: symmetry <q, K p> = <p, K q> and positivity <p, K p> > 0,
    properties of the exact operator at any size."""
    N, delta = 2048, 1.0 / 2048
    with bem.Kernel(N, delta, 16 * delta, 2.0, 0.3, 1.0, 0.3, precision="fp64") as k:
        g = torch.Generator(device=cuda).manual_seed(1)
        p = torch.randn((N, N), dtype=torch.float64, device=cuda, generator=g)
        q = torch.randn((N, N), dtype=torch.float64, device=cuda, generator=g)
        Kp, Kq = k.matvec(p), k.matvec(q)
        a, b = float((q * Kp).sum()), float((p * Kq).sum())
        assert abs(a - b) <= 1e-12 * float((p * Kp).sum())
        assert float((p * Kp).sum()) > 0 and float((q * Kq).sum()) > 0


def test_matvec_is_deterministic(cuda):
    N = 256
    pr = torch.randn((N, N), dtype=torch.float32, device=cuda)
    with bem.Kernel(N, 1.0 / N, 0.05, 1.0, 0.3, 2.0, 0.3, precision="fp32") as k:
        a = k.matvec(pr).clone()
        b = k.matvec(pr).clone()
    assert torch.equal(a, b)


@pytest.mark.parametrize("N,precision", [(64, "fp64"), (64, "fp32"), (2048, "fp32")])
def test_back_to_back_products_equal_isolated_ones(cuda, N, precision):
    """The passes of consecutive products are launched with programmatic dependent
    launch (each may be scheduled while its predecessor finishes).  A chain of products
    on one stream without any synchronisation, u_{i+1} = K u_i (every product reading
    what the one before wrote), equals the same chain with a full device
    synchronisation after every product, bit for bit."""
    dt = torch.float64 if precision == "fp64" else torch.float32
    s = torch.cuda.Stream(device=cuda)
    with bem.Kernel(N, 1.0 / N, 2.0 / N, 3.0, 0.3, 1.0, 0.4, precision=precision) as k:
        x0 = torch.tensor(np.random.default_rng(N).random((N, N)), dtype=dt, device=cuda)
        with torch.cuda.stream(s):
            chain = [x0]
            for _ in range(12):
                chain.append(k.matvec(chain[-1], torch.empty_like(x0), stream=s))
            s.synchronize()
            ref = [x0]
            for _ in range(12):
                torch.cuda.synchronize()
                ref.append(k.matvec(ref[-1], torch.empty_like(x0), stream=s))
                torch.cuda.synchronize()
    assert all(bool(torch.isfinite(a).all()) for a in chain)
    for a, b in zip(chain, ref):
        assert torch.equal(a, b)
