"""FFT radix choices of the register passes (bem_set_radix) and their autotuner
(bem_autotune): every choice keeps parity with the oracle's product, a changed
choice rebuilds the handle's captured iteration graph, invalid choices are refused."""
import numpy as np
import pytest
import torch

from oracle import contact, operator
from paper_1807_01885_gb300 import bem, inputs

pytestmark = pytest.mark.gpu

LAYER = (0.5, 4.0, 0.3, 1.0, 0.3)   # h, E1, nu1, E2, nu2 (delta = 1/N)


def _ref_product(N, pr):
    return operator.matvec_fft(operator.khat_grid(N, 1.0 / N, *LAYER), pr)


@pytest.mark.parametrize("N", [16, 256])
@pytest.mark.parametrize("rows,cols", [(3, 3), (3, 4), (4, 3), (4, 4)])
def test_every_radix_choice_keeps_parity(cuda, N, rows, cols):
    rng = np.random.default_rng(100 + N)
    pr = rng.standard_normal((N, N))
    ref = _ref_product(N, pr)
    with bem.Kernel(N, 1.0 / N, *LAYER, precision="fp32") as k:
        k.set_radix(rows, cols)
        u = k.matvec(torch.tensor(pr, device=cuda, dtype=torch.float32)).double().cpu().numpy()
    assert np.linalg.norm(u - ref) / np.linalg.norm(ref) < 2e-6


@pytest.mark.parametrize("N,precision", [(512, "fp32"), (64, "fp64"), (8, "fp32")])
def test_autotune_choice_and_parity(cuda, N, precision):
    rng = np.random.default_rng(7)
    pr = rng.standard_normal((N, N))
    ref = _ref_product(N, pr)
    with bem.Kernel(N, 1.0 / N, *LAYER, precision=precision) as k:
        rows, cols = k.autotune(reps=3)
        u = k.matvec(torch.tensor(pr, device=cuda, dtype=k.torch_dtype)).double().cpu().numpy()
    allowed = {3, 4} if precision == "fp32" else {3}
    assert rows in allowed and cols in allowed
    tol = 2e-6 if precision == "fp32" else 1e-12
    assert np.linalg.norm(u - ref) / np.linalg.norm(ref) < tol


def test_invalid_radix_refused(cuda):
    with bem.Kernel(64, 1.0 / 64, *LAYER, precision="fp64") as k:
        with pytest.raises(bem.BemError) as e:
            k.set_radix(4, 3)
        assert e.value.status == bem.BEM_EINVAL
    with bem.Kernel(64, 1.0 / 64, *LAYER, precision="fp32") as k:
        for bad in [(5, 4), (4, 2), (0, 0)]:
            with pytest.raises(bem.BemError):
                k.set_radix(*bad)


def test_radix_change_rebuilds_captured_graph(cuda):
    """Solves on a non-default stream replay the captured iteration graph.  After a
    radix change the next solve must capture the new kernels: it agrees with the
    oracle, and switching back reproduces the first result bit for bit."""
    N = 128
    inst = inputs.batch_instance(20260300, sizes=(N,))
    Kg = operator.khat_grid(N, inst["delta"], inst["h"], inst["E1"], inst["nu1"], inst["E2"], inst["nu2"])
    ref = contact.solve_nonadhesive(lambda p: operator.matvec_fft(Kg, p), inst["height"], inst["delta"], "force",
                                    inst["force"], tol=1e-13)
    s = torch.cuda.Stream()
    with bem.Kernel(N, inst["delta"], inst["h"], inst["E1"], inst["nu1"], inst["E2"], inst["nu2"],
                    precision="fp32") as k, torch.cuda.stream(s):
        ht = torch.tensor(inst["height"], device=cuda, dtype=torch.float32)
        results = []
        for choice in [(4, 4), (4, 4), (3, 3), (4, 4)]:
            k.set_radix(*choice, stream=s)
            p, res = k.solve(ht, "force", inst["force"], tol=1e-8, stream=s)
            s.synchronize()
            assert res["status"] == 0
            err = np.linalg.norm(p.double().cpu().numpy() - ref["p"]) / np.linalg.norm(ref["p"])
            assert err < 2e-4
            results.append((p.clone(), res["iters"]))
    assert torch.equal(results[0][0], results[1][0]) and results[0][1] == results[1][1]
    assert torch.equal(results[0][0], results[3][0]) and results[0][1] == results[3][1]
