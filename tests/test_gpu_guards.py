"""Workspace guard zones (a debugging aid beside the parity tests): after every kind
of call the library makes on a handle (products from host and device arrays, solves
under both controls, an adhesive step, a batch, a rebuild, each FFT radix), the
256-byte pattern zones around the handle's arrays are intact; a byte overwritten from
the host (fault injection, no kernel) is counted."""
import numpy as np
import pytest
import torch

from paper_1807_01885_gb300 import bem, inputs

pytestmark = pytest.mark.gpu


@pytest.mark.parametrize("N,precision", [(4, "fp64"), (16, "fp32"), (64, "fp64"), (512, "fp32"), (256, "fp64")])
def test_guards_intact_after_every_call(cuda, N, precision):
    dt = torch.float64 if precision == "fp64" else torch.float32
    delta = 1.0 / N
    f = torch.tensor(inputs.sphere_height(N, delta, 1.0), dtype=dt, device=cuda)
    rng = np.random.default_rng(N)
    # a compliant coating: the operator stays positive definite on every window size
    ks = [bem.Kernel(N, delta, 0.2, 0.5, 0.3, 1.0, 0.4, precision=precision) for _ in range(3)]
    k = ks[0]
    p = torch.tensor(rng.random((N, N)), dtype=dt, device=cuda)
    k.matvec(p)
    k.matvec(p.cpu().numpy())
    F = 1e-4
    k.solve(f, "force", F, tol=1e-8)
    k.solve(f, "depth", 1e-3, tol=1e-8)
    mask = torch.zeros((N, N), dtype=torch.uint8, device=cuda)
    k.solve(f, "depth", 2e-3, dgamma=1e-4, tol=1e-8, contact_mask=mask)
    probs = [bem.make_problem(f, bem.BEM_CTRL_FORCE, F * (1 + i), tol=1e-8, max_iter=5000) for i in range(3)]
    outs = [torch.empty_like(f) for _ in range(3)]
    bem.bem_solve_batch([x.handle for x in ks], probs, outs)
    k.rebuild(delta, 0.1, 0.8, 0.25, 1.0, 0.3)
    if N >= 16:
        radices = [(3, 3)] if precision == "fp64" else [(4, 4), (3, 4), (4, 3), (3, 3)]
        for r in radices:
            k.set_radix(*r)
            k.matvec(p)
        k.autotune(reps=2)
    torch.cuda.synchronize()
    for x in ks:
        assert x.check_guards() == 0
        x.close()


def test_guard_check_counts_an_injected_byte(cuda):
    with bem.Kernel(32, 1.0 / 32, 0.2, 3.0, 0.3, 1.0, 0.4) as k:
        assert k.check_guards() == 0
        bem._check(bem.load().bem_debug_poke_guard(k.handle, 0))
        assert k.check_guards() == 1
        bem._check(bem.load().bem_debug_poke_guard(k.handle, 3))
        assert k.check_guards() == 2
        with pytest.raises(bem.BemError) as e:
            bem._check(bem.load().bem_debug_poke_guard(k.handle, 99))
        assert e.value.status == bem.BEM_EINVAL
