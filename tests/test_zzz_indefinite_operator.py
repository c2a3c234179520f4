"""A coated half-space whose operator is indefinite on the contact set (the k = 0
reading of Eq. 11: a thick coating ten times stiffer than its substrate, h = 10 a,
on a window L = 4 a).  The solve must refuse it with BEM_ENAN in both precisions,
as the oracle refuses it (NotPositiveDefinite), instead of returning an empty
contact set; the same stack with the literal k = 0 rule is positive definite and
solves to the oracle's pressure."""
import numpy as np
import pytest
import torch

from oracle import contact, operator
from paper_1807_01885_gb300 import bem, inputs

pytestmark = pytest.mark.gpu

N, DELTA, A = 64, 1.0, 16.0
H, E1, NU1, E2, NU2 = 10 * A, 10.0, 0.3, 1.0, 0.45
D = 1e-3 * A


@pytest.mark.parametrize("precision", ["fp64", "fp32"])
def test_indefinite_operator_refused(cuda, precision):
    f = inputs.flat_punch_height(N, DELTA, A)
    with bem.Kernel(N, DELTA, H, E1, NU1, E2, NU2, precision=precision) as k:
        with pytest.raises(bem.BemError) as e:
            k.solve(torch.tensor(f, device=cuda, dtype=k.torch_dtype), "depth", D, tol=1e-10)
    assert e.value.status == bem.BEM_ENAN


def test_literal_dc_rule_solves_the_same_stack(cuda):
    f = inputs.flat_punch_height(N, DELTA, A)
    Kg = operator.khat_grid(N, DELTA, H, E1, NU1, E2, NU2, dc_mode=1)
    ref = contact.solve_nonadhesive(lambda p: operator.matvec_fft(Kg, p), f, DELTA, "depth", D, tol=1e-13)
    with bem.Kernel(N, DELTA, H, E1, NU1, E2, NU2, precision="fp64", dc_mode=bem.BEM_DC_ZERO) as k:
        p, res = k.solve(torch.tensor(f, device=cuda), "depth", D, tol=1e-13)
    assert res["status"] == 0
    err = np.linalg.norm(p.cpu().numpy() - ref["p"]) / np.linalg.norm(ref["p"])
    assert err < 1e-10
    assert res["force"] / ref["force"] == pytest.approx(1.0, rel=1e-10)
