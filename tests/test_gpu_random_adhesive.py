"""Seeded random sweep of adhesive steps (Sec. 2 procedure, Eq. 12) against the
oracle: coating, substrate, sphere radius, work of adhesion and the loads drawn per
case.  Each case runs a displacement-controlled loading step from no contact, an
unloading step from that state, and a force-controlled step from the loaded state
(the force may be tensile); the FP64 path must give the oracle's contact area cell
for cell, its pressure and depth, or detach where the oracle detaches."""
import numpy as np
import pytest
import torch

from oracle import contact, kernel as okernel, operator
from paper_1807_01885_gb300 import bem, inputs

pytestmark = pytest.mark.gpu

CASES = 20


def draw(i):
    rng = np.random.default_rng(8300 + i)
    N = int(rng.choice([16, 32]))
    delta = 1.0 / N
    R = float(np.exp(rng.uniform(np.log(0.5), np.log(2.0))))
    h = delta * float(np.exp(rng.uniform(np.log(1.0), np.log(20.0))))
    E1 = float(np.exp(rng.uniform(np.log(0.3), np.log(3.0))))
    E2 = float("inf") if rng.random() < 0.3 else 1.0
    nu1, nu2 = (float(x) for x in rng.uniform(0.2, 0.45, size=2))
    a_d = delta * float(rng.uniform(2.0, 4.0))
    dg = a_d ** 3 * 8 * okernel.e_star(E1, nu1) / (np.pi * R * R) * 10 ** float(rng.uniform(-2.5, 0.0))
    d1 = float(rng.uniform(0.3, 1.0)) * (1.2 * a_d) ** 2 / R
    d2 = d1 * float(rng.uniform(0.2, 0.8))
    ffrac = float(rng.uniform(-4.0, 0.8))
    return dict(N=N, delta=delta, R=R, h=h, E1=E1, E2=E2, nu1=nu1, nu2=nu2, dg=dg, d1=d1, d2=d2, ffrac=ffrac)


def rel(a, b):
    return np.linalg.norm(a - b) / max(np.linalg.norm(b), 1e-300)


@pytest.mark.parametrize("i", range(CASES))
def test_random_adhesive_steps_match_oracle(cuda, i):
    c = draw(i)
    N, delta = c["N"], c["delta"]
    f = inputs.sphere_height(N, delta, c["R"])
    Kg = operator.khat_grid(N, delta, c["h"], c["E1"], c["nu1"], c["E2"], c["nu2"], 1)
    mv = lambda p: operator.matvec_fft(Kg, p)
    sc = contact.sigma_c(c["E1"], c["nu1"], c["dg"], delta)
    empty = np.zeros((N, N), dtype=bool)
    p1, C1, _, _ = contact.adhesive_step(mv, f, c["d1"], empty, sc, tol=1e-12)
    p2, C2, _, _ = contact.adhesive_step(mv, f, c["d2"], C1, sc, p_prev=p1, tol=1e-12)
    F1 = float(delta * delta * p1.sum())
    Ft = c["ffrac"] * F1
    try:
        p3, C3, d3, _, _ = contact.adhesive_step_force(mv, f, Ft, delta, C1, sc, tol=1e-12)
    except contact.Detached:
        p3 = None
    ft = torch.tensor(f, dtype=torch.float64, device=cuda)
    with bem.Kernel(N, delta, c["h"], c["E1"], c["nu1"], c["E2"], c["nu2"], dc_mode=1) as k:
        m1 = torch.zeros((N, N), dtype=torch.uint8, device=cuda)
        g1, r1 = k.solve(ft, "depth", c["d1"], dgamma=c["dg"], tol=1e-12, max_iter=20000, contact_mask=m1)
        assert r1["status"] == 0
        assert np.array_equal(m1.cpu().numpy().astype(bool), C1)
        assert rel(g1.cpu().numpy(), p1) < 1e-8
        m2 = m1.clone()
        g2, r2 = k.solve(ft, "depth", c["d2"], dgamma=c["dg"], tol=1e-12, max_iter=20000, p_init=g1,
                         contact_mask=m2)
        assert r2["status"] == 0
        assert np.array_equal(m2.cpu().numpy().astype(bool), C2)
        if C2.any():
            assert rel(g2.cpu().numpy(), p2) < 1e-8
        m3 = m1.clone()
        g3, r3 = k.solve(ft, "force", Ft, dgamma=c["dg"], tol=1e-12, max_iter=20000, p_init=g1, contact_mask=m3)
        if p3 is None:
            assert r3["status"] == bem.BEM_EDETACHED
        else:
            assert r3["status"] == 0
            assert np.array_equal(m3.cpu().numpy().astype(bool), C3)
            assert rel(g3.cpu().numpy(), p3) < 1e-8
            assert r3["depth"] == pytest.approx(d3, rel=1e-8, abs=1e-12)
