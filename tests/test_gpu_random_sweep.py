"""Seeded random sweep of contact solves against the oracle: grid size, coating
(thickness, modulus ratio, Poisson ratios, rigid or elastic base), DC rule, indenter
(sphere, rough surface, flat punch), control (depth or force), precision and
warm start drawn per case.  Each case is either solved by both sides (pressure,
force and contact count compared at the precision's tolerance) or refused by both:
an operator that the oracle finds indefinite on the contact set must end the GPU
solve with BEM_ENAN, never with a pressure."""
import numpy as np
import pytest
import torch

from oracle import contact, operator
from paper_1807_01885_gb300 import bem, inputs

pytestmark = pytest.mark.gpu

CASES = 40


def draw(i):
    rng = np.random.default_rng(7100 + i)
    N = int(rng.choice([8, 16, 32, 64]))
    delta = 1.0 / N
    h = delta * float(np.exp(rng.uniform(np.log(0.5), np.log(40.0))))
    E1 = float(np.exp(rng.uniform(np.log(0.1), np.log(10.0))))
    E2 = float("inf") if rng.random() < 0.2 else 1.0
    nu1, nu2 = (float(x) for x in rng.uniform(0.15, 0.48, size=2))
    dc_mode = int(rng.random() < 0.3)
    shape = str(rng.choice(["sphere", "rough", "punch"]))
    control = str(rng.choice(["depth", "force"]))
    precision = str(rng.choice(["fp64", "fp32"]))
    warm = bool(rng.random() < 0.3)
    if shape == "sphere":
        f = inputs.sphere_height(N, delta, 1.0)
    elif shape == "rough":
        f = inputs.rough_surface(N, delta, seed=9000 + i)
    else:
        f = inputs.flat_punch_height(N, delta, 0.25)
    return dict(N=N, delta=delta, h=h, E1=E1, E2=E2, nu1=nu1, nu2=nu2, dc_mode=dc_mode, shape=shape,
                control=control, precision=precision, warm=warm, f=f, rng=rng)


@pytest.mark.parametrize("i", range(CASES))
def test_random_case_matches_oracle(cuda, i):
    c = draw(i)
    N, delta, f = c["N"], c["delta"], c["f"]
    Kg = operator.khat_grid(N, delta, c["h"], c["E1"], c["nu1"], c["E2"], c["nu2"], c["dc_mode"])
    mv = lambda p: operator.matvec_fft(Kg, p)
    # a load that presses a few to most cells into contact: the force of a uniform
    # depth of a quarter of the height range over the window's mean compliance
    span = float(f.max() - f.min())
    d = 1e-3 * N * delta if c["shape"] == "punch" else 0.25 * span
    if c["control"] == "depth":
        target = d
    else:
        u1 = mv(np.ones((N, N)))
        target = float(d / u1.mean() * (N * delta) ** 2) * 0.5
    p0 = None
    if c["warm"]:
        p0 = np.abs(c["rng"].standard_normal((N, N))) * (target if c["control"] == "force" else 1.0)
    refused = False
    try:
        ref = contact.solve_nonadhesive(mv, f, delta, c["control"], target, tol=1e-12, p0=p0)
    except contact.NotPositiveDefinite:
        refused = True
    dt = torch.float64 if c["precision"] == "fp64" else torch.float32
    tol = 1e-12 if c["precision"] == "fp64" else 1e-8
    with bem.Kernel(N, delta, c["h"], c["E1"], c["nu1"], c["E2"], c["nu2"], precision=c["precision"],
                    dc_mode=c["dc_mode"]) as k:
        pi = None if p0 is None else torch.tensor(p0, dtype=dt, device=cuda)
        if refused:
            with pytest.raises(bem.BemError) as e:
                k.solve(torch.tensor(f, dtype=dt, device=cuda), c["control"], target, tol=tol, max_iter=20000,
                        p_init=pi)
            assert e.value.status == bem.BEM_ENAN, c
            return
        p, res = k.solve(torch.tensor(f, dtype=dt, device=cuda), c["control"], target, tol=tol, max_iter=20000,
                         p_init=pi)
    assert res["status"] == 0, (res, {k_: v for k_, v in c.items() if k_ not in ("f", "rng")})
    p = p.double().cpu().numpy()
    tp, tf = (1e-9, 1e-9) if c["precision"] == "fp64" else (2e-3, 1e-5)
    scale = np.linalg.norm(ref["p"])
    assert np.linalg.norm(p - ref["p"]) <= tp * scale + 1e-300, c["precision"]
    assert res["force"] == pytest.approx(ref["force"], rel=tf, abs=1e-300)
    if c["precision"] == "fp64":   # cells at the contact edge may carry p ~ 0 on either side
        assert abs(res["n_contact"] - ref["n_contact"]) <= max(1, 0.01 * ref["n_contact"])


STACK_CASES = 16


def draw_variant(i):
    """A coating stack of two or three layers (dc_mode 1) or the open-plane operator of a
    homogeneous half-space, with a random indenter, control and precision."""
    rng = np.random.default_rng(7700 + i)
    N = int(rng.choice([8, 16, 32, 64]))
    delta = 1.0 / N
    kind = "open" if i % 4 == 3 else "stack"
    layers = [(delta * float(np.exp(rng.uniform(np.log(0.5), np.log(10.0)))),
               float(np.exp(rng.uniform(np.log(0.2), np.log(5.0)))), float(rng.uniform(0.15, 0.45)))
              for _ in range(int(rng.integers(2, 4)))]
    E_sub = float("inf") if rng.random() < 0.25 else 1.0
    nu_sub = float(rng.uniform(0.15, 0.45))
    shape = str(rng.choice(["sphere", "rough"]))
    control = str(rng.choice(["depth", "force"]))
    precision = str(rng.choice(["fp64", "fp32"]))
    f = inputs.sphere_height(N, delta, 1.0) if shape == "sphere" else inputs.rough_surface(N, delta, seed=9500 + i)
    return dict(N=N, delta=delta, kind=kind, layers=layers, E_sub=E_sub, nu_sub=nu_sub, E=layers[0][1],
                nu=layers[0][2], shape=shape, control=control, precision=precision, f=f)


@pytest.mark.parametrize("i", range(STACK_CASES))
def test_random_stack_or_open_case_matches_oracle(cuda, i):
    from oracle import influence
    c = draw_variant(i)
    N, delta, f = c["N"], c["delta"], c["f"]
    if c["kind"] == "stack":
        Kg = operator.khat_grid_layers(N, delta, c["layers"], c["E_sub"], c["nu_sub"], dc_mode=1)
        mv = lambda p: operator.matvec_fft(Kg, p)
    else:
        G = influence.influence_love(N, delta, c["E"], c["nu"])
        mv = lambda p: influence.matvec_fft_np(G, p)
    d = 0.25 * float(f.max() - f.min())
    if c["control"] == "depth":
        target = d
    else:
        target = float(d / mv(np.ones((N, N))).mean() * (N * delta) ** 2) * 0.5
    ref = contact.solve_nonadhesive(mv, f, delta, c["control"], target, tol=1e-12)
    dt = torch.float64 if c["precision"] == "fp64" else torch.float32
    tol = 1e-12 if c["precision"] == "fp64" else 1e-8
    if c["kind"] == "stack":
        k = bem.Kernel(N, delta, layers=c["layers"], E2=c["E_sub"], nu2=c["nu_sub"], precision=c["precision"],
                       dc_mode=1)
    else:
        k = bem.Kernel(N, delta, np.inf, c["E"], c["nu"], c["E"], c["nu"], precision=c["precision"],
                       op_kind=bem.BEM_OP_OPEN)
    with k:
        p, res = k.solve(torch.tensor(f, dtype=dt, device=cuda), c["control"], target, tol=tol, max_iter=20000)
    assert res["status"] == 0, (res, c["kind"], c["precision"])
    p = p.double().cpu().numpy()
    tp, tf = (1e-9, 1e-9) if c["precision"] == "fp64" else (2e-3, 1e-5)
    assert np.linalg.norm(p - ref["p"]) <= tp * np.linalg.norm(ref["p"]), (c["kind"], c["precision"])
    assert res["force"] == pytest.approx(ref["force"], rel=tf)


def test_random_mixed_batch_equals_single_solves(cuda):
    """One bem_solve_batch call over a seeded mix: grid sizes 16 to 128, both precisions,
    depth and force control, cold and warm starts, one adhesive step, and an instance
    whose iteration limit is too small.  Every instance equals its own single solve bit
    for bit (pressure, iterations, products, status)."""
    rng = np.random.default_rng(4242)
    ks, probs, outs, singles, keep = [], [], [], [], []
    for i in range(14):
        N = int(rng.choice([16, 32, 64, 128]))
        delta = 1.0 / N
        precision = str(rng.choice(["fp64", "fp32"]))
        dt = torch.float64 if precision == "fp64" else torch.float32
        E1 = float(np.exp(rng.uniform(np.log(0.3), np.log(3.0))))
        k = bem.Kernel(N, delta, delta * float(rng.uniform(1, 10)), E1, 0.3, 1.0, 0.35, precision=precision,
                       dc_mode=1)
        f = torch.tensor(inputs.rough_surface(N, delta, seed=600 + i), dtype=dt, device=cuda)
        span = float(f.max() - f.min())
        adhesive = i == 5
        control = "depth" if (adhesive or rng.random() < 0.5) else "force"
        target = 0.25 * span if control == "depth" else 1e-3 * span
        p0 = torch.tensor(np.abs(rng.standard_normal((N, N))) * 1e-3, dtype=dt, device=cuda) if rng.random() < 0.3 \
            else None
        max_iter = 3 if i == 9 else 20000
        dg = 1e-4 if adhesive else 0.0
        mask = torch.zeros((N, N), dtype=torch.uint8, device=cuda) if adhesive else None
        p, r = k.solve(f, control, target, dgamma=dg, tol=1e-10 if precision == "fp64" else 1e-8, max_iter=max_iter,
                       p_init=p0, contact_mask=None if mask is None else mask.clone())
        singles.append((p.clone(), r))
        ctrl = bem.BEM_CTRL_DEPTH if control == "depth" else bem.BEM_CTRL_FORCE
        bmask = None if mask is None else mask.clone()   # kept alive below: the problem holds its address
        probs.append(bem.make_problem(f, ctrl, target, dg, 1e-10 if precision == "fp64" else 1e-8, max_iter, p0,
                                      bmask))
        keep.append((f, p0, bmask))
        ks.append(k)
        outs.append(torch.empty_like(f))
    st, res = bem.bem_solve_batch([k.handle for k in ks], probs, outs)
    assert st in (bem.BEM_OK, bem.BEM_ENOCONV)
    for (p, r), o, rb in zip(singles, outs, res):
        assert rb["status"] == r["status"]
        assert rb["iters"] == r["iters"] and rb["matvecs"] == r["matvecs"]
        assert torch.equal(p, o)
    assert res[9]["status"] == bem.BEM_ENOCONV
    for k in ks:
        k.close()
