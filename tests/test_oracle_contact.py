"""Pins of the oracle's contact solvers against brute force and the paper's closed forms.

Solution-level pins hold within discretisation error, so each tolerance is set from
the grid (stated per test); the thick-layer test shows the pin is sharp by checking
that plain Hertz (no layer correction) would fail it.
"""
import numpy as np
import pytest
from scipy.optimize import brentq, nnls

from oracle import analytic, contact, kernel, operator
from paper_1807_01885_gb300 import inputs


def _mv(N, delta, h, E1, nu1, E2, nu2, dc_mode=0):
    Kg = operator.khat_grid(N, delta, h, E1, nu1, E2, nu2, dc_mode)
    return Kg, (lambda p: operator.matvec_fft(Kg, p))


def test_pk_matches_nnls_brute_force():
    """Depth control is the QP min 1/2 p'Kp - p'(d - f), p >= 0; with K = L L' it is
    the NNLS problem min ||L' p - L^{-1}(d - f)||, solved by an active-set library
    routine that shares nothing with the CG."""
    N, delta = 8, 0.1
    Kg, mv = _mv(N, delta, 0.15, 2.0, 0.3, 1.0, 0.4)
    Km = operator.dense_matrix(Kg)
    f = inputs.sphere_height(N, delta, 0.5) + 0.002 * np.random.default_rng(3).standard_normal((N, N))
    f -= f.min()
    d = 0.02
    Lc = np.linalg.cholesky(Km)
    b = np.linalg.solve(Lc, (d - f).reshape(-1))
    p_ref, _ = nnls(Lc.T, b, maxiter=10000)
    s = contact.solve_nonadhesive(mv, f, delta, "depth", d, tol=1e-13)
    np.testing.assert_allclose(s["p"].reshape(-1), p_ref, atol=1e-9 * p_ref.max())
    assert contact.kkt_violation(mv, s["p"], f, d) < 1e-11


def test_load_control_equals_depth_control():
    N, delta = 32, 0.05
    _, mv = _mv(N, delta, 0.2, 0.5, 0.3, 1.0, 0.45)
    f = inputs.rough_surface(N, delta, seed=11)
    s1 = contact.solve_nonadhesive(mv, f, delta, "force", 2e-3, tol=1e-13)
    assert s1["force"] == pytest.approx(2e-3, rel=1e-12)
    s2 = contact.solve_nonadhesive(mv, f, delta, "depth", s1["d"], tol=1e-13)
    np.testing.assert_allclose(s2["p"], s1["p"], atol=1e-9 * s1["p"].max())
    assert contact.kkt_violation(mv, s1["p"], f, s1["d"]) < 1e-10


def test_hertz_homogeneous_load_control():
    """E1 = E2: Hertz contact radius a = (3FR/4E*)^(1/3) and pressure
    p0 sqrt(1 - r^2/a^2) (Eq. 22 at epsilon = 0, no adhesion).  Load control keeps
    the result free of the DC offset of the periodic operator.  a = 16 cells."""
    N, R, E, nu = 64, 1.0, 1.0, 0.3
    aH = 0.1
    delta = 4 * aH / N
    Es = kernel.e_star(E, nu)
    _, mv = _mv(N, delta, np.inf, E, nu, E, nu)
    f = inputs.sphere_height(N, delta, R)
    F = analytic.hertz(aH, R, Es)[0]
    s = contact.solve_nonadhesive(mv, f, delta, "force", F, tol=1e-12)
    a_num = np.sqrt(s["n_contact"] * delta ** 2 / np.pi)
    assert a_num == pytest.approx(aH, rel=0.02)
    x, y = inputs.cell_centres(N, delta)
    ph = analytic.hertz_pressure(np.hypot(x, y), aH, R, Es)
    assert np.linalg.norm(s["p"] - ph) / np.linalg.norm(ph) < 0.02


@pytest.mark.parametrize("a_over_h,tol", [(10, 0.03), (20, 0.01)])
def test_thin_layer_flat_punch_stiffness(a_over_h, tol):
    """Rigid base, a >> h: k = pi a^2 E~1 / h (Eqs. 14/15).  Edge effects are
    O(h/a), so the tolerance tightens as a/h grows."""
    N, delta, E1, nu1 = 128, 1.0, 1.0, 0.3
    a = N / 4
    h = a / a_over_h
    _, mv = _mv(N, delta, h, E1, nu1, np.inf, 0.3)
    f = inputs.flat_punch_height(N, delta, a)
    d = 1e-3
    s = contact.solve_nonadhesive(mv, f, delta, "depth", d, tol=1e-12)
    a_eff = np.sqrt(s["n_contact"] / np.pi) * delta
    assert s["force"] / d == pytest.approx(analytic.thin_layer_stiffness(a_eff, h, E1, nu1), rel=tol)


@pytest.mark.parametrize("h", [32.0, 64.0])
def test_thick_layer_series_eq22_23(h):
    """Rigid base, a < h: F(d) from Eqs. (22)/(23) at dgamma = 0, with a0, a1 of
    Eq. (24).  The layer correction is 10-40 % here, so Hertz alone fails."""
    N, delta, R, E1, nu1 = 128, 1.0, 400.0, 1.0, 0.3
    Es = kernel.e_star(E1, nu1)
    _, mv = _mv(N, delta, h, E1, nu1, np.inf, 0.3)
    f = inputs.sphere_height(N, delta, R)
    for d in (0.1, 0.2):
        s = contact.solve_nonadhesive(mv, f, delta, "depth", d, tol=1e-11)
        a = brentq(lambda a: analytic.thick_layer_sphere(a, R, h, E1, nu1, 0.0)[1] - d, 1e-3, h)
        F_ser = analytic.thick_layer_sphere(a, R, h, E1, nu1, 0.0)[0]
        F_hertz = 4.0 / 3.0 * Es * np.sqrt(R) * d ** 1.5
        assert s["force"] == pytest.approx(F_ser, rel=5e-3)
        assert abs(s["force"] / F_hertz - 1) > 0.05


def test_boundary_cells():
    C = np.zeros((6, 6), dtype=bool)
    C[1:5, 1:5] = True
    B = contact.boundary_cells(C)
    assert B.sum() == 12 and not B[2, 2] and not B[3, 3] and B[1, 1] and B[4, 2]
    full = np.ones((3, 3), dtype=bool)
    assert contact.boundary_cells(full).sum() == 8     # the window edge counts as outside


def test_jkr_pull_off_homogeneous():
    """E1 = E2, displacement-controlled pull-off with the criterion of Eq. (12):
    the force minimum approaches the JKR value -(3/2) pi R dgamma (minimum of F(a)
    from Eqs. 22/23 at epsilon = 0) and the contact recedes before the jump-off
    (the JKR jump-off radius is 5 cells here, the force minimum at 10)."""
    N, R, E, nu = 64, 1.0, 1.0, 0.3
    delta = 0.5 / N
    Es = kernel.e_star(E, nu)
    a_d = 5 * delta
    dg = a_d ** 3 * 8 * Es / (np.pi * R * R)
    a_F = 9 ** (1 / 3) * a_d
    _, mv = _mv(N, delta, np.inf, E, nu, E, nu)
    f = inputs.sphere_height(N, delta, R)
    sc = contact.sigma_c(E, nu, dg, delta)
    d_max = (1.4 * a_F) ** 2 / R
    d_jump = analytic.jkr_jump_off(R, Es, dg)[2]
    depths = np.concatenate([np.linspace(0, d_max, 6), np.linspace(d_max, 1.3 * d_jump, 60)])
    out = contact.adhesive_ramp(mv, f, delta, depths, sc, tol=1e-10)
    Fmin = min(o["force"] for o in out)
    assert Fmin / analytic.jkr_pull_off_force(R, dg) == pytest.approx(1.0, abs=0.15)
    n = [o["n_contact"] for o in out[6:]]
    assert n[-1] == 0 and max(n) > 3 * min(x for x in n if x > 0)


def test_sigma_c_constant_from_paper():
    """Eq. (12) with the printed constant 0.473201 (tests/golden/paper_parameters.json)."""
    import json, os
    g = json.load(open(os.path.join(os.path.dirname(__file__), "golden", "paper_parameters.json")))
    c = g["eq12_constant"]["value"]
    E1, nu1, dg, delta = 2.0, 0.3, 0.01, 0.05
    s = contact.sigma_c(E1, nu1, dg, delta)
    assert s * s * c * delta == pytest.approx(E1 / (1 - nu1 ** 2) * dg, rel=1e-14)


def test_pk_matches_active_set_enumeration():
    """Brute force on a 4 x 4 window: of the 65536 candidate contact sets S, exactly one
    gives p_S = K_SS^{-1} (d - f)_S >= 0 with no penetration outside S (the QP's
    unique solution, K being positive definite); the CG returns that pressure."""
    import itertools
    N, delta = 4, 0.15
    Kg, mv = _mv(N, delta, 0.3, 2.0, 0.3, 1.0, 0.4)
    Km = operator.dense_matrix(Kg)
    rng = np.random.default_rng(8)
    f = inputs.sphere_height(N, delta, 0.4) + 0.004 * rng.standard_normal((N, N))
    f -= f.min()
    d = 0.03
    b = (d - f).reshape(-1)
    found = []
    for mask in itertools.product([False, True], repeat=N * N):
        S = np.array(mask)
        p = np.zeros(N * N)
        if S.any():
            p[S] = np.linalg.solve(Km[np.ix_(S, S)], b[S])
        g = Km @ p - b
        if p.min() >= -1e-12 * max(p.max(), 1e-300) and g[~S].min(initial=0.0) >= -1e-12 * np.abs(b).max():
            found.append((S, p))
    assert len(found) == 1
    S_ref, p_ref = found[0]
    assert 0 < S_ref.sum() < N * N                     # a partial contact, not a trivial case
    s = contact.solve_nonadhesive(mv, f, delta, "depth", d, tol=1e-14)
    np.testing.assert_allclose(s["p"].reshape(-1), p_ref, atol=1e-10 * p_ref.max())


def test_adhesive_steps_are_fixed_points_of_the_rules():
    """Every step of an oracle pull-off ramp (N = 16, homogeneous) satisfies the rules
    of the Sec. 2 procedure, checked with the dense matrix of Eq. (1): on C the
    displacement is exactly d - f (dense solve of K_CC p_C = (d - f)_C), p = 0 off C,
    no cell off C penetrates, and no boundary cell of C carries a tension above
    sigma_c (Eq. 12).  The ramp must reach tension and detach cells, so the rules
    that matter in adhesion are exercised."""
    N, R, E, nu = 16, 1.0, 1.0, 0.3
    delta = 0.5 / N
    Kg, mv = _mv(N, delta, np.inf, E, nu, E, nu)
    Km = operator.dense_matrix(Kg)
    Es = kernel.e_star(E, nu)
    dg = (2 * delta) ** 3 * 8 * Es / (np.pi * R * R)
    sc = contact.sigma_c(E, nu, dg, delta)
    f = inputs.sphere_height(N, delta, R)
    d_max = (3.5 * delta) ** 2 / R
    depths = np.concatenate([np.linspace(0, d_max, 4), np.linspace(d_max, -d_max, 16)[1:]])
    out = contact.adhesive_ramp(mv, f, delta, depths, sc, tol=1e-13)
    saw_tension = False
    for o in out:
        C, p, d = o["C"].reshape(-1), o["p"].reshape(-1), o["d"]
        b = (d - f).reshape(-1)
        assert np.all(p[~C] == 0.0)
        if C.any():
            pc = np.linalg.solve(Km[np.ix_(C, C)], b[C])
            np.testing.assert_allclose(p[C], pc, atol=1e-9 * np.abs(pc).max())
        g = Km @ p - b
        assert g[~C].min(initial=0.0) >= -1e-10 * max(np.abs(b).max(), 1e-300)
        B = contact.boundary_cells(o["C"]).reshape(-1)
        assert np.all(-p[B] <= sc)
        saw_tension |= bool((p < 0).any())
    assert saw_tension
    n = [o["n_contact"] for o in out]
    assert max(n) > 0 and n[-1] < max(n)


def test_fixed_set_force_solves_the_bordered_system():
    """Load control on a fixed area against brute force: the bordered (KKT) system
    [[K_CC, -1], [1', 0]] [p_C; d] = [-f_C; F/delta^2] solved densely on an 8 x 8
    window, a layered operator, a random area and random heights."""
    N, delta = 8, 0.2
    Kg, mv = _mv(N, delta, 0.3, 3.0, 0.25, 1.0, 0.4)
    K = operator.dense_matrix(Kg)
    rng = np.random.default_rng(11)
    f = rng.random((N, N))
    C = rng.random((N, N)) < 0.45
    P = 2.5
    c = C.reshape(-1)
    m = int(c.sum())
    A = np.zeros((m + 1, m + 1))
    A[:m, :m] = K[np.ix_(c, c)]
    A[:m, m] = -1.0
    A[m, :m] = 1.0
    sol = np.linalg.solve(A, np.concatenate([-f.reshape(-1)[c], [P]]))
    p, d, _ = contact.solve_fixed_set_force(mv, C, f, P, tol=1e-14)
    assert d == pytest.approx(sol[m], rel=1e-10)
    np.testing.assert_allclose(p.reshape(-1)[c], sol[:m], rtol=0, atol=1e-10 * np.abs(sol[:m]).max())
    assert np.all(p[~C] == 0.0)


def _jkr_loaded(N=64):
    """JKR sphere on a homogeneous half-space (jump-off radius 5 cells) after a
    displacement-controlled loading ramp: (mv, f, delta, sigma_c, Es, dgamma, last)."""
    R, E, nu = 1.0, 1.0, 0.3
    delta = 0.5 / N
    Es = kernel.e_star(E, nu)
    a_d = 5 * delta
    dg = a_d ** 3 * 8 * Es / (np.pi * R * R)
    a_F = 9 ** (1 / 3) * a_d
    _, mv = _mv(N, delta, np.inf, E, nu, E, nu)
    f = inputs.sphere_height(N, delta, R)
    sc = contact.sigma_c(E, nu, dg, delta)
    d_max = (1.4 * a_F) ** 2 / R
    last = contact.adhesive_ramp(mv, f, delta, np.linspace(0, d_max, 6), sc, tol=1e-10)[-1]
    return mv, f, delta, sc, Es, dg, last, d_max


def test_load_controlled_step_is_a_fixed_point_of_the_depth_step():
    """A load-controlled adhesive step ends in a state that the displacement-controlled
    step at the depth it found leaves unchanged: same area after one outer pass, same
    force, for an unloading target (half the loaded force) and a tensile one."""
    mv, f, delta, sc, Es, dg, last, d_max = _jkr_loaded(N=32)
    Fj = analytic.jkr_pull_off_force(1.0, dg)
    for F in (0.5 * last["force"], 0.5 * Fj):
        p, C, d, outer, _ = contact.adhesive_step_force(mv, f, F, delta, last["C"], sc, tol=1e-12)
        assert delta * delta * p.sum() == pytest.approx(F, rel=1e-9)
        assert C.any() and d < d_max
        p2, C2, outer2, _ = contact.adhesive_step(mv, f, d, C, sc, p_prev=p, tol=1e-12)
        assert outer2 == 1 and np.array_equal(C2, C)
        assert delta * delta * p2.sum() == pytest.approx(F, rel=1e-8)


def test_load_controlled_pull_off_is_jkr():
    """Load-controlled pull-off by the oracle's own load-controlled steps (N = 64,
    jump-off radius 5 cells): decreasing targets are carried until one detaches the
    whole area; the last carried force is the minimum of the branch followed in small
    depth steps (within the few cells by which the two paths detach differently, 3 %
    of the pull-off force) and the JKR pull-off force -(3/2) pi R dgamma within this
    grid's discretisation error (15 %)."""
    mv, f, delta, sc, Es, dg, last, d_max = _jkr_loaded(N=64)
    Fj = analytic.jkr_pull_off_force(1.0, dg)
    spacing = 0.05 * abs(Fj)
    targets = np.concatenate([np.linspace(last["force"], 0.7 * Fj, 6)[1:], 0.7 * Fj - spacing * np.arange(1, 15)])
    C, carried, depths = last["C"], [], []
    with pytest.raises(contact.Detached):
        for F in targets:
            p, C, d, _, _ = contact.adhesive_step_force(mv, f, F, delta, C, sc, tol=1e-10)
            carried.append(F)
            depths.append(d)
    assert 0 < len(carried) < len(targets)
    assert all(b < a for a, b in zip(depths, depths[1:]))
    d_end = 1.3 * analytic.jkr_jump_off(1.0, Es, dg)[2]
    disp = contact.adhesive_ramp(mv, f, delta, np.linspace(d_max, d_end, 61)[1:], sc, C0=last["C"], tol=1e-10)
    F_min = min(o["force"] for o in disp)
    assert F_min - 0.03 * abs(Fj) <= carried[-1] < F_min + spacing + 0.03 * abs(Fj)
    assert carried[-1] / Fj == pytest.approx(1.0, abs=0.15)


def test_indefinite_operator_is_refused():
    """Polonsky-Keer CG needs K positive definite on the contact set.  A thick stiff
    coating (h = 10 a, E1/E2 = 10) on a 2N period makes the finite-part DC value of
    the k = 0 term strongly negative (reading of Eq. 11 at k = 0) and K indefinite on
    the punch: the dense matrix shows a negative eigenvalue, and the solve must stop
    with NotPositiveDefinite instead of returning a pressure.  The same stack with
    the literal DC rule (K^(0) = 0) stays positive definite and solves."""
    N, delta, a = 64, 1.0, 16.0
    f = inputs.flat_punch_height(N, delta, a)
    C = (f == 0).ravel()
    Kg, mv = _mv(N, delta, 10 * a, 10.0, 0.3, 1.0, 0.45)
    assert Kg[0, 0] < 0
    assert np.linalg.eigvalsh(operator.dense_matrix(Kg)[np.ix_(C, C)])[0] < 0
    with pytest.raises(contact.NotPositiveDefinite):
        contact.solve_nonadhesive(mv, f, delta, "depth", 1e-3 * a, tol=1e-12)
    Kz, mz = _mv(N, delta, 10 * a, 10.0, 0.3, 1.0, 0.45, dc_mode=1)
    assert np.linalg.eigvalsh(operator.dense_matrix(Kz)[np.ix_(C, C)])[0] > 0
    s = contact.solve_nonadhesive(mz, f, delta, "depth", 1e-3 * a, tol=1e-12)
    assert s["force"] > 0 and contact.kkt_violation(mz, s["p"], f, 1e-3 * a) < 1e-9


def test_flat_punch_stiffness_sweep_bracketed():
    """Flat punch on a coating (L = 4a, N = 64, nu1 = 0.3, nu2 = 0.45), h/a in
    {0.1, 0.3, 1, 3, 10}, E1/E2 in {0.1, 0.5, 2, 10}.  Stiffness F/d is normalised by
    the same grid's homogeneous value (the period's images and the zero-mean datum
    stiffen every punch alike, here by 1.43).  With the literal k = 0 rule (K^(0) = 0)
    the operator stays ordered between the two homogeneous ones, so each normalised
    stiffness lies between the substrate's and the coating's Boussinesq values
    2aE2* and 2aE1*, moves monotonically from the first towards the second as h/a
    grows, and reaches the coating's within 1 % at h/a = 10 (the layer then holds the
    whole response at the window's scale)."""
    N, delta, a = 64, 1.0, 16.0
    f = inputs.flat_punch_height(N, delta, a)
    E2, nu1, nu2 = 1.0, 0.3, 0.45
    d = 1e-3 * a

    def stiffness(h, E1, n1, Es, ns):
        _, mv = _mv(N, delta, h, E1, n1, Es, ns, dc_mode=1)
        return contact.solve_nonadhesive(mv, f, delta, "depth", d, tol=1e-12)["force"] / d

    k_hom = stiffness(np.inf, 1.0, 0.3, 1.0, 0.3) / analytic.flat_punch_stiffness(a, kernel.e_star(1.0, 0.3))
    assert 1.2 < k_hom < 1.6
    for r in (0.1, 0.5, 2.0, 10.0):
        lo, hi = sorted([1.0, kernel.e_star(r, nu1) / kernel.e_star(E2, nu2)])
        ks = [stiffness(hoa * a, r * E2, nu1, E2, nu2) / (k_hom * analytic.flat_punch_stiffness(a, kernel.e_star(E2, nu2)))
              for hoa in (0.1, 0.3, 1.0, 3.0, 10.0)]
        assert all(lo * (1 - 1e-6) <= k <= hi * (1 + 1e-6) for k in ks), (r, ks)
        steps = np.diff(ks)
        assert np.all(steps > 0) if r > 1 else np.all(steps < 0), (r, ks)
        coat = kernel.e_star(r, nu1) / kernel.e_star(E2, nu2)
        assert ks[-1] == pytest.approx(coat, rel=0.01), (r, ks)
