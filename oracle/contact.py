"""Contact solves on top of the discrete operator (Sec. 2, inverse problem and adhesion).

Test infrastructure (see ``oracle/__init__``).  Plain FP64 numpy; ``matvec`` is any
callable p -> K p (``operator.matvec_fft`` or ``operator.matvec_dense`` bound to a
sampled kernel).

Conventions (Sec. 2, condition (c)): p > 0 is compressive, tension is p < 0; u is the
surface displacement into the body; f is the indenter height above its lowest
point; d is the indentation depth; the gap is g = u + f - d.  Non-adhesive contact
(Sec. 2: the pressures for a prescribed surface displacement, found by the
conjugate-gradient method of the paper's reference [8]) means p >= 0, g >= 0,
p g = 0; the total force is F = delta^2 sum p.

* ``solve_nonadhesive``  Polonsky-Keer constrained conjugate gradients, the method
  the paper cites as [8], under depth control (d given) or load control (F given,
  d is the multiplier).  Two operator products per iteration, written plainly.
* ``kkt_violation``      complementarity check of a computed solution.
* ``sigma_c``            Eq. (12), the mesh-dependent detachment stress.
* ``boundary_cells``     cells of a contact set with a 4-neighbour outside it (the
  window edge counts as outside): the cells on the rim of the contact area to
  which Sec. 2 applies the detachment test.
* ``solve_fixed_set``    the inverse problem on a fixed contact area, p free in sign.
* ``adhesive_step``      one displacement-controlled step of Sec. 2's adhesive
  procedure: solve on the fixed area, add penetrating cells, detach boundary cells
  whose tension exceeds sigma_c (all at once), repeat until the area is unchanged.
* ``adhesive_ramp``      a sequence of such steps over a list of depths.
* ``solve_fixed_set_force``  the fixed-area problem under load control: the sum of
  p is given and d is unknown (the multiplier of that constraint), by superposition
  of two fixed-area solves (linearity of K).
* ``adhesive_step_force``   the same procedure as ``adhesive_step`` with every
  fixed-area solve carrying the given force; raises ``Detached`` when an area update
  leaves no contact (the force is below what the contact can carry).

Parity status: pinned by tests (KKT, enumeration of every contact set of a tiny
window, NNLS, Hertz, flat punch, thin layer, JKR, Eq. 16, fixed points of the
adhesive rules) - see tests/test_oracle_contact.py.
"""
import numpy as np


class NoConvergence(RuntimeError):
    pass


class Detached(NoConvergence):
    """Under load control the adhesive contact area vanished: the given force is below
    what the contact can carry (the indenter jumps off)."""


class NotPositiveDefinite(NoConvergence):
    """A search direction with non-positive curvature t'Kt <= 0: the operator is not
    positive definite on the contact set, the minimisation has no unique solution and
    the conjugate-gradient steps are undefined (e.g. a negative DC value, reading of
    the k = 0 term, on a period that is small compared with the coating)."""


def _initial_depth_control(matvec, f, d):
    q = np.maximum(d - f, 0.0)
    if not np.any(q > 0):
        return np.zeros_like(f)
    Kq = matvec(q)
    curv = np.sum(q * Kq)
    if not curv > 0.0:
        raise NotPositiveDefinite("non-positive curvature of the initial direction")
    s = np.sum(q * (d - f)) / curv
    return s * q


def solve_nonadhesive(matvec, f, delta, control="depth", target=0.0, tol=1e-12,
                      max_iter=20000, p0=None):
    """Polonsky-Keer CG.  Returns dict(p, d, force, iters, residual, n_contact).

    Iteration (depth control drops the mean shifts and the load rescale):
      Ic = {p > 0};  u = K p;  g = u + f - d
      load control: gbar = mean_Ic g;  g -= gbar;  d += gbar
      G = sum_Ic g^2;  t = g + delta_flag (G/G_old) t on Ic, 0 elsewhere
      r = K t;  load control: r -= mean_Ic r on Ic
      tau = sum_Ic g t / sum_Ic r t
      p -= tau t on Ic;  p[p < 0] = 0
      Iol = {p = 0, g < 0}: delta_flag = 0 and p -= tau g on Iol if Iol non-empty
      load control: p *= F / (delta^2 sum p)
    Stop at the start of an iteration when sqrt(G)/||u||_Ic <= tol and the previous
    iteration changed no cell of the contact set.
    """
    f = np.asarray(f, dtype=np.float64)
    load = control == "force"
    if load:
        W = float(target)
        d = 0.0
        p = np.full_like(f, W / (delta * delta * f.size)) if p0 is None else np.array(p0, dtype=np.float64)
        p *= W / (delta * delta * p.sum())
    else:
        d = float(target)
        p = _initial_depth_control(matvec, f, d) if p0 is None else np.maximum(np.array(p0, dtype=np.float64), 0.0)
    t = np.zeros_like(f)
    G_old = 1.0
    flag = 0.0
    set_changed = True
    res = np.inf
    for it in range(1, max_iter + 1):
        Ic = p > 0
        if not np.any(Ic):
            if load:
                raise NoConvergence("empty contact set under load control")
            return dict(p=p, d=d, force=0.0, iters=it - 1, residual=0.0, n_contact=0)
        u = matvec(p)
        g = u + f - d
        if load:
            gbar = g[Ic].mean()
            g -= gbar
            d += gbar
        G = np.sum(g[Ic] ** 2)
        unorm = np.sqrt(np.sum(u[Ic] ** 2))
        res = np.sqrt(G) / unorm if unorm > 0 else 0.0
        if res <= tol and not set_changed:
            return dict(p=p, d=d, force=delta * delta * p.sum(), iters=it - 1,
                        residual=res, n_contact=int(Ic.sum()))
        t = np.where(Ic, g + flag * (G / G_old) * t, 0.0)
        G_old = G
        r = matvec(t)
        if load:
            r[Ic] -= r[Ic].mean()
        curv = np.sum(r[Ic] * t[Ic])
        if not np.any(t[Ic] != 0.0):
            tau = 0.0                       # the gap is exactly level on the set: no step
        elif not curv > 0.0:
            raise NotPositiveDefinite(f"non-positive curvature t'Kt = {curv:.3e} at iteration {it}")
        else:
            tau = np.sum(g[Ic] * t[Ic]) / curv
        p = np.where(Ic, p - tau * t, p)
        neg = p < 0
        p[neg] = 0.0
        Iol = (p == 0) & (g < 0)
        if np.any(Iol):
            flag = 0.0
            p[Iol] -= tau * g[Iol]
        else:
            flag = 1.0
        set_changed = bool(np.any(neg) or np.any(Iol))
        if load:
            p *= W / (delta * delta * p.sum())
    raise NoConvergence(f"PK-CG: residual {res:.3e} after {max_iter} iterations")


def kkt_violation(matvec, p, f, d):
    """Max violation of p >= 0, g >= 0, p g = 0 relative to max|u| (and the tension)."""
    u = matvec(p)
    g = u + f - d
    scale = max(np.abs(u).max(), 1e-300)
    pscale = max(np.abs(p).max(), 1e-300)
    v_p = max(0.0, -p.min()) / pscale
    v_g = max(0.0, -g.min()) / scale
    v_c = np.abs(g[p > 0]).max() / scale if np.any(p > 0) else 0.0
    return max(v_p, v_g, v_c)


def sigma_c(E1, nu1, dgamma, delta):
    """Eq. (12): sqrt(E1* dgamma / (0.473201 delta)), E1* = E1/(1-nu1^2)."""
    return np.sqrt(E1 / (1.0 - nu1 * nu1) * dgamma / (0.473201 * delta))


def boundary_cells(C):
    """Cells of C with at least one von Neumann neighbour outside C (window edge = outside)."""
    pad = np.zeros((C.shape[0] + 2, C.shape[1] + 2), dtype=bool)
    pad[1:-1, 1:-1] = C
    inner = pad[:-2, 1:-1] & pad[2:, 1:-1] & pad[1:-1, :-2] & pad[1:-1, 2:]
    return C & ~inner


def solve_fixed_set(matvec, C, b, tol=1e-13, max_iter=20000, p0=None):
    """Plain CG for K_CC p_C = b_C with p = 0 outside C (p unrestricted in sign)."""
    p = np.zeros_like(b) if p0 is None else np.where(C, p0, 0.0)
    r = np.where(C, b - matvec(p), 0.0)
    bnorm = np.sqrt(np.sum(b[C] ** 2))
    if bnorm == 0.0:
        return np.zeros_like(b), 0
    s = r.copy()
    rr = np.sum(r * r)
    for it in range(max_iter):
        if np.sqrt(rr) <= tol * bnorm:
            return p, it
        Ks = np.where(C, matvec(s), 0.0)
        curv = np.sum(s * Ks)
        if not curv > 0.0:
            raise NotPositiveDefinite(f"non-positive curvature on the fixed set at iteration {it}")
        a = rr / curv
        p = p + a * s
        r = r - a * Ks
        rr_new = np.sum(r * r)
        s = r + (rr_new / rr) * s
        rr = rr_new
    raise NoConvergence("fixed-set CG did not converge")


def adhesive_step(matvec, f, d, C, sig_c, p_prev=None, tol=1e-13, max_outer=1000):
    """One displacement-controlled step of the adhesive procedure of Sec. 2.

    With the contact area C held fixed the pressure that gives u = d - f on C is
    found (p free in sign); cells outside C that penetrate (g < 0) join; boundary
    cells of C whose tension -p exceeds sigma_c (Eq. 12, strict '>') leave, all at
    once; this repeats until the area does not change.  Returns (p, C, outer, cg_iters).
    """
    C = C.copy()
    seen = set()
    p = p_prev
    total = 0
    for outer in range(1, max_outer + 1):
        p, its = solve_fixed_set(matvec, C, d - f, tol=tol, p0=p)
        total += its
        g = matvec(p) + f - d
        add = ~C & (g < 0)
        detach = boundary_cells(C) & (-p > sig_c)
        if not np.any(add) and not np.any(detach):
            return p, C, outer, total
        key = (C | add) & ~detach
        h = key.tobytes()
        if h in seen:
            raise NoConvergence("contact set cycles")
        seen.add(h)
        C = key
    raise NoConvergence("adhesive outer loop did not settle")


def adhesive_ramp(matvec, f, delta, depths, sig_c, C0=None, tol=1e-13):
    """Run ``adhesive_step`` over the given depths, carrying (p, C) between steps.

    Returns a list of dicts with d, force = delta^2 sum p, n_contact and the
    equivalent contact radius a_eq = sqrt(n delta^2 / pi).
    """
    C = np.zeros(f.shape, dtype=bool) if C0 is None else C0.copy()
    p = None
    out = []
    for d in depths:
        p, C, outer, its = adhesive_step(matvec, f, d, C, sig_c, p_prev=p, tol=tol)
        n = int(C.sum())
        out.append(dict(d=float(d), force=float(delta * delta * p.sum()), n_contact=n,
                        a_eq=float(np.sqrt(n * delta * delta / np.pi)), outer=outer,
                        cg_iters=its, p=p.copy(), C=C.copy()))
    return out


def solve_fixed_set_force(matvec, C, f, P, tol=1e-13):
    """Load control on a fixed area C: p (free in sign, 0 outside C) and d with
    K_CC p_C = (d - f)_C and sum_C p = P (P = F / delta^2).  K is linear, so
    p = p_f + d p_1 with K_CC p_f = -f_C and K_CC p_1 = 1_C, and the sum fixes
    d = (P - sum p_f) / sum p_1 (sum p_1 = 1' K_CC^-1 1 > 0).  Returns (p, d, cg_iters)."""
    pf, i1 = solve_fixed_set(matvec, C, -f, tol=tol)
    p1, i2 = solve_fixed_set(matvec, C, np.ones_like(f), tol=tol)
    d = (P - pf[C].sum()) / p1[C].sum()
    return pf + d * p1, float(d), i1 + i2


def adhesive_step_force(matvec, f, force, delta, C, sig_c, tol=1e-13, max_outer=1000):
    """One load-controlled step of the adhesive procedure of Sec. 2: as ``adhesive_step``
    (solve on the fixed area, add penetrating cells, detach boundary cells whose tension
    exceeds sigma_c, repeat until the area is unchanged) with every fixed-area solve
    carrying the total force F = delta^2 sum p, the depth following from it.  Starts
    from the non-empty area C.  Returns (p, C, d, outer, cg_iters); raises ``Detached``
    when an update leaves no contact."""
    C = C.copy()
    if not C.any():
        raise ValueError("load control needs a non-empty starting area")
    P = force / (delta * delta)
    seen = set()
    total = 0
    for outer in range(1, max_outer + 1):
        p, d, its = solve_fixed_set_force(matvec, C, f, P, tol=tol)
        total += its
        g = matvec(p) + f - d
        add = ~C & (g < 0)
        detach = boundary_cells(C) & (-p > sig_c)
        if not np.any(add) and not np.any(detach):
            return p, C, d, outer, total
        key = (C | add) & ~detach
        if not key.any():
            raise Detached("the contact area vanished under the given force")
        h = key.tobytes()
        if h in seen:
            raise NoConvergence("contact set cycles")
        seen.add(h)
        C = key
    raise NoConvergence("adhesive outer loop did not settle")
