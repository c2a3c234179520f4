"""Displacement-controlled adhesive ramps (loading, then pull-off), as in Sec. 2.

Orchestration only: each step is one bem_solve_contact call with dgamma > 0 at the
step's depth; the pressure and the contact mask carry over from step to step.  The
ramp state can be saved every few steps and a saved ramp resumed: the resumed steps
repeat the same trajectory (same inputs, same device-side arithmetic).
"""
import numpy as np
import torch


def depth_schedule(d_max, d_min, n_load, n_unload):
    """Depths of a loading phase 0 -> d_max and a pull-off phase d_max -> d_min."""
    return np.concatenate([np.linspace(0.0, d_max, n_load), np.linspace(d_max, d_min, n_unload + 1)[1:]])


def run(kernel, height, depths, dgamma, tol=1e-8, max_iter=20000, state=None, checkpoint=None, every=25,
        stream=None, with_state=False):
    """Runs the ramp; returns a list of per-step records (d, force, area, a_eq, n_contact,
    iterations, outer iterations, status).  ``state`` = (step, p, mask) resumes a saved
    ramp; ``checkpoint`` is a path for np.savez every ``every`` steps.  The solves run
    on ``stream`` (default: a stream of the ramp's own, on which the library replays
    its captured iteration graphs; every solve synchronises its stream).
    ``with_state``: return (records, (p, mask)) with the device state after the last
    step, e.g. to continue under force control (``force_run``)."""
    if stream is None:
        stream = torch.cuda.Stream(device=height.device)
    with torch.cuda.stream(stream):
        out, p, mask = _run(kernel, height, depths, dgamma, tol, max_iter, state, checkpoint, every, stream)
    return (out, (p, mask)) if with_state else out


def _run(kernel, height, depths, dgamma, tol, max_iter, state, checkpoint, every, stream):
    N = kernel.N
    dev = height.device
    if state is None:
        start = 0
        p = torch.zeros((N, N), dtype=kernel.torch_dtype, device=dev)
        mask = torch.zeros((N, N), dtype=torch.uint8, device=dev)
    else:
        start = int(state[0])
        p = torch.as_tensor(state[1], dtype=kernel.torch_dtype, device=dev).clone()
        mask = torch.as_tensor(state[2], dtype=torch.uint8, device=dev).clone()
    out = []
    for i in range(start, len(depths)):
        p_new, res = kernel.solve(height, "depth", float(depths[i]), dgamma=dgamma, tol=tol, max_iter=max_iter,
                                  p_init=p, contact_mask=mask, stream=stream)
        p = p_new
        rec = dict(step=i, d=float(depths[i]), force=res["force"], area=res["area"], a_eq=res["a_eq"],
                   n_contact=res["n_contact"], iters=res["iters"], outer=res["outer_iters"], status=res["status"])
        out.append(rec)
        if checkpoint is not None and (i + 1) % every == 0:
            np.savez(checkpoint, step=i + 1, p=p.cpu().numpy(), mask=mask.cpu().numpy(), depths=np.asarray(depths))
    return out, p, mask


def load_state(path):
    z = np.load(path)
    return int(z["step"]), z["p"], z["mask"]


def force_pull_off(solve_depth, forces, d0, state0, F0, stiffness, rtol=2e-3, max_step=np.inf, max_trials=400,
                   max_halvings=14):
    """Force-controlled pull-off over decreasing force targets, as a search over the
    depth-controlled steps of the Sec. 2 procedure.

    ``solve_depth(d, state) -> (state', F, n_contact)`` runs one displacement-controlled
    adhesive step at depth d starting from ``state`` (which it must not modify).  The
    procedure depends on the path (cells detach irreversibly, all boundary cells above
    sigma_c at once), so the search moves the way a slowly released load does: every
    trial starts from the last state whose force is still above the target, and no
    step lowers the depth by more than ``max_step``.  Per target F_t: steps downward
    (secant-sized) until F(d) <= F_t, then false position (Illinois) between the last
    state above and the trial below until |F - F_t| <= rtol * max(|F_t|, |F0|).  A
    step whose force rose (a detachment event) is passed through like any state above
    the target.  A step that loses the whole contact is halved towards the last state;
    when ``max_halvings`` halvings in a row still lose it, the contact cannot carry
    F_t: under force control the indenter jumps off.  ``stiffness`` (dF/dd > 0) sizes
    the first step.

    Returns (records, jumped): one record per reached target (target, d, force,
    n_contact, trials) and whether the jump-off was reached before the targets ran out.
    Raises RuntimeError if a target takes more than ``max_trials`` steps.
    """
    d, state, F, k = float(d0), state0, float(F0), float(stiffness)
    out = []
    for Ft in forces:
        Ft = float(Ft)
        if not Ft < F:
            raise ValueError("force targets must decrease below the current force")
        scale = rtol * max(abs(Ft), abs(F0))
        hi = [d, F, state]                  # last state with F > Ft: every trial starts here
        f_hi = F                            # its force as false position sees it (Illinois-scaled)
        lo = None                           # trial below the target: (d, F as scaled)
        side = 0
        dn = d - min((F - Ft) / k, max_step)
        halvings, trials, done = 0, 0, None
        while True:
            if trials >= max_trials:
                raise RuntimeError(f"force target {Ft} not reached in {max_trials} steps")
            st, Fn, nc = solve_depth(dn, hi[2])
            trials += 1
            if nc == 0:
                halvings += 1
                if halvings > max_halvings:
                    break
                dn = 0.5 * (hi[0] + dn)
                continue
            halvings = 0
            if abs(Fn - Ft) <= scale:
                done = (dn, Fn, st, nc)
                break
            if Fn > Ft:
                if lo is None:              # still above the target: move on down the branch
                    if Fn < hi[1]:
                        k = (hi[1] - Fn) / (hi[0] - dn)
                    hi, f_hi = [dn, Fn, st], Fn
                    dn = dn - min((Fn - Ft) / k, max_step)
                    continue
                hi, f_hi = [dn, Fn, st], Fn
                if side == 1:
                    lo = (lo[0], 0.5 * (lo[1] + Ft))
                side = 1
            else:
                lo = (dn, Fn)
                if side == -1:
                    f_hi = 0.5 * (f_hi + Ft)
                side = -1
            dn = hi[0] + (Ft - f_hi) * (lo[0] - hi[0]) / (lo[1] - f_hi)
        if done is None:
            return out, True
        d, F, state = float(done[0]), done[1], done[2]
        out.append(dict(target=Ft, d=d, force=F, n_contact=done[3], trials=trials))
    return out, False


def force_run(kernel, height, forces, dgamma, d0, p0, mask0, F0, stiffness, tol=1e-9, max_iter=20000, rtol=2e-3,
              max_step=np.inf, stream=None):
    """``force_pull_off`` on the library's depth-controlled adhesive solves: the state is
    the (pressure, contact mask) pair of the last accepted step, copied for every
    trial.  Start from a loaded state (d0, p0, mask0, force F0), e.g. the last step of
    ``run``.  Returns (records, jumped)."""
    if stream is None:
        stream = torch.cuda.Stream(device=height.device)

    def solve_depth(d, state):
        p, mask = state
        m = mask.clone()
        p_new, res = kernel.solve(height, "depth", float(d), dgamma=dgamma, tol=tol, max_iter=max_iter,
                                  p_init=p, contact_mask=m, stream=stream)
        if res["status"] != 0:
            raise RuntimeError(f"adhesive step failed: {res}")
        return (p_new, m), res["force"], res["n_contact"]

    with torch.cuda.stream(stream):
        return force_pull_off(solve_depth, forces, d0, (p0, mask0.clone()), F0, stiffness, rtol=rtol,
                              max_step=max_step)
