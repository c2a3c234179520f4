"""Displacement-controlled adhesive ramps (loading, then pull-off), as in Sec. 2.

Orchestration only: each step is one bem_solve_contact call with dgamma > 0 at the
step's depth (``run``) or force (``force_steps``, the force control inside the
library); the pressure and the contact mask carry over from step to step.  The
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
    step, e.g. to continue under force control (``force_steps``)."""
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


def force_steps(kernel, height, forces, dgamma, p0, mask0, tol=1e-9, max_iter=20000, stream=None):
    """Load-controlled adhesive steps with the force control inside the library: one
    bem_solve_contact call under force control per target (in the given order), each
    starting from the previous step's pressure and contact mask, the first from (p0,
    mask0), e.g. the state after the last step of ``run``.  Returns (records, jumped):
    one record per carried target (target, d, force, area, a_eq, n_contact, iters,
    outer, status) and whether a target detached the whole area (BEM_EDETACHED: under
    load control the indenter jumps off there)."""
    if stream is None:
        stream = torch.cuda.Stream(device=height.device)
    from . import bem
    p, mask = p0, mask0.clone()
    out = []
    with torch.cuda.stream(stream):
        for Ft in forces:
            m = mask.clone()
            p_new, res = kernel.solve(height, "force", float(Ft), dgamma=dgamma, tol=tol, max_iter=max_iter,
                                      p_init=p, contact_mask=m, stream=stream)
            if res["status"] == bem.BEM_EDETACHED:
                return out, True
            out.append(dict(target=float(Ft), d=res["depth"], force=res["force"], area=res["area"],
                            a_eq=res["a_eq"], n_contact=res["n_contact"], iters=res["iters"],
                            outer=res["outer_iters"], status=res["status"]))
            p, mask = p_new, m
    return out, False
