"""Learned warm start: solver-generated training data, training, prediction.

Orchestration only: every numerical step runs in libbem.so (contact solves, feature
construction, network forward/backward/Adam, target and pressure scaling); this
module moves device tensors between those calls and picks minibatches.

The network predicts q = p / pbar (pbar = F / L^2, the mean pressure) from the height
map and the layer parameters; the warm start handed to the solver is p_init = pbar q
on the cells where q exceeds a cut (1 by default: the network's confident contact
cells), 0 elsewhere, which the force-controlled solve then rescales to F exactly.
"""
import numpy as np
import torch

from . import bem, inputs


def instance_tensors(insts, device):
    """Stacks same-size instances: heights [B, N, N] float32, params [B, 4] float64
    (h/delta, E1/E2, nu1, nu2), pbar [B] float64 — all on the device."""
    N = insts[0]["N"]
    assert all(i["N"] == N for i in insts)
    heights = torch.tensor(np.stack([i["height"] for i in insts]), dtype=torch.float32, device=device)
    params = torch.tensor([[i["h"] / i["delta"], i["E1"] / i["E2"], i["nu1"], i["nu2"]] for i in insts],
                          dtype=torch.float64, device=device)
    pbar = torch.tensor([i["force"] / (i["N"] * i["delta"]) ** 2 for i in insts], dtype=torch.float64,
                        device=device)
    return heights, params, pbar


def solve_all(insts, heights, p_init=None, tol=1e-8, max_iter=5000, stream=None, kernels=None):
    """Solves every instance (force control, float) with one batched call; returns
    (pressures [B, N, N], results).  ``kernels``: reusable float handles of the grid
    size (rebuilt in place for each instance); by default one handle per instance."""
    own = kernels is None
    if own:
        ks = [bem.Kernel(i["N"], i["delta"], i["h"], i["E1"], i["nu1"], i["E2"], i["nu2"], precision="fp32")
              for i in insts]
    else:
        ks = kernels[:len(insts)]
        for k, i in zip(ks, insts):
            k.rebuild(i["delta"], i["h"], i["E1"], i["nu1"], i["E2"], i["nu2"])
    outs = torch.empty_like(heights)
    probs = [bem.make_problem(heights[b], bem.BEM_CTRL_FORCE, insts[b]["force"], tol=tol, max_iter=max_iter,
                              p_init=None if p_init is None else p_init[b]) for b in range(len(insts))]
    st, res = bem.bem_solve_batch([k.handle for k in ks], probs, [outs[b] for b in range(len(insts))],
                                  stream=stream)
    if own:
        for k in ks:
            k.close()
    return outs, res


def make_dataset(fno, insts, device, tol=1e-8, kernels=None):
    """Features x [B, 7, N, N] and targets q [B, N, N] from solver solutions; ``kernels``
    (optional, at least B handles of the grid size) are rebuilt in place instead of
    creating one handle per instance."""
    heights, params, pbar = instance_tensors(insts, device)
    p, res = solve_all(insts, heights, tol=tol, kernels=kernels)
    B, N = heights.shape[0], heights.shape[-1]
    x = torch.empty((B, 7, N, N), dtype=torch.float32, device=device)
    fno.features(B, N, heights, params, x)
    q = torch.empty_like(heights)
    fno.target(B, N, p, pbar, q)
    torch.cuda.synchronize(device)
    return x, q, res


def train(fno, x, q, steps, batch, lr, seed=0, lr_final=None):
    """Adam on minibatches drawn without replacement per epoch; returns the losses.
    The learning rate decays geometrically to lr_final (if given)."""
    rng = np.random.default_rng(seed)
    B, N = x.shape[0], x.shape[-1]
    losses = []
    order = rng.permutation(B)
    pos = 0
    for s in range(steps):
        if pos + batch > B:
            order = rng.permutation(B)
            pos = 0
        idx = torch.as_tensor(order[pos:pos + batch], device=x.device)
        pos += batch
        xb = x.index_select(0, idx).contiguous()
        qb = q.index_select(0, idx).contiguous()
        rate = lr if lr_final is None else lr * (lr_final / lr) ** (s / max(steps - 1, 1))
        losses.append(fno.train_step(batch, N, xb, qb, rate))
    return losses


# cells per network call in prediction (bounds the network's activation buffers)
PREDICT_CELLS = 1 << 22


def predict(fno, heights, params, pbar, q_min=1.0):
    """Warm-start pressures p_init [B, N, N] for stacked instances: the network runs
    on as many samples per call as PREDICT_CELLS allows; cells with q <= q_min get 0."""
    B, N = heights.shape[0], heights.shape[-1]
    x = torch.empty((B, 7, N, N), dtype=torch.float32, device=heights.device)
    fno.features(B, N, heights, params, x)
    out = torch.empty_like(heights)
    p = torch.empty_like(heights)
    step = max(1, PREDICT_CELLS // (N * N))
    for b0 in range(0, B, step):
        b1 = min(B, b0 + step)
        fno.forward(b1 - b0, N, x[b0:b1], out[b0:b1])
    fno.pressure(B, N, out, pbar, p, q_min=q_min)
    return p


def default_instances(count, N, seed0, workers=None):
    """Rough-surface batch-workload instances at one grid size (height maps included)."""
    heights, insts = inputs.batch_heights(count, N, seed0, workers)
    for b, inst in enumerate(insts):
        inst["height"] = heights[b]
    return insts
