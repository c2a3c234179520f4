#!/usr/bin/env python
"""Benchmark of the FFT-BEM hot path on one GB300 (or N independent replicas).

Workload (one step): a cold-start FP32 contact solve at N = 2048 (4096^2 padded
period) of a seeded self-affine rough surface (Hurst 0.7, rms slope 0.1, roll-off
L/8) pressed into a coated half-space drawn from the rough-surface batch
distribution, under force control, to a relative gap residual of 1e-8.  Every
row of the hot path runs inside the step: the operator products (row FFT, fused
column FFT x K^ x inverse FFT, inverse row FFT), the constrained-CG sweeps with
double reductions, and the force/area outputs.  The compliance table is built
once per instance before timing.

value = operator products per second over the whole job (all ranks); the step
time is the time to converge.  Extra keys: matvec-only throughput on 8 distinct
inputs (larger than L2), the roofline of the dominant pass, the end-to-end number
through the C ABI with host buffers, the CPU oracle timed on a bounded sample, the
256-instance batch of uneven grids (batched vs one after another), the adhesive
ramp (200 displacement steps at N = 512) and the learned warm start.  A comparison
line times the same products through torch.fft (cuFFT R2C, pointwise K^, C2R); it
is never part of the library's path.

--impl reference times the CPU FP64 oracle (the method written plainly, see
oracle/) on the same workload: each step is one N = 2048 operator product.
"""
import argparse
import json
import os
import statistics
import subprocess
import sys
import tempfile
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

from paper_1807_01885_gb300.tuning import RadixCache  # noqa: E402  (no GPU or library needed)

METRIC = "FFT-BEM matvecs/s at N=2048; time-to-converge: warm-start+batch vs plain"
UNIT = "matvecs/s"
N_GRID = 2048
N_INST = 2
SEED0 = 40000000
TOL = 1e-8


def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=20)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--batch", type=int, default=256, help="instances of the batch workload (0: skip)")
    ap.add_argument("--warmstart-steps", type=int, default=2000, help="training steps of the learned warm start")
    ap.add_argument("--warmstart-test", type=int, default=16, help="held-out N=2048 instances of the warm start")
    ap.add_argument("--warmstart", type=int, default=20000,
                    help="training solutions for the learned warm start (0: skip)")
    ap.add_argument("--adhesive", type=int, default=1,
                    help="run the adhesive ramp workload (N=512, 200 steps, FP32; 0: skip)")
    ap.add_argument("--punch", type=int, default=1,
                    help="run the flat-punch stiffness sweep (N=256, 20 cells, FP64 and FP32; 0: skip)")
    ap.add_argument("--radix", default=None, metavar="ROWS,COLS",
                    help="log2 FFT radices to use instead of the autotuner's choice (e.g. 4,4); for "
                         "profiling runs, where the autotuner's timings would be taken under the profiler")
    ap.add_argument("--probe-matvec", type=int, default=0, metavar="K",
                    help="only run K operator products at N=2048 (FP32) and exit: the small case "
                         "that the ncu summaries under profiles/ capture")
    ap.add_argument("--probe-fno", type=int, default=0, metavar="K",
                    help="only run K forwards of the warm-start network (width 32, 16 modes, 4 layers) on one "
                         "N=2048 sample and exit: the case of the network's ncu launch list")
    return ap.parse_args()


def aggregate_ranks(torch, ms, units, device):
    """Whole-job figures of a timed region run on every rank: the slowest rank's
    time (max) and the units all ranks processed (sum).  Returns (ms, units); a
    single process returns its own values."""
    if not (torch.distributed.is_available() and torch.distributed.is_initialized()):
        return float(ms), float(units)
    t = torch.tensor([float(ms), float(units)], dtype=torch.float64, device=device)
    tm, tu = t[0:1].clone(), t[1:2].clone()
    torch.distributed.all_reduce(tm, op=torch.distributed.ReduceOp.MAX)
    torch.distributed.all_reduce(tu, op=torch.distributed.ReduceOp.SUM)
    return float(tm[0]), float(tu[0])


def dist_env():
    rank = int(os.environ.get("RANK", "0"))
    world = int(os.environ.get("WORLD_SIZE", "1"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return rank, world, local


def peaks():
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as fh:
            d = json.load(fh)
        return float(d["hbm_gbs"]), "measured"
    except Exception:
        return 6800.0, "fallback"


def alg_bytes(N, elem=4):
    """Algorithmic DRAM bytes of one product (pruned, padded half never stored):
    rows fwd: read p 4N^2, write spectrum 8N(N+1); columns: read+write spectrum
    16N(N+1), read table 4(N+1)^2; rows inv: read spectrum 8N(N+1), write u 4N^2."""
    c = 2 * elem
    row_fwd = elem * N * N + c * N * (N + 1)
    col = 2 * c * N * (N + 1) + elem * (N + 1) ** 2
    row_inv = c * N * (N + 1) + elem * N * N
    return row_fwd, col, row_inv


def library_fft_khat(torch, table, N, dtype):
    """K^ on the half grid M x (N+1) of a length-M real FFT along rows (M = 2N), from
    the folded (N+1) x (N+1) table the library exports: period row i is table row
    min(i, M - i).  For the comparison line only."""
    return torch.cat([table, table[1:N].flip(0)], 0).to(dtype).contiguous()


def library_fft_matvec(torch, khat_half, p, pad):
    """u = K p by the vendor FFT behind torch.fft (cuFFT on a GPU): copy p into the
    zero-padded M x M buffer ``pad`` (zero outside the window), R2C, multiply by K^,
    C2R with the 1/M^2 normalisation, crop.  The comparison line of the benchmark,
    never the product path."""
    N = p.shape[0]
    pad[:N, :N].copy_(p)
    U = torch.fft.irfft2(torch.fft.rfft2(pad) * khat_half, s=tuple(pad.shape))
    return U[:N, :N]


def library_fft_bench(torch, k, P, U, stream, reps=100):
    """Products per second of the torch.fft comparison on the inputs of the
    matvec-only loop, and its relative L2 difference from the library's product."""
    N = P[0].shape[0]
    kh = library_fft_khat(torch, k.table(device=P[0].device), N, torch.float32)
    pad = torch.zeros((2 * N, 2 * N), dtype=torch.float32, device=P[0].device)
    out = [library_fft_matvec(torch, kh, x, pad).clone() for x in P]
    rel = max(float(torch.linalg.vector_norm((a - b).double()) / torch.linalg.vector_norm(b.double()))
              for a, b in zip(out, U))
    torch.cuda.synchronize()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    for j in range(reps):
        library_fft_matvec(torch, kh, P[j % len(P)], pad)
    e1.record(stream)
    torch.cuda.synchronize()
    ms = e0.elapsed_time(e1) / reps
    return {"impl": "torch.fft rfft2 x K^ x irfft2 (cuFFT), FP32, zero-padded 2N x 2N",
            "value": 1000.0 / ms, "unit": UNIT, "ms_per_matvec": ms, "rel_l2_vs_library": rel}


def fft_nominal_flops(N):
    """Nominal flops of one product (5 M log2 M per complex length-M transform, a real
    one counted as half): two row passes of N real transforms, and N + 1 columns of a
    forward and an inverse complex transform, M = 2N."""
    M = 2 * N
    c = 5.0 * M * np.log2(M)
    return 2 * N * (c / 2) + (N + 1) * 2 * c


def fp64_bench(torch, bem, inst, stream, reps=20):
    """The FP64 product at N = 2048 against a cuBLAS DGEMM timed in the same run: the
    double path is bound by the FP64 pipe, so its roofline is a flop rate."""
    N = inst["N"]
    k = bem.Kernel(N, inst["delta"], inst["h"], inst["E1"], inst["nu1"], inst["E2"], inst["nu2"], precision="fp64")
    try:
        dev = torch.device("cuda", torch.cuda.current_device())
        P = [torch.rand((N, N), dtype=torch.float64, device=dev) for _ in range(2)]
        U = [torch.empty_like(x) for x in P]
        for j in range(2):
            k.matvec(P[j], U[j])
        torch.cuda.synchronize()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        for j in range(reps):
            k.matvec(P[j % 2], U[j % 2])
        e1.record(stream)
        torch.cuda.synchronize()
        ms = e0.elapsed_time(e1) / reps
    finally:
        k.close()
    n = 4096
    A = torch.randn((n, n), dtype=torch.float64, device=dev)
    B = torch.randn((n, n), dtype=torch.float64, device=dev)
    for _ in range(2):
        torch.matmul(A, B)
    torch.cuda.synchronize()
    e0.record(stream)
    for _ in range(10):
        torch.matmul(A, B)
    e1.record(stream)
    torch.cuda.synchronize()
    gemm = 2.0 * n ** 3 / (e0.elapsed_time(e1) / 10 * 1e-3) / 1e12
    tf = fft_nominal_flops(N) / (ms * 1e-3) / 1e12
    return {"ms_per_matvec": ms, "nominal_gflop": fft_nominal_flops(N) / 1e9, "tflops": tf,
            "dgemm_tflops_measured": gemm, "frac_of_dgemm": tf / gemm,
            "note": "FP64 product (nominal transform flops) against cuBLAS DGEMM 4096^3 in the same run"}


class Clocks:
    """nvidia-smi sampling of SM clocks and throttle reasons during the timed region."""

    def __init__(self, index):
        self.index = index
        self.proc = None
        self.path = None

    def start(self):
        q = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
             "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
             "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")
        fd, self.path = tempfile.mkstemp(suffix=".csv")
        os.close(fd)
        try:
            self.proc = subprocess.Popen(["nvidia-smi", "-i", str(self.index), f"--query-gpu={q}",
                                          "--format=csv,noheader,nounits", "-lms", "200"],
                                         stdout=open(self.path, "w"), stderr=subprocess.DEVNULL)
        except (OSError, FileNotFoundError):
            self.proc = None

    def stop(self):
        if self.proc is None:
            return None
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except subprocess.TimeoutExpired:
            self.proc.kill()
        rows = []
        for line in open(self.path):
            parts = [x.strip() for x in line.split(",")]
            if len(parts) < 9:
                continue
            try:
                rows.append(parts)
            except ValueError:
                pass
        os.unlink(self.path)
        if not rows:
            return None
        sm = [float(r[1]) for r in rows if r[1].replace(".", "").isdigit()]
        mx = [float(r[2]) for r in rows if r[2].replace(".", "").isdigit()]
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        reasons = sorted({names[i] for r in rows for i in range(4) if "Active" in r[5 + i] and "Not" not in r[5 + i]})
        return {"sm_mhz": statistics.median(sm) if sm else None, "sm_max_mhz": max(mx) if mx else None,
                "reasons": reasons, "samples": len(rows)}


PROFILE = os.path.join(ROOT, "profiles", "col_pass_pair_N2048_fp32.md")
# the sources of the three FFT passes (the column pass, its FFT and its launch);
# a change to any of them invalidates the captured traffic
PROFILED_SOURCES = ["paper_1807_01885_gb300/csrc/matvec_reg.cuh", "paper_1807_01885_gb300/csrc/fft_reg.cuh",
                    "paper_1807_01885_gb300/csrc/fft_pair.cuh", "paper_1807_01885_gb300/csrc/matvec_f32.cu"]


def profiled_traffic():
    """DRAM bytes per launch of the column pass from the committed ncu summary, or None
    when the kernel sources changed since that capture."""
    import hashlib
    try:
        text = open(PROFILE).read()
    except OSError:
        return None
    fields = dict(line.strip().split(": ", 1) for line in text.splitlines()
                  if line.strip().startswith(("traffic_bytes_per_launch:", "source_sha256:")))
    h = hashlib.sha256()
    for f in PROFILED_SOURCES:
        h.update(open(os.path.join(ROOT, f), "rb").read())
    if fields.get("source_sha256") != h.hexdigest():
        return None
    return int(fields["traffic_bytes_per_launch"])


def make_instances(torch, dev, bem, inputs, radix):
    out = []
    for i in range(N_INST):
        inst = inputs.batch_instance(SEED0 + i, sizes=(N_GRID,))
        k = bem.Kernel(N_GRID, inst["delta"], inst["h"], inst["E1"], inst["nu1"], inst["E2"], inst["nu2"],
                       precision="fp32")
        radix.apply(k)
        f = torch.tensor(inst["height"], dtype=torch.float32, device=dev)
        out.append(dict(inst=inst, kernel=k, f=f, p=torch.empty_like(f)))
    return out


BATCH_SEED0 = 20260000


def batch_bench(torch, dev, bem, inputs, n_inst, radix):
    """Rough-surface batch workload: n_inst instances, N drawn from {128, 256, 512, 1024},
    FP32, force control to 1e-8; one bem_solve_batch call against the same instances
    solved one after another on one stream (both replay the handles' iteration graphs)."""
    insts = [inputs.batch_instance(BATCH_SEED0 + i) for i in range(n_inst)]
    ks, probs, hts, outs = [], [], [], []
    for inst in insts:
        k = bem.Kernel(inst["N"], inst["delta"], inst["h"], inst["E1"], inst["nu1"], inst["E2"], inst["nu2"],
                       precision="fp32")
        radix.apply(k)
        ht = torch.tensor(inst["height"], dtype=torch.float32, device=dev)
        ks.append(k)
        hts.append(ht)
        outs.append(torch.empty_like(ht))
        probs.append(bem.make_problem(ht, bem.BEM_CTRL_FORCE, inst["force"], tol=TOL, max_iter=5000))
    s = torch.cuda.Stream(device=dev)
    handles = [k.handle for k in ks]
    with torch.cuda.stream(s):
        st, _ = bem.bem_solve_batch(handles, probs, outs, stream=s)          # warm-up: graphs captured
        s.synchronize()
        t0 = time.perf_counter()
        st, res = bem.bem_solve_batch(handles, probs, outs, stream=s)
        s.synchronize()
        t_batch = time.perf_counter() - t0
        # warm-up of the one-after-another path (each handle's own loop graph)
        for k, pr, o in zip(ks, probs, outs):
            bem.bem_solve_contact(k.handle, pr, o, stream=s)
        s.synchronize()
        t0 = time.perf_counter()
        seq = [bem.bem_solve_contact(k.handle, pr, o, stream=s) for k, pr, o in zip(ks, probs, outs)]
        s.synchronize()
        t_seq = time.perf_counter() - t0
    mv = sum(r["matvecs"] for r in res)
    sizes = {}
    for inst in insts:
        sizes[inst["N"]] = sizes.get(inst["N"], 0) + 1
    for k in ks:
        k.close()
    return {"instances": n_inst, "sizes": {str(a): b for a, b in sorted(sizes.items())}, "status": int(st),
            "all_converged": all(r["status"] == 0 for r in res),
            "batch_wall_ms": 1000 * t_batch, "sequential_wall_ms": 1000 * t_seq,
            "speedup": t_seq / t_batch, "instances_per_s": n_inst / t_batch,
            "matvecs": mv, "matvecs_per_s": mv / t_batch,
            "fft_log2_radix": {str(n): list(radix.by_size[n]) for n in sorted(sizes)},
            "seeds": f"{BATCH_SEED0}..{BATCH_SEED0 + n_inst - 1}"}


def adhesive_bench(torch, dev, bem, inputs):
    """Adhesive ramp (Sec. 2 procedure, Eq. 12): sphere R = 1 on a coating E1 = 0.2,
    h = a_max/2, over E2 = 1, nu = 0.3; N = 512, L = 4 a_max with a_max = 0.1; the work
    of adhesion from a Tabor parameter of 5 with z0 = delta; 100 loading steps to
    d_max = a_max^2/R, then 100 unloading steps to -d_max; FP32, tol 1e-7.  Timed on
    one stream (the ramp driver's own): wall time of the 200 steps."""
    from paper_1807_01885_gb300 import ramp
    N, R, E1, E2, nu = 512, 1.0, 0.2, 1.0, 0.3
    a_max = 0.1
    delta = 4 * a_max / N
    h = 0.5 * a_max
    E1s = E1 / (1 - nu * nu)
    mu = 5.0
    dg = E1s * np.sqrt(mu ** 3 * delta ** 3 / R)
    d_max = a_max ** 2 / R
    f = torch.tensor(inputs.sphere_height(N, delta, R), device=dev, dtype=torch.float32)
    depths = np.concatenate([np.linspace(0, d_max, 101)[1:], np.linspace(d_max, -d_max, 101)[1:]])
    s = torch.cuda.Stream(device=dev)
    with bem.Kernel(N, delta, h, E1, nu, E2, nu, precision="fp32") as k:
        ramp.run(k, f, depths[:5], dg, tol=1e-7, stream=s)              # graph capture, warm caches
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        out = ramp.run(k, f, depths, dg, tol=1e-7, stream=s)
        torch.cuda.synchronize()
        dt = time.perf_counter() - t0
    return {"N": N, "steps": len(depths), "wall_s": dt, "ms_per_step": 1000 * dt / len(depths),
            "cg_iters": int(sum(r["iters"] for r in out)), "outer_passes": int(sum(r["outer"] for r in out)),
            "pull_off_force": float(min(r["force"] for r in out)),
            "all_converged": all(r["status"] == 0 for r in out),
            "contact_lost_after_step": int(max([i for i, r in enumerate(out) if r["n_contact"] > 0], default=-1)),
            "dtype": "f32", "tabor": mu}


def punch_sweep_bench(torch, dev, bem, inputs):
    """Flat-punch stiffness sweep: rigid cylindrical punch of radius a = 64 cells on a
    coating, L = 4a, N = 256, nu1 = 0.3, nu2 = 0.45, h/a in {0.1, 0.3, 1, 3, 10} x E1/E2
    in {0.1, 0.5, 2, 10}, depth control, FP64 and FP32 (literal k = 0 rule).  Stiffness
    F/d normalised by the same grid's homogeneous punch and by 2aE2*; wall time of the
    20 solves per precision (tables built inside the timed loop, one handle per cell)."""
    N, delta, a = 256, 1.0, 64.0
    E2, nu1, nu2 = 1.0, 0.3, 0.45
    d = 1e-3 * a
    hoa, ratios = (0.1, 0.3, 1.0, 3.0, 10.0), (0.1, 0.5, 2.0, 10.0)
    f = inputs.flat_punch_height(N, delta, a)
    es2 = E2 / (1 - nu2 * nu2)
    out = {"N": N, "a_cells": a, "h_over_a": list(hoa), "E1_over_E2": list(ratios), "dc_mode": 1}
    s = torch.cuda.Stream(device=dev)
    for precision, dt in (("fp64", torch.float64), ("fp32", torch.float32)):
        fd = torch.tensor(f, device=dev, dtype=dt)
        tol = 1e-12 if precision == "fp64" else 1e-8

        def stiff(h, E1, n1, Es, ns):
            with bem.Kernel(N, delta, h, E1, n1, Es, ns, precision=precision, dc_mode=bem.BEM_DC_ZERO,
                            stream=s) as k:
                _, res = k.solve(fd, "depth", d, tol=tol, stream=s)
            return res["force"] / d, res["status"]

        k_hom, _ = stiff(np.inf, 1.0, 0.3, 1.0, 0.3)
        norm = k_hom / (2 * a * 1.0 / (1 - 0.09))
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        table, ok = [], True
        for r in ratios:
            row = []
            for x in hoa:
                kv, st = stiff(x * a, r * E2, nu1, E2, nu2)
                ok = ok and st == 0
                row.append(kv / (norm * 2 * a * es2))
            table.append(row)
        torch.cuda.synchronize()
        out[precision] = {"wall_ms": 1000 * (time.perf_counter() - t0), "solves": len(ratios) * len(hoa),
                          "stiffness_over_2aE2star": table, "homogeneous_grid_factor": norm, "all_converged": ok}
    out["fp32_vs_fp64_max_rel"] = float(max(abs(a_ / b_ - 1) for ra, rb in zip(out["fp32"]["stiffness_over_2aE2star"],
                                                                             out["fp64"]["stiffness_over_2aE2star"])
                                        for a_, b_ in zip(ra, rb)))
    return out


WS_TRAIN_SEED0 = 30000000
WS_TEST_SEED0 = 40000000


def warm_start_bench(torch, dev, bem, n_train, steps, n_test, batch=16):
    """Learned warm start (the learned-warm-start workload): the network (4 layers,
    width 32, 16 modes) is trained here on n_train solver solutions at N = 256 of the
    rough-surface workload (seeds 30000000 + i), then seeds FP32 force-controlled solves
    to 1e-8 of n_test held-out N = 2048 instances (seeds 40000000 + i).  Timed on one
    stream: cold and seeded solves one after another and batched, the network's
    inference separately; and the same at the training resolution (32 instances)."""
    from paper_1807_01885_gb300 import warmstart
    net = bem.Fno(width=32, modes=16, layers=4, hidden=64)
    rng = np.random.default_rng(7)
    cnt = net.count
    init = np.concatenate([rng.standard_normal(32 * 7) / np.sqrt(7), np.zeros(32),
                           rng.random(2 * 4 * 32 * 32 * 32 * 16) / (32 * 32),
                           rng.standard_normal(4 * 32 * 32) / np.sqrt(32), np.zeros(4 * 32),
                           rng.standard_normal(64 * 32) / np.sqrt(32), np.zeros(64),
                           rng.standard_normal(64) / 8.0, np.zeros(1)]).astype(np.float32)
    assert init.size == cnt
    net.set_params(torch.tensor(init, device=dev))
    Nt = 256
    t0 = time.perf_counter()
    insts = warmstart.default_instances(n_train, Nt, WS_TRAIN_SEED0)
    t_gen = time.perf_counter() - t0
    # training set: solver solutions of every instance, a pool of handles rebuilt in place
    t0 = time.perf_counter()
    chunk = 256
    pool = [bem.Kernel(Nt, 1.0 / Nt, 0.1, 1.0, 0.3, 1.0, 0.3, precision="fp32") for _ in range(min(chunk, n_train))]
    x = torch.empty((n_train, 7, Nt, Nt), dtype=torch.float32, device=dev)
    q = torch.empty((n_train, Nt, Nt), dtype=torch.float32, device=dev)
    iters_train = []
    for c in range(0, n_train, chunk):
        xc, qc, res = warmstart.make_dataset(net, insts[c:c + chunk], dev, kernels=pool)
        x[c:c + xc.shape[0]].copy_(xc)
        q[c:c + qc.shape[0]].copy_(qc)
        iters_train += [r["iters"] for r in res]
        del xc, qc
    for k in pool:
        k.close()
    torch.cuda.synchronize()
    t_data = time.perf_counter() - t0
    t0 = time.perf_counter()
    losses = warmstart.train(net, x, q, steps=steps, batch=batch, lr=2e-3, lr_final=1e-4)
    torch.cuda.synchronize()
    t_train = time.perf_counter() - t0
    del x, q
    torch.cuda.empty_cache()
    test = warmstart.default_instances(n_test, N_GRID, WS_TEST_SEED0)
    heights, params, pbar = warmstart.instance_tensors(test, dev)
    s = torch.cuda.Stream(device=dev)
    ks = [bem.Kernel(i["N"], i["delta"], i["h"], i["E1"], i["nu1"], i["E2"], i["nu2"], precision="fp32")
          for i in test]
    outs = torch.empty_like(heights)

    def one_by_one(p_init=None):
        rs = []
        for kk, i, b in zip(ks, test, range(len(test))):
            rs.append(kk.solve(heights[b], "force", i["force"], tol=TOL, p_init=None if p_init is None else p_init[b],
                               p_out=outs[b], stream=s)[1])
        s.synchronize()
        return rs

    def batched(p_init=None):
        probs = [bem.make_problem(heights[b], bem.BEM_CTRL_FORCE, test[b]["force"], tol=TOL, max_iter=5000,
                                  p_init=None if p_init is None else p_init[b]) for b in range(len(test))]
        _, rs = bem.bem_solve_batch([kk.handle for kk in ks], probs, [outs[b] for b in range(len(test))], stream=s)
        s.synchronize()
        return rs

    with torch.cuda.stream(s):
        one_by_one()                                                     # graph capture, warm caches
        batched()
        p_w = warmstart.predict(net, heights, params, pbar)
        one_by_one(p_w)
        batched(p_w)
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        r_cold = one_by_one()
        t_cold = time.perf_counter() - t0
        t0 = time.perf_counter()
        rb_cold = batched()
        t_cold_b = time.perf_counter() - t0
        t0 = time.perf_counter()
        p_init = warmstart.predict(net, heights, params, pbar)
        torch.cuda.synchronize()
        t_pred = time.perf_counter() - t0
        t0 = time.perf_counter()
        r_warm = one_by_one(p_init)
        t_warm = time.perf_counter() - t0
        t0 = time.perf_counter()
        p_init = warmstart.predict(net, heights, params, pbar)
        rb_warm = batched(p_init)
        t_warm_b = time.perf_counter() - t0
        # the same at the training resolution: 32 held-out N = 256 instances, solved
        # in one batch call on a pool of handles rebuilt in place for each instance
        # (the rebuild is inside both timed regions)
        small = warmstart.default_instances(32, Nt, WS_TEST_SEED0)
        hs, ps, pbs = warmstart.instance_tensors(small, dev)
        spool = [bem.Kernel(Nt, 1.0 / Nt, 0.1, 1.0, 0.3, 1.0, 0.3, precision="fp32") for _ in small]
        warmstart.solve_all(small, hs, stream=s, kernels=spool)
        warmstart.solve_all(small, hs, p_init=warmstart.predict(net, hs, ps, pbs), stream=s, kernels=spool)
        s.synchronize()
        t0 = time.perf_counter()
        _, rs_cold = warmstart.solve_all(small, hs, stream=s, kernels=spool)
        s.synchronize()
        ts_cold = time.perf_counter() - t0
        t0 = time.perf_counter()
        ps_init = warmstart.predict(net, hs, ps, pbs)
        s.synchronize()
        ts_pred = time.perf_counter() - t0
        t0 = time.perf_counter()
        ps_init = warmstart.predict(net, hs, ps, pbs)
        _, rs_warm = warmstart.solve_all(small, hs, p_init=ps_init, stream=s, kernels=spool)
        s.synchronize()
        ts_warm = time.perf_counter() - t0
    for kk in ks + spool:
        kk.close()
    net.close()
    it = lambda rs: [r["iters"] for r in rs]
    return {"train_samples": n_train, "train_N": Nt, "train_steps": steps, "batch": batch,
            "train_seeds": f"{WS_TRAIN_SEED0}..{WS_TRAIN_SEED0 + n_train - 1}", "q_min": 1.0,
            "generate_s": t_gen, "data_s": t_data, "train_s": t_train,
            "train_solve_iters_mean": float(np.mean(iters_train)),
            "loss_first20": float(np.mean(losses[:20])), "loss_last20": float(np.mean(losses[-20:])),
            "test_N": N_GRID, "test_instances": n_test, "test_seeds": f"{WS_TEST_SEED0}..{WS_TEST_SEED0 + n_test - 1}",
            "inference_ms_per_instance": 1000 * t_pred / n_test,
            "one_after_another": {"cold_ms_per_solve": 1000 * t_cold / n_test,
                                  "warm_plus_inference_ms_per_solve": 1000 * (t_warm + t_pred) / n_test,
                                  "cold_iters_mean": float(np.mean(it(r_cold))),
                                  "warm_iters_mean": float(np.mean(it(r_warm)))},
            "batched": {"cold_ms_per_solve": 1000 * t_cold_b / n_test,
                        "warm_plus_inference_ms_per_solve": 1000 * t_warm_b / n_test,
                        "cold_iters_mean": float(np.mean(it(rb_cold))),
                        "warm_iters_mean": float(np.mean(it(rb_warm)))},
            "at_training_resolution": {"N": Nt, "instances": len(small),
                                       "cold_batch_ms": 1000 * ts_cold, "inference_batch_ms": 1000 * ts_pred,
                                       "warm_plus_inference_batch_ms": 1000 * ts_warm,
                                       "cold_iters_mean": float(np.mean(it(rs_cold))),
                                       "warm_iters_mean": float(np.mean(it(rs_warm)))},
            "all_converged": all(r["status"] == 0 for r in r_cold + r_warm + rb_cold + rb_warm + rs_cold + rs_warm)}


_ORACLE_CASE = {}


def _oracle_case(N=N_GRID):
    """The oracle's padded K^ grid of the first timed instance and a pressure field."""
    if N not in _ORACLE_CASE:
        from oracle import operator
        from paper_1807_01885_gb300 import inputs
        inst = inputs.batch_instance(SEED0, sizes=(N,))
        Kg = operator.khat_grid(N, inst["delta"], inst["h"], inst["E1"], inst["nu1"], inst["E2"], inst["nu2"])
        _ORACLE_CASE[N] = (Kg, np.random.default_rng(0).random((N, N)))
    return _ORACLE_CASE[N]


def cpu_oracle_matvecs():
    """One N = 2048 product of the FP64 oracle (its own radix-2 FFT), timed."""
    from oracle import operator
    Kg, p = _oracle_case()
    t0 = time.perf_counter()
    operator.matvec_fft(Kg, p)
    return time.perf_counter() - t0


def cpu_library_fft(reps=4, N=N_GRID):
    """The same FP64 product through scipy's FFT (pocketfft) on every host core: the
    'reasonable CPU' comparison next to the one-thread oracle.  Returns a JSON dict."""
    import scipy.fft as sfft
    from oracle import operator
    Kg, p = _oracle_case(N)
    M = 2 * N
    kh = np.ascontiguousarray(Kg[:, :N + 1])
    pad = np.zeros((M, M))
    cores = os.cpu_count() or 1

    def product():
        pad[:N, :N] = p
        return sfft.irfft2(sfft.rfft2(pad, workers=cores) * kh, s=(M, M), workers=cores)[:N, :N]

    u = product()
    ref = operator.matvec_fft(Kg, p) if N <= 256 else None
    t0 = time.perf_counter()
    for _ in range(reps):
        product()
    dt = (time.perf_counter() - t0) / reps
    out = {"kind": "library FFT (scipy.fft pocketfft, FP64), not the oracle", "value": 1.0 / dt, "unit": UNIT,
           "cores": cores, "sample": f"{reps} FP64 products at N={N} after 1 untimed"}
    if ref is not None:
        out["rel_l2_vs_oracle"] = float(np.linalg.norm(u - ref) / np.linalg.norm(ref))
    return out


def run_reference(args):
    rank, world, _ = dist_env()
    if world > 1 and rank != 0:
        return
    # every requested step is one full N = 2048 oracle product (about 7 s on one Grace
    # core): 20 steps and 3 warm-up steps take under three minutes
    n_warm = args.warmup
    n_timed = max(1, args.steps)
    for _ in range(n_warm):
        cpu_oracle_matvecs()
    times = [cpu_oracle_matvecs() for _ in range(n_timed)]
    total = sum(times)
    value = n_timed / total
    line = {
        "impl": "reference", "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": args.gpus,
        "steps": n_timed, "warmup": n_warm, "ms_per_step": 1000 * total / n_timed,
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
        "data": "synthetic",
        "config": {"workload": f"oracle FFT-BEM operator product, N={N_GRID} (4096^2 period), rough-surface "
                               "pressures, coated half-space", "N": N_GRID},
        "cpu_baseline": {"value": value, "unit": UNIT, "cores": 1, "kind": "oracle",
                         "sample": f"{n_timed} timed FP64 products at N={N_GRID} after {n_warm} untimed "
                                   "(one product per step; numpy radix-2 FFT, one thread)"},
        "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }
    print(json.dumps(line), flush=True)


def run_ours(args):
    import torch
    rank, world, local = dist_env()
    from paper_1807_01885_gb300 import bem, build, inputs
    if local == 0 or world == 1:
        build.build()
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl", init_method="env://")
        dist.barrier()
        build.build()
    dev = torch.device(f"cuda:{local}")
    torch.cuda.set_device(dev)
    # a non-default stream: solves replay their captured CG iteration graphs
    stream = torch.cuda.Stream(device=dev)
    torch.cuda.set_stream(stream)
    radix = RadixCache(tuple(int(x) for x in args.radix.split(",")) if args.radix else None)
    insts = make_instances(torch, dev, bem, inputs, radix)

    def step(i):
        c = insts[i % N_INST]
        _, res = c["kernel"].solve(c["f"], "force", c["inst"]["force"], tol=TOL, max_iter=5000, p_out=c["p"],
                                   stream=stream)
        if res["status"] != 0:
            raise RuntimeError(f"solve failed: {res}")
        return res

    for i in range(args.warmup):
        step(i)
    # timed region (pass timing off: nothing but the solves runs in it)
    clocks = Clocks(local)
    if world > 1:
        torch.distributed.barrier()
    torch.cuda.synchronize()
    clocks.start()
    launches0 = bem.bem_launch_count()
    ev0 = torch.cuda.Event(enable_timing=True)
    ev1 = torch.cuda.Event(enable_timing=True)
    ev0.record(stream)
    results = [step(i) for i in range(args.steps)]
    ev1.record(stream)
    torch.cuda.synchronize()
    launches = bem.bem_launch_count() - launches0
    ms = ev0.elapsed_time(ev1)
    if world > 1:
        torch.distributed.barrier()
    clk = clocks.stop()
    mv = sum(r["matvecs"] for r in results)
    iters = sum(r["iters"] for r in results)
    ms_max, mv_all = aggregate_ranks(torch, ms, mv, dev)
    value = mv_all / (ms_max / 1000.0)

    # second timed region, same steps with the library recording CUDA events around
    # every pass on the launching stream (plain launches): the per-pass durations
    for c in insts:
        bem.bem_set_pass_timing(c["kernel"].handle, True)
        bem.bem_pass_timing(c["kernel"].handle, reset=True)
    torch.cuda.synchronize()
    for i in range(args.steps):
        step(i)
    torch.cuda.synchronize()
    pass_ms, pass_n = [0.0, 0.0, 0.0], [0, 0, 0]
    for c in insts:
        m_, n_ = bem.bem_pass_timing(c["kernel"].handle, reset=True)
        bem.bem_set_pass_timing(c["kernel"].handle, False)
        pass_ms = [a + b for a, b in zip(pass_ms, m_)]
        pass_n = [a + b for a, b in zip(pass_n, n_)]
    pass_mean = [pass_ms[i] / max(pass_n[i], 1) for i in range(3)]

    # matvec-only throughput: 8 distinct inputs and outputs (268 MB > L2)
    k0 = insts[0]["kernel"]
    P = [torch.rand((N_GRID, N_GRID), dtype=torch.float32, device=dev) for _ in range(8)]
    U = [torch.empty_like(x) for x in P]
    for j in range(8):
        k0.matvec(P[j], U[j])
    torch.cuda.synchronize()
    reps = 200
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    for j in range(reps):
        k0.matvec(P[j % 8], U[j % 8])
    e1.record(stream)
    torch.cuda.synchronize()
    mv_ms = e0.elapsed_time(e1) / reps
    # comparison only: the same products through torch.fft (cuFFT) on the same inputs
    try:
        lib_fft = library_fft_bench(torch, k0, P, U, stream)
    except Exception as exc:                    # a comparison line never fails the bench
        lib_fft = {"error": f"{type(exc).__name__}: {exc}"}
    try:
        fp64 = fp64_bench(torch, bem, insts[0]["inst"], stream)
    except Exception as exc:
        fp64 = {"error": f"{type(exc).__name__}: {exc}"}

    # dominant pass: mean duration over its launches inside the timed region (CUDA
    # events recorded by the library on the launching stream around every pass)
    rb = alg_bytes(N_GRID)
    hbm, src = peaks()
    dom = int(np.argmax(pass_ms))
    names = ["row_fwd_r2c", "col_fft_kmul_ifft", "row_inv_c2r"]
    achieved = rb[dom] / (pass_mean[dom] * 1e-3) / 1e9
    traffic = profiled_traffic() if dom == 1 else None

    # end-to-end through the C ABI with host buffers (pinned), copies inside the timed region
    e2e_mv = 0
    hosts = [(torch.tensor(c["inst"]["height"], dtype=torch.float32).pin_memory(),
              torch.empty((N_GRID, N_GRID), dtype=torch.float32).pin_memory()) for c in insts]
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    for i in range(max(1, args.steps)):
        c = insts[i % N_INST]
        fh, ph = hosts[i % N_INST]
        _, res = c["kernel"].solve(fh, "force", c["inst"]["force"], tol=TOL, max_iter=5000, p_out=ph, stream=stream)
        e2e_mv += res["matvecs"]
    torch.cuda.synchronize()
    e2e_s = time.perf_counter() - t0
    e2e_ms, e2e_all = aggregate_ranks(torch, 1000.0 * e2e_s, e2e_mv, dev)
    e2e_value = e2e_all / (e2e_ms / 1000.0)

    line = {
        "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": ms_max / args.steps, "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None, "dtype": "f32", "data": "synthetic",
        "config": {
            "workload": f"FP32 force-controlled contact solve, N={N_GRID} (4096^2 period), seeded rough surface "
                        "(H=0.7, rms slope 0.1, roll-off L/8) on a coated half-space, cold start, CG to 1e-8",
            "N": N_GRID, "instances": N_INST, "seeds": [SEED0 + i for i in range(N_INST)],
            "parallelism": f"replicas x{world}" if world > 1 else "single GPU",
            "l2": "working set ~170 MB per solve > 129 MB L2 (no flush needed); matvec-only loop cycles 8 "
                  "distinct 16.8 MB inputs",
            "fft_log2_radix": {"rows": radix.by_size[N_GRID][0], "cols": radix.by_size[N_GRID][1],
                               "picked_by": "--radix" if args.radix else "bem_autotune"},
        },
        "time_to_converge_ms": ms_max / args.steps,
        "cg_iters_per_solve": iters / args.steps,
        "matvecs_per_solve": mv / args.steps,
        "matvec_only": {"value": 1000.0 / mv_ms, "unit": UNIT, "ms_per_matvec": mv_ms,
                        "alg_bytes": sum(rb), "gbs": sum(rb) / (mv_ms * 1e-3) / 1e9},
        "library_fft_comparison": lib_fft,
        "fp64_product": fp64,
        "passes_ms_mean": dict(zip(names, pass_mean)),
        "passes_timing_region": "a second run of the same steps with CUDA events around every pass",
        "passes_launches": dict(zip(names, pass_n)),
        "roofline": {"bound": "hbm", "kernel": names[dom], "achieved": achieved, "peak": hbm,
                     "peak_source": f"{src} (MEASURED_PEAKS.json hbm_gbs)" if src == "measured" else src,
                     "unit": "GB/s", "frac": achieved / hbm, "traffic": traffic,
                     "traffic_source": "profiles/col_pass_pair_N2048_fp32.md (ncu, cold cache)" if traffic else None,
                     "alg_bytes_per_launch": rb[dom]},
        "e2e": {"value": e2e_value, "unit": UNIT, "h2d_bytes_per_step": 4 * N_GRID * N_GRID,
                "d2h_bytes_per_step": 4 * N_GRID * N_GRID + 96},
        "gpu_launches": int(launches),
        "clocks": clk,
    }
    if args.batch > 0:
        line["batch"] = batch_bench(torch, dev, bem, inputs, args.batch, radix)
    if args.adhesive > 0:
        line["adhesive_ramp"] = adhesive_bench(torch, dev, bem, inputs)
    if args.punch > 0:
        line["punch_sweep"] = punch_sweep_bench(torch, dev, bem, inputs)
    if args.warmstart > 0:
        line["warm_start"] = warm_start_bench(torch, dev, bem, args.warmstart, args.warmstart_steps, args.warmstart_test)
    if rank == 0 and world == 1 and not args.no_cpu_baseline:
        dt = cpu_oracle_matvecs()
        line["cpu_baseline"] = {"value": 1.0 / dt, "unit": UNIT, "cores": 1, "kind": "oracle",
                                "sample": f"1 FP64 product at N={N_GRID} (oracle radix-2 FFT, numpy, one thread)"}
        try:
            line["cpu_library_fft"] = cpu_library_fft()
        except Exception as exc:                # a comparison line never fails the bench
            line["cpu_library_fft"] = {"error": f"{type(exc).__name__}: {exc}"}
    if rank == 0:
        print(json.dumps(line), flush=True)
    for c in insts:
        c["kernel"].close()
    if world > 1:
        torch.distributed.destroy_process_group()


def probe_matvec(count):
    """K products u = K p of one N = 2048 FP32 operator (h/delta = 16, E1/E2 = 2,
    nu = 0.3) on four random pressure fields; prints nothing but 'ok'."""
    import torch
    from paper_1807_01885_gb300 import bem, build
    build.build()
    N = N_GRID
    k = bem.Kernel(N, 1.0 / N, 16.0 / N, 2.0, 0.3, 1.0, 0.3, precision="fp32")
    gen = torch.Generator(device="cuda").manual_seed(1)
    P = [torch.rand((N, N), dtype=torch.float32, device="cuda", generator=gen) for _ in range(4)]
    U = [torch.empty_like(x) for x in P]
    for it in range(count):
        k.matvec(P[it % 4], U[it % 4])
    torch.cuda.synchronize()
    k.close()
    print("ok")


def probe_fno(count):
    """K forwards of the warm-start network on one random N = 2048 feature map; prints 'ok'."""
    import torch
    from paper_1807_01885_gb300 import bem, build
    build.build()
    net = bem.Fno(width=32, modes=16, layers=4, hidden=64)
    gen = torch.Generator(device="cuda").manual_seed(1)
    x = torch.randn((1, 7, N_GRID, N_GRID), dtype=torch.float32, device="cuda", generator=gen)
    out = torch.empty((1, N_GRID, N_GRID), dtype=torch.float32, device="cuda")
    for _ in range(count):
        net.forward(1, N_GRID, x, out)
    torch.cuda.synchronize()
    net.close()
    print("ok")


def main():
    args = parse()
    if args.probe_matvec > 0:
        probe_matvec(args.probe_matvec)
        return
    if args.probe_fno > 0:
        probe_fno(args.probe_fno)
        return
    if args.impl == "reference":
        run_reference(args)
    else:
        run_ours(args)


if __name__ == "__main__":
    main()
