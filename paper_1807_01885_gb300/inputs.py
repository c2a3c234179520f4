"""Seeded synthetic inputs shaped like the paper's workloads.

Holds no arithmetic of the method itself: only indenter height maps and parameter
draws.  Both the CUDA path's tests/benchmark and the CPU oracle take their inputs
from here.

Grid convention: N x N cells of side ``delta`` (Sec. 2, Fig. 2), row-major, cell
(r, c) centred at ((c + 0.5) delta - L/2, (r + 0.5) delta - L/2), L = N delta.
Heights f are measured upward from the indenter's lowest point (f >= 0).
"""
import numpy as np


def cell_centres(N, delta):
    x = (np.arange(N) + 0.5) * delta - 0.5 * N * delta
    return x[None, :], x[:, None]


def sphere_height(N, delta, R):
    """Paraboloid f = r^2/(2R) (the 'parabolic indenter' of Sec. 3.1)."""
    x, y = cell_centres(N, delta)
    return (x * x + y * y) / (2.0 * R)


def flat_punch_height(N, delta, a, lift=None):
    """Flat cylindrical punch of radius a: f = 0 for r <= a, ``lift`` outside.

    ``lift`` defaults to 10 L, far above any surface displacement, so cells outside
    the punch face never touch."""
    x, y = cell_centres(N, delta)
    lift = 10.0 * N * delta if lift is None else lift
    return np.where(x * x + y * y <= a * a, 0.0, lift)


def rough_surface(N, delta, seed, hurst=0.7, rms_slope=0.1, rolloff_frac=1.0 / 8.0):
    """Self-affine Gaussian random surface by spectral synthesis (periodic, N x N).

    Power spectrum flat below the roll-off q_r = 2 pi / (L rolloff_frac), falling as
    q^{-2(1+H)} above it up to the Nyquist wave number pi/delta, zero above; random
    Gaussian amplitudes and uniform phases from ``numpy.random.default_rng(seed)``;
    zero mean; scaled so that the rms of its central-difference slope equals
    ``rms_slope``.  Returned as the indenter height f = max(z) - z >= 0 (summits at
    f = 0).
    """
    rng = np.random.default_rng(seed)
    L = N * delta
    q1 = 2.0 * np.pi * np.fft.fftfreq(N, d=delta)
    qx, qy = np.meshgrid(q1, q1, indexing="xy")
    q = np.sqrt(qx * qx + qy * qy)
    qr = 2.0 * np.pi / (L * rolloff_frac)
    qs = np.pi / delta
    psd = np.where(q < qr, 1.0, (np.maximum(q, qr) / qr) ** (-2.0 * (1.0 + hurst)))
    psd[q > qs] = 0.0
    psd[0, 0] = 0.0
    amp = np.sqrt(psd) * (rng.standard_normal((N, N)) + 1j * rng.standard_normal((N, N)))
    z = np.real(np.fft.ifft2(amp))
    z -= z.mean()
    gx = (np.roll(z, -1, axis=1) - np.roll(z, 1, axis=1)) / (2.0 * delta)
    gy = (np.roll(z, -1, axis=0) - np.roll(z, 1, axis=0)) / (2.0 * delta)
    slope = np.sqrt(np.mean(gx * gx + gy * gy))
    z *= rms_slope / slope
    return z.max() - z


def batch_instance(seed, sizes=(128, 256, 512, 1024)):
    """One instance of the heterogeneous rough-surface batch workload.

    Draws N uniformly from ``sizes``, h/delta log-uniform in [2, 200], E1/E2
    log-uniform in [0.05, 20], nu1 and nu2 uniform in [0.2, 0.49]; E2 = 1, L = 1.
    The load is a mean pressure 0.025 * h'_rms * min(E1*, E2*) with h'_rms the rms
    slope (0.1), which gives a contact area of a few per cent.
    """
    rng = np.random.default_rng(seed)
    N = int(sizes[rng.integers(len(sizes))])
    delta = 1.0 / N
    h = delta * float(np.exp(rng.uniform(np.log(2.0), np.log(200.0))))
    E2 = 1.0
    E1 = E2 * float(np.exp(rng.uniform(np.log(0.05), np.log(20.0))))
    nu1 = float(rng.uniform(0.2, 0.49))
    nu2 = float(rng.uniform(0.2, 0.49))
    f = rough_surface(N, delta, seed=seed + 7919)
    es = min(E1 / (1 - nu1 * nu1), E2 / (1 - nu2 * nu2))
    pbar = 0.025 * 0.1 * es
    force = pbar * (N * delta) ** 2
    return dict(N=N, delta=delta, h=h, E1=E1, nu1=nu1, E2=E2, nu2=nu2, height=f, force=force)


def _heights_chunk(args):
    """Worker of ``batch_heights``: instances [i0, i1) at grid size N; the height maps
    go into the named shared-memory array, the scalars come back."""
    from multiprocessing import shared_memory
    name, count, N, seed0, i0, i1 = args
    shm = shared_memory.SharedMemory(name=name)
    try:
        out = np.ndarray((count, N, N), dtype=np.float32, buffer=shm.buf)
        scalars = []
        for i in range(i0, i1):
            inst = batch_instance(seed0 + i, sizes=(N,))
            out[i] = inst.pop("height")
            scalars.append(inst)
        del out
        return scalars
    finally:
        shm.close()


def batch_heights(count, N, seed0, workers=None, timeout=900.0):
    """``count`` instances of the batch workload at grid size N (seeds seed0 + i), the
    same draws as ``batch_instance``, made on the host cores in parallel: returns
    (heights float32 [count, N, N], per-instance scalar dicts).  Workers start with
    'spawn' (the caller may hold a CUDA context) and write into shared memory; a
    failed pool or one slower than ``timeout`` seconds raises."""
    import concurrent.futures as cf
    import multiprocessing
    import os
    from multiprocessing import shared_memory
    workers = workers or max(1, min(16, os.cpu_count() or 1))
    if workers == 1 or count * N * N < (1 << 21):
        insts = [batch_instance(seed0 + i, sizes=(N,)) for i in range(count)]
        return np.stack([i.pop("height") for i in insts]).astype(np.float32), insts
    shm = shared_memory.SharedMemory(create=True, size=count * N * N * 4)
    try:
        bounds = np.linspace(0, count, 4 * workers + 1).astype(int)
        jobs = [(shm.name, count, N, seed0, int(a), int(b)) for a, b in zip(bounds[:-1], bounds[1:]) if b > a]
        with cf.ProcessPoolExecutor(workers, mp_context=multiprocessing.get_context("spawn")) as ex:
            futs = [ex.submit(_heights_chunk, j) for j in jobs]
            parts = [f.result(timeout=timeout) for f in futs]
        heights = np.ndarray((count, N, N), dtype=np.float32, buffer=shm.buf).copy()
    finally:
        shm.close()
        shm.unlink()
    return heights, [inst for part in parts for inst in part]
