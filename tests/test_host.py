"""Host-side logic on the CPU: the seeded input generators keep the statistics their
recipe states, the adhesive ramp's depth schedule, and the benchmark's bookkeeping
(algorithmic bytes, the gating of the committed ncu traffic on the kernel sources,
the per-size FFT radix cache, the command-line defaults)."""
import os
import sys

import numpy as np
import pytest

from paper_1807_01885_gb300 import inputs

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


# ---------------------------------------------------------------- input generators

def _radial_psd(z, delta):
    N = z.shape[0]
    Z = np.fft.fft2(z)
    q1 = 2.0 * np.pi * np.fft.fftfreq(N, d=delta)
    q = np.hypot(q1[None, :], q1[:, None])
    return q.ravel(), (np.abs(Z) ** 2).ravel()


def test_rough_surface_is_seeded_and_nonnegative():
    a = inputs.rough_surface(128, 1.0 / 128, seed=3)
    b = inputs.rough_surface(128, 1.0 / 128, seed=3)
    c = inputs.rough_surface(128, 1.0 / 128, seed=4)
    assert np.array_equal(a, b)
    assert not np.array_equal(a, c)
    assert a.min() == 0.0 and (a >= 0).all()


@pytest.mark.parametrize("hurst", [0.5, 0.7, 0.9])
def test_rough_surface_power_law_exponent(hurst):
    """Above the roll-off the radially averaged spectrum falls as q^{-2(1+H)}: the
    log-log slope over [2 q_r, q_s / 2] recovers the exponent."""
    N, delta = 512, 1.0 / 512
    f = inputs.rough_surface(N, delta, seed=11, hurst=hurst)
    q, P = _radial_psd(f, delta)
    qr = 2.0 * np.pi / (N * delta / 8.0)
    qs = np.pi / delta
    edges = np.geomspace(2 * qr, qs / 2, 25)
    idx = np.digitize(q, edges)
    qm, Pm = [], []
    for b in range(1, len(edges)):
        sel = idx == b
        if sel.sum() > 20:
            qm.append(np.mean(q[sel]))
            Pm.append(np.mean(P[sel]))
    slope = np.polyfit(np.log(qm), np.log(Pm), 1)[0]
    assert slope == pytest.approx(-2.0 * (1.0 + hurst), abs=0.05)


def test_rough_surface_band_limits_and_slope():
    """Flat spectrum below the roll-off (ratio of band means near 1), nothing beyond the
    Nyquist circle, and the stated rms slope of the central differences."""
    N, delta = 256, 1.0 / 256
    f = inputs.rough_surface(N, delta, seed=5, rms_slope=0.1)
    q, P = _radial_psd(f, delta)
    qr = 2.0 * np.pi / (N * delta / 8.0)
    qs = np.pi / delta
    assert P[q > qs * (1 + 1e-9)].max() < 1e-20 * P.max()
    low = P[(q > 0) & (q < qr / 2)]
    mid = P[(q >= qr / 2) & (q < qr)]
    # flat plateau: both bands hold exponential(|Z|^2) samples of one variance
    assert np.mean(mid) / np.mean(low) == pytest.approx(1.0, abs=0.5)
    gx = (np.roll(f, -1, 1) - np.roll(f, 1, 1)) / (2 * delta)
    gy = (np.roll(f, -1, 0) - np.roll(f, 1, 0)) / (2 * delta)
    assert np.sqrt(np.mean(gx ** 2 + gy ** 2)) == pytest.approx(0.1, rel=1e-12)


def test_sphere_and_punch_geometry():
    N, delta, R, a = 64, 1.0 / 64, 0.5, 0.2
    f = inputs.sphere_height(N, delta, R)
    assert np.array_equal(f, f.T) and np.array_equal(f, f[::-1, ::-1])
    # the four centre cells sit at (+-delta/2, +-delta/2)
    c = N // 2
    assert f[c, c] == pytest.approx((delta * delta / 2) / (2 * R), rel=1e-14)
    assert f.min() == f[c, c]
    g = inputs.flat_punch_height(N, delta, a)
    face = g == 0.0
    assert face.sum() * delta ** 2 == pytest.approx(np.pi * a * a, rel=0.05)
    assert (g[~face] == 10.0 * N * delta).all()


def test_batch_instance_parameter_ranges():
    sizes = (128, 256, 512, 1024)
    seen = {inputs.batch_instance(s, sizes=sizes)["N"] for s in range(40)}
    assert seen == set(sizes)
    for s in range(6):
        d = inputs.batch_instance(s, sizes=(64,))
        assert d["N"] == 64 and d["delta"] == 1.0 / 64 and d["E2"] == 1.0
        assert 2.0 <= d["h"] / d["delta"] <= 200.0
        assert 0.05 <= d["E1"] <= 20.0
        assert 0.2 <= d["nu1"] <= 0.49 and 0.2 <= d["nu2"] <= 0.49
        es = min(d["E1"] / (1 - d["nu1"] ** 2), 1.0 / (1 - d["nu2"] ** 2))
        assert d["force"] == pytest.approx(0.025 * 0.1 * es, rel=1e-14)
        assert d["height"].shape == (64, 64) and d["height"].min() == 0.0
    a, b = inputs.batch_instance(9, sizes=(64,)), inputs.batch_instance(9, sizes=(64,))
    assert np.array_equal(a["height"], b["height"]) and a["E1"] == b["E1"]


# ---------------------------------------------------------------- adhesive ramp

def test_depth_schedule_loads_then_pulls_off():
    ramp = pytest.importorskip("paper_1807_01885_gb300.ramp")
    d = ramp.depth_schedule(0.3, -0.1, 4, 5)
    assert len(d) == 9
    assert d[0] == 0.0 and d[3] == 0.3 and d[-1] == pytest.approx(-0.1)
    assert (np.diff(d[:4]) > 0).all() and (np.diff(d[3:]) < 0).all()
    assert np.count_nonzero(d == 0.3) == 1


# ---------------------------------------------------------------- benchmark bookkeeping

@pytest.fixture(scope="module")
def bench():
    sys.path.insert(0, ROOT)
    import bench as b
    return b


def test_alg_bytes_counts_stored_arrays(bench):
    """Each pass's algorithmic bytes: the arrays it must read and write once, counted
    from their shapes (pressure/displacement N x N real, half spectrum N x (N+1)
    complex, compliance table (N+1) x (N+1) real)."""
    for N, elem in ((2048, 4), (256, 8)):
        real = np.empty((N, N), dtype=np.float32 if elem == 4 else np.float64).nbytes
        spec = np.empty((N, N + 1), dtype=np.complex64 if elem == 4 else np.complex128).nbytes
        table = np.empty((N + 1, N + 1), dtype=np.float32 if elem == 4 else np.float64).nbytes
        assert bench.alg_bytes(N, elem) == (real + spec, 2 * spec + table, spec + real)
    assert bench.alg_bytes(2048)[1] == 83_935_236


def test_profiled_traffic_gated_on_sources(bench, tmp_path, monkeypatch):
    """The ncu traffic figure is used only while the profiled sources hash to the value
    recorded beside it: a summary written for the current sources gives its figure,
    any other hash (a kernel edit since the capture) gives None."""
    import hashlib
    h = hashlib.sha256()
    for f in bench.PROFILED_SOURCES:
        h.update(open(os.path.join(ROOT, f), "rb").read())
    text = f"notes\n\n    traffic_bytes_per_launch: 12345\n    source_sha256: {h.hexdigest()}\n"
    cur = tmp_path / "cur.md"
    cur.write_text(text)
    monkeypatch.setattr(bench, "PROFILE", str(cur))
    assert bench.profiled_traffic() == 12345
    # a different source hash (any kernel edit since the capture) voids the figure
    bad = tmp_path / "p.md"
    bad.write_text(text.replace("source_sha256: ", "source_sha256: 0"))
    monkeypatch.setattr(bench, "PROFILE", str(bad))
    assert bench.profiled_traffic() is None
    monkeypatch.setattr(bench, "PROFILE", str(tmp_path / "missing.md"))
    assert bench.profiled_traffic() is None


def test_profiled_traffic_tracks_a_source_edit(bench, tmp_path, monkeypatch):
    """Copies of the profiled sources with one byte appended no longer match."""
    import hashlib
    root = tmp_path / "r"
    h = hashlib.sha256()
    for f in bench.PROFILED_SOURCES:
        dst = root / f
        dst.parent.mkdir(parents=True, exist_ok=True)
        data = open(os.path.join(ROOT, f), "rb").read()
        dst.write_bytes(data)
        h.update(data)
    prof = tmp_path / "prof.md"
    prof.write_text(f"    traffic_bytes_per_launch: 777\n    source_sha256: {h.hexdigest()}\n")
    monkeypatch.setattr(bench, "ROOT", str(root))
    monkeypatch.setattr(bench, "PROFILE", str(prof))
    assert bench.profiled_traffic() == 777
    with open(root / bench.PROFILED_SOURCES[0], "ab") as fh:
        fh.write(b"\n")
    assert bench.profiled_traffic() is None


class _FakeKernel:
    def __init__(self, N):
        self.N = N
        self.calls = []

    def set_radix(self, rows, cols, stream=None):
        self.calls.append(("set", rows, cols))

    def autotune(self, reps=5, stream=None):
        self.calls.append(("tune",))
        return (4, 3)


def test_radix_cache_tunes_once_per_size(bench):
    rc = bench.RadixCache()
    a, b, c = _FakeKernel(512), _FakeKernel(512), _FakeKernel(1024)
    assert rc.apply(a) == (4, 3) and a.calls == [("tune",)]
    assert rc.apply(b) == (4, 3) and b.calls == [("set", 4, 3)]
    assert rc.apply(c) == (4, 3) and c.calls == [("tune",)]
    assert rc.by_size == {512: (4, 3), 1024: (4, 3)}   # what the bench line reports per size
    fixed = bench.RadixCache(fixed=(4, 4))
    d = _FakeKernel(512)
    assert fixed.apply(d) == (4, 4) and d.calls == [("set", 4, 4)]
    assert fixed.by_size == {512: (4, 4)}


def test_radix_cache_file_is_reused(tmp_path):
    """An on-disk cache tunes a (device, N, precision) once across processes: a second
    cache reading the same file applies the stored choice without timing."""
    from paper_1807_01885_gb300 import tuning
    path = str(tmp_path / "sub" / "radix.json")
    first = tuning.RadixCache(path=path, device="GB300")
    a = _FakeKernel(2048)
    assert first.apply(a) == (4, 3) and a.calls == [("tune",)]
    second = tuning.RadixCache(path=path, device="GB300")
    b = _FakeKernel(2048)
    assert second.apply(b) == (4, 3) and b.calls == [("set", 4, 3)]
    other = tuning.RadixCache(path=path, device="B200")
    c = _FakeKernel(2048)
    assert other.apply(c) == (4, 3) and c.calls == [("tune",)]
    with open(path, "w") as fh:
        fh.write("not json")
    broken = tuning.RadixCache(path=path, device="GB300")
    d = _FakeKernel(2048)
    assert broken.apply(d) == (4, 3) and d.calls == [("tune",)]


def test_bench_defaults(bench, monkeypatch):
    monkeypatch.setattr(sys, "argv", ["bench.py"])
    a = bench.parse()
    assert a.gpus == 1 and a.warmup >= 3 and a.steps >= 1 and a.impl == "ours"
    monkeypatch.setattr(sys, "argv", ["bench.py", "--impl", "reference", "--gpus", "2"])
    a = bench.parse()
    assert a.impl == "reference" and a.gpus == 2


def test_peaks_read_measured_file(bench):
    hbm, kind = bench.peaks()
    if os.path.exists(os.path.join(ROOT, "MEASURED_PEAKS.json")):
        assert kind == "measured" and hbm > 1000
    else:
        assert (hbm, kind) == (6800.0, "fallback")


def test_library_fft_comparison_matches_oracle_operator(bench):
    """The benchmark's torch.fft comparison line computes the same operator as the
    oracle's Eq. (11) product: the half-grid K^ unfolded from an (N+1)^2 table equals
    the oracle's padded grid, and the product agrees on a ragged rough pressure field."""
    import torch
    from oracle import operator as oop
    N, delta = 24, 1.0 / 24
    Kg = oop.khat_grid(N, delta, 0.1, 3.0, 0.3, 1.0, 0.45)
    table = torch.tensor(Kg[:N + 1, :N + 1])
    kh = bench.library_fft_khat(torch, table, N, torch.float64)
    assert kh.shape == (2 * N, N + 1)
    np.testing.assert_array_equal(kh.numpy(), Kg[:, :N + 1])
    rng = np.random.default_rng(4)
    p = np.maximum(rng.standard_normal((N, N)), 0.0)
    pad = torch.zeros((2 * N, 2 * N), dtype=torch.float64)
    u = bench.library_fft_matvec(torch, kh, torch.tensor(p), pad).numpy()
    ref = oop.matvec_dense(Kg, p)
    assert np.linalg.norm(u - ref) / np.linalg.norm(ref) < 1e-13
    # the buffer outside the window stays zero, so a second call gives the same product
    u2 = bench.library_fft_matvec(torch, kh, torch.tensor(p), pad).numpy()
    np.testing.assert_array_equal(u, u2)


def test_cpu_library_fft_line_matches_oracle(bench):
    """The multi-core scipy FFT comparison computes the oracle's product (N = 64)."""
    pytest.importorskip("scipy.fft")
    out = bench.cpu_library_fft(reps=1, N=64)
    assert out["rel_l2_vs_oracle"] < 1e-13
    assert out["value"] > 0 and out["cores"] >= 1


def test_fft_nominal_flops(bench):
    """5 M log2 M per complex transform of length M = 2N, a real transform as half:
    1.51 GFLOP per product at N = 2048, four times as much per doubling of N (plus
    the log factor)."""
    assert bench.fft_nominal_flops(2048) == pytest.approx(1.51044096e9, rel=1e-12)
    M = 16
    c = 5 * M * 4
    assert bench.fft_nominal_flops(8) == 2 * 8 * c / 2 + 9 * 2 * c


def test_reference_arm_line_contract(bench, monkeypatch, capsys):
    """`bench.py --impl reference` prints one JSON line with the keys the benchmark
    contract needs; the oracle product is replaced by a fixed 0.5 s stand-in so the
    line's arithmetic can be checked.  Every requested step is timed and the line's
    step counts are the ones that ran."""
    import json
    calls = []
    monkeypatch.setattr(bench, "cpu_oracle_matvecs", lambda: calls.append(1) or 0.5)
    monkeypatch.setattr(sys, "argv", ["bench.py", "--impl", "reference", "--steps", "40", "--warmup", "3"])
    monkeypatch.delenv("WORLD_SIZE", raising=False)
    bench.run_reference(bench.parse())
    lines = [ln for ln in capsys.readouterr().out.splitlines() if ln.strip()]
    assert len(lines) == 1
    d = json.loads(lines[0])
    for key in ("metric", "value", "unit", "n_gpus", "steps", "warmup", "ms_per_step", "higher_is_better",
                "scaling", "vs_baseline", "dtype", "data", "config", "cpu_baseline", "e2e"):
        assert key in d, key
    assert d["impl"] == "reference" and d["metric"] == bench.METRIC and d["unit"] == bench.UNIT
    assert d["value"] == pytest.approx(2.0) and d["ms_per_step"] == pytest.approx(500.0)
    assert d["higher_is_better"] is True and d["steps"] == 40 and d["warmup"] == 3
    assert "workload" in d["config"]
    cb = d["cpu_baseline"]
    assert cb["kind"] == "oracle" and cb["cores"] >= 1 and cb["value"] == d["value"] and "40 timed" in cb["sample"]
    assert len(calls) == 43
    assert d["e2e"] == {"value": d["value"], "unit": d["unit"], "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}


def test_reference_arm_other_ranks_do_nothing(bench, monkeypatch, capsys):
    """Under a multi-process launch only rank 0 runs and prints the reference arm."""
    calls = []
    monkeypatch.setattr(bench, "cpu_oracle_matvecs", lambda: calls.append(1) or 0.5)
    monkeypatch.setattr(sys, "argv", ["bench.py", "--impl", "reference", "--gpus", "2"])
    monkeypatch.setenv("RANK", "1")
    monkeypatch.setenv("WORLD_SIZE", "2")
    bench.run_reference(bench.parse())
    assert capsys.readouterr().out.strip() == "" and not calls
