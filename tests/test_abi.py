"""CPU-side checks of the C ABI library: it builds for sm_103a, loads, and exports
every entry point include/bem.h declares (no compute calls without a GPU)."""
import ctypes
import os
import re

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def declared_entry_points():
    src = open(os.path.join(ROOT, "include", "bem.h")).read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    return sorted(set(re.findall(r"\b(bem_[a-z_0-9]+)\s*\(", src)))


def test_header_declares_the_boundary():
    names = declared_entry_points()
    for n in ("bem_make_kernel", "bem_matvec", "bem_solve_contact", "bem_solve_batch"):
        assert n in names


def test_library_exports_every_declared_symbol(bemlib):
    from paper_1807_01885_gb300 import bem
    for name in declared_entry_points():
        assert hasattr(bemlib, name), name
        assert name in bem.EXPORTS, name
    assert bem.bem_version() == 100


def test_struct_layouts_match_header():
    from paper_1807_01885_gb300 import bem
    assert ctypes.sizeof(bem.KernelDesc) == 4 * 4 + 6 * 8
    assert ctypes.sizeof(bem.Problem) == 3 * 8 + 2 * 4 + 3 * 8
    assert ctypes.sizeof(bem.Result) == 6 * 8 + 6 * 4


def test_invalid_descriptor_rejected_without_gpu(bemlib):
    """Argument checks run before any device call, so they work on a CPU host."""
    from paper_1807_01885_gb300 import bem
    for kw in (dict(N=48), dict(N=8192), dict(nu1=0.5), dict(h=-1.0), dict(E1=0.0), dict(delta=0.0)):
        args = dict(N=64, delta=0.1, h=1.0, E1=1.0, nu1=0.3, E2=1.0, nu2=0.3)
        args.update(kw)
        with pytest.raises(bem.BemError) as e:
            bem.bem_make_kernel(**args)
        assert e.value.status == bem.BEM_EINVAL


def test_missing_library_fails_loudly(tmp_path, monkeypatch):
    from paper_1807_01885_gb300 import bem
    monkeypatch.setattr(bem, "_lib", None)
    with pytest.raises(RuntimeError, match="no CPU fallback"):
        bem.load(str(tmp_path / "libbem.so"))
