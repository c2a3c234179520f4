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


def test_status_codes_match_header():
    """Every bem_status value of include/bem.h has the same number and name in the
    binding (statuses are compared by value on both sides of the ABI)."""
    from paper_1807_01885_gb300 import bem
    src = open(os.path.join(ROOT, "include", "bem.h")).read()
    body = re.search(r"typedef enum \{(.*?)\} bem_status;", src, flags=re.S).group(1)
    body = re.sub(r"/\*.*?\*/", "", body, flags=re.S)
    codes = {name: int(val) for name, val in re.findall(r"(BEM_[A-Z]+)\s*=\s*(\d+)", body)}
    assert codes and len(codes) == len(bem.STATUS_NAMES)
    for name, val in codes.items():
        assert getattr(bem, name) == val, name
        assert bem.STATUS_NAMES[val] == name


def test_struct_layouts_match_header():
    from paper_1807_01885_gb300 import bem
    assert ctypes.sizeof(bem.KernelDesc) == 4 * 4 + 6 * 8
    assert ctypes.sizeof(bem.Problem) == 3 * 8 + 2 * 4 + 3 * 8
    assert ctypes.sizeof(bem.Result) == 6 * 8 + 6 * 4
    assert ctypes.sizeof(bem.Layer) == 3 * 8


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


def declared_signatures():
    """(return type, name, [parameter types]) of every prototype in include/bem.h."""
    src = open(os.path.join(ROOT, "include", "bem.h")).read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    src = re.sub(r"//[^\n]*", "", src)
    out = []
    for m in re.finditer(r"([A-Za-z_][A-Za-z_0-9 \*]*?)\s*\b(bem_[a-z_0-9]+)\s*\(([^)]*)\)\s*;", src):
        params = [] if m.group(3).strip() == "void" else [p.strip() for p in m.group(3).split(",")]
        # drop the parameter name, keep the type (with its stars)
        types = [re.sub(r"\s*\b[A-Za-z_][A-Za-z_0-9]*$", "", p).strip() for p in params]
        out.append((m.group(1).strip(), m.group(2), types))
    return out


def _expected(ctype):
    """ctypes the binding may use for a C type of the header: scalars exactly, data
    pointers as c_void_p or a POINTER of the pointee, opaque handles as c_void_p."""
    from paper_1807_01885_gb300 import bem
    scalars = {"int32_t": ctypes.c_int32, "int64_t": ctypes.c_int64, "float": ctypes.c_float,
               "double": ctypes.c_double, "bem_status": ctypes.c_int32, "const char*": ctypes.c_char_p}
    structs = {"bem_kernel_desc": bem.KernelDesc, "bem_problem": bem.Problem, "bem_result": bem.Result,
               "bem_fno_desc": getattr(bem, "FnoDesc", None), "bem_layer": bem.Layer}
    t = " ".join(ctype.replace("*", " * ").split())
    t = t.replace(" *", "*")
    if t in scalars:
        return {scalars[t]}
    if t in ("bem_kernel", "bem_fno"):
        return {ctypes.c_void_p}
    if "*" in t:
        bare = re.sub(r"\bconst\b", "", t).replace(" ", "")
        base, stars = bare.rstrip("*"), len(bare) - len(bare.rstrip("*"))
        ok = {ctypes.c_void_p}
        if stars == 1 and base in scalars:
            ok.add(ctypes.POINTER(scalars[base]))
        if stars == 1 and structs.get(base) is not None:
            ok.add(ctypes.POINTER(structs[base]))
        if (stars == 1 and base in ("bem_kernel", "bem_fno")) or bare == "void**":
            ok.add(ctypes.POINTER(ctypes.c_void_p))
        return ok
    raise AssertionError(f"unmapped C type {ctype!r}")


def test_binding_signatures_match_header(bemlib):
    """Every prototype's arity, argument types and return type agree with the ctypes
    declarations of the binding: a drifted signature would pass arguments wrongly
    without any error at the call."""
    sigs = declared_signatures()
    assert sorted(n for _, n, _ in sigs) == declared_entry_points()
    for ret, name, params in sigs:
        fn = getattr(bemlib, name)
        assert fn.argtypes is not None, f"{name}: argtypes not set"
        assert len(fn.argtypes) == len(params), (name, params, fn.argtypes)
        for i, (c, py) in enumerate(zip(params, fn.argtypes)):
            assert py in _expected(c), f"{name} argument {i}: header {c!r}, binding {py}"
        assert fn.restype in _expected(ret), f"{name} return: header {ret!r}, binding {fn.restype}"


def test_argument_errors_before_any_device_call(bemlib):
    """Entry points check their arguments before touching a device, so the statuses and
    the thread's error message can be checked on a CPU host (no call here reaches CUDA)."""
    import numpy as np
    from paper_1807_01885_gb300 import bem
    import ctypes
    p = np.zeros((4, 4), np.float32)
    u = np.zeros_like(p)

    def static(N, p_, u_, nu1=0.3, E1=1.0, precision=bem.BEM_FP32):
        d = bem.KernelDesc(N=N, precision=precision, dc_mode=0, op_kind=0, delta=0.1, h=1.0, E1=E1, nu1=nu1,
                           E2=1.0, nu2=0.3)
        st = bemlib.bem_matvec_static(ctypes.byref(d), bem._ptr(p_), bem._ptr(u_), None)
        return st, bemlib.bem_last_error().decode()

    st, msg = static(512, p, u)
    assert st == bem.BEM_EINVAL and "power of two" in msg and str(bem.BEM_STATIC_MAX_N) in msg
    st, msg = static(64, None, u)
    assert st == bem.BEM_EINVAL and "NULL" in msg
    # the operator checks are those of bem_make_kernel (Poisson ratio, infinite E1)
    st, msg = static(64, p, u, nu1=0.5)
    assert st == bem.BEM_EINVAL and "Poisson" in msg
    st, msg = static(64, p, u, E1=float("inf"))
    assert st == bem.BEM_EINVAL and "E1" in msg
    st, msg = static(64, p, u, precision=bem.BEM_FP64)
    assert st == bem.BEM_EINVAL and "FP32" in msg
    # the binding rejects a wrong dtype or size before the call
    with pytest.raises(ValueError, match="float32"):
        bem.bem_matvec_static(4, 0.1, 1.0, 1.0, 0.3, 1.0, 0.3, p.astype(np.float64), u)
    with pytest.raises(ValueError, match="N\\*N"):
        bem.bem_matvec_static(8, 0.1, 1.0, 1.0, 0.3, 1.0, 0.3, p, u)
    # coating stacks: layer count, thickness, modulus, Poisson ratio, total thickness
    for layers, msg in (([], "n_layers"), ([(0.1, 1.0, 0.3)] * 9, "BEM_MAX_LAYERS"),
                        ([(0.1, 1.0, 0.3), (-0.1, 1.0, 0.3)], "layer 1"),
                        ([(0.1, float("inf"), 0.3)], "layer 0"), ([(0.1, 1.0, 0.5)], "layer 0"),
                        ([(0.0, 1.0, 0.3)], "total thickness")):
        with pytest.raises(bem.BemError, match=msg) as e:
            bem.bem_make_kernel_layers(16, 0.1, layers, 1.0, 0.3)
        assert e.value.status == bem.BEM_EINVAL
    # the open-plane operator is built for a homogeneous half-space only
    with pytest.raises(bem.BemError, match="homogeneous") as e:
        bem.bem_make_kernel(16, 0.1, 0.3, 4.0, 0.3, 1.0, 0.3, op_kind=bem.BEM_OP_OPEN)
    assert e.value.status == bem.BEM_EUNSUPPORTED
    with pytest.raises(bem.BemError, match="homogeneous") as e:
        bem.bem_make_kernel_layers(16, 0.1, [(0.3, 4.0, 0.3)], 1.0, 0.3, op_kind=bem.BEM_OP_OPEN)
    assert e.value.status == bem.BEM_EUNSUPPORTED
    with pytest.raises(bem.BemError, match="op_kind") as e:
        bem.bem_make_kernel(16, 0.1, 0.3, 4.0, 0.3, 1.0, 0.3, op_kind=7)
    assert e.value.status == bem.BEM_EINVAL
    # batch: an empty batch is a no-op; a negative count is rejected with a message
    st, res = bem.bem_solve_batch([], [], [])
    assert st == bem.BEM_OK and res == []
    assert bemlib.bem_solve_batch(-1, None, None, None, None, None) == bem.BEM_EINVAL
    assert b"invalid batch" in bemlib.bem_last_error()
    # network descriptor: widths from the list, modes >= 1, 1 <= layers <= 16
    for kw in (dict(width=5), dict(hidden=3), dict(modes=0), dict(layers=0), dict(layers=17)):
        args = dict(width=8, modes=2, layers=1, hidden=8)
        args.update(kw)
        with pytest.raises(bem.BemError) as e:
            bem.Fno(**args)
        assert e.value.status == bem.BEM_EINVAL, kw
    # NULL handles: destroy is a no-op, the parameter count is -1
    assert bemlib.bem_fno_param_count(None) == -1
    assert bemlib.bem_fno_destroy(None) == bem.BEM_OK
    assert bemlib.bem_destroy_kernel(None) == bem.BEM_OK
