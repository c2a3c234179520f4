"""ctypes binding of libbem.so (include/bem.h): argument marshalling only.

Every computation happens in the CUDA library; this module converts Python values
to the C structs, passes tensor/array data pointers and CUDA stream handles, and
turns status codes into exceptions.  There is no CPU fallback: if the library is
missing the first call raises.

Arrays may be torch tensors (CUDA or CPU) or numpy arrays, row-major, N x N, of the
kernel's dtype (float64 for "fp64", float32 for "fp32"); the library detects
device versus host pointers itself.
"""
import ctypes
import os

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "libbem.so")

(BEM_OK, BEM_EINVAL, BEM_ENOMEM, BEM_ECUDA, BEM_ENOCONV, BEM_ETIMEOUT, BEM_ENAN, BEM_ECYCLE, BEM_EUNSUPPORTED,
 BEM_EDETACHED) = range(10)
STATUS_NAMES = ["BEM_OK", "BEM_EINVAL", "BEM_ENOMEM", "BEM_ECUDA", "BEM_ENOCONV", "BEM_ETIMEOUT", "BEM_ENAN",
                "BEM_ECYCLE", "BEM_EUNSUPPORTED", "BEM_EDETACHED"]
BEM_FP64, BEM_FP32 = 0, 1
BEM_CTRL_DEPTH, BEM_CTRL_FORCE = 0, 1
BEM_DC_FINITE_PART, BEM_DC_ZERO = 0, 1
BEM_OP_PERIODIC, BEM_OP_OPEN = 0, 1

# entry points declared in include/bem.h
EXPORTS = ("bem_make_kernel", "bem_destroy_kernel", "bem_kernel_table", "bem_matvec", "bem_solve_contact",
           "bem_solve_batch", "bem_matvec_static", "bem_profile_passes", "bem_set_pass_timing", "bem_pass_timing",
           "bem_launch_count", "bem_last_error", "bem_version", "bem_fno_create", "bem_fno_destroy",
           "bem_check_guards", "bem_debug_poke_guard", "bem_fno_param_count", "bem_fno_set_params", "bem_fno_get_params", "bem_fno_get_state",
           "bem_fno_set_state", "bem_fno_features", "bem_fno_forward",
           "bem_fno_gradients", "bem_fno_train_step", "bem_fno_target", "bem_fno_pressure", "bem_set_radix",
           "bem_autotune", "bem_make_kernel_layers", "bem_rebuild_kernel")
BEM_MAX_LAYERS = 8
BEM_STATIC_MAX_N = 256


class BemError(RuntimeError):
    def __init__(self, status, msg):
        super().__init__(f"{STATUS_NAMES[status] if 0 <= status < len(STATUS_NAMES) else status}: {msg}")
        self.status = status


class KernelDesc(ctypes.Structure):
    _fields_ = [("N", ctypes.c_int32), ("precision", ctypes.c_int32), ("dc_mode", ctypes.c_int32),
                ("op_kind", ctypes.c_int32), ("delta", ctypes.c_double), ("h", ctypes.c_double),
                ("E1", ctypes.c_double), ("nu1", ctypes.c_double), ("E2", ctypes.c_double), ("nu2", ctypes.c_double)]


class Layer(ctypes.Structure):
    _fields_ = [("h", ctypes.c_double), ("E", ctypes.c_double), ("nu", ctypes.c_double)]


class FnoDesc(ctypes.Structure):
    _fields_ = [("width", ctypes.c_int32), ("modes", ctypes.c_int32), ("layers", ctypes.c_int32),
                ("hidden", ctypes.c_int32)]


class Problem(ctypes.Structure):
    _fields_ = [("height", ctypes.c_void_p), ("p_init", ctypes.c_void_p), ("contact_mask", ctypes.c_void_p),
                ("control", ctypes.c_int32), ("max_iter", ctypes.c_int32), ("target", ctypes.c_double),
                ("dgamma", ctypes.c_double), ("tol", ctypes.c_double)]


class Result(ctypes.Structure):
    _fields_ = [("force", ctypes.c_double), ("depth", ctypes.c_double), ("area", ctypes.c_double),
                ("a_eq", ctypes.c_double), ("residual", ctypes.c_double), ("err_est", ctypes.c_double),
                ("iters", ctypes.c_int32), ("outer_iters", ctypes.c_int32), ("n_contact", ctypes.c_int32),
                ("status", ctypes.c_int32), ("matvecs", ctypes.c_int32), ("reserved", ctypes.c_int32)]

    def as_dict(self):
        return {name: getattr(self, name) for name, _ in self._fields_ if name != "reserved"}


_lib = None


def load(path=None):
    """Loads libbem.so (once).  Raises if it has not been built."""
    global _lib
    if _lib is not None:
        return _lib
    path = path or LIB_PATH
    if not os.path.exists(path):
        raise RuntimeError(f"{path} is missing: build it with `python -m paper_1807_01885_gb300.build` "
                           "(there is no CPU fallback)")
    lib = ctypes.CDLL(path)
    vp, i32 = ctypes.c_void_p, ctypes.c_int32
    lib.bem_make_kernel.argtypes = [ctypes.POINTER(KernelDesc), vp, ctypes.POINTER(vp)]
    lib.bem_make_kernel_layers.argtypes = [ctypes.POINTER(KernelDesc), i32, ctypes.POINTER(Layer), vp,
                                           ctypes.POINTER(vp)]
    lib.bem_make_kernel_layers.restype = i32
    lib.bem_rebuild_kernel.argtypes = [vp, ctypes.POINTER(KernelDesc), vp]
    lib.bem_rebuild_kernel.restype = i32
    lib.bem_destroy_kernel.argtypes = [vp]
    lib.bem_kernel_table.argtypes = [vp, vp, vp]
    lib.bem_check_guards.argtypes = [vp, ctypes.POINTER(ctypes.c_int64), vp]
    lib.bem_check_guards.restype = i32
    lib.bem_debug_poke_guard.argtypes = [vp, i32]
    lib.bem_debug_poke_guard.restype = i32
    lib.bem_matvec.argtypes = [vp, vp, vp, vp]
    lib.bem_solve_contact.argtypes = [vp, ctypes.POINTER(Problem), vp, ctypes.POINTER(Result), vp]
    lib.bem_solve_batch.argtypes = [i32, ctypes.POINTER(vp), ctypes.POINTER(Problem), ctypes.POINTER(vp),
                                    ctypes.POINTER(Result), vp]
    for name in ("bem_make_kernel", "bem_destroy_kernel", "bem_kernel_table", "bem_matvec", "bem_solve_contact",
                 "bem_solve_batch"):
        getattr(lib, name).restype = i32
    lib.bem_last_error.restype = ctypes.c_char_p
    lib.bem_last_error.argtypes = []
    lib.bem_version.restype = i32
    lib.bem_version.argtypes = []
    lib.bem_profile_passes.argtypes = [vp, vp, vp, i32, ctypes.POINTER(ctypes.c_float), vp]
    lib.bem_profile_passes.restype = i32
    lib.bem_launch_count.argtypes = []
    lib.bem_matvec_static.argtypes = [ctypes.POINTER(KernelDesc), vp, vp, vp]
    i64, dbl = ctypes.c_int64, ctypes.POINTER(ctypes.c_double)
    lib.bem_fno_create.argtypes = [ctypes.POINTER(FnoDesc), ctypes.POINTER(vp)]
    lib.bem_fno_destroy.argtypes = [vp]
    lib.bem_fno_param_count.argtypes = [vp]
    lib.bem_fno_param_count.restype = i64
    lib.bem_fno_set_params.argtypes = [vp, vp, i64, vp]
    lib.bem_fno_get_params.argtypes = [vp, vp, i64, i32, vp]
    lib.bem_fno_get_state.argtypes = [vp, vp, vp, i64, ctypes.POINTER(i32), vp]
    lib.bem_fno_set_state.argtypes = [vp, vp, vp, i64, i32, vp]
    lib.bem_fno_features.argtypes = [vp, i32, i32, vp, vp, vp, vp]
    lib.bem_fno_forward.argtypes = [vp, i32, i32, vp, vp, vp]
    lib.bem_fno_gradients.argtypes = [vp, i32, i32, vp, vp, vp, dbl, vp]
    lib.bem_fno_train_step.argtypes = [vp, i32, i32, vp, vp, ctypes.c_float, dbl, vp]
    lib.bem_fno_target.argtypes = [vp, i32, i32, vp, vp, vp, vp]
    lib.bem_fno_pressure.argtypes = [vp, i32, i32, vp, vp, ctypes.c_float, vp, vp]
    for name in ("bem_fno_create", "bem_fno_destroy", "bem_fno_set_params", "bem_fno_get_params", "bem_fno_get_state",
                 "bem_fno_set_state", "bem_fno_features",
                 "bem_fno_forward", "bem_fno_gradients", "bem_fno_train_step", "bem_fno_target", "bem_fno_pressure"):
        getattr(lib, name).restype = i32
    lib.bem_set_pass_timing.argtypes = [vp, i32]
    lib.bem_set_radix.argtypes = [vp, i32, i32, vp]
    lib.bem_set_radix.restype = i32
    lib.bem_autotune.argtypes = [vp, i32, ctypes.POINTER(i32), vp]
    lib.bem_autotune.restype = i32
    lib.bem_set_pass_timing.restype = i32
    lib.bem_pass_timing.argtypes = [vp, ctypes.POINTER(ctypes.c_double), ctypes.POINTER(ctypes.c_int64), i32]
    lib.bem_pass_timing.restype = i32
    lib.bem_matvec_static.restype = i32
    lib.bem_launch_count.restype = ctypes.c_int64
    _lib = lib
    return lib


def _check(status, allow=()):
    if status != BEM_OK and status not in allow:
        raise BemError(status, load().bem_last_error().decode())
    return status


def _ptr(x):
    """Data pointer of a torch tensor or numpy array (None -> NULL)."""
    if x is None:
        return None
    if hasattr(x, "data_ptr"):
        if not x.is_contiguous():
            raise ValueError("array must be contiguous")
        return x.data_ptr()
    if isinstance(x, np.ndarray):
        if not x.flags.c_contiguous:
            raise ValueError("array must be C-contiguous")
        return x.ctypes.data
    raise TypeError(f"unsupported array type {type(x)}")


def _stream(stream):
    if stream is None:
        try:
            import torch
            if torch.cuda.is_available():
                return torch.cuda.current_stream().cuda_stream
        except ImportError:
            pass
        return None
    return stream.cuda_stream if hasattr(stream, "cuda_stream") else int(stream)


# ---------------------------------------------------------------------------
# the C entry points, one to one

def bem_make_kernel(N, delta, h, E1, nu1, E2, nu2, precision=BEM_FP64, dc_mode=BEM_DC_FINITE_PART, stream=None,
                    op_kind=BEM_OP_PERIODIC):
    lib = load()
    d = KernelDesc(N=N, precision=precision, dc_mode=dc_mode, op_kind=op_kind, delta=delta, h=h, E1=E1, nu1=nu1,
                   E2=E2, nu2=nu2)
    out = ctypes.c_void_p()
    _check(lib.bem_make_kernel(ctypes.byref(d), _stream(stream), ctypes.byref(out)))
    return out.value


def bem_make_kernel_layers(N, delta, layers, E2, nu2, precision=BEM_FP64, dc_mode=BEM_DC_FINITE_PART, stream=None,
                           op_kind=BEM_OP_PERIODIC):
    """Operator of a stack of bonded layers ``layers`` = [(h, E, nu), ...] from the
    surface down, on the substrate (E2, nu2)."""
    lib = load()
    d = KernelDesc(N=N, precision=precision, dc_mode=dc_mode, op_kind=op_kind, delta=delta, h=0.0, E1=1.0, nu1=0.0,
                   E2=E2, nu2=nu2)
    n = len(layers)
    arr = (Layer * max(n, 1))(*[Layer(h=float(h), E=float(E), nu=float(nu)) for h, E, nu in layers])
    out = ctypes.c_void_p()
    _check(lib.bem_make_kernel_layers(ctypes.byref(d), n, arr, _stream(stream), ctypes.byref(out)))
    return out.value


def bem_rebuild_kernel(k, N, delta, h, E1, nu1, E2, nu2, precision=BEM_FP64, dc_mode=BEM_DC_FINITE_PART,
                       stream=None, op_kind=BEM_OP_PERIODIC):
    d = KernelDesc(N=N, precision=precision, dc_mode=dc_mode, op_kind=op_kind, delta=delta, h=h, E1=E1, nu1=nu1,
                   E2=E2, nu2=nu2)
    _check(load().bem_rebuild_kernel(k, ctypes.byref(d), _stream(stream)))


def bem_destroy_kernel(k):
    _check(load().bem_destroy_kernel(k))


def bem_kernel_table(k, out, stream=None):
    _check(load().bem_kernel_table(k, _ptr(out), _stream(stream)))
    return out


def bem_matvec(k, p, u, stream=None):
    _check(load().bem_matvec(k, _ptr(p), _ptr(u), _stream(stream)))
    return u


def make_problem(height, control=BEM_CTRL_DEPTH, target=0.0, dgamma=0.0, tol=1e-10, max_iter=10000,
                 p_init=None, contact_mask=None):
    return Problem(height=_ptr(height), p_init=_ptr(p_init), contact_mask=_ptr(contact_mask), control=control,
                   max_iter=max_iter, target=target, dgamma=dgamma, tol=tol)


def bem_solve_contact(k, prob, p_out, stream=None, allow=(BEM_ENOCONV, BEM_EDETACHED)):
    res = Result()
    st = load().bem_solve_contact(k, ctypes.byref(prob), _ptr(p_out), ctypes.byref(res), _stream(stream))
    _check(st, allow)
    return res.as_dict()


def bem_solve_batch(kernels, probs, p_outs, stream=None):
    n = len(kernels)
    karr = (ctypes.c_void_p * n)(*kernels)
    parr = (Problem * n)(*probs)
    oarr = (ctypes.c_void_p * n)(*[_ptr(p) for p in p_outs])
    rarr = (Result * n)()
    st = load().bem_solve_batch(n, karr, parr, oarr, rarr, _stream(stream))
    return st, [r.as_dict() for r in rarr]


def bem_version():
    return load().bem_version()


def bem_profile_passes(k, p, u, reps, stream=None):
    ms = (ctypes.c_float * 3)()
    _check(load().bem_profile_passes(k, _ptr(p), _ptr(u), reps, ms, _stream(stream)))
    return [ms[0], ms[1], ms[2]]


def bem_matvec_static(N, delta, h, E1, nu1, E2, nu2, p, u, dc_mode=BEM_DC_FINITE_PART, stream=None):
    """u = K p through the entry point that allocates nothing (float32 device arrays,
    N <= BEM_STATIC_MAX_N); for callers that may not allocate device memory."""
    for name, x in (("p", p), ("u", u)):
        if x is None:
            continue
        dtype = getattr(x, "dtype", None)
        if str(dtype) not in ("torch.float32", "float32"):
            raise ValueError(f"bem_matvec_static: {name} must be float32, got {dtype}")
        size = x.numel() if hasattr(x, "numel") else x.size
        if size != N * N:
            raise ValueError(f"bem_matvec_static: {name} must hold N*N = {N * N} values, got {size}")
        if getattr(x, "is_cuda", False):      # a torch tensor on a GPU
            import torch
            if x.device.index != torch.cuda.current_device():
                raise ValueError(f"bem_matvec_static: {name} is on {x.device}, the current device is "
                                 f"cuda:{torch.cuda.current_device()}")
    d = KernelDesc(N=N, precision=BEM_FP32, dc_mode=dc_mode, op_kind=0, delta=delta, h=h, E1=E1, nu1=nu1,
                   E2=E2, nu2=nu2)
    _check(load().bem_matvec_static(ctypes.byref(d), _ptr(p), _ptr(u), _stream(stream)))
    return u


def bem_set_radix(k, row_log2_radix, col_log2_radix, stream=None):
    _check(load().bem_set_radix(k, row_log2_radix, col_log2_radix, _stream(stream)))


def bem_autotune(k, reps=10, stream=None):
    """Times the allowed FFT radices of the row and column passes and keeps the
    fastest; returns (rows, columns) as log2 of the radix."""
    c = (ctypes.c_int32 * 2)()
    _check(load().bem_autotune(k, reps, c, _stream(stream)))
    return int(c[0]), int(c[1])


def bem_set_pass_timing(k, on):
    _check(load().bem_set_pass_timing(k, 1 if on else 0))


def bem_pass_timing(k, reset=False):
    """(ms_total[3], launches[3]) of the timed passes (rows fwd, columns, rows inv)."""
    ms = (ctypes.c_double * 3)()
    n = (ctypes.c_int64 * 3)()
    _check(load().bem_pass_timing(k, ms, n, 1 if reset else 0))
    return list(ms), list(n)


def bem_launch_count():
    return load().bem_launch_count()


# ---------------------------------------------------------------------------
class Kernel:
    """Owning wrapper of a bem_kernel handle (same parameters as bem_kernel_desc)."""

    def __init__(self, N, delta, h=None, E1=None, nu1=None, E2=1.0, nu2=0.3, precision="fp64",
                 dc_mode=BEM_DC_FINITE_PART, stream=None, layers=None, op_kind=BEM_OP_PERIODIC):
        """One coating (h, E1, nu1) on the substrate (E2, nu2), or, with ``layers`` =
        [(h, E, nu), ...] from the surface down, a stack of coatings on it.  op_kind
        BEM_OP_OPEN selects the non-periodic operator (homogeneous half-space only)."""
        self.N, self.delta = N, delta
        self.precision = precision
        prec = BEM_FP64 if precision == "fp64" else BEM_FP32
        if layers is not None:
            self.params = dict(layers=[tuple(x) for x in layers], E2=E2, nu2=nu2)
            self.handle = bem_make_kernel_layers(N, delta, layers, E2, nu2, prec, dc_mode, stream, op_kind)
        else:
            self.params = dict(h=h, E1=E1, nu1=nu1, E2=E2, nu2=nu2)
            self.handle = bem_make_kernel(N, delta, h, E1, nu1, E2, nu2, prec, dc_mode, stream, op_kind)

    @property
    def torch_dtype(self):
        import torch
        return torch.float64 if self.precision == "fp64" else torch.float32

    @property
    def np_dtype(self):
        return np.float64 if self.precision == "fp64" else np.float32

    def table(self, device="cuda"):
        import torch
        out = torch.empty((self.N + 1, self.N + 1), dtype=torch.float64, device=device)
        return bem_kernel_table(self.handle, out)

    def matvec(self, p, u=None, stream=None):
        if u is None:
            import torch
            u = torch.empty_like(p) if hasattr(p, "data_ptr") else np.empty_like(p)
        return bem_matvec(self.handle, p, u, stream)

    def solve(self, height, control="depth", target=0.0, dgamma=0.0, tol=1e-10, max_iter=10000, p_init=None,
              contact_mask=None, p_out=None, stream=None):
        ctrl = BEM_CTRL_DEPTH if control == "depth" else BEM_CTRL_FORCE
        if p_out is None:
            import torch
            p_out = torch.empty_like(height) if hasattr(height, "data_ptr") else np.empty_like(height)
        prob = make_problem(height, ctrl, target, dgamma, tol, max_iter, p_init, contact_mask)
        res = bem_solve_contact(self.handle, prob, p_out, stream)
        return p_out, res

    def rebuild(self, delta, h, E1, nu1, E2, nu2, dc_mode=BEM_DC_FINITE_PART, stream=None,
                op_kind=BEM_OP_PERIODIC):
        """New operator parameters on the same grid size and precision, in place."""
        prec = BEM_FP64 if self.precision == "fp64" else BEM_FP32
        bem_rebuild_kernel(self.handle, self.N, delta, h, E1, nu1, E2, nu2, prec, dc_mode, stream, op_kind)
        self.delta = delta
        self.params = dict(h=h, E1=E1, nu1=nu1, E2=E2, nu2=nu2)

    def check_guards(self, stream=None):
        """Bytes of the workspace guard zones that lost their pattern (0: no kernel wrote
        outside its arrays)."""
        bad = ctypes.c_int64()
        _check(load().bem_check_guards(self.handle, ctypes.byref(bad), _stream(stream)))
        return bad.value

    def set_radix(self, rows, cols, stream=None):
        """log2 of the FFT radix of the row and column passes (3 or 4; 3 only in fp64)."""
        bem_set_radix(self.handle, rows, cols, stream)

    def autotune(self, reps=10, stream=None):
        return bem_autotune(self.handle, reps, stream)

    def close(self):
        if getattr(self, "handle", None):
            bem_destroy_kernel(self.handle)
            self.handle = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def __enter__(self):
        return self

    def __exit__(self, *a):
        self.close()


class Fno:
    """Owning wrapper of a bem_fno handle (the warm-start network)."""

    def __init__(self, width=32, modes=16, layers=4, hidden=64):
        self.desc = FnoDesc(width=width, modes=modes, layers=layers, hidden=hidden)
        out = ctypes.c_void_p()
        _check(load().bem_fno_create(ctypes.byref(self.desc), ctypes.byref(out)))
        self.handle = out.value
        self.count = load().bem_fno_param_count(self.handle)

    def set_params(self, w, stream=None):
        _check(load().bem_fno_set_params(self.handle, _ptr(w), self.count, _stream(stream)))

    def get_params(self, out, rounded=False, stream=None):
        _check(load().bem_fno_get_params(self.handle, _ptr(out), self.count, 1 if rounded else 0, _stream(stream)))
        return out

    def save(self, path):
        """Checkpoint: the float master parameters, Adam's moments and step count, and the
        network's sizes, in one .npz file."""
        w, m1, m2 = (np.empty(self.count, dtype=np.float32) for _ in range(3))
        self.get_params(w)
        step = ctypes.c_int32()
        _check(load().bem_fno_get_state(self.handle, _ptr(m1), _ptr(m2), self.count, ctypes.byref(step), None))
        d = self.desc
        np.savez(path, desc=np.array([d.width, d.modes, d.layers, d.hidden], dtype=np.int64), params=w, m1=m1, m2=m2,
                 step=np.int64(step.value))

    @classmethod
    def load(cls, path):
        """A network restored from ``save``: the same parameters and optimiser state."""
        z = np.load(path)
        width, modes, layers, hidden = (int(v) for v in z["desc"])
        net = cls(width=width, modes=modes, layers=layers, hidden=hidden)
        w = np.ascontiguousarray(z["params"], dtype=np.float32)
        m1 = np.ascontiguousarray(z["m1"], dtype=np.float32)
        m2 = np.ascontiguousarray(z["m2"], dtype=np.float32)
        net.set_params(w)
        _check(load().bem_fno_set_state(net.handle, _ptr(m1), _ptr(m2), net.count, int(z["step"]), None))
        return net

    def features(self, B, N, heights, params, x, stream=None):
        _check(load().bem_fno_features(self.handle, B, N, _ptr(heights), _ptr(params), _ptr(x), _stream(stream)))
        return x

    def forward(self, B, N, x, out, stream=None):
        _check(load().bem_fno_forward(self.handle, B, N, _ptr(x), _ptr(out), _stream(stream)))
        return out

    def gradients(self, B, N, x, target, grad=None, stream=None):
        loss = ctypes.c_double()
        _check(load().bem_fno_gradients(self.handle, B, N, _ptr(x), _ptr(target), _ptr(grad), ctypes.byref(loss),
                                        _stream(stream)))
        return loss.value

    def train_step(self, B, N, x, target, lr, stream=None):
        loss = ctypes.c_double()
        _check(load().bem_fno_train_step(self.handle, B, N, _ptr(x), _ptr(target), ctypes.c_float(lr),
                                         ctypes.byref(loss), _stream(stream)))
        return loss.value

    def target(self, B, N, p, pbar, q, stream=None):
        _check(load().bem_fno_target(self.handle, B, N, _ptr(p), _ptr(pbar), _ptr(q), _stream(stream)))
        return q

    def pressure(self, B, N, out, pbar, p, q_min=0.0, stream=None):
        _check(load().bem_fno_pressure(self.handle, B, N, _ptr(out), _ptr(pbar), float(q_min), _ptr(p),
                                       _stream(stream)))
        return p

    def close(self):
        if getattr(self, "handle", None):
            _check(load().bem_fno_destroy(self.handle))
            self.handle = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass
