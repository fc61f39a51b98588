"""Thin ctypes binding of the C ABI in ``include/lbm.h`` (library ``liblbm.so``).

Argument marshalling only: every step of the solver runs in the CUDA kernels of
``csrc/``.  The module-level functions carry the C names; :class:`Solver` wraps a
handle.  Device arrays are passed as raw pointers (``tensor.data_ptr()``), host
arrays as numpy buffers.  There is no CPU fallback: if the library is missing or
no GPU is present the calls raise.
"""
from __future__ import annotations

import ctypes as C
import os
import threading

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(HERE, "liblbm.so")

LBM_OK, LBM_ERR_INVALID, LBM_ERR_CUDA, LBM_ERR_OOM, LBM_ERR_DIVERGED, LBM_ERR_TIMEOUT = range(6)
LBM_ANNULUS, LBM_ANNULUS_PERIODIC_Z, LBM_PIPE_PERIODIC_Z, LBM_PIPE_INFLOW = 0, 1, 2, 3
LBM_F32, LBM_F16, LBM_BF16 = 0, 1, 2
LBM_MRT, LBM_BGK = 0, 1
LBM_FLUID, LBM_WALL_IN, LBM_WALL_OUT, LBM_BOTTOM, LBM_TOP, LBM_AXIS, LBM_INLET, LBM_OUTLET = range(8)
STORAGE = {"f32": LBM_F32, "f16": LBM_F16, "bf16": LBM_BF16}


class LbmError(RuntimeError):
    def __init__(self, code: int, msg: str):
        super().__init__(f"lbm error {code}: {msg}")
        self.code = code


class lbm_params(C.Structure):
    _fields_ = [
        ("nr", C.c_int32), ("nz", C.c_int32), ("geometry", C.c_int32), ("storage", C.c_int32),
        ("radius_ratio", C.c_double),
        ("Ra", C.c_double), ("Da", C.c_double), ("Pr", C.c_double), ("J", C.c_double), ("lam", C.c_double),
        ("Ma", C.c_double), ("tau_nu", C.c_double), ("F_eps", C.c_double), ("eps_mean", C.c_double),
        ("T_hot", C.c_double), ("T_cold", C.c_double), ("body_accel_z", C.c_double),
        ("init_noise", C.c_double), ("seed", C.c_uint64), ("u_in", C.c_double),
        ("heater_len", C.c_double), ("heater_center", C.c_double),
        ("collision", C.c_int32), ("inplace", C.c_int32),
    ]


class lbm_info(C.Structure):
    _fields_ = [
        ("L", C.c_double), ("H", C.c_double), ("r0", C.c_double), ("tau_nu", C.c_double), ("tau_T", C.c_double),
        ("nu_e", C.c_double), ("nu", C.c_double), ("gbeta", C.c_double), ("T0", C.c_double), ("Ma", C.c_double),
        ("Kbar", C.c_double), ("steps", C.c_int64), ("bytes_per_step", C.c_int64),
    ]


_lock = threading.Lock()
_lib = None

_vp = C.c_void_p
_SIGS = {
    "lbm_params_default": (None, [C.POINTER(lbm_params)]),
    "lbm_derive": (C.c_int, [C.POINTER(lbm_params), C.POINTER(lbm_info)]),
    "lbm_create": (C.c_int, [C.POINTER(lbm_params), C.POINTER(_vp)]),
    "lbm_set_stream": (C.c_int, [_vp, _vp]),
    "lbm_set_porosity": (C.c_int, [_vp, _vp, C.c_int]),
    "lbm_init_fields": (C.c_int, [_vp, _vp, _vp, _vp, C.c_int]),
    "lbm_step": (C.c_int, [_vp, C.c_int64]),
    "lbm_moments": (C.c_int, [_vp, _vp, _vp, _vp, _vp, C.c_int]),
    "lbm_nusselt": (C.c_int, [_vp, C.POINTER(C.c_double), C.POINTER(C.c_double)]),
    "lbm_pipe_nusselt": (C.c_int, [_vp, _vp, C.c_int32]),
    "lbm_heater_nusselt": (C.c_int, [_vp, C.POINTER(C.c_double), _vp]),
    "lbm_stream_function": (C.c_int, [_vp, _vp, C.c_int, C.POINTER(C.c_double)]),
    "lbm_nusselt_async": (C.c_int, [_vp, _vp]),
    "lbm_sync": (C.c_int, [_vp]),
    "lbm_residual": (C.c_int, [_vp, C.POINTER(C.c_double), C.POINTER(C.c_double)]),
    "lbm_run": (C.c_int, [_vp, C.c_int64, C.c_int64, C.c_double, C.POINTER(C.c_int64), C.POINTER(C.c_double)]),
    "lbm_rebase": (C.c_int, [_vp]),
    "lbm_set_porosity_async": (C.c_int, [_vp, _vp]),
    "lbm_porosity_errors": (C.c_int, [_vp, C.POINTER(C.c_uint32), C.c_int]),
    "lbm_node_class": (C.c_int, [_vp, _vp]),
    "lbm_export_populations": (C.c_int, [_vp, C.c_int32, C.c_int32, _vp, _vp]),
    "lbm_get_info": (C.c_int, [_vp, C.POINTER(lbm_info)]),
    "lbm_set_timing": (C.c_int, [_vp, C.c_int]),
    "lbm_set_wait_limit": (C.c_int, [_vp, C.c_int]),
    "lbm_wait_status": (C.c_int, [_vp, C.c_int]),
    "lbm_batch_set_wait_limit": (C.c_int, [_vp, C.c_int]),
    "lbm_set_staging": (C.c_int, [_vp, C.c_int]),
    "lbm_batch_set_staging": (C.c_int, [_vp, C.c_int]),
    "lbm_batch_wait_status": (C.c_int, [_vp, C.c_int]),
    "lbm_kernel_times": (C.c_int, [_vp, C.POINTER(C.c_double), C.POINTER(C.c_int64), C.POINTER(C.c_double),
                                   C.POINTER(C.c_int64)]),
    "lbm_field_residual_noalloc": (C.c_int, [C.c_int32, C.c_int32, C.c_int32, C.c_double, _vp, _vp, C.c_int64,
                                             C.POINTER(C.c_double), C.POINTER(C.c_double), _vp]),
    "lbm_batch_create": (C.c_int, [C.POINTER(lbm_params), C.c_int32, C.POINTER(_vp)]),
    "lbm_batch_set_stream": (C.c_int, [_vp, _vp]),
    "lbm_batch_set_porosity": (C.c_int, [_vp, C.c_int32, _vp, C.c_int]),
    "lbm_batch_init_fields": (C.c_int, [_vp, C.c_int32, _vp, _vp, _vp, C.c_int]),
    "lbm_batch_step": (C.c_int, [_vp, C.c_int64]),
    "lbm_batch_run": (C.c_int, [_vp, C.c_int64, C.c_int64, C.c_double, _vp, _vp]),
    "lbm_batch_rebase": (C.c_int, [_vp]),
    "lbm_batch_pipe_nusselt": (C.c_int, [_vp, C.c_int32, _vp, C.c_int32]),
    "lbm_batch_nusselt": (C.c_int, [_vp, _vp, _vp]),
    "lbm_batch_moments": (C.c_int, [_vp, C.c_int32, _vp, _vp, _vp, _vp, C.c_int]),
    "lbm_batch_tune": (C.c_int, [_vp, C.c_int32, C.POINTER(C.c_int32), C.POINTER(C.c_int32),
                                 C.POINTER(C.c_float)]),
    "lbm_batch_get_info": (C.c_int, [_vp, C.c_int32, C.POINTER(lbm_info)]),
    "lbm_batch_destroy": (C.c_int, [_vp]),
    "lbm_destroy": (C.c_int, [_vp]),
    "lbm_last_error": (C.c_char_p, []),
}


def load(path: str | None = None):
    """Load liblbm.so (building it first if it is absent and nvcc is available)."""
    global _lib
    with _lock:
        if _lib is not None:
            return _lib
        p = path or LIB_PATH
        if not os.path.exists(p):
            from . import build as _b

            _b.build()
        lib = C.CDLL(p)
        for name, (res, args) in _SIGS.items():
            fn = getattr(lib, name)
            fn.restype = res
            fn.argtypes = args
        _lib = lib
        return lib


def _check(rc: int):
    if rc != LBM_OK:
        raise LbmError(rc, load().lbm_last_error().decode())


def _ptr(a):
    """Raw pointer of a numpy array, a torch tensor, an int address, or None."""
    if a is None:
        return None
    if isinstance(a, int):
        return a
    if isinstance(a, np.ndarray):
        return a.ctypes.data
    return a.data_ptr()


# ---- C-named wrappers -------------------------------------------------------
def lbm_params_default(**overrides) -> lbm_params:
    p = lbm_params()
    load().lbm_params_default(C.byref(p))
    for k, v in overrides.items():
        if k == "storage" and isinstance(v, str):
            v = STORAGE[v]
        if not hasattr(p, k):
            raise KeyError(k)
        setattr(p, k, v)
    return p


def lbm_derive(p: lbm_params) -> lbm_info:
    info = lbm_info()
    _check(load().lbm_derive(C.byref(p), C.byref(info)))
    return info


def lbm_create(p: lbm_params) -> int:
    h = _vp()
    _check(load().lbm_create(C.byref(p), C.byref(h)))
    return h.value


def lbm_set_stream(h, stream: int | None):
    _check(load().lbm_set_stream(h, stream))


def lbm_set_porosity(h, phi, on_device: bool):
    _check(load().lbm_set_porosity(h, _ptr(phi), int(on_device)))


def lbm_init_fields(h, ur, uz, T, on_device: bool):
    _check(load().lbm_init_fields(h, _ptr(ur), _ptr(uz), _ptr(T), int(on_device)))


def lbm_step(h, nsteps: int):
    _check(load().lbm_step(h, int(nsteps)))


def lbm_moments(h, rho, ur, uz, T, on_device: bool):
    _check(load().lbm_moments(h, _ptr(rho), _ptr(ur), _ptr(uz), _ptr(T), int(on_device)))


def lbm_heater_nusselt(h, nz: int):
    """(mean over the heater, Nu(z) with NaN off the heater) of Eq. 43-44."""
    m = C.c_double()
    out = np.zeros(nz, np.float64)
    _check(load().lbm_heater_nusselt(h, C.byref(m), out.ctypes.data))
    return m.value, out


def lbm_nusselt_async(h, out):
    """Enqueue the Nusselt numbers of the current state into out (2 float64, host memory:
    a pinned tensor or a numpy array); valid after lbm_sync."""
    _check(load().lbm_nusselt_async(h, _ptr(out)))


def lbm_sync(h):
    _check(load().lbm_sync(h))


def lbm_stream_function(h, psi, on_device: bool):
    """Stokes stream function (lattice units) into psi (nr*nz floats, or None);
    returns max |psi|."""
    m = C.c_double()
    _check(load().lbm_stream_function(h, _ptr(psi), int(on_device), C.byref(m)))
    return m.value


def lbm_pipe_nusselt(h, nz: int):
    out = np.zeros(nz, np.float64)
    _check(load().lbm_pipe_nusselt(h, out.ctypes.data, int(nz)))
    return out


def lbm_nusselt(h):
    a, b = C.c_double(), C.c_double()
    _check(load().lbm_nusselt(h, C.byref(a), C.byref(b)))
    return a.value, b.value


def lbm_residual(h):
    a, b = C.c_double(), C.c_double()
    _check(load().lbm_residual(h, C.byref(a), C.byref(b)))
    return a.value, b.value


def lbm_run(h, max_steps: int, check_every: int, tol: float):
    n, r = C.c_int64(), C.c_double()
    _check(load().lbm_run(h, int(max_steps), int(check_every), float(tol), C.byref(n), C.byref(r)))
    return n.value, r.value


def lbm_set_porosity_async(h, phi_ptr: int):
    """phi_ptr: address of nr*nz float32 in host memory (pinned for an asynchronous copy)."""
    _check(load().lbm_set_porosity_async(h, phi_ptr))


def lbm_porosity_errors(h, clear: bool = True) -> int:
    n = C.c_uint32()
    _check(load().lbm_porosity_errors(h, C.byref(n), int(clear)))
    return n.value


def lbm_rebase(h):
    _check(load().lbm_rebase(h))


def lbm_node_class(h, out: np.ndarray):
    _check(load().lbm_node_class(h, _ptr(out)))


def lbm_export_populations(h, row0: int, nrows: int, nz: int):
    f = np.empty((9, nrows, nz), np.float64)
    g = np.empty((5, nrows, nz), np.float64)
    _check(load().lbm_export_populations(h, int(row0), int(nrows), f.ctypes.data, g.ctypes.data))
    return f, g


def lbm_get_info(h) -> lbm_info:
    info = lbm_info()
    _check(load().lbm_get_info(h, C.byref(info)))
    return info


def lbm_set_timing(h, enable: bool):
    _check(load().lbm_set_timing(h, int(enable)))


def lbm_set_wait_limit(h, rounds: int):
    _check(load().lbm_set_wait_limit(h, int(rounds)))


def lbm_wait_status(h, clear: bool = False) -> int:
    """LBM_OK, or LBM_ERR_TIMEOUT if a bounded wait of the staged bulk kernel ran out."""
    rc = load().lbm_wait_status(h, int(clear))
    if rc not in (LBM_OK, LBM_ERR_TIMEOUT):
        _check(rc)
    return rc


def lbm_set_staging(h, enable: bool):
    _check(load().lbm_set_staging(h, int(enable)))


def lbm_batch_set_staging(b, enable: bool):
    _check(load().lbm_batch_set_staging(b, int(enable)))


def lbm_batch_set_wait_limit(b, rounds: int):
    _check(load().lbm_batch_set_wait_limit(b, int(rounds)))


def lbm_batch_wait_status(b, clear: bool = False) -> int:
    """LBM_OK, or LBM_ERR_TIMEOUT if a bounded wait of the staged batch kernel ran out."""
    rc = load().lbm_batch_wait_status(b, int(clear))
    if rc not in (LBM_OK, LBM_ERR_TIMEOUT):
        _check(rc)
    return rc


def lbm_kernel_times(h):
    a, b, c, d = C.c_double(), C.c_int64(), C.c_double(), C.c_int64()
    _check(load().lbm_kernel_times(h, C.byref(a), C.byref(b), C.byref(c), C.byref(d)))
    return a.value, b.value, c.value, d.value


def _device_ptr(a, name):
    """Address of a CUDA tensor, or an int taken as a device address (checked by the library)."""
    if isinstance(a, int):
        return a
    if getattr(a, "is_cuda", False):
        return a.data_ptr()
    raise TypeError(f"{name}: a CUDA tensor or a device address is required")


def lbm_field_residual_noalloc(geometry: int, nr: int, nz: int, r0: float, cur, prev, field_stride: int,
                               stream=None):
    """Residual and mass from device field snapshots without any device allocation."""
    a, b = C.c_double(), C.c_double()
    _check(load().lbm_field_residual_noalloc(int(geometry), int(nr), int(nz), float(r0), _device_ptr(cur, "cur"),
                                             _device_ptr(prev, "prev"), int(field_stride), C.byref(a), C.byref(b),
                                             stream))
    return a.value, b.value


def lbm_destroy(h):
    _check(load().lbm_destroy(h))


# ---- convenience wrapper ----------------------------------------------------
class Solver:
    """One problem on the current CUDA device."""

    def __init__(self, params: lbm_params | None = None, **kw):
        self.params = params if params is not None else lbm_params_default(**kw)
        self.h = lbm_create(self.params)
        self.nr, self.nz = self.params.nr, self.params.nz

    def close(self):
        if self.h:
            lbm_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def set_stream(self, stream):
        lbm_set_stream(self.h, stream)

    def set_porosity(self, phi):
        if isinstance(phi, np.ndarray):
            phi = np.ascontiguousarray(phi, dtype=np.float32)
            lbm_set_porosity(self.h, phi, False)
        else:
            lbm_set_porosity(self.h, phi, True)

    def init_fields(self, ur=None, uz=None, T=None):
        on_dev = not any(isinstance(a, np.ndarray) for a in (ur, uz, T))
        if not on_dev:
            ur, uz, T = (None if a is None else np.ascontiguousarray(a, dtype=np.float32) for a in (ur, uz, T))
        lbm_init_fields(self.h, ur, uz, T, on_dev)

    def step(self, n: int = 1):
        lbm_step(self.h, n)

    def moments(self):
        out = [np.empty((self.nr, self.nz), np.float32) for _ in range(4)]
        lbm_moments(self.h, *out, False)
        return out

    def nusselt(self):
        return lbm_nusselt(self.h)

    def pipe_nusselt(self):
        return lbm_pipe_nusselt(self.h, self.nz)

    def heater_nusselt(self):
        return lbm_heater_nusselt(self.h, self.nz)

    def stream_function(self):
        """(psi[nr, nz], max |psi|) of the current state, lattice units."""
        psi = np.empty((self.nr, self.nz), np.float32)
        m = lbm_stream_function(self.h, psi, False)
        return psi, m

    def residual(self):
        return lbm_residual(self.h)

    def run(self, max_steps, check_every=100, tol=1e-8):
        return lbm_run(self.h, max_steps, check_every, tol)

    def rebase(self):
        lbm_rebase(self.h)

    def node_class(self):
        out = np.empty((self.nr, self.nz), np.uint8)
        lbm_node_class(self.h, out)
        return out

    def export_populations(self, row0: int = 0, nrows: int | None = None):
        return lbm_export_populations(self.h, row0, self.nr - row0 if nrows is None else nrows, self.nz)

    def info(self) -> lbm_info:
        return lbm_get_info(self.h)


# ---- batches ----------------------------------------------------------------
def lbm_batch_create(params) -> int:
    arr = (lbm_params * len(params))(*params)
    h = _vp()
    _check(load().lbm_batch_create(arr, len(params), C.byref(h)))
    return h.value


def lbm_batch_set_stream(b, stream):
    _check(load().lbm_batch_set_stream(b, stream))


def lbm_batch_set_porosity(b, i: int, phi, on_device: bool):
    _check(load().lbm_batch_set_porosity(b, int(i), _ptr(phi), int(on_device)))


def lbm_batch_init_fields(b, i: int, ur, uz, T, on_device: bool):
    _check(load().lbm_batch_init_fields(b, int(i), _ptr(ur), _ptr(uz), _ptr(T), int(on_device)))


def lbm_batch_step(b, nsteps: int):
    _check(load().lbm_batch_step(b, int(nsteps)))


def lbm_batch_run(b, n: int, max_steps: int, check_every: int, tol: float):
    steps = np.zeros(n, np.int64)
    res = np.zeros(n, np.float64)
    _check(load().lbm_batch_run(b, int(max_steps), int(check_every), float(tol), steps.ctypes.data, res.ctypes.data))
    return steps, res


def lbm_batch_rebase(b):
    _check(load().lbm_batch_rebase(b))


def lbm_batch_pipe_nusselt(b, i: int, nz: int):
    out = np.zeros(nz, np.float64)
    _check(load().lbm_batch_pipe_nusselt(b, int(i), out.ctypes.data, int(nz)))
    return out


def lbm_batch_nusselt(b, n: int):
    a = np.zeros(n, np.float64)
    c = np.zeros(n, np.float64)
    _check(load().lbm_batch_nusselt(b, a.ctypes.data, c.ctypes.data))
    return a, c


def lbm_batch_moments(b, i: int, rho, ur, uz, T, on_device: bool):
    _check(load().lbm_batch_moments(b, int(i), _ptr(rho), _ptr(ur), _ptr(uz), _ptr(T), int(on_device)))


def lbm_batch_tune(b, steps: int):
    cz, rw, ms = C.c_int32(), C.c_int32(), C.c_float()
    _check(load().lbm_batch_tune(b, int(steps), C.byref(cz), C.byref(rw), C.byref(ms)))
    return cz.value, rw.value, ms.value


def lbm_batch_get_info(b, i: int) -> lbm_info:
    info = lbm_info()
    _check(load().lbm_batch_get_info(b, int(i), C.byref(info)))
    return info


def lbm_batch_destroy(b):
    _check(load().lbm_batch_destroy(b))


class Batch:
    """Independent problems advanced together on the current CUDA device."""

    def __init__(self, params):
        self.params = list(params)
        self.n = len(self.params)
        self.b = lbm_batch_create(self.params)

    def close(self):
        if self.b:
            lbm_batch_destroy(self.b)
            self.b = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def set_porosity(self, i, phi):
        lbm_batch_set_porosity(self.b, i, np.ascontiguousarray(phi, dtype=np.float32), False)

    def init_fields(self, i, ur=None, uz=None, T=None):
        ur, uz, T = (None if a is None else np.ascontiguousarray(a, dtype=np.float32) for a in (ur, uz, T))
        lbm_batch_init_fields(self.b, i, ur, uz, T, False)

    def step(self, n=1):
        lbm_batch_step(self.b, n)

    def run(self, max_steps, check_every=1000, tol=1e-8):
        return lbm_batch_run(self.b, self.n, max_steps, check_every, tol)

    def rebase(self):
        lbm_batch_rebase(self.b)

    def pipe_nusselt(self, i):
        return lbm_batch_pipe_nusselt(self.b, i, self.params[i].nz)

    def nusselt(self):
        return lbm_batch_nusselt(self.b, self.n)

    def moments(self, i):
        p = self.params[i]
        out = [np.empty((p.nr, p.nz), np.float32) for _ in range(4)]
        lbm_batch_moments(self.b, i, *out, False)
        return out

    def tune(self, steps=10):
        return lbm_batch_tune(self.b, steps)

    def info(self, i) -> lbm_info:
        return lbm_batch_get_info(self.b, i)
