"""ctypes wrapper of the FP64 CPU oracle (``lbm_oracle.c``).

Test infrastructure only: the test suite, the smoke check and the CPU-baseline leg
of the benchmark may import this module; the library package never does.  The
oracle shares no code with the CUDA path.

Every array is float64, population-major, z fastest: ``f[i, kr, kz]`` for the
nine D2Q9 populations and ``g[i, kr, kz]`` for the five D2Q5 ones (Eq. 14, 34).
"""
from __future__ import annotations

import ctypes as C
import os
import subprocess
import threading

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
SRC = os.path.join(HERE, "lbm_oracle.c")
LIB = os.path.join(HERE, "liblbm_oracle.so")

ANNULUS, ANNULUS_PERIODIC_Z, PIPE_PERIODIC_Z, PIPE_INFLOW = 0, 1, 2, 3
FLUID, WALL_IN, WALL_OUT, BOTTOM, TOP, AXIS, INLET, OUTLET = 0, 1, 2, 3, 4, 5, 6, 7

_lock = threading.Lock()
_lib = None


def build(force: bool = False) -> str:
    """Compile the oracle with gcc (plain C99, OpenMP over rows, no FMA contraction
    so that x86 and Arm hosts round identically)."""
    if not force and os.path.exists(LIB) and os.path.getmtime(LIB) >= os.path.getmtime(SRC):
        return LIB
    tmp = LIB + f".tmp{os.getpid()}"
    cmd = ["gcc", "-O2", "-std=c99", "-fPIC", "-shared", "-fopenmp", "-ffp-contract=off",
           "-o", tmp, SRC, "-lm"]
    subprocess.run(cmd, check=True)
    os.replace(tmp, LIB)
    return LIB


class Params(C.Structure):
    _fields_ = [
        ("nr", C.c_int32), ("nz", C.c_int32), ("geometry", C.c_int32), ("collision", C.c_int32),
        ("radius_ratio", C.c_double),
        ("Ra", C.c_double), ("Da", C.c_double), ("Pr", C.c_double), ("J", C.c_double),
        ("lam", C.c_double), ("Ma", C.c_double), ("tau_nu", C.c_double),
        ("F_eps", C.c_double), ("eps_mean", C.c_double),
        ("T_hot", C.c_double), ("T_cold", C.c_double), ("body_accel_z", C.c_double),
        ("init_noise", C.c_double), ("seed", C.c_uint64), ("u_in", C.c_double),
        ("heater_len", C.c_double), ("heater_center", C.c_double),
    ]


def params(**kw) -> Params:
    """Parameters with the porous-annulus defaults (R* = 2, eps = 0.6, Da = 1e-2,
    Ra = 1e3, Pr = 1, J = lambda = 1, Ma = 0.1, Ergun F_eps, T_hot = 1, T_cold = 0)."""
    d = dict(nr=48, nz=96, geometry=ANNULUS, collision=0, radius_ratio=2.0, Ra=1e3, Da=1e-2, Pr=1.0, J=1.0,
             lam=1.0, Ma=0.1, tau_nu=0.0, F_eps=-1.0, eps_mean=0.6, T_hot=1.0, T_cold=0.0,
             body_accel_z=0.0, init_noise=1e-3, seed=1, u_in=0.0, heater_len=0.0, heater_center=0.5)
    for k in kw:
        if k not in d:
            raise KeyError(k)
    d.update(kw)
    p = Params()
    for k, v in d.items():
        setattr(p, k, v)
    return p


def lib():
    global _lib
    with _lock:
        if _lib is None:
            build()
            L = C.CDLL(LIB)
            dp = C.POINTER(C.c_double)
            pp = C.POINTER(Params)
            L.orc_derive_export.argtypes = [pp, dp]
            L.orc_matrices.argtypes = [dp, dp]
            L.orc_feq.argtypes = [C.c_double] * 5 + [dp]
            L.orc_meq.argtypes = [C.c_double] * 5 + [dp]
            L.orc_source.argtypes = [C.c_double] * 7 + [dp]
            L.orc_init.argtypes = [pp, dp, dp, dp, dp, dp, dp]
            L.orc_run.argtypes = [pp, dp, dp, dp, C.c_int64, C.c_int]
            L.orc_moments.argtypes = [pp, dp, dp, dp, dp, dp, dp, dp]
            L.orc_nusselt.argtypes = [pp, dp, dp, dp]
            L.orc_pipe_nusselt.argtypes = [pp, dp, dp, dp]
            L.orc_heater_nusselt.argtypes = [pp, dp, dp, dp]
            L.orc_stream_function.argtypes = [pp, dp, dp, dp]
            L.orc_residual.argtypes = [pp] + [dp] * 9
            L.orc_node_class.argtypes = [pp, C.POINTER(C.c_uint8)]
            L.orc_splitmix64.argtypes = [C.c_uint64, C.c_uint64]
            L.orc_splitmix64.restype = C.c_uint64
            L.orc_collide_node.argtypes = [pp, dp, C.c_int, C.c_double, C.c_double, dp, dp, C.c_int,
                                           C.c_double, dp, dp, dp]
            L.orc_node_update.argtypes = [pp, dp, dp, dp, C.c_int, C.c_int, dp, dp, dp]
            _lib = L
    return _lib


def _d(a):
    return a.ctypes.data_as(C.POINTER(C.c_double))


def _f64(a):
    return np.ascontiguousarray(a, dtype=np.float64)


def derive(p: Params) -> dict:
    out = np.zeros(11)
    rc = lib().orc_derive_export(C.byref(p), _d(out))
    if rc:
        raise ValueError("invalid oracle parameters")
    keys = ["L", "H", "r0", "tau", "tauT", "nu_e", "nu", "gbeta", "T0", "Ma", "Kbar"]
    return dict(zip(keys, out.tolist()))


def matrices():
    M = np.zeros((9, 9))
    Mi = np.zeros((9, 9))
    lib().orc_matrices(_d(M), _d(Mi))
    return M, Mi


def feq(r, rho, ur, uz, phi):
    out = np.zeros(9)
    lib().orc_feq(r, rho, ur, uz, phi, _d(out))
    return out


def meq(r, rho, ur, uz, phi):
    out = np.zeros(9)
    lib().orc_meq(r, rho, ur, uz, phi, _d(out))
    return out


def source(r, rho, ur, uz, phi, Ftr, Ftz):
    out = np.zeros(9)
    lib().orc_source(r, rho, ur, uz, phi, Ftr, Ftz, _d(out))
    return out


def splitmix64(seed: int, n: int) -> int:
    return int(lib().orc_splitmix64(seed, n))


def node_class(p: Params) -> np.ndarray:
    out = np.zeros((p.nr, p.nz), dtype=np.uint8)
    lib().orc_node_class(C.byref(p), out.ctypes.data_as(C.POINTER(C.c_uint8)))
    return out


def collide_node(p: Params, r, phi, f, g, s=None, cartesian=False, wall=False, T_wall=0.0):
    """One collision at one node; returns (f+, g+, (rho, u_r, u_z, T))."""
    f = _f64(f)
    g = _f64(g)
    fo = np.zeros(9)
    go = np.zeros(5)
    mo = np.zeros(4)
    sp = None
    if s is not None:
        s = _f64(s)
        sp = _d(s)
    rc = lib().orc_collide_node(C.byref(p), sp, int(cartesian), r, phi, _d(f), _d(g), int(wall),
                                T_wall, _d(fo), _d(go), _d(mo))
    if rc:
        raise ValueError("invalid oracle parameters")
    return fo, go, mo


class State:
    """Post-collision populations of the whole grid plus the porosity field."""

    def __init__(self, p: Params, phi=None, ur=None, uz=None, T=None):
        self.p = p
        n = (p.nr, p.nz)
        self.phi = _f64(np.full(n, p.eps_mean) if phi is None else phi).reshape(n)
        self.f = np.zeros((9,) + n)
        self.g = np.zeros((5,) + n)
        args = [None if a is None else _f64(a).reshape(n) for a in (ur, uz, T)]
        ptrs = [None if a is None else _d(a) for a in args]
        rc = lib().orc_init(C.byref(p), _d(self.phi), ptrs[0], ptrs[1], ptrs[2], _d(self.f), _d(self.g))
        if rc:
            raise ValueError("invalid oracle parameters")
        self.steps = 0

    def run(self, nsteps: int, threads: int | None = None):
        if threads is None:
            threads = os.cpu_count() or 1
        rc = lib().orc_run(C.byref(self.p), _d(self.phi), _d(self.f), _d(self.g), int(nsteps), int(threads))
        if rc:
            raise RuntimeError("oracle run failed")
        self.steps += nsteps
        return self

    def moments(self):
        n = (self.p.nr, self.p.nz)
        rho, ur, uz, T = (np.zeros(n) for _ in range(4))
        lib().orc_moments(C.byref(self.p), _d(self.phi), _d(self.f), _d(self.g), _d(rho), _d(ur), _d(uz), _d(T))
        return rho, ur, uz, T

    def nusselt(self, T=None):
        if T is None:
            T = self.moments()[3]
        T = _f64(T)
        a = C.c_double()
        b = C.c_double()
        lib().orc_nusselt(C.byref(self.p), _d(T), C.byref(a), C.byref(b))
        return a.value, b.value

    def heater_nusselt(self):
        return heater_nusselt(self.p, self.moments()[3])

    def stream_function(self):
        """(psi field, max |psi|) of the current state, lattice units."""
        return stream_function(self.p, self.moments()[2])

    def pipe_nusselt(self):
        """Local wall Nusselt number Nu(z) of Eq. 40 with the mixing-cup bulk
        temperature (pipe with inlet and outlet)."""
        m = self.moments()
        return pipe_nusselt(self.p, m[2], m[3])


def heater_nusselt(p: Params, T):
    """Eq. 43-44: (mean over the heater, local Nu(z) with NaN off the heater)."""
    T = _f64(T)
    m = C.c_double()
    nz = np.zeros(p.nz)
    if lib().orc_heater_nusselt(C.byref(p), _d(T), C.byref(m), _d(nz)):
        raise ValueError("heater_nusselt needs heater_len > 0")
    return m.value, nz


def stream_function(p: Params, uz):
    """Stokes stream function psi(r, z) = int r' u_z dr' from the inner wall (annulus)
    or the axis (pipes), trapezoid rule; returns (psi[nr, nz], max |psi|)."""
    uz = _f64(uz)
    psi = np.zeros((p.nr, p.nz))
    m = C.c_double()
    if lib().orc_stream_function(C.byref(p), _d(uz), _d(psi), C.byref(m)):
        raise ValueError("invalid parameters")
    return psi, m.value


def pipe_nusselt(p: Params, uz, T):
    uz, T = _f64(uz), _f64(T)
    out = np.zeros(p.nz)
    if lib().orc_pipe_nusselt(C.byref(p), _d(uz), _d(T), _d(out)):
        raise ValueError("pipe_nusselt needs the pipe with inlet and outlet")
    return out


def node_update(p: Params, phi, f, g, kr: int, kz: int):
    """Update of one node from a state given as full float64 arrays phi[nr, nz],
    f[9, nr, nz], g[5, nr, nz]; only rows kr-2..kr+2 are read.
    Returns (f+, g+, (rho, u_r, u_z, T))."""
    for a in (phi, f, g):
        assert a.dtype == np.float64 and a.flags.c_contiguous
    fo, go, mo = np.zeros(9), np.zeros(5), np.zeros(4)
    rc = lib().orc_node_update(C.byref(p), _d(phi), _d(f), _d(g), int(kr), int(kz), _d(fo), _d(go), _d(mo))
    if rc:
        raise ValueError("invalid oracle parameters")
    return fo, go, mo


def residual(p: Params, cur, prev):
    """cur = (rho, u_r, u_z, T) of state n, prev = same of state n - 1."""
    rho, ur, uz, T = (_f64(a) for a in cur)
    _, urp, uzp, Tp = (_f64(a) for a in prev)
    res = C.c_double()
    mass = C.c_double()
    lib().orc_residual(C.byref(p), _d(rho), _d(ur), _d(uz), _d(T), _d(urp), _d(uzp), _d(Tp),
                       C.byref(res), C.byref(mass))
    return res.value, mass.value
