"""CPU oracle for the HGKS hot path: a plain FP64 statement of the scheme.

TEST INFRASTRUCTURE.  Only the test-suite, ``__graft_entry__.smoke()`` and the
benchmark's CPU-baseline leg may import this package.  It shares no code with
the GPU library (``paper_2407_00656_b300``); both read the same seeded input
arrays and nothing else.

The C++ source (``hgks_oracle.cpp``) is compiled with g++ on first use into
``oracle/_build/liboracle.so`` and driven through ctypes.
"""
from __future__ import annotations

import ctypes as C
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "hgks_oracle.cpp")
_OUT = os.path.join(_HERE, "_build", "liboracle.so")
_lock = threading.Lock()
_lib = None

PARAM_KEYS = ("gamma", "mu_ref", "T_ref", "visc_exp", "Pr", "cfl", "tau_c", "eps", "glin")
DEFAULTS = dict(gamma=1.4, mu_ref=0.0, T_ref=1.0, visc_exp=0.0, Pr=1.0, cfl=0.4, tau_c=0.0,
                eps=1e-8, glin=0.025, qinf=(1.0, 0.0, 0.0, 0.0, 2.5))


def build(force: bool = False) -> str:
    """Compile the oracle shared library (g++, FP64, OpenMP) if out of date."""
    os.makedirs(os.path.dirname(_OUT), exist_ok=True)
    if force or not os.path.exists(_OUT) or os.path.getmtime(_OUT) < os.path.getmtime(_SRC):
        tmp = _OUT + f".{os.getpid()}.tmp"
        cmd = ["g++", "-O2", "-std=c++17", "-fopenmp", "-fPIC", "-shared", "-fno-fast-math",
               "-ffp-contract=off", _SRC, "-o", tmp]
        subprocess.run(cmd, check=True)
        os.replace(tmp, _OUT)
    return _OUT


def _load():
    global _lib
    with _lock:
        if _lib is None:
            lib = C.CDLL(build())
            P = C.c_void_p
            d = C.POINTER(C.c_double)
            i64 = C.POINTER(C.c_int64)
            i32 = C.POINTER(C.c_int32)
            lib.o_create.restype = P
            lib.o_create.argtypes = [C.c_int64, d, C.c_int64, i32, C.c_int32, i64, i64, C.c_int64, i64, i32, d, d,
                                     C.c_char_p, C.c_int]
            lib.o_destroy.argtypes = [P]
            lib.o_set_params.argtypes = [P, d]
            lib.o_set_threads.argtypes = [C.c_int]
            lib.o_get_threads.restype = C.c_int
            lib.o_n_faces.restype = C.c_int64
            lib.o_n_faces.argtypes = [P]
            lib.o_set_state.argtypes = [P, d, C.c_double]
            lib.o_get_state.argtypes = [P, d, d, i64]
            lib.o_step.restype = C.c_int
            lib.o_step.argtypes = [P, C.c_int, C.c_double, C.c_double]
            lib.o_time_step.restype = C.c_double
            lib.o_time_step.argtypes = [P]
            lib.o_cell_geometry.argtypes = [P, d, d, d, d]
            lib.o_stencil_info.argtypes = [P, C.c_int, C.POINTER(C.c_int), C.POINTER(C.c_int)]
            lib.o_stencil.argtypes = [P, C.c_int, C.POINTER(C.c_int), C.POINTER(C.c_int), d]
            lib.o_reconstruct.argtypes = [P, C.c_int]
            lib.o_recon_eval.argtypes = [P, C.c_int, d, d, d]
            lib.o_recon_weights.argtypes = [P, C.c_int, d]
            lib.o_operator.argtypes = [P, C.c_double, d, d]
            lib.o_flux_point.argtypes = [d, d, d, d, d, d, C.c_double, d, d]
            lib.o_gauss_moments.argtypes = [C.c_double, C.c_double, C.c_int, d]
            lib.o_micro_slope.argtypes = [C.c_double, d, d, d]
            lib.o_boundary_state.argtypes = [d, C.c_int, d, d, d]
            lib.o_boundary_flux.argtypes = [d, C.c_int, d, d, d, C.c_double, d, d, d, d]
            lib.o_s2o4_linear.argtypes = [C.c_int, d, C.c_double, C.c_double]
            _lib = lib
    return _lib


def _dp(a):
    return a.ctypes.data_as(C.POINTER(C.c_double))


def _f64(a):
    return np.ascontiguousarray(a, dtype=np.float64)


def param_array(**kw) -> np.ndarray:
    p = dict(DEFAULTS)
    p.update(kw)
    arr = [float(p[k]) for k in PARAM_KEYS] + [float(x) for x in p["qinf"]]
    return np.array(arr, dtype=np.float64)


def set_threads(n: int) -> None:
    _load().o_set_threads(int(n))


def get_threads() -> int:
    return int(_load().o_get_threads())


class Oracle:
    """One mesh and state on the CPU oracle."""

    def __init__(self, xyz, cells, periods=None, bface_nodes=None, bface_tag=None, **params):
        lib = _load()
        xyz = _f64(xyz)
        cells = np.ascontiguousarray(cells, dtype=np.int64)
        self.n_cells = cells.shape[0]
        self.params = param_array(**params)
        nb = 0 if bface_nodes is None else len(bface_nodes)
        bfn = np.ascontiguousarray(bface_nodes if nb else np.zeros((1, 4)), dtype=np.int64)
        if nb and bfn.shape[1] == 3:
            bfn = np.ascontiguousarray(np.concatenate([bfn, -np.ones((nb, 1), dtype=np.int64)], axis=1))
        bft = np.ascontiguousarray(bface_tag if nb else np.zeros(1), dtype=np.int32)
        per = None if periods is None else _f64(periods)
        err = C.create_string_buffer(256)
        self._h = lib.o_create(
            len(xyz), _dp(xyz), self.n_cells, None, int(cells.shape[1]), None,
            cells.ctypes.data_as(C.POINTER(C.c_int64)), nb, bfn.ctypes.data_as(C.POINTER(C.c_int64)),
            bft.ctypes.data_as(C.POINTER(C.c_int32)), None if per is None else _dp(per), _dp(self.params), err, 256)
        if not self._h:
            raise ValueError("oracle mesh build failed: " + err.value.decode())
        self._lib = lib

    def __del__(self):
        h = getattr(self, "_h", None)
        if h:
            self._lib.o_destroy(h)
            self._h = None

    @property
    def n_faces(self) -> int:
        return int(self._lib.o_n_faces(self._h))

    def set_state(self, q, t: float = 0.0):
        q = _f64(q).reshape(self.n_cells, 5)
        self._lib.o_set_state(self._h, _dp(q), float(t))

    def get_state(self):
        q = np.empty((self.n_cells, 5))
        t = C.c_double()
        s = C.c_int64()
        self._lib.o_get_state(self._h, _dp(q), C.byref(t), C.byref(s))
        return q, t.value, s.value

    def step(self, n: int = 1, t_end: float = 0.0, dt_fixed: float = 0.0) -> None:
        rc = self._lib.o_step(self._h, int(n), float(t_end), float(dt_fixed))
        if rc != 0:
            raise FloatingPointError(f"oracle step failed with status {rc}")

    def time_step(self) -> float:
        return float(self._lib.o_time_step(self._h))

    def geometry(self):
        n = self.n_cells
        vol, cen, mom, hdt = np.empty(n), np.empty((n, 3)), np.empty((n, 6)), np.empty(n)
        self._lib.o_cell_geometry(self._h, _dp(vol), _dp(cen), _dp(mom), _dp(hdt))
        return vol, cen, mom, hdt

    def stencil(self, c: int):
        K, M = C.c_int(), C.c_int()
        self._lib.o_stencil_info(self._h, int(c), C.byref(K), C.byref(M))
        kind = (C.c_int * K.value)()
        ids = (C.c_int * K.value)()
        cen = np.empty((K.value, 3))
        self._lib.o_stencil(self._h, int(c), kind, ids, _dp(cen))
        return np.array(kind), np.array(ids), cen, M.value

    def reconstruct(self, force_linear: bool = False):
        self._lib.o_reconstruct(self._h, 1 if force_linear else 0)

    def recon_eval(self, c: int, x):
        x = _f64(x)
        val = np.empty(5)
        grad = np.empty((5, 3))
        self._lib.o_recon_eval(self._h, int(c), _dp(x), _dp(val), _dp(grad))
        return val, grad

    def recon_weights(self, c: int):
        _, _, _, M = self.stencil(c)
        w = np.empty((5, M + 1))
        self._lib.o_recon_weights(self._h, int(c), _dp(w))
        return w

    def operator(self, dt: float):
        L = np.empty((self.n_cells, 5))
        dL = np.empty((self.n_cells, 5))
        self._lib.o_operator(self._h, float(dt), _dp(L), _dp(dL))
        return L, dL


def flux_point(n, ql, gl, qr, gr, dt, **params):
    """Gas-kinetic flux F^n and dF/dt at one point with unit normal n (global frame)."""
    lib = _load()
    p = param_array(**params)
    F = np.empty(5)
    dF = np.empty(5)
    n, ql, gl, qr, gr = (_f64(a) for a in (n, ql, gl, qr, gr))
    lib.o_flux_point(_dp(p), _dp(n), _dp(ql), _dp(gl), _dp(qr), _dp(gr), float(dt), _dp(F), _dp(dF))
    return F, dF


def gauss_moments(U: float, lam: float, half: int):
    m = np.empty(12)
    _load().o_gauss_moments(float(U), float(lam), int(half), _dp(m))
    return m


def micro_slope(q, b, gamma: float = 1.4):
    a = np.empty(5)
    q, b = _f64(q), _f64(b)
    _load().o_micro_slope(float(gamma), _dp(q), _dp(b), _dp(a))
    return a


def boundary_state(kind: int, n, q, **params):
    p = param_array(**params)
    o = np.empty(5)
    n, q = _f64(n), _f64(q)
    _load().o_boundary_state(_dp(p), int(kind), _dp(n), _dp(q), _dp(o))
    return o


def boundary_flux(kind: int, n, ql, gl, dt, **params):
    """Flux F^n, dF/dt at a boundary Gauss point (kind 2 far field, 3 wall)
    as the stage operator forms it, with the far side (qr, gr) it used."""
    lib = _load()
    p = param_array(**params)
    F, dF, qr, gr = np.empty(5), np.empty(5), np.empty(5), np.empty((5, 3))
    n, ql, gl = (_f64(a) for a in (n, ql, gl))
    lib.o_boundary_flux(_dp(p), int(kind), _dp(n), _dp(ql), _dp(gl), float(dt), _dp(F), _dp(dF), _dp(qr), _dp(gr))
    return F, dF, qr, gr


def s2o4_linear(q, lam: float, dt: float):
    """One S2O4 step of dQ/dt = lam Q through the oracle's S2O4 routine."""
    q = _f64(q).copy()
    _load().o_s2o4_linear(len(q), _dp(q), float(lam), float(dt))
    return q
