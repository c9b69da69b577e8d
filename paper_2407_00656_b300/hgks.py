"""ctypes binding of libhgks (include/hgks.h): the same entry points, with
argument marshalling only.  Every step of the scheme runs in the library's
CUDA kernels; nothing here computes.

The library is loaded from this package directory (``libhgks.so``, built by
``paper_2407_00656_b300.build``).  A missing library raises ImportError at
first use: there is no fallback path.
"""
from __future__ import annotations

import ctypes as C
import os
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "libhgks.so")

HGKS_OK, HGKS_EINVAL, HGKS_ENOMEM, HGKS_EMESH, HGKS_ECUDA, HGKS_ENONFINITE, HGKS_ETIMEOUT = 0, -1, -2, -3, -4, -5, -6
HGKS_TET4, HGKS_HEX8 = 4, 8
HGKS_BC_PERIODIC, HGKS_BC_FARFIELD, HGKS_BC_WALL = 1, 2, 3
HGKS_FP64, HGKS_FP32_MIXED = 0, 1

_ERRNAMES = {0: "HGKS_OK", -1: "HGKS_EINVAL", -2: "HGKS_ENOMEM", -3: "HGKS_EMESH", -4: "HGKS_ECUDA",
             -5: "HGKS_ENONFINITE", -6: "HGKS_ETIMEOUT"}


class hgks_mesh_desc(C.Structure):
    _fields_ = [
        ("n_nodes", C.c_int64),
        ("xyz", C.POINTER(C.c_double)),
        ("n_cells", C.c_int64),
        ("cell_type", C.c_int32),
        ("sfc_reorder", C.c_int32),
        ("cell_nodes", C.POINTER(C.c_int64)),
        ("n_bfaces", C.c_int64),
        ("bface_nodes", C.POINTER(C.c_int64)),
        ("bface_tag", C.POINTER(C.c_int32)),
        ("periods", C.POINTER(C.c_double)),
    ]


class hgks_params(C.Structure):
    _fields_ = [
        ("gamma", C.c_double), ("mu_ref", C.c_double), ("T_ref", C.c_double), ("visc_exp", C.c_double),
        ("Pr", C.c_double), ("cfl", C.c_double), ("tau_num_c", C.c_double), ("weno_eps", C.c_double),
        ("weno_gamma_lin", C.c_double), ("q_inf", C.c_double * 5), ("precision", C.c_int32),
        ("use_graph", C.c_int32), ("autotune", C.c_int32), ("persistent", C.c_int32), ("stream", C.c_void_p),
    ]


class HGKSError(RuntimeError):
    def __init__(self, code: int, where: str, msg: str):
        super().__init__(f"{where}: {_ERRNAMES.get(code, code)}: {msg}")
        self.code = code


_lib = None
_lock = threading.Lock()
EXPORTS = ("hgks_params_default", "hgks_mesh_create", "hgks_mesh_destroy", "hgks_mesh_clone", "hgks_mesh_geometry", "hgks_mesh_info",
           "hgks_init",
           "hgks_batch_init", "hgks_members", "hgks_write", "hgks_member_write", "hgks_step", "hgks_query",
           "hgks_sync", "hgks_read", "hgks_member_read", "hgks_stage_operator", "hgks_profile", "hgks_solver_bytes",
           "hgks_tuning", "hgks_set_tuning", "hgks_destroy", "hgks_last_error", "hgks_cfl_dt_noalloc",
           "hgks_dmesh_create", "hgks_dmesh_release", "hgks_dmesh_info", "hgks_init_shared",
           "hgks_test_barrier_limit", "hgks_test_fail_alloc", "hgks_test_erfcx")


def lib():
    """Load libhgks.so (raises ImportError when it has not been built)."""
    global _lib
    with _lock:
        if _lib is None:
            if not os.path.exists(LIB_PATH):
                raise ImportError(f"libhgks.so not found at {LIB_PATH}; run python -m paper_2407_00656_b300.build")
            L = C.CDLL(LIB_PATH)
            vp, dp = C.c_void_p, C.POINTER(C.c_double)
            L.hgks_params_default.argtypes = [C.POINTER(hgks_params)]
            L.hgks_params_default.restype = None
            L.hgks_mesh_create.argtypes = [C.POINTER(hgks_mesh_desc), C.POINTER(vp)]
            L.hgks_mesh_destroy.argtypes = [vp]
            L.hgks_mesh_destroy.restype = None
            L.hgks_mesh_geometry.argtypes = [vp, dp, dp]
            L.hgks_mesh_geometry.restype = C.c_int
            L.hgks_mesh_clone.argtypes = [vp, C.POINTER(vp)]
            L.hgks_mesh_clone.restype = C.c_int
            L.hgks_mesh_info.argtypes = [vp, C.c_int]
            L.hgks_mesh_info.restype = C.c_int64
            L.hgks_init.argtypes = [vp, C.POINTER(hgks_params), dp, C.POINTER(vp)]
            L.hgks_write.argtypes = [vp, dp, C.c_double]
            L.hgks_batch_init.argtypes = [C.POINTER(vp), C.c_int, C.POINTER(hgks_params), C.POINTER(dp), C.POINTER(vp)]
            L.hgks_members.argtypes = [vp]
            L.hgks_member_write.argtypes = [vp, C.c_int, dp, C.c_double]
            L.hgks_member_read.argtypes = [vp, C.c_int, dp, dp, C.POINTER(C.c_int64)]
            L.hgks_query.argtypes = [vp]
            L.hgks_solver_bytes.argtypes = [vp]
            L.hgks_solver_bytes.restype = C.c_int64
            L.hgks_tuning.argtypes = [vp, C.POINTER(C.c_int), C.POINTER(C.c_int)]
            L.hgks_tuning.restype = C.c_int
            L.hgks_set_tuning.argtypes = [vp, C.c_int, C.c_int]
            L.hgks_set_tuning.restype = C.c_int
            L.hgks_step.argtypes = [vp, C.c_int, C.c_double, C.c_double]
            L.hgks_sync.argtypes = [vp]
            L.hgks_read.argtypes = [vp, dp, dp, C.POINTER(C.c_int64)]
            L.hgks_stage_operator.argtypes = [vp, C.c_double, dp, dp]
            L.hgks_profile.argtypes = [vp, C.c_int, C.c_double, C.c_double, dp]
            L.hgks_test_barrier_limit.argtypes = [vp, C.c_int64]
            L.hgks_test_barrier_limit.restype = C.c_int
            L.hgks_test_fail_alloc.argtypes = [C.c_int]
            L.hgks_test_fail_alloc.restype = C.c_int
            L.hgks_test_erfcx.argtypes = [dp, dp, C.c_int64]
            L.hgks_test_erfcx.restype = C.c_int
            L.hgks_cfl_dt_noalloc.argtypes = [vp, vp, C.c_int64, C.POINTER(hgks_params), vp, vp]
            L.hgks_cfl_dt_noalloc.restype = C.c_int
            L.hgks_dmesh_create.argtypes = [vp, vp, C.POINTER(vp)]
            L.hgks_dmesh_create.restype = C.c_int
            L.hgks_dmesh_release.argtypes = [vp]
            L.hgks_dmesh_release.restype = None
            L.hgks_dmesh_info.argtypes = [vp, C.c_int]
            L.hgks_dmesh_info.restype = C.c_int64
            L.hgks_init_shared.argtypes = [vp, C.POINTER(hgks_params), dp, C.POINTER(vp)]
            L.hgks_init_shared.restype = C.c_int
            L.hgks_destroy.argtypes = [vp]
            L.hgks_destroy.restype = None
            L.hgks_last_error.restype = C.c_char_p
            for name in ("hgks_mesh_create", "hgks_init", "hgks_write", "hgks_step", "hgks_sync", "hgks_read",
                         "hgks_stage_operator", "hgks_profile", "hgks_batch_init", "hgks_members",
                         "hgks_member_write", "hgks_member_read", "hgks_query"):
                getattr(L, name).restype = C.c_int
            _lib = L
    return _lib


def _check(rc: int, where: str):
    if rc != HGKS_OK:
        raise HGKSError(rc, where, lib().hgks_last_error().decode())


def _dp(a):
    return a.ctypes.data_as(C.POINTER(C.c_double))


def params_default() -> hgks_params:
    p = hgks_params()
    lib().hgks_params_default(C.byref(p))
    return p


def make_params(**kw) -> hgks_params:
    """hgks_params with defaults overridden by keyword (q_inf a 5-sequence)."""
    p = params_default()
    for k, v in kw.items():
        if k == "q_inf":
            for i in range(5):
                p.q_inf[i] = float(v[i])
        elif k == "stream":
            p.stream = C.c_void_p(v)
        else:
            setattr(p, k, v)
    return p


def cfl_dt_noalloc(q_ptr: int, hdt_ptr: int, n_cells: int, params: hgks_params, dt_ptr: int, stream: int = 0):
    """hgks_cfl_dt_noalloc on caller-owned device buffers (raw device addresses):
    q [n][5], hdt [n], result written to dt_ptr on the GPU."""
    _check(lib().hgks_cfl_dt_noalloc(C.c_void_p(q_ptr), C.c_void_p(hdt_ptr), int(n_cells), C.byref(params),
                                     C.c_void_p(dt_ptr), C.c_void_p(stream or None)), "hgks_cfl_dt_noalloc")


def test_fail_alloc(n: int) -> None:
    """hgks_test_fail_alloc: make the library's n-th device allocation from now
    on fail (n = 0: the next one); n < 0 switches the hook off."""
    _check(lib().hgks_test_fail_alloc(int(n)), "hgks_test_fail_alloc")


def test_erfcx(x) -> np.ndarray:
    """hgks_test_erfcx: the binary64 flux's erfcx on the values x."""
    x = np.ascontiguousarray(x, dtype=np.float64).ravel()
    y = np.empty_like(x)
    _check(lib().hgks_test_erfcx(_dp(x), _dp(y), x.size), "hgks_test_erfcx")
    return y


class Mesh:
    """hgks_mesh_create / hgks_mesh_destroy."""

    def __init__(self, xyz, cells, periods=None, bface_nodes=None, bface_tag=None, sfc_reorder: bool = True):
        self._keep = []
        xyz = np.ascontiguousarray(xyz, dtype=np.float64)
        cells = np.ascontiguousarray(cells, dtype=np.int64)
        d = hgks_mesh_desc()
        d.n_nodes = len(xyz)
        d.xyz = _dp(xyz)
        d.n_cells = len(cells)
        d.cell_type = cells.shape[1]
        d.sfc_reorder = 1 if sfc_reorder else 0
        d.cell_nodes = cells.ctypes.data_as(C.POINTER(C.c_int64))
        self._keep += [xyz, cells]
        if bface_nodes is not None and len(bface_nodes):
            bfn = np.asarray(bface_nodes, dtype=np.int64)
            if bfn.shape[1] == 3:
                bfn = np.concatenate([bfn, -np.ones((len(bfn), 1), dtype=np.int64)], axis=1)
            bfn = np.ascontiguousarray(bfn)
            bft = np.ascontiguousarray(bface_tag, dtype=np.int32)
            d.n_bfaces = len(bfn)
            d.bface_nodes = bfn.ctypes.data_as(C.POINTER(C.c_int64))
            d.bface_tag = bft.ctypes.data_as(C.POINTER(C.c_int32))
            self._keep += [bfn, bft]
        if periods is not None:
            per = np.ascontiguousarray(periods, dtype=np.float64)
            d.periods = _dp(per)
            self._keep.append(per)
        h = C.c_void_p()
        _check(lib().hgks_mesh_create(C.byref(d), C.byref(h)), "hgks_mesh_create")
        self._h = h
        self._keep = []

    def info(self, what: int) -> int:
        return int(lib().hgks_mesh_info(self._h, what))

    @property
    def n_cells(self):
        return self.info(0)

    @property
    def n_faces(self):
        return self.info(1)

    @property
    def n_ghosts(self):
        return self.info(2)

    @property
    def stencil_size(self):
        return self.info(3)

    def device_bytes(self, precision: int = HGKS_FP64) -> int:
        return self.info(5 if precision == HGKS_FP64 else 6)

    @property
    def static_bytes(self) -> int:
        """Device bytes of the mesh arrays alone (a DeviceMesh)."""
        return self.info(7)

    def work_bytes(self, precision: int = HGKS_FP64) -> int:
        """Device bytes of one solver's own arrays over a DeviceMesh."""
        return self.info(8 if precision == HGKS_FP64 else 9)

    def geometry(self):
        """(cell volumes, 3|cell|/|surface|) in caller order."""
        vol = np.empty(self.n_cells)
        hdt = np.empty(self.n_cells)
        _check(lib().hgks_mesh_geometry(self._h, _dp(vol), _dp(hdt)), "hgks_mesh_geometry")
        return vol, hdt

    def clone(self) -> "Mesh":
        """hgks_mesh_clone: an independent copy of the built mesh."""
        h = C.c_void_p()
        _check(lib().hgks_mesh_clone(self._h, C.byref(h)), "hgks_mesh_clone")
        m = Mesh.__new__(Mesh)
        m._keep = []
        m._h = h
        return m

    def release(self):
        """Hand ownership to a solver (hgks_init took it)."""
        h, self._h = self._h, None
        return h

    def __del__(self):
        h = getattr(self, "_h", None)
        if h:
            lib().hgks_mesh_destroy(h)
            self._h = None


class DeviceMesh:
    """hgks_dmesh_create / hgks_dmesh_release: a mesh resident in device
    memory, shared by the solvers created over it (Solver(dmesh, q0, ...))."""

    def __init__(self, mesh: Mesh, stream: int = 0):
        h = C.c_void_p()
        _check(lib().hgks_dmesh_create(mesh._h, C.c_void_p(stream or None), C.byref(h)), "hgks_dmesh_create")
        self._h = h

    def info(self, what: int) -> int:
        return int(lib().hgks_dmesh_info(self._h, what))

    @property
    def n_cells(self):
        return self.info(0)

    @property
    def bytes(self) -> int:
        return self.info(5)

    def work_bytes(self, precision: int = HGKS_FP64) -> int:
        return self.info(6 if precision == HGKS_FP64 else 7)

    @property
    def solvers(self) -> int:
        return self.info(8)

    def release(self):
        h, self._h = getattr(self, "_h", None), None
        if h:
            lib().hgks_dmesh_release(h)

    def __del__(self):
        self.release()


class Solver:
    """hgks_init / hgks_step / hgks_read / hgks_destroy on one mesh,
    hgks_batch_init on a list of meshes (one launch per kernel for all), or
    hgks_init_shared on a DeviceMesh (the mesh is not consumed)."""

    def __init__(self, mesh, q0, params: hgks_params | None = None, **kw):
        p = params if params is not None else make_params(**kw)
        h = C.c_void_p()
        if isinstance(mesh, DeviceMesh):
            self.member_cells = [mesh.n_cells]
            q0 = np.ascontiguousarray(q0, dtype=np.float64).reshape(mesh.n_cells, 5)
            _check(lib().hgks_init_shared(mesh._h, C.byref(p), _dp(q0), C.byref(h)), "hgks_init_shared")
        elif isinstance(mesh, (list, tuple)):
            meshes = list(mesh)
            self.member_cells = [m.n_cells for m in meshes]
            qs = [np.ascontiguousarray(q, dtype=np.float64).reshape(n, 5) for q, n in zip(q0, self.member_cells)]
            harr = (C.c_void_p * len(meshes))(*[m._h for m in meshes])
            qarr = (C.POINTER(C.c_double) * len(qs))(*[_dp(q) for q in qs])
            _check(lib().hgks_batch_init(harr, len(meshes), C.byref(p), qarr, C.byref(h)), "hgks_batch_init")
            for m in meshes:
                m.release()
        else:
            self.member_cells = [mesh.n_cells]
            q0 = np.ascontiguousarray(q0, dtype=np.float64).reshape(mesh.n_cells, 5)
            _check(lib().hgks_init(mesh._h, C.byref(p), _dp(q0), C.byref(h)), "hgks_init")
            mesh.release()
        self.n_cells = self.member_cells[0]
        self._h = h
        self.params = p

    @property
    def members(self) -> int:
        return len(self.member_cells)

    def member_read(self, i: int, out=None):
        q = out if out is not None else np.empty((self.member_cells[i], 5))
        t = C.c_double()
        s = C.c_int64()
        _check(lib().hgks_member_read(self._h, int(i), _dp(q), C.byref(t), C.byref(s)), "hgks_member_read")
        return q, t.value, s.value

    def member_write(self, i: int, q, t: float = 0.0):
        q = np.ascontiguousarray(q, dtype=np.float64).reshape(self.member_cells[i], 5)
        _check(lib().hgks_member_write(self._h, int(i), _dp(q), float(t)), "hgks_member_write")

    def query(self) -> bool:
        rc = lib().hgks_query(self._h)
        if rc < 0:
            _check(rc, "hgks_query")
        return rc == 1

    @property
    def device_bytes(self) -> int:
        return int(lib().hgks_solver_bytes(self._h))

    @property
    def tuning(self):
        """(flux_variant, recon_variant) in use."""
        f, r = C.c_int(), C.c_int()
        _check(lib().hgks_tuning(self._h, C.byref(f), C.byref(r)), "hgks_tuning")
        return f.value, r.value

    def set_tuning(self, flux_variant: int, recon_variant: int):
        _check(lib().hgks_set_tuning(self._h, int(flux_variant), int(recon_variant)), "hgks_set_tuning")

    def step(self, n: int = 1, t_end: float = 0.0, dt_fixed: float = 0.0):
        _check(lib().hgks_step(self._h, int(n), float(t_end), float(dt_fixed)), "hgks_step")

    def test_barrier_limit(self, cycles: int):
        """hgks_test_barrier_limit: wait limit (clock cycles) of the persistent
        launch's grid barriers; negative restores the default."""
        _check(lib().hgks_test_barrier_limit(self._h, int(cycles)), "hgks_test_barrier_limit")

    def sync(self):
        _check(lib().hgks_sync(self._h), "hgks_sync")

    def write(self, q, t: float = 0.0):
        q = np.ascontiguousarray(q, dtype=np.float64).reshape(self.n_cells, 5)
        _check(lib().hgks_write(self._h, _dp(q), float(t)), "hgks_write")

    def read(self, out=None):
        q = out if out is not None else np.empty((self.n_cells, 5))
        t = C.c_double()
        s = C.c_int64()
        _check(lib().hgks_read(self._h, _dp(q), C.byref(t), C.byref(s)), "hgks_read")
        return q, t.value, s.value

    def stage_operator(self, dt: float):
        L = np.empty((self.n_cells, 5))
        dL = np.empty((self.n_cells, 5))
        _check(lib().hgks_stage_operator(self._h, float(dt), _dp(L), _dp(dL)), "hgks_stage_operator")
        return L, dL

    def profile(self, n: int, t_end: float = 0.0, dt_fixed: float = 0.0):
        """Average ms per step in (finalize, ghost+recon, flux, update)."""
        ms = np.empty(4)
        _check(lib().hgks_profile(self._h, int(n), float(t_end), float(dt_fixed), _dp(ms)), "hgks_profile")
        return ms

    def close(self):
        h = getattr(self, "_h", None)
        if h:
            lib().hgks_destroy(h)
            self._h = None

    def __del__(self):
        self.close()
