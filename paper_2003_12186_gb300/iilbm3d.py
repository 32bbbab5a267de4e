"""Python binding of the three-dimensional (D3Q19) II-LBM C ABI (include/iilbm3d.h).

Argument marshalling only: every step of the method runs in the CUDA library
(libiilbm.so, built in-tree for sm_103a).  Arrays are numpy (host) or torch (host or
CUDA) FP64, checked for size and layout before the library touches them.
"""
from __future__ import annotations

import ctypes as C

import numpy as np

from . import iilbm
from .iilbm import (BF16, F16, F32, F64, FORCE_GUO, FORCE_SIMPLE, MRT, SRT, STORAGE,  # noqa: F401
                    IilbmError, _check, _current_device, _ptr)

# stored value = df * 2^k for 16-bit storage: FP16 keeps the small shifted deviations in
# its normal range; BF16 has FP32's exponent range
DEFAULT_SCALE_LOG2 = {F64: 0, F32: 0, F16: 12, BF16: 0}

PRESCRIBED, TENSION = 0, 1


class iilbm3d_config(C.Structure):
    _fields_ = [("nx", C.c_int32), ("ny", C.c_int32), ("nz", C.c_int32),
                ("collision", C.c_int32), ("storage", C.c_int32), ("jump", C.c_int32),
                ("force", C.c_int32), ("storage_scale_log2", C.c_int32), ("tau", C.c_double),
                ("s", C.c_double * 19), ("rho0", C.c_double), ("body", C.c_double * 3),
                ("stream", C.c_void_p)]


class iilbm3d_surface_params(C.Structure):
    _fields_ = [("model", C.c_int32), ("moves", C.c_int32), ("gamma", C.c_double)]


_H = C.c_void_p
_P = C.c_void_p

SIGNATURES3 = {
    "iilbm3d_create": [C.POINTER(_H), C.POINTER(iilbm3d_config)],
    "iilbm3d_destroy": [_H],
    "iilbm3d_set_surface": [_H, _P, C.c_int32, _P, C.c_int32, C.POINTER(iilbm3d_surface_params),
                            _P],
    "iilbm3d_init_equilibrium": [_H, _P, _P, _P, _P],
    "iilbm3d_set_populations": [_H, _P],
    "iilbm3d_get_populations": [_H, _P],
    "iilbm3d_step": [_H, C.c_int32],
    "iilbm3d_get_macros": [_H, _P, _P, _P, _P],
    "iilbm3d_get_markers": [_H, _P, _P, _P, _P],
    "iilbm3d_get_jump": [_H, _P],
    "iilbm3d_get_cut_link_count": [_H, C.POINTER(C.c_int32)],
    "iilbm3d_set_timing": [_H, C.c_int32],
    "iilbm3d_get_timing": [_H, C.POINTER(C.c_double), C.POINTER(C.c_int32), C.POINTER(C.c_int64)],
    "iilbm3d_synchronize": [_H],
}

_bound = None


def load():
    """The library with the 3-D entry points typed."""
    global _bound
    L = iilbm.load()
    if _bound is not L:
        for name, args in SIGNATURES3.items():
            fn = getattr(L, name)
            fn.argtypes = args
            fn.restype = C.c_int
        _bound = L
    return L


def paper_rates(tau: float):
    """The D3Q19 MRT rates of section 2.2.1 in the d'Humieres moment order."""
    s = [0.0] * 19
    s[1] = 1.19
    s[2] = s[10] = s[12] = 1.4
    s[4] = s[6] = s[8] = 1.2
    s[9] = s[11] = s[13] = s[14] = s[15] = 1.0 / tau
    s[16] = s[17] = s[18] = 1.98
    return s


class Lattice3D:
    """One D3Q19 II-LBM lattice (handle of iilbm3d_create)."""

    def __init__(self, nx, ny, nz, collision=MRT, storage=F32, tau=0.8, s=None, rho0=1.0,
                 jump=1, force=FORCE_GUO, body=(0.0, 0.0, 0.0), stream=None,
                 storage_scale_log2=None):
        L = load()
        c = iilbm3d_config()
        c.nx, c.ny, c.nz = nx, ny, nz
        c.collision = collision
        c.storage = STORAGE[storage] if isinstance(storage, str) else storage
        c.jump, c.force = jump, force
        c.storage_scale_log2 = (DEFAULT_SCALE_LOG2.get(c.storage, 0) if storage_scale_log2 is None
                                else storage_scale_log2)
        c.tau, c.rho0 = tau, rho0
        rates = s if s is not None else paper_rates(tau)
        for r in range(19):
            c.s[r] = rates[r]
        for d in range(3):
            c.body[d] = body[d]
        c.stream = stream
        self.cfg = c
        self.nx, self.ny, self.nz = nx, ny, nz
        self.N = nx * ny * nz
        self.n = self.m = 0
        self.device = _current_device()
        h = _H()
        _check("iilbm3d_create", L.iilbm3d_create(C.byref(h), C.byref(c)))
        self._h, self._L = h, L

    def close(self):
        if getattr(self, "_h", None):
            self._L.iilbm3d_destroy(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def _p(self, a, count):
        return _ptr(a, count, self.device)

    def set_surface(self, X, tri, model=PRESCRIBED, moves=False, gamma=0.0, G=None):
        p = iilbm3d_surface_params(int(model), int(moves), float(gamma))
        if X is None or len(X) == 0:
            _check("iilbm3d_set_surface",
                   self._L.iilbm3d_set_surface(self._h, None, 0, None, 0, C.byref(p), None))
            self.n = self.m = 0
            return
        X = np.ascontiguousarray(np.asarray(X, np.float64)).reshape(-1, 3)
        tri = np.ascontiguousarray(np.asarray(tri, np.int32)).reshape(-1, 3)
        Gp = None if G is None else np.ascontiguousarray(np.asarray(G, np.float64)).reshape(-1, 3)
        _check("iilbm3d_set_surface", self._L.iilbm3d_set_surface(
            self._h, X.ctypes.data, len(X), tri.ctypes.data, len(tri), C.byref(p),
            None if Gp is None else _ptr(Gp, 3 * len(X))))
        self.n, self.m = len(X), len(tri)

    def init_equilibrium(self, drho=None, ux=None, uy=None, uz=None):
        arr = [None if a is None else np.ascontiguousarray(np.asarray(a, np.float64))
               for a in (drho, ux, uy, uz)]
        _check("iilbm3d_init_equilibrium", self._L.iilbm3d_init_equilibrium(
            self._h, *[None if a is None else self._p(a, self.N) for a in arr]))

    def set_populations(self, df):
        if not hasattr(df, "data_ptr"):
            df = np.ascontiguousarray(np.asarray(df, np.float64))
        _check("iilbm3d_set_populations",
               self._L.iilbm3d_set_populations(self._h, self._p(df, 19 * self.N)))

    def get_populations(self, out=None):
        out = np.zeros((19, self.nz, self.ny, self.nx)) if out is None else out
        _check("iilbm3d_get_populations",
               self._L.iilbm3d_get_populations(self._h, self._p(out, 19 * self.N)))
        return out

    def step(self, n=1):
        _check("iilbm3d_step", self._L.iilbm3d_step(self._h, int(n)))

    def get_macros(self):
        shp = (self.nz, self.ny, self.nx)
        out = [np.zeros(shp) for _ in range(4)]
        _check("iilbm3d_get_macros",
               self._L.iilbm3d_get_macros(self._h, *[self._p(a, self.N) for a in out]))
        return tuple(out)

    def get_markers(self):
        n = self.n
        X, G, U, Fn = np.zeros((n, 3)), np.zeros((n, 3)), np.zeros((n, 3)), np.zeros(n)
        _check("iilbm3d_get_markers", self._L.iilbm3d_get_markers(
            self._h, self._p(X, 3 * n), self._p(G, 3 * n), self._p(U, 3 * n), self._p(Fn, n)))
        return dict(X=X, G=G, U=U, Fn=Fn)

    def get_markers_into(self, X=None, G=None, U=None, Fn=None):
        """The vertex arrays into caller buffers (numpy or torch, host or the lattice's
        device; None skips one)."""
        n = self.n
        _check("iilbm3d_get_markers", self._L.iilbm3d_get_markers(
            self._h, self._p(X, 3 * n), self._p(G, 3 * n), self._p(U, 3 * n), self._p(Fn, n)))

    def get_jump(self, out=None):
        out = np.zeros((18, self.nz, self.ny, self.nx)) if out is None else out
        _check("iilbm3d_get_jump", self._L.iilbm3d_get_jump(self._h, self._p(out, 18 * self.N)))
        return out

    def get_cut_link_count(self):
        c = C.c_int32()
        _check("iilbm3d_get_cut_link_count",
               self._L.iilbm3d_get_cut_link_count(self._h, C.byref(c)))
        return c.value

    def set_timing(self, enable=True):
        _check("iilbm3d_set_timing", self._L.iilbm3d_set_timing(self._h, int(enable)))

    def get_timing(self):
        ms, n, k = C.c_double(), C.c_int32(), C.c_int64()
        _check("iilbm3d_get_timing",
               self._L.iilbm3d_get_timing(self._h, C.byref(ms), C.byref(n), C.byref(k)))
        return ms.value, n.value, k.value

    def synchronize(self):
        _check("iilbm3d_synchronize", self._L.iilbm3d_synchronize(self._h))
