"""FP64 CPU oracle of the three-dimensional (D3Q19) II-LBM time step -- ctypes wrapper.

TEST INFRASTRUCTURE ONLY: imported by ``tests/``, ``__graft_entry__.smoke()`` and the
CPU-baseline leg of ``bench.py``; never by the product package.  The oracle is
``iilbm3d_oracle.c`` in this directory, compiled by :func:`build` with gcc alone; it
shares no code with the CUDA library or with the two-dimensional oracle.

Every function maps onto a routine of ``iilbm3d_oracle.c``, where the paper passages
each follows are cited.  Pins: ``tests/test_oracle_3d.py`` checks each routine against
a closed form, an invariant, a special case, or exact rational arithmetic.
"""
from __future__ import annotations

import ctypes as C
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "iilbm3d_oracle.c")
_LIB = os.path.join(_HERE, "_build", "liboracle_iilbm3d.so")
_LIB_OMP = os.path.join(_HERE, "_build", "liboracle_iilbm3d_omp.so")
_lock = threading.Lock()
_libs = {}

SRT, MRT = 0, 1
FORCE_GUO, FORCE_SIMPLE = 0, 1
PRESCRIBED, TENSION = 0, 1
QSCALE = float(1 << 20)


def paper_rates(tau: float):
    """The D3Q19 MRT rates of section 2.2.1 in the d'Humieres moment order: s1 = 1.19,
    s2 = s10 = s12 = 1.4, s4 = s6 = s8 = 1.2, s9 = s11 = s13 = s14 = s15 = 1/tau,
    s16 = s17 = s18 = 1.98, conserved moments 0."""
    s = [0.0] * 19
    s[1] = 1.19
    s[2] = s[10] = s[12] = 1.4
    s[4] = s[6] = s[8] = 1.2
    s[9] = s[11] = s[13] = s[14] = s[15] = 1.0 / tau
    s[16] = s[17] = s[18] = 1.98
    return s


def build(force: bool = False, parallel: bool = False):
    """Compile the oracle with gcc (no fused multiply-adds); parallel=True builds the same
    source with OpenMP.  Returns the path, or None when OpenMP is unavailable."""
    out = _LIB_OMP if parallel else _LIB
    os.makedirs(os.path.dirname(out), exist_ok=True)
    if force or not os.path.exists(out) or os.path.getmtime(out) < os.path.getmtime(_SRC):
        tmp = out + f".tmp{os.getpid()}"
        cmd = ["gcc", "-O2", "-fPIC", "-shared", "-ffp-contract=off", "-fno-fast-math",
               "-std=c11", *(["-fopenmp"] if parallel else []), _SRC, "-o", tmp, "-lm"]
        try:
            subprocess.check_call(cmd, stderr=subprocess.DEVNULL if parallel else None)
        except subprocess.CalledProcessError:
            if parallel:
                return None
            raise
        os.replace(tmp, out)
    return out


class _Cfg(C.Structure):
    _fields_ = [("nx", C.c_int), ("ny", C.c_int), ("nz", C.c_int), ("collision", C.c_int),
                ("tau", C.c_double), ("s", C.c_double * 19), ("rho0", C.c_double),
                ("body", C.c_double * 3), ("jump", C.c_int), ("force", C.c_int)]


_D = C.POINTER(C.c_double)
_I = C.POINTER(C.c_int)
_L64 = C.POINTER(C.c_int64)
_LONG = C.POINTER(C.c_long)


def _bind(L):
    sig = {
        "o3_create": ([C.POINTER(_Cfg)], C.c_void_p),
        "o3_destroy": ([C.c_void_p], None),
        "o3_set_df": ([C.c_void_p, _D], None),
        "o3_get_df": ([C.c_void_p, _D], None),
        "o3_init_equilibrium": ([C.c_void_p, _D, _D, _D, _D], None),
        "o3_set_surface": ([C.c_void_p, _D, C.c_int, _I, C.c_int, C.c_int, C.c_int, C.c_double,
                            _D], C.c_int),
        "o3_step": ([C.c_void_p, C.c_int], C.c_int),
        "o3_prepare": ([C.c_void_p], C.c_int),
        "o3_current_macros": ([C.c_void_p, _D, _D, _D, _D], C.c_int),
        "o3_get_markers": ([C.c_void_p, _D, _D, _D, _D], None),
        "o3_cut_link_count": ([C.c_void_p], C.c_int),
        "o3_get_ref_area": ([C.c_void_p, _D], None),
        "o3_jump_field": ([C.c_void_p, _D], C.c_int),
        "o3_volume": ([_D, _I, C.c_int], C.c_double),
        "o3_mrt_matrix": ([_D], None),
        "o3_mrt_inverse": ([_D, _D], None),
        "o3_feq_shifted": ([C.c_double, C.c_double, C.c_double, C.c_double, C.c_double, _D],
                           None),
        "o3_guo_source": ([C.c_double] * 6 + [_D], None),
        "o3_collide_cell": ([C.POINTER(_Cfg), _D, _D, _D, C.c_double, C.c_double, C.c_double,
                             _D], None),
        "o3_phi": ([C.c_double], C.c_double),
        "o3_spread": ([C.POINTER(_Cfg), _D, C.c_int, _D, _D, _D, _D], None),
        "o3_interp": ([C.POINTER(_Cfg), _D, C.c_int, _D, _D, _D, _D], None),
        "o3_surface_geometry": ([_D, C.c_int, _I, C.c_int, _D, _D], None),
        "o3_tension_forces": ([_D, C.c_int, _I, C.c_int, _D, C.c_double, _D], None),
        "o3_normal_split": ([_D, C.c_int, _D, _D, _D, _D, _D], None),
        "o3_quantize": ([C.c_double], C.c_int64),
        "o3_link_crosses": ([_L64, _L64, _L64, C.c_int, C.c_int, C.c_int, C.c_int, _D], C.c_int),
        "o3_cut_links": ([C.POINTER(_Cfg), _D, _I, C.c_int, _D, _LONG, _I, _D, C.c_int], C.c_int),
        "o3_inside": ([_D, C.c_int, _I, C.c_int, C.c_int, C.c_int, C.c_int], C.c_int),
        "o3_opp": ([C.c_int], C.c_int),
        "o3_lattice": ([_I, _I, _I, _D], None),
    }
    for name, (args, res) in sig.items():
        fn = getattr(L, name)
        fn.argtypes = args
        fn.restype = res
    return L


def lib(parallel: bool = False):
    with _lock:
        if parallel not in _libs:
            path = build(parallel=parallel)
            if path is None:
                raise RuntimeError("the OpenMP build of the 3-D oracle is unavailable")
            _libs[parallel] = _bind(C.CDLL(path))
        return _libs[parallel]


def omp_threads() -> int:
    """Threads the OpenMP build uses (OMP_NUM_THREADS, else the host's cores)."""
    v = os.environ.get("OMP_NUM_THREADS")
    return int(v) if v and v.isdigit() else (os.cpu_count() or 1)


def _f64(a):
    return np.ascontiguousarray(np.asarray(a, dtype=np.float64))


def _p(a):
    return None if a is None else a.ctypes.data_as(_D)


def _pi(a):
    return a.ctypes.data_as(_I)


def make_cfg(nx, ny, nz, collision=MRT, tau=0.8, s=None, rho0=1.0, body=(0.0, 0.0, 0.0),
             jump=1, force=FORCE_GUO):
    c = _Cfg()
    c.nx, c.ny, c.nz, c.collision, c.tau, c.rho0 = nx, ny, nz, collision, tau, rho0
    rates = s if s is not None else paper_rates(tau)
    for i in range(19):
        c.s[i] = rates[i]
    for d in range(3):
        c.body[d] = body[d]
    c.jump, c.force = jump, force
    return c


class Oracle3D:
    """One D3Q19 lattice of the oracle with an optional triangulated surface."""

    def __init__(self, nx, ny, nz, parallel=False, **kw):
        self._L = lib(parallel)
        self.nx, self.ny, self.nz = nx, ny, nz
        self.N = nx * ny * nz
        self.cfg = make_cfg(nx, ny, nz, **kw)
        self._h = self._L.o3_create(C.byref(self.cfg))
        self.n = self.m = 0
        self._tri = None

    def __del__(self):
        if getattr(self, "_h", None):
            self._L.o3_destroy(self._h)
            self._h = None

    def set_df(self, df):
        df = _f64(df).reshape(19, self.N)
        self._L.o3_set_df(self._h, _p(df))

    def get_df(self):
        out = np.zeros((19, self.nz, self.ny, self.nx))
        self._L.o3_get_df(self._h, _p(out))
        return out

    def init_equilibrium(self, drho=None, ux=None, uy=None, uz=None):
        keep = [None if a is None else _f64(a).ravel() for a in (drho, ux, uy, uz)]
        self._L.o3_init_equilibrium(self._h, *[_p(k) for k in keep])

    def set_surface(self, X, tri, model=PRESCRIBED, moves=False, gamma=0.0, G=None):
        X, tri = _f64(X).reshape(-1, 3), np.ascontiguousarray(np.asarray(tri, np.int32)).reshape(-1, 3)
        Gp = None if G is None else _f64(G).reshape(-1, 3)
        rc = self._L.o3_set_surface(self._h, _p(X), len(X), _pi(tri), len(tri), model,
                                    int(moves), float(gamma), _p(Gp))
        if rc != 0:
            raise ValueError("invalid surface (degenerate triangle or edge >= 8)")
        self.n, self.m, self._tri = len(X), len(tri), tri

    def step(self, n=1):
        if self._L.o3_step(self._h, int(n)) != 0:
            raise RuntimeError("cut-link capacity exceeded")

    def current_macros(self):
        shp = (self.nz, self.ny, self.nx)
        d, ux, uy, uz = (np.zeros(shp) for _ in range(4))
        if self._L.o3_current_macros(self._h, _p(d), _p(ux), _p(uy), _p(uz)) != 0:
            raise RuntimeError("cut-link capacity exceeded")
        return d, ux, uy, uz

    def markers(self):
        n = self.n
        X, G, U, Fn = np.zeros((n, 3)), np.zeros((n, 3)), np.zeros((n, 3)), np.zeros(n)
        self._L.o3_get_markers(self._h, _p(X), _p(G), _p(U), _p(Fn))
        return dict(X=X, G=G, U=U, Fn=Fn)

    def ref_area(self):
        out = np.zeros(self.n)
        self._L.o3_get_ref_area(self._h, _p(out))
        return out

    def cut_link_count(self):
        return self._L.o3_cut_link_count(self._h)

    def jump_field(self):
        J = np.zeros((18, self.nz, self.ny, self.nx))
        r = self._L.o3_jump_field(self._h, _p(J))
        return J, r

    def volume(self):
        return volume(self.markers()["X"], self._tri)


# ---- free functions on arrays (pins) ---------------------------------------------------
def lattice():
    ex, ey, ez = (np.zeros(19, np.int32) for _ in range(3))
    w = np.zeros(19)
    lib().o3_lattice(_pi(ex), _pi(ey), _pi(ez), _p(w))
    return np.stack([ex, ey, ez], axis=1), w


def opp(i):
    return lib().o3_opp(int(i))


def mrt_matrix():
    M = np.zeros(19 * 19)
    lib().o3_mrt_matrix(_p(M))
    return M.reshape(19, 19)


def mrt_inverse(M):
    M = _f64(M)
    out = np.zeros(19 * 19)
    lib().o3_mrt_inverse(_p(M), _p(out))
    return out.reshape(19, 19)


def feq(drho, rho0, u):
    out = np.zeros(19)
    lib().o3_feq_shifted(float(drho), float(rho0), float(u[0]), float(u[1]), float(u[2]), _p(out))
    return out


def guo_source(u, g):
    out = np.zeros(19)
    lib().o3_guo_source(*[float(v) for v in (*u, *g)], _p(out))
    return out


def collide(cfg, dfc, g):
    M = mrt_matrix()
    Mi = mrt_inverse(M)
    M, Mi, dfc = _f64(M), _f64(Mi), _f64(dfc)
    out = np.zeros(19)
    lib().o3_collide_cell(C.byref(cfg), _p(M), _p(Mi), _p(dfc), float(g[0]), float(g[1]),
                          float(g[2]), _p(out))
    return out


def phi(r):
    return lib().o3_phi(float(r))


def spread(cfg, X, P):
    X, P = _f64(X).reshape(-1, 3), _f64(P).reshape(-1, 3)
    shp = (cfg.nz, cfg.ny, cfg.nx)
    gx, gy, gz = (np.zeros(shp) for _ in range(3))
    lib().o3_spread(C.byref(cfg), _p(X), len(X), _p(P), _p(gx), _p(gy), _p(gz))
    return gx, gy, gz


def interp(cfg, X, ux, uy, uz):
    X = _f64(X).reshape(-1, 3)
    U = np.zeros((len(X), 3))
    lib().o3_interp(C.byref(cfg), _p(X), len(X), _p(_f64(ux)), _p(_f64(uy)), _p(_f64(uz)), _p(U))
    return U


def surface_geometry(X, tri):
    X = _f64(X).reshape(-1, 3)
    tri = np.ascontiguousarray(np.asarray(tri, np.int32))
    nrm, area = np.zeros((len(X), 3)), np.zeros(len(X))
    lib().o3_surface_geometry(_p(X), len(X), _pi(tri), len(tri), _p(nrm), _p(area))
    return nrm, area


def tension_forces(X, tri, Aref, gamma):
    X = _f64(X).reshape(-1, 3)
    tri = np.ascontiguousarray(np.asarray(tri, np.int32))
    G = np.zeros((len(X), 3))
    lib().o3_tension_forces(_p(X), len(X), _pi(tri), len(tri), _p(_f64(Aref)), float(gamma), _p(G))
    return G


def normal_split(G, nrm, area, Aref):
    G = _f64(G).reshape(-1, 3)
    n = len(G)
    Fn, Gpar = np.zeros(n), np.zeros((n, 3))
    lib().o3_normal_split(_p(G), n, _p(_f64(nrm)), _p(_f64(area)), _p(_f64(Aref)), _p(Fn), _p(Gpar))
    return Fn, Gpar


def quantize(v):
    return lib().o3_quantize(float(v))


def link_crosses(A, B, Cq, x, y, z, i):
    """(sign, barycentric coordinates) of the link of direction i into node (x, y, z)
    against the snapped triangle A, B, Cq (int64 triples)."""
    a, b, c = (np.ascontiguousarray(np.asarray(v, np.int64)) for v in (A, B, Cq))
    lam = np.zeros(3)
    s = lib().o3_link_crosses(a.ctypes.data_as(_L64), b.ctypes.data_as(_L64),
                              c.ctypes.data_as(_L64), int(x), int(y), int(z), int(i), _p(lam))
    return s, lam


def cut_links(cfg, X, tri, Fn, cap=None):
    X = _f64(X).reshape(-1, 3)
    tri = np.ascontiguousarray(np.asarray(tri, np.int32))
    cap = cap or 256 * len(tri) + 64
    cell, d, coef = np.zeros(cap, np.int64), np.zeros(cap, np.int32), np.zeros(cap)
    r = lib().o3_cut_links(C.byref(cfg), _p(X), _pi(tri), len(tri), _p(_f64(Fn)),
                           cell.ctypes.data_as(_LONG), _pi(d), _p(coef), cap)
    if r < 0:
        raise RuntimeError("capacity")
    return cell[:r], d[:r], coef[:r]


def inside(X, tri, x, y, z):
    X = _f64(X).reshape(-1, 3)
    tri = np.ascontiguousarray(np.asarray(tri, np.int32))
    return lib().o3_inside(_p(X), len(X), _pi(tri), len(tri), int(x), int(y), int(z))


def volume(X, tri):
    X = _f64(X).reshape(-1, 3)
    tri = np.ascontiguousarray(np.asarray(tri, np.int32))
    return lib().o3_volume(_p(X), _pi(tri), len(tri))
