"""FP64 CPU oracle of the II-LBM time step -- ctypes wrapper.

TEST INFRASTRUCTURE ONLY: imported by ``tests/``, ``__graft_entry__.smoke()`` and
the CPU-baseline leg of ``bench.py``; never by the product package.  The oracle is
``iilbm_oracle.c`` in this directory, compiled by :func:`build` with gcc alone.  It
shares no code with the CUDA library.

Every function maps one-to-one onto a routine of ``iilbm_oracle.c``; the paper
passages each follows are cited there.  Parity pins: every routine here is pinned
by a test in ``tests/test_oracle_*.py`` against a closed form, an invariant, a
special case or a brute-force / exact-rational computation (see the test
docstrings); none is "parity unpinned".
"""
from __future__ import annotations

import ctypes as C
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "iilbm_oracle.c")
_LIB = os.path.join(_HERE, "_build", "liboracle_iilbm.so")
_LIB_OMP = os.path.join(_HERE, "_build", "liboracle_iilbm_omp.so")
_lock = threading.Lock()
_lib = None
_lib_omp = None

SRT, MRT = 0, 1
BC_PERIODIC, BC_WALLS_Y, BC_CHANNEL, BC_BOX_OUTFLOW, BC_BOX_WALL = 0, 1, 2, 3, 4
FORCE_GUO, FORCE_SIMPLE = 0, 1
SPRING, SPRING_REST, PRESCRIBED, DIRECT = 0, 1, 2, 3
BODY_PRESCRIBED_X, BODY_FREE = 1, 2
# Lallemand-Luo D2Q9 rates quoted in section 2.2.1 (s7 = s8 = 1/tau set per case)
PAPER_MRT_RATES = (0.0, 1.63, 1.14, 0.0, 1.92, 0.0, 1.92, None, None)


def build(force: bool = False, parallel: bool = False) -> str:
    """Compile the oracle with gcc (no fused multiply-add contraction); parallel=True
    builds the same source with OpenMP (per-node loops on all host cores, identical
    results).  Returns the library path, or None for a parallel build that this gcc
    cannot make (no OpenMP runtime)."""
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
    _fields_ = [("nx", C.c_int), ("ny", C.c_int), ("collision", C.c_int), ("tau", C.c_double),
                ("s", C.c_double * 9), ("rho0", C.c_double), ("bc", C.c_int),
                ("u_max", C.c_double), ("body_x", C.c_double), ("body_y", C.c_double),
                ("jump", C.c_int), ("force", C.c_int)]


_D = C.POINTER(C.c_double)
_I = C.POINTER(C.c_int)


def lib(parallel: bool = False):
    """The oracle library (serial, or the OpenMP build with parallel=True)."""
    global _lib, _lib_omp
    with _lock:
        if parallel and _lib_omp is None:
            path = build(parallel=True)
            if path is None:
                raise RuntimeError("the OpenMP build of the oracle is unavailable")
            _lib_omp = _bind(C.CDLL(path))
        if not parallel and _lib is None:
            _lib = _bind(C.CDLL(build()))
        return _lib_omp if parallel else _lib


def _bind(L):
    """Declare the argument and result types of every oracle routine."""
    L.orc_create.restype = C.c_void_p
    L.orc_create.argtypes = [C.POINTER(_Cfg)]
    L.orc_destroy.argtypes = [C.c_void_p]
    L.orc_set_df.argtypes = [C.c_void_p, _D]
    L.orc_get_df.argtypes = [C.c_void_p, _D]
    L.orc_init_equilibrium.argtypes = [C.c_void_p, _D, _D, _D]
    L.orc_set_interface.argtypes = [C.c_void_p, _D, C.c_int, C.c_int, C.c_int, C.c_double,
                                    C.c_double, C.c_double, C.c_double, C.c_int,
                                    C.c_double, _D, _D]
    L.orc_step.argtypes = [C.c_void_p]
    L.orc_prepare.argtypes = [C.c_void_p]
    L.orc_cut_link_count.argtypes = [C.c_void_p]
    L.orc_run.argtypes = [C.c_void_p, C.c_int]
    L.orc_get_step_macros.argtypes = [C.c_void_p, _D, _D, _D]
    L.orc_get_markers.argtypes = [C.c_void_p, _D, _D, _D, _D]
    L.orc_mdf_iters.argtypes = [C.c_void_p]
    L.orc_set_ws_previous.argtypes = [C.c_void_p, C.c_int]
    L.orc_get_ustar.argtypes = [C.c_void_p, _D]
    L.orc_mdf_residual.argtypes = [C.c_void_p]
    L.orc_mdf_residual.restype = C.c_double
    L.orc_polygon_area.argtypes = [_D, C.c_int]
    L.orc_polygon_area.restype = C.c_double
    L.orc_phi.argtypes = [C.c_double]
    L.orc_phi.restype = C.c_double
    L.orc_mrt_matrix.argtypes = [_D]
    L.orc_invert9.argtypes = [_D, _D]
    L.orc_mrt_inverse.argtypes = [_D, _D]
    L.orc_feq_shifted.argtypes = [C.c_double, C.c_double, C.c_double, C.c_double, _D]
    L.orc_guo_source.argtypes = [C.c_double] * 4 + [_D]
    L.orc_collide_cell.argtypes = [C.POINTER(_Cfg), _D, _D, _D, C.c_double, C.c_double, _D]
    L.orc_cut_links.argtypes = [C.POINTER(_Cfg), _D, C.c_int, _D, _I, _I, _D, C.c_int]
    L.orc_winding.argtypes = [_D, C.c_int, C.c_int, C.c_int]
    L.orc_spread.argtypes = [C.POINTER(_Cfg), _D, C.c_int, _D, _D, _D]
    L.orc_interp.argtypes = [C.POINTER(_Cfg), _D, C.c_int, _D, _D, _D]
    L.orc_spring_forces_arr.argtypes = [_D, C.c_int, C.c_int, C.c_double, C.c_double,
                                        C.c_double, _D]
    L.orc_normal_split_arr.argtypes = [_D, C.c_int, C.c_int, C.c_double, _D, _D, _D, _D,
                                       C.c_int]
    L.orc_set_curve.argtypes = [C.c_void_p, C.c_int]
    L.orc_set_body.argtypes = [C.c_void_p, C.c_int, C.c_int, C.c_double, C.c_double, C.c_double,
                               C.c_double, C.c_double, _D, _D]
    L.orc_get_body.argtypes = [C.c_void_p, _D]
    L.orc_spline_coeffs.argtypes = [_D, C.c_int, C.c_int, _D]
    L.orc_spline_eval.argtypes = [_D, C.c_int, C.c_int, C.c_double, C.c_int]
    L.orc_spline_eval.restype = C.c_double
    L.orc_cut_links_spline.argtypes = [C.POINTER(_Cfg), _D, C.c_int, _D, C.c_int, _I, _I, _D,
                                       C.c_int]
    return L


def omp_threads() -> int:
    """Threads the OpenMP build runs with (OMP_NUM_THREADS, else every host core)."""
    v = os.environ.get("OMP_NUM_THREADS")
    return int(v) if v and v.isdigit() else (os.cpu_count() or 1)


def _p(a: np.ndarray):
    return a.ctypes.data_as(_D)


def _f64(a) -> np.ndarray:
    return np.ascontiguousarray(np.asarray(a, dtype=np.float64))


def make_cfg(nx, ny, collision=SRT, tau=0.8, s=None, rho0=1.0, bc=BC_PERIODIC, u_max=0.0,
             body=(0.0, 0.0), jump=1, force=FORCE_GUO) -> _Cfg:
    c = _Cfg()
    c.nx, c.ny, c.collision, c.tau, c.rho0, c.bc, c.u_max = nx, ny, collision, tau, rho0, bc, u_max
    c.body_x, c.body_y = body
    c.jump = jump
    c.force = force
    rates = mrt_rates(tau) if s is None else s
    for i in range(9):
        c.s[i] = rates[i]
    return c


def mrt_rates(tau: float, paper: bool = True):
    """Section 2.2.1 D2Q9 rates with s7 = s8 = 1/tau (paper=True), else all 1/tau."""
    if not paper:
        return [1.0 / tau] * 9
    r = list(PAPER_MRT_RATES)
    r[7] = r[8] = 1.0 / tau
    return r


# ---------------------------------------------------------------- primitives
def phi(r: float) -> float:
    return lib().orc_phi(float(r))


def mrt_matrix():
    """(M, M^-1) as the oracle's collision uses them (orthogonal-basis inverse)."""
    M = np.zeros(81)
    lib().orc_mrt_matrix(_p(M))
    Mi = np.zeros(81)
    lib().orc_mrt_inverse(_p(M), _p(Mi))
    return M.reshape(9, 9), Mi.reshape(9, 9)


def invert9(A):
    """General 9x9 inverse (Gauss-Jordan) -- an independent check of mrt_matrix()."""
    A = _f64(A).ravel()
    out = np.zeros(81)
    if lib().orc_invert9(_p(A), _p(out)) != 0:
        raise ValueError("singular")
    return out.reshape(9, 9)


def feq_shifted(rho, rho0, ux, uy):
    """Shifted equilibrium of Eq. 23 at density rho (passed to C as rho - rho0)."""
    out = np.zeros(9)
    lib().orc_feq_shifted(rho - rho0, rho0, ux, uy, _p(out))
    return out


def guo_source(ux, uy, gx, gy):
    out = np.zeros(9)
    lib().orc_guo_source(ux, uy, gx, gy, _p(out))
    return out


def collide_cell(cfg: _Cfg, df, gx=0.0, gy=0.0):
    M, Mi = mrt_matrix()
    M, Mi = _f64(M.ravel()), _f64(Mi.ravel())
    df = _f64(df)
    out = np.zeros(9)
    lib().orc_collide_cell(C.byref(cfg), _p(M), _p(Mi), _p(df), gx, gy, _p(out))
    return out


def cut_links(cfg: _Cfg, X, Fn, cap=None):
    """Cut-link records (cell, dir, coef) of the closed polygon X with jump strengths Fn."""
    X = _f64(X).reshape(-1, 2)
    Fn = _f64(Fn)
    n = X.shape[0]
    cap = cap or 64 * n + 64
    cell = np.zeros(cap, np.int32)
    d = np.zeros(cap, np.int32)
    coef = np.zeros(cap)
    m = lib().orc_cut_links(C.byref(cfg), _p(X), n, _p(Fn), cell.ctypes.data_as(_I),
                            d.ctypes.data_as(_I), _p(coef), cap)
    if m < 0:
        raise RuntimeError("cut-link capacity exceeded")
    return cell[:m].copy(), d[:m].copy(), coef[:m].copy()


def winding(X, px: int, py: int) -> int:
    X = _f64(X).reshape(-1, 2)
    return lib().orc_winding(_p(X), X.shape[0], int(px), int(py))


def spread(cfg: _Cfg, X, P):
    X = _f64(X).reshape(-1, 2)
    P = _f64(P).reshape(-1, 2)
    gx = np.zeros(cfg.nx * cfg.ny)
    gy = np.zeros(cfg.nx * cfg.ny)
    lib().orc_spread(C.byref(cfg), _p(X), X.shape[0], _p(P), _p(gx), _p(gy))
    return gx.reshape(cfg.ny, cfg.nx), gy.reshape(cfg.ny, cfg.nx)


def interp(cfg: _Cfg, X, ux, uy):
    X = _f64(X).reshape(-1, 2)
    U = np.zeros((X.shape[0], 2))
    lib().orc_interp(C.byref(cfg), _p(X), X.shape[0], _p(_f64(ux).ravel()),
                     _p(_f64(uy).ravel()), _p(U))
    return U


def spring_forces(X, model=SPRING, kappa=1.0, dX=1.0, l0=1.0):
    X = _f64(X).reshape(-1, 2)
    G = np.zeros_like(X)
    lib().orc_spring_forces_arr(_p(X), X.shape[0], model, kappa, dX, l0, _p(G))
    return G


def normal_split(X, G, moves=True, dX=1.0, curve=0):
    """(Fn, Gpar, normals) of Eqs. 31-32 and 46 (curve > 0: from the spline interface)."""
    X = _f64(X).reshape(-1, 2)
    G = _f64(G).reshape(-1, 2)
    n = X.shape[0]
    Fn, Gpar, nrm = np.zeros(n), np.zeros((n, 2)), np.zeros((n, 2))
    lib().orc_normal_split_arr(_p(X), n, int(moves), dX, _p(G), _p(Fn), _p(Gpar), _p(nrm),
                               int(curve))
    return Fn, Gpar, nrm


def spline_coeffs(v):
    """B-spline coefficients of the periodic cubic spline through v[k] (k < n)."""
    v = _f64(v).ravel()
    c = np.zeros_like(v)
    lib().orc_spline_coeffs(_p(v), v.size, 1, _p(c))
    return c


def spline_eval(c, s, deriv=0):
    c = _f64(c).ravel()
    return lib().orc_spline_eval(_p(c), c.size, 1, float(s), int(deriv))


def cut_links_spline(cfg: _Cfg, X, Fn, m, cap=None):
    """Cut-link records of the spline interface through the markers X (m chords per
    segment), jump strengths from the spline of Fn."""
    X = _f64(X).reshape(-1, 2)
    Fn = _f64(Fn)
    n = X.shape[0]
    cap = cap or 64 * n * m + 64
    cell = np.zeros(cap, np.int32)
    d = np.zeros(cap, np.int32)
    coef = np.zeros(cap)
    k = lib().orc_cut_links_spline(C.byref(cfg), _p(X), n, _p(Fn), int(m),
                                   cell.ctypes.data_as(_I), d.ctypes.data_as(_I), _p(coef), cap)
    if k < 0:
        raise RuntimeError("cut-link capacity exceeded")
    return cell[:k].copy(), d[:k].copy(), coef[:k].copy()


def polygon_area(X) -> float:
    X = _f64(X).reshape(-1, 2)
    return lib().orc_polygon_area(_p(X), X.shape[0])


# -------------------------------------------------------------- simulation
class Oracle:
    """One lattice with at most one immersed interface, stepped on the CPU in FP64."""

    def __init__(self, nx, ny, parallel=False, **kw):
        """parallel=True steps with the OpenMP build (identical results, all cores)."""
        self.cfg = make_cfg(nx, ny, **kw)
        self.nx, self.ny = nx, ny
        self._L = lib(parallel)
        self._h = self._L.orc_create(C.byref(self.cfg))
        self.n_markers = 0

    def close(self):
        if self._h:
            self._L.orc_destroy(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    # state
    def init_equilibrium(self, rho=None, ux=None, uy=None):
        keep = [None if a is None else _f64(a).ravel() for a in (rho, ux, uy)]
        self._L.orc_init_equilibrium(self._h, *[None if k is None else _p(k) for k in keep])

    def set_df(self, df):
        df = _f64(df).reshape(9, self.ny, self.nx)
        self._L.orc_set_df(self._h, _p(df))

    def get_df(self):
        df = np.zeros((9, self.ny, self.nx))
        self._L.orc_get_df(self._h, _p(df))
        return df

    def set_interface(self, X, model=SPRING, moves=True, kappa=0.0, dX=1.0, l0=1.0, eta=2.0,
                      mdf_iters=0, mdf_tol=0.0, G=None, UD=None, curve=0):
        X = _f64(X).reshape(-1, 2)
        n = X.shape[0]
        Gp = None if G is None else _f64(G).reshape(n, 2)
        UDa = None if UD is None else _f64(UD).reshape(n, 2)
        self._L.orc_set_interface(self._h, _p(X), n, model, int(moves), kappa, dX, l0, eta,
                                mdf_iters, mdf_tol, None if Gp is None else _p(Gp),
                                None if UDa is None else _p(UDa))
        self._L.orc_set_curve(self._h, int(curve))
        self.n_markers = n

    def step(self, n=1):
        if self._L.orc_run(self._h, int(n)) != 0:
            raise RuntimeError("oracle step failed (cut-link capacity)")

    def step_macros(self, deviation=False):
        """rho (or rho - rho0 if deviation), ux, uy used by the most recent step's
        collision (Eq. 24 at time t)."""
        N = self.nx * self.ny
        r, ux, uy = np.zeros(N), np.zeros(N), np.zeros(N)
        self._L.orc_get_step_macros(self._h, _p(r), _p(ux), _p(uy))
        s = (self.ny, self.nx)
        if not deviation:
            r = r + self.cfg.rho0
        return r.reshape(s), ux.reshape(s), uy.reshape(s)

    def current_macros(self, deviation=True):
        """drho (or rho), ux, uy of the current state: what the next collision uses
        (items 1-4 of the step, without advancing)."""
        if self._L.orc_prepare(self._h) != 0:
            raise RuntimeError("oracle prepare failed (cut-link capacity)")
        return self.step_macros(deviation=deviation)

    def cut_link_count(self):
        return self._L.orc_cut_link_count(self._h)

    def markers(self):
        n = self.n_markers
        X, G, U, Fn = np.zeros((n, 2)), np.zeros((n, 2)), np.zeros((n, 2)), np.zeros(n)
        self._L.orc_get_markers(self._h, _p(X), _p(G), _p(U), _p(Fn))
        return dict(X=X, G=G, U=U, Fn=Fn)

    def set_ws_previous(self, on=True):
        """Direct forcing starts from the force the previous iteration ended with."""
        self._L.orc_set_ws_previous(self._h, int(on))

    def unforced_velocity(self):
        """U*_k = interp(u*) of the most recent force iteration."""
        out = np.zeros((self.n_markers, 2))
        self._L.orc_get_ustar(self._h, _p(out))
        return out

    def mdf_stats(self):
        return self._L.orc_mdf_iters(self._h), self._L.orc_mdf_residual(self._h)

    def set_body(self, mode, dof=0, A=0.0, umax=0.0, mass=1.0, inertia=1.0, volume=0.0,
                 spring=(0.0, 0.0, 0.0), damping=(0.0, 0.0, 0.0)):
        """Make the directly forced interface a rigid body (section 2.3)."""
        k, c = _f64(spring), _f64(damping)
        if self._L.orc_set_body(self._h, mode, dof, A, umax, mass, inertia, volume, _p(k),
                                _p(c)) != 0:
            raise RuntimeError("a rigid body needs a directly forced interface")

    def body(self):
        """(X_c, Y_c, theta, U_x, U_y, W, F_x, F_y, T) of the rigid body."""
        out = np.zeros(9)
        self._L.orc_get_body(self._h, _p(out))
        return out
