"""Thin Python binding of the C ABI in include/iilbm.h (argument marshalling only).

Every function has the name of its C entry point; every step of the method runs in
the CUDA library ``lib/libiilbm.so``.  There is no CPU fallback: if the library is
missing or no sm_103a GPU is present, calls raise.

Array arguments may be numpy arrays (host) or CUDA torch tensors (device); both are
passed as raw pointers, and the library copies with cudaMemcpyDefault.
"""
from __future__ import annotations

import ctypes as C
import os
import threading

import numpy as np

from . import build as _build

OK = 0
(ERR_INVALID_ARG, ERR_OOM, ERR_CUDA, ERR_DEVICE_TIMEOUT, ERR_NONFINITE, ERR_INTERFACE,
 ERR_CAPACITY, ERR_NO_DEVICE) = range(-1, -9, -1)
SRT, MRT = 0, 1
F64, F32, F16, BF16 = 0, 1, 2, 3
BC_PERIODIC, BC_WALLS_Y, BC_CHANNEL, BC_BOX_OUTFLOW, BC_BOX_WALL = 0, 1, 2, 3, 4
FORCE_GUO, FORCE_SIMPLE = 0, 1
SPRING, SPRING_REST, PRESCRIBED, DIRECT = 0, 1, 2, 3
OPT_CUDA_GRAPH, OPT_OVERLAP, OPT_VECTOR_KERNEL, OPT_FORCED_BLOCKS, OPT_TMA_KERNEL = 0, 1, 2, 3, 4
WS_GIVEN, WS_PREVIOUS, WS_MLP = 0, 1, 2
MLP_PARAMS, MLP_FEATURES = 10434, 30
BODY_PRESCRIBED_X, BODY_FREE = 1, 2
STORAGE = {"f64": F64, "f32": F32, "f16": F16, "bf16": BF16}
STORAGE_BYTES = {F64: 8, F32: 4, F16: 2, BF16: 2}


class IilbmError(RuntimeError):
    def __init__(self, fn: str, code: int):
        self.code = code
        super().__init__(f"{fn} failed: {code} ({error_string(code)})")


class iilbm_config(C.Structure):
    _fields_ = [("nx", C.c_int32), ("ny", C.c_int32), ("collision", C.c_int32),
                ("storage", C.c_int32), ("bc", C.c_int32), ("jump", C.c_int32),
                ("storage_scale_log2", C.c_int32), ("force", C.c_int32),
                ("tau", C.c_double), ("s", C.c_double * 9), ("rho0", C.c_double),
                ("u_max", C.c_double), ("body", C.c_double * 2), ("stream", C.c_void_p)]


class iilbm_interface_params(C.Structure):
    _fields_ = [("model", C.c_int32), ("moves", C.c_int32), ("stiffness", C.c_double),
                ("dX", C.c_double), ("rest_length", C.c_double), ("eta", C.c_double),
                ("mdf_iters", C.c_int32), ("curve", C.c_int32), ("mdf_tol", C.c_double)]


class iilbm_body_params(C.Structure):
    _fields_ = [("mode", C.c_int32), ("dof", C.c_int32), ("amplitude", C.c_double),
                ("u_max", C.c_double), ("mass", C.c_double), ("inertia", C.c_double),
                ("volume", C.c_double), ("spring", C.c_double * 3),
                ("damping", C.c_double * 3)]


_lib = None
_lock = threading.Lock()
_H = C.c_void_p
_P = C.c_void_p

SIGNATURES = {
    "iilbm_create_lattice": [C.POINTER(_H), C.POINTER(iilbm_config)],
    "iilbm_destroy": [_H],
    "iilbm_set_interface": [_H, _P, C.c_int32, C.POINTER(iilbm_interface_params), _P],
    "iilbm_init_equilibrium": [_H, _P, _P, _P],
    "iilbm_set_populations": [_H, _P],
    "iilbm_get_populations": [_H, _P],
    "iilbm_step": [_H, C.c_int32],
    "iilbm_get_macros": [_H, _P, _P, _P],
    "iilbm_get_markers": [_H, _P, _P, _P, _P],
    "iilbm_get_mdf_stats": [_H, C.POINTER(C.c_int32), C.POINTER(C.c_double)],
    "iilbm_set_warm_start": [_H, _P],
    "iilbm_set_warm_start_mode": [_H, C.c_int32],
    "iilbm_set_warm_start_mlp": [_H, _H, C.c_double],
    "iilbm_get_df_features": [_H, C.c_double, _P],
    "iilbm_mlp_create": [C.POINTER(_H), _P],
    "iilbm_mlp_destroy": [_H],
    "iilbm_mlp_set_params": [_H, _P],
    "iilbm_mlp_get_params": [_H, _P],
    "iilbm_mlp_set_normalization": [_H, _P, _P, _P, _P],
    "iilbm_mlp_forward": [_H, _P, C.c_int32, _P],
    "iilbm_mlp_gradient": [_H, _P, _P, C.c_int32, _P, _P],
    "iilbm_mlp_train": [_H, _P, _P, C.c_int32, _P, C.c_int32, C.c_int32, C.c_float, C.c_float,
                        C.c_float, C.c_float, _P],
    "iilbm_get_unforced_velocity": [_H, _P],
    "iilbm_get_body_force": [_H, C.POINTER(C.c_double)],
    "iilbm_set_rigid_body": [_H, C.POINTER(iilbm_body_params)],
    "iilbm_get_rigid_body": [_H, C.POINTER(C.c_double)],
    "iilbm_get_cut_link_count": [_H, C.POINTER(C.c_int32)],
    "iilbm_get_jump": [_H, _P],
    "iilbm_set_timing": [_H, C.c_int32],
    "iilbm_get_timing": [_H, C.POINTER(C.c_double), C.POINTER(C.c_int32),
                         C.POINTER(C.c_int64), C.POINTER(C.c_int64)],
    "iilbm_set_option": [_H, C.c_int32, C.c_int32],
    "iilbm_get_macros_noalloc": [_H, _P, _P, _P],
    "iilbm_synchronize": [_H],
    "iilbm_error_string": [C.c_int],
    "iilbm_create_batch": [C.POINTER(_H), C.POINTER(_H), C.c_int32, _P],
    "iilbm_destroy_batch": [_H],
    "iilbm_batch_step": [_H, C.c_int32],
    "iilbm_batch_set_variant": [_H, C.c_int32],
    "iilbm_batch_autotune": [_H, C.c_int32, C.POINTER(C.c_int32), C.POINTER(C.c_double)],
    "iilbm_batch_set_timing": [_H, C.c_int32],
    "iilbm_batch_get_timing": [_H, C.POINTER(C.c_double), C.POINTER(C.c_int32),
                               C.POINTER(C.c_int64)],
    "iilbm_batch_synchronize": [_H],
}

# stream-collide variants of a batch (iilbm_batch_set_variant)
BATCH_VARIANTS = tuple(f"npt{n}-b{b}-{g}" for n, b in ((4, 3), (4, 2), (2, 3), (2, 2), (1, 3),
                                                       (4, "3o2"))
                       for g in ("per-item", "persistent"))


def library_path() -> str:
    return _build.LIB


def load(build_if_missing: bool = True) -> C.CDLL:
    """Load libiilbm.so (building it with nvcc first if it is missing or stale)."""
    global _lib
    with _lock:
        if _lib is None:
            path = _build.build() if build_if_missing else _build.LIB
            if not os.path.exists(path):
                raise RuntimeError(f"II-LBM CUDA library not built: {path}")
            L = C.CDLL(path)
            for name, args in SIGNATURES.items():
                fn = getattr(L, name)
                fn.argtypes = args
                fn.restype = C.c_char_p if name == "iilbm_error_string" else C.c_int
            _lib = L
    return _lib


def error_string(code: int) -> str:
    return load().iilbm_error_string(int(code)).decode()


def _check(fn: str, rc: int):
    if rc != OK:
        raise IilbmError(fn, rc)


def _ptr(a, count=None, device=None, dtype="float64"):
    """Raw pointer of a numpy array or a torch tensor (None -> NULL).

    The library reads or writes exactly `count` elements of `dtype` there, so the buffer
    is checked first: C-contiguous, of that dtype and element count, and -- for a torch
    tensor -- on the host or on CUDA device `device` (the lattice's).  Raises ValueError,
    which `python -O` keeps, instead of letting a copy run past the end of a buffer."""
    if a is None:
        return None
    if isinstance(a, np.ndarray):
        if not a.flags["C_CONTIGUOUS"] or a.dtype != np.dtype(dtype):
            raise ValueError(f"need a C-contiguous {dtype} array, got {a.dtype}")
        if count is not None and a.size != count:
            raise ValueError(f"need {count} elements, got {a.size} (shape {a.shape})")
        return a.ctypes.data
    if not hasattr(a, "data_ptr"):
        raise ValueError(f"need a numpy array or a torch tensor, got {type(a).__name__}")
    if not a.is_contiguous() or str(a.dtype) != f"torch.{dtype}":
        raise ValueError(f"need a contiguous {dtype} tensor, got {a.dtype}")
    if count is not None and a.numel() != count:
        raise ValueError(f"need {count} elements, got {a.numel()} (shape {tuple(a.shape)})")
    if a.device.type == "cuda":
        if device is not None and a.device.index != device:
            raise ValueError(f"tensor on cuda:{a.device.index}, lattice on cuda:{device}")
    elif a.device.type != "cpu":
        raise ValueError(f"tensor on {a.device}, need the host or a CUDA device")
    return a.data_ptr()


def _host(a, shape):
    a = np.ascontiguousarray(np.asarray(a, dtype=np.float64))
    if a.size != int(np.prod(shape)):
        raise ValueError(f"expected {shape}, got {a.shape}")
    return a


def _current_device():
    """The current CUDA device as torch sees it (the one the library creates handles
    on), or None when torch is not in use."""
    import sys
    torch = sys.modules.get("torch")
    if torch is None:
        return None
    try:
        return torch.cuda.current_device() if torch.cuda.is_available() else None
    except Exception:
        return None


class Lattice:
    """One II-LBM lattice (handle of iilbm_create_lattice)."""

    def __init__(self, nx, ny, collision=MRT, storage=F32, tau=0.8, s=None, rho0=1.0,
                 bc=BC_PERIODIC, jump=1, u_max=0.0, body=(0.0, 0.0), stream=None,
                 storage_scale_log2=None, force=FORCE_GUO):
        L = load()
        cfg = iilbm_config()
        cfg.nx, cfg.ny = nx, ny
        cfg.collision = collision
        cfg.storage = STORAGE[storage] if isinstance(storage, str) else storage
        cfg.bc, cfg.jump = bc, jump
        if storage_scale_log2 is None:
            storage_scale_log2 = {F64: 0, F32: 0, F16: 12, BF16: 0}[cfg.storage]
        cfg.storage_scale_log2 = storage_scale_log2
        cfg.force = force
        cfg.tau, cfg.rho0, cfg.u_max = tau, rho0, u_max
        rates = s if s is not None else [0.0, 1.63, 1.14, 0.0, 1.92, 0.0, 1.92, 1 / tau, 1 / tau]
        for i in range(9):
            cfg.s[i] = rates[i]
        cfg.body[0], cfg.body[1] = body
        cfg.stream = stream
        self.cfg = cfg
        self.nx, self.ny = nx, ny
        self.n_markers = 0
        self.device = _current_device()
        h = _H()
        _check("iilbm_create_lattice", L.iilbm_create_lattice(C.byref(h), C.byref(cfg)))
        self._h = h
        self._L = L

    def close(self):
        if getattr(self, "_h", None):
            self._L.iilbm_destroy(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    @property
    def handle(self):
        return self._h

    # ---------------------------------------------------------------- state
    def iilbm_set_interface(self, X, model=SPRING, moves=True, stiffness=0.0, dX=1.0,
                            rest_length=1.0, eta=2.0, mdf_iters=0, mdf_tol=0.0, aux=None,
                            curve=0):
        p = iilbm_interface_params()
        p.curve = curve
        p.model, p.moves, p.stiffness, p.dX, p.rest_length = model, int(moves), stiffness, dX, \
            rest_length
        p.eta, p.mdf_iters, p.mdf_tol = eta, mdf_iters, mdf_tol
        if X is None or (hasattr(X, "__len__") and len(X) == 0):
            _check("iilbm_set_interface", self._L.iilbm_set_interface(self._h, None, 0, C.byref(p),
                                                                      None))
            self.n_markers = 0
            return
        n = len(X)
        Xh = X if not isinstance(X, np.ndarray) and hasattr(X, "data_ptr") else _host(X, (n, 2))
        A = None if aux is None else (aux if hasattr(aux, "data_ptr") else _host(aux, (n, 2)))
        _check("iilbm_set_interface",
               self._L.iilbm_set_interface(self._h, self._p(Xh, 2 * n), n, C.byref(p),
                                           self._p(A, 2 * n)))
        self.n_markers = n

    set_interface = iilbm_set_interface

    def _p(self, a, count):
        return _ptr(a, count, self.device)

    def iilbm_init_equilibrium(self, rho=None, ux=None, uy=None):
        N = (self.ny, self.nx)
        arrs = [None if a is None else _host(a, N) for a in (rho, ux, uy)]
        _check("iilbm_init_equilibrium",
               self._L.iilbm_init_equilibrium(self._h, *[self._p(a, self.nx * self.ny)
                                                         for a in arrs]))

    init_equilibrium = iilbm_init_equilibrium

    def iilbm_set_populations(self, df):
        d = df if hasattr(df, "data_ptr") else _host(df, (9, self.ny, self.nx))
        _check("iilbm_set_populations",
               self._L.iilbm_set_populations(self._h, self._p(d, 9 * self.nx * self.ny)))

    set_populations = iilbm_set_populations

    def iilbm_get_populations(self, out=None):
        out = np.zeros((9, self.ny, self.nx)) if out is None else out
        _check("iilbm_get_populations",
               self._L.iilbm_get_populations(self._h, self._p(out, 9 * self.nx * self.ny)))
        return out

    get_populations = iilbm_get_populations

    def iilbm_step(self, n=1):
        _check("iilbm_step", self._L.iilbm_step(self._h, int(n)))

    step = iilbm_step

    def iilbm_get_macros(self, drho=None, ux=None, uy=None, want=(True, True, True)):
        """drho, ux, uy of the current state (host numpy unless device tensors given)."""
        outs = []
        for a, w in zip((drho, ux, uy), want):
            outs.append(a if a is not None else (np.zeros((self.ny, self.nx)) if w else None))
        N = self.nx * self.ny
        _check("iilbm_get_macros",
               self._L.iilbm_get_macros(self._h, *[self._p(a, N) for a in outs]))
        return tuple(outs)

    get_macros = iilbm_get_macros

    def iilbm_get_macros_noalloc(self, drho=None, ux=None, uy=None, want=(True, True, True)):
        """As iilbm_get_macros, staged through the library's static device array (no
        device allocation; lattices up to 2^18 nodes)."""
        outs = []
        for a, w in zip((drho, ux, uy), want):
            outs.append(a if a is not None else (np.zeros((self.ny, self.nx)) if w else None))
        N = self.nx * self.ny
        _check("iilbm_get_macros_noalloc",
               self._L.iilbm_get_macros_noalloc(self._h, *[self._p(a, N) for a in outs]))
        return tuple(outs)

    def iilbm_get_markers(self):
        n = self.n_markers
        X, G, U, Fn = np.zeros((n, 2)), np.zeros((n, 2)), np.zeros((n, 2)), np.zeros(n)
        self.iilbm_get_markers_into(X, G, U, Fn)
        return dict(X=X, G=G, U=U, Fn=Fn)

    get_markers = iilbm_get_markers

    def iilbm_get_markers_into(self, X=None, G=None, U=None, Fn=None):
        n = self.n_markers
        _check("iilbm_get_markers",
               self._L.iilbm_get_markers(self._h, self._p(X, 2 * n), self._p(G, 2 * n),
                                         self._p(U, 2 * n), self._p(Fn, n)))

    def iilbm_get_mdf_stats(self):
        it, res = C.c_int32(), C.c_double()
        _check("iilbm_get_mdf_stats",
               self._L.iilbm_get_mdf_stats(self._h, C.byref(it), C.byref(res)))
        return it.value, res.value

    def iilbm_set_warm_start(self, G0=None):
        G = None if G0 is None else (G0 if hasattr(G0, "data_ptr") else
                                     _host(G0, (self.n_markers, 2)))
        _check("iilbm_set_warm_start",
               self._L.iilbm_set_warm_start(self._h, self._p(G, 2 * self.n_markers)))

    def iilbm_set_warm_start_mode(self, mode):
        _check("iilbm_set_warm_start_mode", self._L.iilbm_set_warm_start_mode(self._h, int(mode)))

    def iilbm_get_unforced_velocity(self, out=None):
        """U*_k [n][2] of the most recent force iteration (numpy, or into `out`)."""
        o = out if out is not None else np.zeros((self.n_markers, 2))
        _check("iilbm_get_unforced_velocity",
               self._L.iilbm_get_unforced_velocity(self._h, self._p(o, 2 * self.n_markers)))
        return o

    def iilbm_set_warm_start_mlp(self, mlp, re):
        _check("iilbm_set_warm_start_mlp",
               self._L.iilbm_set_warm_start_mlp(self._h, mlp.handle, float(re)))
        self._mlp = mlp  # kept alive while attached

    def iilbm_get_df_features(self, re):
        """Raw features [n][30] (FP32) of the most recent force iteration."""
        F = np.zeros((self.n_markers, 30), dtype=np.float32)
        _check("iilbm_get_df_features",
               self._L.iilbm_get_df_features(self._h, float(re), F.ctypes.data))
        return F

    def iilbm_get_body_force(self):
        F = (C.c_double * 2)()
        _check("iilbm_get_body_force", self._L.iilbm_get_body_force(self._h, F))
        return F[0], F[1]

    def iilbm_set_rigid_body(self, mode, dof=0, amplitude=0.0, u_max=0.0, mass=1.0,
                             inertia=1.0, volume=0.0, spring=(0.0, 0.0, 0.0),
                             damping=(0.0, 0.0, 0.0)):
        """Make the directly forced interface a rigid body (section 2.3): BODY_PRESCRIBED_X
        (harmonic translation of section 4.4) or BODY_FREE (Eqs. 27-29 with springs and
        dampers on the degrees of freedom in dof: 1 x, 2 y, 4 rotation)."""
        bp = iilbm_body_params(int(mode), int(dof), float(amplitude), float(u_max),
                               float(mass), float(inertia), float(volume),
                               (C.c_double * 3)(*[float(v) for v in spring]),
                               (C.c_double * 3)(*[float(v) for v in damping]))
        _check("iilbm_set_rigid_body", self._L.iilbm_set_rigid_body(self._h, C.byref(bp)))

    def iilbm_get_rigid_body(self):
        """Body state: dict of Xc, Yc, theta, Ux, Uy, W, Fx, Fy, T (the last F_ext, T_ext)."""
        v = (C.c_double * 9)()
        _check("iilbm_get_rigid_body", self._L.iilbm_get_rigid_body(self._h, v))
        return dict(zip(("Xc", "Yc", "theta", "Ux", "Uy", "W", "Fx", "Fy", "T"), list(v)))

    def iilbm_get_jump(self, out=None):
        """Jump field J[8][ny][nx] (directions 1..8) of the current state's interface."""
        out = np.zeros((8, self.ny, self.nx)) if out is None else out
        _check("iilbm_get_jump",
               self._L.iilbm_get_jump(self._h, self._p(out, 8 * self.nx * self.ny)))
        return out

    def iilbm_get_cut_link_count(self):
        c = C.c_int32()
        _check("iilbm_get_cut_link_count", self._L.iilbm_get_cut_link_count(self._h, C.byref(c)))
        return c.value

    def iilbm_set_timing(self, enable=True):
        _check("iilbm_set_timing", self._L.iilbm_set_timing(self._h, int(enable)))

    def iilbm_get_timing(self, with_tiles=False):
        """(lean stream-collide ms summed, its launches, library kernel launches[,
        flagged tiles summed])."""
        ms, n, k, t = C.c_double(), C.c_int32(), C.c_int64(), C.c_int64()
        _check("iilbm_get_timing", self._L.iilbm_get_timing(self._h, C.byref(ms), C.byref(n),
                                                            C.byref(k), C.byref(t)))
        return (ms.value, n.value, k.value, t.value) if with_tiles else (ms.value, n.value,
                                                                          k.value)

    def iilbm_set_option(self, option, value):
        _check("iilbm_set_option", self._L.iilbm_set_option(self._h, int(option), int(value)))

    set_option = iilbm_set_option

    def iilbm_synchronize(self):
        _check("iilbm_synchronize", self._L.iilbm_synchronize(self._h))

    synchronize = iilbm_synchronize


class Batch:
    """Many lattices advanced together (handle of iilbm_create_batch).  Holds references
    to its lattices so that they outlive it."""

    def __init__(self, lattices, stream=None):
        L = load()
        self.lattices = list(lattices)
        arr = (_H * len(self.lattices))(*[g.handle for g in self.lattices])
        h = _H()
        _check("iilbm_create_batch",
               L.iilbm_create_batch(C.byref(h), arr, len(self.lattices), stream))
        self._h = h
        self._L = L

    def close(self):
        if getattr(self, "_h", None):
            self._L.iilbm_destroy_batch(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def __enter__(self):
        return self

    def __exit__(self, *exc):
        self.close()

    def iilbm_batch_step(self, n=1):
        _check("iilbm_batch_step", self._L.iilbm_batch_step(self._h, int(n)))

    step = iilbm_batch_step

    def iilbm_batch_set_variant(self, variant):
        if isinstance(variant, str):
            variant = BATCH_VARIANTS.index(variant)
        _check("iilbm_batch_set_variant", self._L.iilbm_batch_set_variant(self._h, int(variant)))

    def iilbm_batch_autotune(self, steps=64):
        """Time every stream-collide variant on the batch itself (the lattices advance);
        returns (variant chosen, us per step)."""
        v, us = C.c_int32(), C.c_double()
        _check("iilbm_batch_autotune",
               self._L.iilbm_batch_autotune(self._h, int(steps), C.byref(v), C.byref(us)))
        return v.value, us.value

    autotune = iilbm_batch_autotune

    def iilbm_batch_set_timing(self, enable=True):
        _check("iilbm_batch_set_timing", self._L.iilbm_batch_set_timing(self._h, int(enable)))

    def iilbm_batch_get_timing(self):
        ms, n, k = C.c_double(), C.c_int32(), C.c_int64()
        _check("iilbm_batch_get_timing",
               self._L.iilbm_batch_get_timing(self._h, C.byref(ms), C.byref(n), C.byref(k)))
        return ms.value, n.value, k.value

    def iilbm_batch_synchronize(self):
        _check("iilbm_batch_synchronize", self._L.iilbm_batch_synchronize(self._h))

    synchronize = iilbm_batch_synchronize


def _f32(a, shape=None):
    """Contiguous FP32 host array (or a contiguous float32 CUDA tensor, passed as is)."""
    if a is not None and not isinstance(a, np.ndarray) and hasattr(a, "data_ptr"):
        _ptr(a, None if shape is None else int(np.prod(shape)), dtype="float32")
        return a
    a = np.ascontiguousarray(np.asarray(a, dtype=np.float32))
    if shape is not None and a.size != int(np.prod(shape)):
        raise ValueError(f"expected {shape}, got {a.shape}")
    return a


def _fptr(a):
    return a.ctypes.data if isinstance(a, np.ndarray) else a.data_ptr()


class Mlp:
    """The learned warm start's network (handle of iilbm_mlp_create)."""

    def __init__(self, params=None, stream=None):
        L = load()
        h = _H()
        _check("iilbm_mlp_create", L.iilbm_mlp_create(C.byref(h), stream))
        self._h, self._L = h, L
        if params is not None:
            self.iilbm_mlp_set_params(params)

    @property
    def handle(self):
        return self._h

    def close(self):
        if getattr(self, "_h", None):
            self._L.iilbm_mlp_destroy(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def iilbm_mlp_set_params(self, params):
        p = _f32(params, (MLP_PARAMS,))
        _check("iilbm_mlp_set_params", self._L.iilbm_mlp_set_params(self._h, _fptr(p)))

    def iilbm_mlp_get_params(self):
        p = np.zeros(MLP_PARAMS, dtype=np.float32)
        _check("iilbm_mlp_get_params", self._L.iilbm_mlp_get_params(self._h, p.ctypes.data))
        return p

    def iilbm_mlp_set_normalization(self, in_mean, in_istd, out_mean, out_scale):
        a = [_f32(v, (n,)) for v, n in ((in_mean, 30), (in_istd, 30), (out_mean, 2), (out_scale, 2))]
        _check("iilbm_mlp_set_normalization",
               self._L.iilbm_mlp_set_normalization(self._h, *[x.ctypes.data for x in a]))

    def iilbm_mlp_forward(self, X):
        X = _f32(X)
        N = X.shape[0] if isinstance(X, np.ndarray) else X.shape[0]
        Y = np.zeros((N, 2), dtype=np.float32)
        _check("iilbm_mlp_forward", self._L.iilbm_mlp_forward(self._h, _fptr(X), N, Y.ctypes.data))
        return Y

    def iilbm_mlp_gradient(self, X, T):
        X, T = _f32(X), _f32(T)
        g = np.zeros(MLP_PARAMS, dtype=np.float32)
        loss = C.c_float()
        _check("iilbm_mlp_gradient",
               self._L.iilbm_mlp_gradient(self._h, _fptr(X), _fptr(T), X.shape[0], g.ctypes.data,
                                          C.byref(loss)))
        return loss.value, g

    def iilbm_mlp_train(self, X, T, order, batch, lr=1e-3, beta1=0.9, beta2=0.999, eps=1e-8):
        """Adam steps over batches order[s*batch:(s+1)*batch]; returns each step's loss."""
        X, T = _f32(X), _f32(T)
        order = np.ascontiguousarray(np.asarray(order, dtype=np.int32))
        steps = order.size // batch
        losses = np.zeros(max(steps, 1), dtype=np.float32)
        _check("iilbm_mlp_train",
               self._L.iilbm_mlp_train(self._h, _fptr(X), _fptr(T), X.shape[0], order.ctypes.data,
                                       steps, batch, lr, beta1, beta2, eps, losses.ctypes.data))
        return losses[:steps]

    forward = iilbm_mlp_forward
    gradient = iilbm_mlp_gradient
    train = iilbm_mlp_train
