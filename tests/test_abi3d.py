"""The library exports and the binding types every entry point include/iilbm3d.h
declares; invalid configurations are rejected on the host before any device use.  CPU
only (no compute)."""
import ctypes as C
import os
import re

import pytest

from paper_2003_12186_gb300 import iilbm3d

HDR = os.path.join(os.path.dirname(os.path.dirname(os.path.abspath(__file__))), "include",
                   "iilbm3d.h")


def declared():
    src = open(HDR).read()
    return sorted(set(re.findall(r"^\s*int\s+(iilbm3d_\w+)\s*\(", src, re.M)))


def test_every_declared_symbol_is_exported_and_bound():
    names = declared()
    for must in ("iilbm3d_create", "iilbm3d_set_surface", "iilbm3d_step", "iilbm3d_get_macros",
                 "iilbm3d_get_jump"):
        assert must in names
    L = iilbm3d.load()
    for name in names:
        assert hasattr(L, name), name
    assert set(names) == set(iilbm3d.SIGNATURES3)


def _cfg(**kw):
    c = iilbm3d.iilbm3d_config()
    base = dict(nx=16, ny=16, nz=16, collision=iilbm3d.MRT, storage=iilbm3d.F32, tau=0.8,
                rho0=1.0, jump=1, force=0)
    base.update(kw)
    for k, v in base.items():
        setattr(c, k, v)
    for r, s in enumerate(iilbm3d.paper_rates(base["tau"])):
        c.s[r] = s
    return c


def test_invalid_configs_rejected_before_device_use():
    L = iilbm3d.load()
    for bad in (dict(nx=2), dict(nz=4096), dict(tau=0.5), dict(storage=4), dict(storage=-1),
                dict(collision=3), dict(jump=2), dict(force=5), dict(rho0=0.0),
                dict(storage_scale_log2=3), dict(storage=iilbm3d.F16, storage_scale_log2=25)):
        h = C.c_void_p()
        assert L.iilbm3d_create(C.byref(h), C.byref(_cfg(**bad))) == -1, bad
        assert not h.value
    c = _cfg()
    c.s[4] = 2.5  # a non-conserved MRT rate outside (0, 2)
    assert L.iilbm3d_create(C.byref(C.c_void_p()), C.byref(c)) == -1
    assert L.iilbm3d_create(None, None) == -1
    assert L.iilbm3d_step(None, 1) == -1
    assert L.iilbm3d_destroy(None) == -1


def test_no_device_is_reported_without_a_gpu():
    torch = pytest.importorskip("torch")
    if torch.cuda.is_available():
        pytest.skip("a GPU is present")
    with pytest.raises(iilbm3d.IilbmError) as e:
        iilbm3d.Lattice3D(8, 8, 8)
    assert e.value.code == -8
