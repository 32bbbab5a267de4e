"""The C-ABI library builds, loads and exports every entry point include/iilbm.h
declares; host-side argument checks work without a GPU.  CPU only (no compute)."""
import ctypes as C
import os
import re

import pytest

from paper_2003_12186_gb300 import iilbm

HDR = os.path.join(os.path.dirname(os.path.dirname(os.path.abspath(__file__))), "include",
                   "iilbm.h")


def declared():
    src = open(HDR).read()
    return sorted(set(re.findall(r"^\s*(?:int|const char \*)\s*(iilbm_\w+)\s*\(", src, re.M)))


def test_header_declares_the_boundary():
    names = declared()
    for must in ("iilbm_create_lattice", "iilbm_set_interface", "iilbm_step",
                 "iilbm_get_macros"):
        assert must in names
    assert len(names) >= 12


def test_library_exports_every_declared_symbol():
    L = iilbm.load()
    for name in declared():
        assert hasattr(L, name), name
    assert set(declared()) <= set(iilbm.SIGNATURES)


def test_error_strings():
    assert iilbm.error_string(0) == "ok"
    assert "invalid" in iilbm.error_string(-1)
    assert iilbm.error_string(-99) == "unknown status"


def test_invalid_configs_rejected_before_device_use():
    L = iilbm.load()
    base = dict(nx=16, ny=16, collision=iilbm.MRT, storage=iilbm.F32, tau=0.8)
    bad = [dict(nx=2), dict(tau=0.5), dict(storage=7), dict(collision=5), dict(ny=100000)]
    for b in bad:
        c = iilbm.iilbm_config()
        kw = dict(base, **b)
        c.nx, c.ny, c.collision, c.storage, c.tau, c.rho0 = (kw["nx"], kw["ny"], kw["collision"],
                                                             kw["storage"], kw["tau"], 1.0)
        for i in range(9):
            c.s[i] = 1.0
        h = C.c_void_p()
        assert L.iilbm_create_lattice(C.byref(h), C.byref(c)) == -1
        assert not h.value
    assert L.iilbm_create_lattice(None, None) == -1
    assert L.iilbm_step(None, 1) == -1
    assert L.iilbm_destroy(None) == -1


def test_no_device_is_reported_without_a_gpu():
    torch = pytest.importorskip("torch")
    if torch.cuda.is_available():
        pytest.skip("a GPU is present")
    with pytest.raises(iilbm.IilbmError) as e:
        iilbm.Lattice(16, 16)
    assert e.value.code == -8


def test_buffer_checks_raise_value_error():
    """The binding checks every buffer the library will read or write (dtype, layout,
    element count, device) and raises ValueError, which `python -O` keeps."""
    import numpy as np
    a = np.zeros(10)
    assert iilbm._ptr(a, 10) == a.ctypes.data
    assert iilbm._ptr(None, 10) is None
    for bad in (dict(a=a, count=11), dict(a=np.zeros(10, np.float32), count=10),
                dict(a=np.zeros((4, 6))[:, ::2], count=12), dict(a=[0.0] * 10, count=10)):
        with pytest.raises(ValueError):
            iilbm._ptr(bad["a"], bad["count"])
    torch = pytest.importorskip("torch")
    t = torch.zeros(10, dtype=torch.float64)
    assert iilbm._ptr(t, 10) == t.data_ptr()
    with pytest.raises(ValueError):
        iilbm._ptr(t, 9)
    with pytest.raises(ValueError):
        iilbm._ptr(t.to(torch.float32), 10)
    with pytest.raises(ValueError):
        iilbm._ptr(torch.zeros(10, dtype=torch.float64, device="meta"), 10)
