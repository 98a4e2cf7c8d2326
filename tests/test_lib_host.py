"""The C-ABI library without a GPU: it loads, exports every entry point that include/cme.h
declares, and rejects invalid arguments on the host before touching CUDA."""
import ctypes
import os
import re

import numpy as np
import pytest

from paper_1307_3428_gb300 import _build, cme

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module")
def lib():
    _build.build()
    return cme.load()


def header_functions():
    names = []
    for fn in os.listdir(os.path.join(ROOT, "include")):
        if fn.endswith(".h"):
            text = open(os.path.join(ROOT, "include", fn)).read()
            text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
            names += re.findall(r"^\s*(?:const\s+)?[A-Za-z_][\w\s\*]*?\b(cme_\w+)\s*\(",
                                text, flags=re.M)
    return sorted(set(names))


def test_header_lists_entry_points():
    names = header_functions()
    for must in ("cme_create", "cme_batch_create", "cme_step", "cme_spectrum", "cme_last_error"):
        assert must in names


def test_library_exports_every_declared_symbol(lib):
    for name in header_functions():
        assert hasattr(lib, name), name
    # and the binding wraps every declared function
    assert set(header_functions()) <= set(cme.exported_names())


def test_create_validates_on_host(lib):
    N = 12
    kap = np.ones(N)
    om = np.zeros(N)
    with pytest.raises(cme.CmeError) as e:
        cme.Instance(N, kap, om, 1.0, 0.5, 1.0, 0.0)
    assert e.value.code == -2
    for bad in (2, 1 << 21, 0, -4):
        with pytest.raises(cme.CmeError) as e:
            cme.Instance(bad, np.ones(max(bad, 1)), np.zeros(max(bad, 1)), 1.0, 0.5, 1.0, 0.0)
        assert e.value.code == -2
    with pytest.raises(cme.CmeError) as e:
        cme.Instance(8, -np.ones(8), np.zeros(8), 1.0, 0.5, 1.0, 0.0)
    assert e.value.code == -1
    with pytest.raises(cme.CmeError) as e:
        cme.Instance(8, np.ones(8), np.full(8, np.nan), 1.0, 0.5, 1.0, 0.0)
    assert e.value.code == -1
    inst = cme.Instance(8, np.ones(8), np.zeros(8), 1.0, 0.5, 1.0, 0.0)
    with pytest.raises(cme.CmeError):
        inst.set_field(np.full(8, np.nan + 0j))


def test_batch_create_rejects_bad_arguments(lib):
    a = cme.Instance(16, np.ones(16), np.zeros(16), 1.0, 0.5, 1.0, 0.0)
    b = cme.Instance(8, np.ones(8), np.zeros(8), 1.0, 0.5, 1.0, 0.0)
    with pytest.raises(cme.CmeError) as e:
        cme.Batch([a, b])            # not ordered by N
    assert e.value.code == -1
    with pytest.raises(cme.CmeError) as e:
        cme.Batch([b], precision=7)
    assert e.value.code == -1
    with pytest.raises(cme.CmeError) as e:
        cme.Batch([b], integrator=5)
    assert e.value.code == -1
    with pytest.raises(cme.CmeError) as e:
        cme.Batch([a], radix=2)      # launch shape not compiled
    assert e.value.code == -1 and b"N=16" in lib.cme_last_error()
    for M in (0, 17, -3):            # physical modes must lie in [1, N]
        with pytest.raises(cme.CmeError) as e:
            a.set_modes(M)
        assert e.value.code == -1 and b"cme_set_modes" in lib.cme_last_error()
    a.set_modes(16)
    a.set_modes(1)
    out = ctypes.c_void_p()
    om = np.zeros(16)
    dp = ctypes.POINTER(ctypes.c_double)
    assert lib.cme_create_eq2(16, None, None, 1.0, 0.0, ctypes.byref(out)) == -1
    assert lib.cme_create_eq2(12, None, om.ctypes.data_as(dp), 1.0, 0.0, ctypes.byref(out)) == -2
    bad = np.full(16, -1.0)
    assert lib.cme_create_eq2(16, bad.ctypes.data_as(dp), om.ctypes.data_as(dp), 1.0, 0.0,
                              ctypes.byref(out)) == -1
    assert b"cme_create_eq2" in lib.cme_last_error()
    cme.Instance.from_eq2(16, om, 1.2 + 0.1j, M=11)
    for c in (3, 16, -1):            # blocks per instance must be 0, 1, 2, 4 or 8
        with pytest.raises(cme.CmeError) as e:
            cme.Batch([a], cluster=c)
        assert e.value.code == -1 and b"cluster" in lib.cme_last_error()
    out = ctypes.c_void_p()
    assert lib.cme_batch_create(None, 0, None, None, ctypes.byref(out)) == -1
    assert lib.cme_step(None, 1e-3, 1) == -1
    assert lib.cme_spectrum(None, 0, 0, None) == -1
    assert b"invalid argument" in lib.cme_last_error()


def test_version_and_counters(lib):
    assert b"sm_103a" in lib.cme_version()
    assert lib.cme_kernel_launches() >= 0
