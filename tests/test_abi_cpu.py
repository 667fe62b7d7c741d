"""CPU-side checks of the C ABI: the library builds, loads and exports every declared symbol."""
import os
import re

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _declared():
    names = set()
    for f in os.listdir(os.path.join(ROOT, "include")):
        if f.endswith(".h"):
            txt = open(os.path.join(ROOT, "include", f)).read()
            txt = re.sub(r"/\*.*?\*/", "", txt, flags=re.S)
            names |= set(re.findall(r"\b(sparc_\w+)\s*\(", txt))
    return names


@pytest.fixture(scope="module")
def lib():
    from paper_1603_04339_gb300 import build, sparc
    build.build()
    return sparc.load()


def test_library_exports_every_declared_entry_point(lib):
    declared = _declared()
    assert {"sparc_apply_H", "sparc_cheb_filter", "sparc_rayleigh_ritz", "sparc_lanczos_bounds"} <= declared
    for name in declared:
        assert hasattr(lib, name), name


def test_binding_declares_the_same_names():
    from paper_1603_04339_gb300 import sparc
    assert set(sparc.EXPORTS) == _declared()


def test_create_without_device_is_an_error_not_a_crash(lib):
    import ctypes
    import torch
    if torch.cuda.is_available():
        pytest.skip("a device is present")
    h = ctypes.c_void_p()
    rc = lib.sparc_create(ctypes.byref(h), 0)
    assert rc != 0 and not h.value


def test_null_arguments_are_rejected(lib):
    import ctypes
    assert lib.sparc_create(None, 0) == 1
    assert lib.sparc_apply_H(None, 0, None, None, 1, 1, None) == 1
    assert lib.sparc_cheb_filter(None, 0, 3, 0.0, 1.0, -1.0, None, None, 1, 1, None) == 1
    assert lib.sparc_rayleigh_ritz(None, 0, None, 2, 1, None, 0, None) == 1
    a, b = ctypes.c_double(), ctypes.c_double()
    assert lib.sparc_lanczos_bounds(None, 10, None, ctypes.byref(a), ctypes.byref(b), None) == 1
