"""CPU checks of the C ABI: the library builds for sm_103a, loads, exports every entry
point declared in include/bp.h, and rejects bad arguments before touching the GPU."""
import ctypes as C
import os
import re

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module")
def lib():
    from paper_2201_02632_gb300 import build

    build.build()
    from paper_2201_02632_gb300 import _lib

    return _lib.load()


def _declared():
    src = open(os.path.join(ROOT, "include", "bp.h")).read()
    return sorted(set(re.findall(r"^(?:int|int64_t|const char\*)\s+(bp_\w+)\(", src, re.M)))


def test_every_declared_symbol_is_exported(lib):
    names = _declared()
    assert len(names) >= 12
    for n in names:
        assert hasattr(lib, n), n
    from paper_2201_02632_gb300 import _lib

    assert sorted(_lib.EXPORTS) == names


def test_null_context_and_bad_parameters_are_rejected(lib):
    from paper_2201_02632_gb300 import _lib

    assert lib.bp_solve_halos(None, 1, None, None, None, None, None, 0, 0.0) == _lib.BP_EINVAL
    assert lib.bp_paste_particles(None, 1, None, None, 0, None, None, None, None) == _lib.BP_EINVAL
    h = C.c_void_p()
    bad = _lib.BpCosmology(Om=-1.0, Ob=0.046, h=0.7, Tcmb=2.726, XH=0.76)
    icm = _lib.BpIcm(1.2, 0.0, 3.97e-6, 0.026, 0.12, 0.18, 0.5, 0.8, 0, 0)
    assert lib.bp_create(C.byref(h), C.byref(bad), C.byref(icm), None) == _lib.BP_EINVAL
    assert b"non-physical" in lib.bp_last_error(None)
    good = _lib.BpCosmology(Om=0.279, Ob=0.046, h=0.7, Tcmb=2.726, XH=0.76)
    badicm = _lib.BpIcm(0.9, 0.0, 3.97e-6, 0.026, 0.12, 0.18, 0.5, 0.8, 0, 0)
    assert lib.bp_create(C.byref(h), C.byref(good), C.byref(badicm), None) == _lib.BP_EINVAL
    assert lib.bp_destroy(None) == _lib.BP_OK


def test_binding_refuses_cpu_tensors():
    import torch

    from paper_2201_02632_gb300 import api

    with pytest.raises(TypeError):
        api._ptr(torch.zeros(3, dtype=torch.float64), torch.float64, "x")


def test_binding_constants_match_the_header():
    """Every BP_* integer constant the binding mirrors has the header's value."""
    from paper_2201_02632_gb300 import _lib

    text = open(os.path.join(os.path.dirname(__file__), "..", "include", "bp.h")).read()
    defs = {m.group(1): int(m.group(2)) for m in
            re.finditer(r"^#define (BP_[A-Z0-9_]+) \(?(-?\d+)\)?", text, re.M)}
    names = [n for n in dir(_lib) if n.startswith("BP_") and isinstance(getattr(_lib, n), int)]
    assert len(names) >= 10
    for n in names:
        assert n in defs, n
        assert getattr(_lib, n) == defs[n], n
