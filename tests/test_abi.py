"""Host-side checks of the C-ABI library: it builds, loads, and exports every
entry point include/ndmg.h declares.  No GPU calls."""
import ctypes
import os
import re

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
LIB = os.path.join(ROOT, "paper_2205_05840_gb300", "libndmg.so")
HEADER = os.path.join(ROOT, "include", "ndmg.h")


def _declared():
    with open(HEADER) as fh:
        txt = fh.read()
    return sorted(set(re.findall(r"^\s*(?:int|const char\s*\*)\s+(ndmg_\w+)\s*\(", txt, flags=re.M)))


@pytest.fixture(scope="module")
def lib():
    if not os.path.exists(LIB):
        from paper_2205_05840_gb300 import build
        build.build()
    return ctypes.CDLL(LIB)


def test_header_declares_the_abi():
    names = _declared()
    for want in ("ndmg_create", "ndmg_destroy", "ndmg_apply", "ndmg_residual", "ndmg_smooth", "ndmg_restrict",
                 "ndmg_prolong_add", "ndmg_coarse_solve", "ndmg_vcycle", "ndmg_solve", "ndmg_grad_alpha",
                 "ndmg_set_alpha", "ndmg_num_dofs", "ndmg_last_error"):
        assert want in names


def test_library_exports_every_declared_symbol(lib):
    missing = [n for n in _declared() if not hasattr(lib, n)]
    assert not missing, missing


def test_opts_default_and_invalid_create_without_gpu(lib):
    # ndmg_opts_default is pure host code; ndmg_create rejects bad options on
    # the host before touching the device
    from paper_2205_05840_gb300 import ndmg
    o = ndmg.Opts()
    assert ndmg._lib.ndmg_opts_default(ctypes.byref(o)) == 0
    assert (o.n, o.n_coarsest, o.m, o.nrhs) == (8, 2, 2, 1)
    assert abs(o.eta - 1 / 9) < 1e-15 and o.L == 1.0
    h = ctypes.c_void_p()
    for field, bad in (("n", 7), ("alpha", -1.0), ("beta", 0.0), ("m", 0), ("L", 0.0), ("n_coarsest", 3)):
        o2 = ndmg.Opts()
        ndmg._lib.ndmg_opts_default(ctypes.byref(o2))
        setattr(o2, field, bad)
        assert ndmg._lib.ndmg_create(ctypes.byref(o2), ctypes.byref(h)) == ndmg.INVALID_ARG
        assert not h.value
    assert ndmg._lib.ndmg_create(None, ctypes.byref(h)) == ndmg.INVALID_ARG
    assert ndmg._lib.ndmg_destroy(None) == 0


def test_binding_signatures_cover_header():
    from paper_2205_05840_gb300 import ndmg
    declared = set(_declared())
    bound = set(ndmg._SIGS) | {"ndmg_last_error"}
    assert declared <= bound, declared - bound
