"""The C ABI library loads and exports every entry point include/sfmm.h
declares; argument validation that needs no GPU."""
import ctypes
import os
import re

import pytest

from paper_2210_07021_gb300 import sfmm

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def declared():
    txt = open(os.path.join(ROOT, "include", "sfmm.h")).read()
    txt = re.sub(r"/\*.*?\*/", "", txt, flags=re.S)
    return sorted(set(re.findall(r"\b(sfmm_[a-z_0-9]+)\s*\(", txt)))


def test_header_and_binding_agree():
    assert declared() == sorted(sfmm.EXPORTS)


def test_library_exports_every_declared_symbol():
    L = sfmm.load()
    for name in declared():
        assert hasattr(L, name), name


def test_default_options():
    L = sfmm.load()
    o = sfmm.Options()
    assert L.sfmm_default_options(ctypes.byref(o)) == sfmm.SFMM_OK
    assert (o.leaf_size, o.c_s, o.c_t, o.precision) == (32, 2.0, 0.5, sfmm.SFMM_FP64)
    assert L.sfmm_default_options(None) == sfmm.SFMM_EINVAL


@pytest.mark.parametrize("depth,p,tol,msg", [
    (30, 10, 0.0, "max_depth"),
    (-1, 10, 0.0, "max_depth"),
    (29, 33, 0.0, "order_p"),
    (29, 0, 0.0, "tol"),
    (29, 0, 1.5, "tol"),
])
def test_plan_rejects_bad_arguments(depth, p, tol, msg):
    L = sfmm.load()
    h = ctypes.c_void_p()
    assert L.sfmm_plan(ctypes.byref(h), depth, p, tol, None) == sfmm.SFMM_EINVAL
    assert h.value is None
    assert msg in L.sfmm_last_error(None).decode()


def test_plan_rejects_bad_mac():
    L = sfmm.load()
    o = sfmm.Options()
    L.sfmm_default_options(ctypes.byref(o))
    o.c_s = 0.9
    h = ctypes.c_void_p()
    assert L.sfmm_plan(ctypes.byref(h), 29, 10, 0.0, ctypes.byref(o)) == sfmm.SFMM_EINVAL
    assert "c_s" in L.sfmm_last_error(None).decode()


def test_null_plan_calls():
    L = sfmm.load()
    assert L.sfmm_potential(None, None, None, 0, None, 0, None) == sfmm.SFMM_EINVAL
    assert L.sfmm_get_stats(None, None) == sfmm.SFMM_EINVAL
    L.sfmm_destroy(None)
