"""The C-ABI library builds, loads and exports every symbol of include/dg.h (no GPU)."""
import ctypes
import os
import re

import pytest

from paper_1305_5536_gb300 import _build, dg

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _declared():
    src = open(os.path.join(ROOT, "include", "dg.h")).read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    return sorted(set(re.findall(r"\b(dg_[a-z_0-9]+)\s*\(", src)))


def test_header_and_binding_agree():
    assert sorted(dg.SYMBOLS) == _declared()


def test_library_exports_every_symbol():
    lib = dg.load()
    for name in _declared():
        assert hasattr(lib, name), name


def test_num_planes_and_validation():
    lib = dg.load()
    for eq, dim, n in ((0, 2, 12), (0, 3, 20), (1, 2, 17), (1, 3, 31)):
        c = dg.make_config("mhd" if eq else "euler", dim, (8, 8, 8))
        assert lib.dg_num_planes(ctypes.byref(c)) == n
    # every equation set takes both integrators and every limiter
    for lim in (0, 1, 2):
        c = dg.make_config("mhd", 3, (8, 8, 8), limiter=lim)
        assert lib.dg_num_planes(ctypes.byref(c)) == 31
        for fp in (0, 1, 2):
            c = dg.make_config("mhd", 3, (8, 8, 8), limiter=lim, integrator="mh", face_points=fp)
            assert lib.dg_num_planes(ctypes.byref(c)) == 31
    # not built: the SSP-RK2 step with the face-centroid rule
    bad = dg.make_config("euler", 2, (8, 8), face_points=1)
    assert lib.dg_num_planes(ctypes.byref(bad)) == -1
    bad = dg.make_config("euler", 2, (8, 8))
    bad.gamma = 1.0
    assert lib.dg_num_planes(ctypes.byref(bad)) == -1


def test_init_rejects_bad_config_without_gpu_work():
    lib = dg.load()
    h = ctypes.c_void_p()
    bad = dg.make_config("euler", 2, (0, 8))
    assert lib.dg_init(ctypes.byref(bad), None, ctypes.byref(h)) == dg.DG_EINVAL
    assert b"grid size" in lib.dg_last_error(None)
    assert not h.value
