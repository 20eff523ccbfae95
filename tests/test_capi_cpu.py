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


def _cfg(**kw):
    """A valid 2D Euler configuration with the given raw fields overwritten."""
    dim = kw.pop("dim", 2)
    n = kw.pop("n", (8, 8, 8))
    mhd = kw.get("eq") == 1
    c = dg.make_config("mhd" if mhd else "euler", dim if dim in (2, 3) else 2, n)
    c.dim = dim
    for k, v in kw.items():
        if k == "box":
            for a, b in enumerate(v):
                c.box[a] = b
        else:
            setattr(c, k, v)
    return c


# every rule of the configuration check, with the fragment of its message
BAD = [
    (dict(eq=2), "eq must be"),
    (dict(dim=1), "dim must be"),
    (dict(n=(0, 8)), "grid size"),
    (dict(n=((1 << 20) + 1, 8)), "grid size"),
    (dict(dim=3, n=(2048, 2048, 512)), "too many cells"),
    (dict(box=(0.0, 1.0)), "box lengths"),
    (dict(box=(float("inf"), 1.0)), "box lengths"),
    (dict(gamma=1.0), "gamma"),
    (dict(gamma=float("nan")), "gamma"),
    (dict(cfl=0.0), "cfl"),
    (dict(cfl=float("inf")), "cfl"),
    (dict(limiter=3), "limiter"),
    (dict(precision=2), "precision"),
    (dict(riemann=1), "exact Riemann"),
    (dict(eq=1, riemann=0), "HLLD"),
    (dict(ckpt_every=-1), "ckpt_every"),
    (dict(integrator=2), "integrator"),
    (dict(integrator=1, face_points=3), "face_points"),
    (dict(face_points=1), "Gauss face rule"),
]


@pytest.mark.parametrize("kw,msg", BAD, ids=[m for _, m in BAD])
def test_every_configuration_rule_rejects_with_its_message(kw, msg):
    lib = dg.load()
    c = _cfg(**kw)
    assert lib.dg_num_planes(ctypes.byref(c)) == -1
    h = ctypes.c_void_p()
    assert lib.dg_init(ctypes.byref(c), None, ctypes.byref(h)) == dg.DG_EINVAL
    assert msg.encode() in lib.dg_last_error(None), lib.dg_last_error(None)
    assert not h.value


def test_largest_accepted_sizes():
    lib = dg.load()
    # the per-axis and total-cell limits themselves are accepted
    assert lib.dg_num_planes(ctypes.byref(_cfg(n=(1 << 20, 8)))) == 12
    assert lib.dg_num_planes(ctypes.byref(_cfg(dim=3, n=(2048, 2048, 476)))) == 20


def test_batch_rules():
    lib = dg.load()
    h = ctypes.c_void_p()
    one = _cfg()
    assert lib.dg_init_batch(ctypes.byref(one), 0, None, ctypes.byref(h)) == dg.DG_EINVAL
    assert b"at least one" in lib.dg_last_error(None)
    arr = (dg.dg_config * 2)(_cfg(), _cfg(cfl=0.4))
    assert lib.dg_init_batch(arr, 2, None, ctypes.byref(h)) == dg.DG_EINVAL
    assert b"must share" in lib.dg_last_error(None)
    arr = (dg.dg_config * 2)(_cfg(), _cfg(limiter=7))
    assert lib.dg_init_batch(arr, 2, None, ctypes.byref(h)) == dg.DG_EINVAL
    assert b"configuration 1" in lib.dg_last_error(None)
    assert not h.value
    assert lib.dg_init(ctypes.byref(one), None, None) == dg.DG_EINVAL
