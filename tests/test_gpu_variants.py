"""Every compiled tile shape of the 2D stage kernels -- per-element staging
(variants 0-2) and the persistent TMA kernels (3, 4) -- against the oracle, on grids
mixing interior tiles (TMA boxes) and tiles at the periodic seams."""
import numpy as np
import pytest

import oracle as O
from paper_1305_5536_gb300 import dg, ics

from helpers import poly_rel_err

pytestmark = pytest.mark.gpu

TOL = {"fp64": 1e-12, "fp32": 1e-5}


def _state(eq, n):
    if eq == "mhd":
        return ics.mhd_random_smooth(n[0], rng=np.random.default_rng(3)) if n[0] == n[1] else \
            ics.orszag_tang(n)
    f = lambda X, Y: (1 + 0.2 * np.sin(2 * np.pi * (X + Y) + 0.31),
                      0.5 + 0.2 * np.sin(2 * np.pi * X + 0.47),
                      -0.3 + 0.2 * np.cos(2 * np.pi * Y + 0.23),
                      1 + 0.1 * np.sin(2 * np.pi * (X - 2 * Y) + 0.11))
    return ics.add_slope_noise(ics.project_2d(f, n), 0, 2, 0.05, np.random.default_rng(4))


@pytest.mark.parametrize("variant", [0, 1, 2, 3, 4])
@pytest.mark.parametrize("prec", ["fp64", "fp32"])
@pytest.mark.parametrize("eq", ["euler", "mhd"])
@pytest.mark.parametrize("n", [(64, 48), (96, 96)])
def test_every_tile_variant_one_and_two_steps(variant, prec, eq, n, monkeypatch):
    monkeypatch.setenv("DG_TILE_VARIANT", str(variant))
    u0 = _state(eq, n)
    P = O.Problem(O.MHD if eq == "mhd" else O.EULER, 2, n)
    dt = 0.5 * P.cfl_dt(u0)[0]
    ref, fl = P.step(u0, dt)
    assert fl == 0
    ref2, fl = P.step(ref, dt)
    s = dg.DGSolver(eq, 2, n, precision=prec)
    s.set_state(u0)
    s.step(1, dt=dt, sync=True)
    err, where = poly_rel_err(s.get_state(), ref, 1 if eq == "mhd" else 0, 2, P.h)
    assert err < TOL[prec], (err, where)
    s.step(1, dt=dt, sync=True)
    err, where = poly_rel_err(s.get_state(), ref2, 1 if eq == "mhd" else 0, 2, P.h)
    assert err < 3 * TOL[prec], (err, where)
    s.close()


@pytest.mark.parametrize("variant", [3, 4])
@pytest.mark.parametrize("prec", ["fp64", "fp32"])
@pytest.mark.parametrize("eq", ["euler", "mhd"])
def test_tma_kernel_many_tiles_per_cta(variant, prec, eq, monkeypatch):
    """The persistent TMA kernels with their grid capped at 3 CTAs (test hook
    DG_TEST_MAX_CTAS): each CTA walks 20-40 tiles, so the next-tile prefetch into
    the raw boxes, the reuse of shared memory across tiles and the seam tiles'
    element-wise staging between TMA tiles all run; the result must still be the
    oracle's."""
    monkeypatch.setenv("DG_TILE_VARIANT", str(variant))
    monkeypatch.setenv("DG_TEST_MAX_CTAS", "3")
    n = (128, 96)
    u0 = _state(eq, n)
    P = O.Problem(O.MHD if eq == "mhd" else O.EULER, 2, n)
    dt = 0.5 * P.cfl_dt(u0)[0]
    ref, fl = P.step(u0, dt)
    assert fl == 0
    ref2, fl = P.step(ref, dt)
    assert fl == 0
    s = dg.DGSolver(eq, 2, n, precision=prec)
    s.set_state(u0)
    assert "stage2d_tma_kernel" in s.kernel_name()
    s.step(1, dt=dt, sync=True)
    err, where = poly_rel_err(s.get_state(), ref, 1 if eq == "mhd" else 0, 2, P.h)
    assert err < TOL[prec], (err, where)
    s.step(1, dt=dt, sync=True)
    err, where = poly_rel_err(s.get_state(), ref2, 1 if eq == "mhd" else 0, 2, P.h)
    assert err < 3 * TOL[prec], (err, where)
    s.close()
