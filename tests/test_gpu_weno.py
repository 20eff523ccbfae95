"""The WENO-type limiter of Sec. 2.5 (limiter = 2) on the GPU against the oracle,
through the C ABI, in every kernel that limits: the SSP-RK2 stages (2D Euler and
MHD, every 2D tile shape including the TMA kernels, 3D Euler), the batched 2D
step, and the MUSCL-Hancock steps (2D and 3D).  FP64 within 1e-12, FP32 within
1e-5 of the variable's scale (tests/helpers.py)."""
import numpy as np
import pytest

import oracle as O
from paper_1305_5536_gb300 import dg, ics

from helpers import poly_rel_err

pytestmark = pytest.mark.gpu

TOL = {"fp64": 1e-12, "fp32": 1e-5}


def _euler2d(n, seed=3):
    f = lambda X, Y: (1 + 0.2 * np.sin(2 * np.pi * (X + Y) + 0.31) + 0.3 * (X > 0.6),
                      0.5 + 0.2 * np.sin(2 * np.pi * X + 0.47),
                      -0.3 + 0.2 * np.cos(2 * np.pi * Y + 0.23),
                      1 + 0.1 * np.sin(2 * np.pi * (X - 2 * Y) + 0.11) + 0.4 * (Y > 0.5))
    return ics.add_slope_noise(ics.project_2d(f, n), 0, 2, 0.2, np.random.default_rng(seed))


def _mhd2d(n, seed=4):
    u = ics.orszag_tang(n)
    rng = np.random.default_rng(seed)
    for pl in (1, 2, 4, 5, 7, 8, 10, 11, 14, 15, 16):
        u[pl] += 0.2 * rng.standard_normal(u.shape[1:])
    return u


def _euler3d(n, seed=5):
    u = ics.kh3d(n, w0=0.1)
    rng = np.random.default_rng(seed)
    for v in range(5):
        for k in range(1, 4):
            u[v * 4 + k] += 0.2 * rng.standard_normal(u.shape[1:]) * (1 + abs(u[v * 4]))
    return u


def _check(eq, dim, n, u0, prec, integrator="rk2", box=None, steps=1):
    box = box or (1.0, 1.0, 1.0)[:dim]
    P = O.Problem(O.MHD if eq == "mhd" else O.EULER, dim, n, box=box, limiter=2)
    dt = 0.5 * P.cfl_dt(u0)[0]
    ref = u0
    for _ in range(steps):
        ref, fl = (P.mh_step(ref, dt) if integrator == "mh" else P.step(ref, dt))
        assert fl == 0
    s = dg.DGSolver(eq, dim, n, box=tuple(box) + (1.0,) * (3 - dim), limiter=2, precision=prec,
                    integrator=integrator)
    s.set_state(u0)
    s.step(steps, dt=dt, sync=True)
    err, where = poly_rel_err(s.get_state(), ref, 1 if eq == "mhd" else 0, dim, P.h)
    s.close()
    assert err < (3 if steps > 1 else 1) * TOL[prec], (err, where)


@pytest.mark.parametrize("integrator", ["rk2", "mh"])
@pytest.mark.parametrize("prec", ["fp64", "fp32"])
@pytest.mark.parametrize("n", [(5, 3), (37, 29), (64, 64), (33, 1)])
def test_weno_euler2d(integrator, prec, n):
    _check("euler", 2, n, _euler2d(n), prec, integrator, box=(1.0, 0.9))


@pytest.mark.parametrize("integrator", ["rk2", "mh"])
@pytest.mark.parametrize("prec", ["fp64", "fp32"])
@pytest.mark.parametrize("n", [(24, 20), (64, 64), (17, 5)])
def test_weno_mhd2d(integrator, prec, n):
    _check("mhd", 2, n, _mhd2d(n), prec, integrator)


@pytest.mark.parametrize("integrator", ["rk2", "mh"])
@pytest.mark.parametrize("prec", ["fp64", "fp32"])
@pytest.mark.parametrize("n", [(8, 8, 8), (12, 10, 6)])
def test_weno_euler3d(integrator, prec, n):
    _check("euler", 3, n, _euler3d(n), prec, integrator, box=(1.0, 0.9, 1.1))


@pytest.mark.parametrize("variant", [0, 1, 2, 3, 4])
@pytest.mark.parametrize("prec", ["fp64", "fp32"])
def test_weno_every_rk_tile_variant(variant, prec, monkeypatch):
    monkeypatch.setenv("DG_TILE_VARIANT", str(variant))
    n = (64, 48)
    _check("mhd", 2, n, _mhd2d(n), prec, steps=2)


@pytest.mark.parametrize("prec", ["fp64", "fp32"])
def test_weno_batch(prec):
    sizes = [(40, 40), (24, 32), (33, 9)]
    states = [_mhd2d(m, seed=i) for i, m in enumerate(sizes)]
    cfgs = [dg.make_config("mhd", 2, m, precision=prec, limiter=2) for m in sizes]
    dt = min(O.Problem(O.MHD, 2, m).cfl_dt(u)[0] for m, u in zip(sizes, states)) * 0.5
    b = dg.DGSolver(configs=cfgs)
    b.set_state(np.concatenate([u.ravel() for u in states]))
    b.step(1, dt=dt, sync=True)
    got = b.get_state()
    b.close()
    off = 0
    for m, u in zip(sizes, states):
        P = O.Problem(O.MHD, 2, m, limiter=2)
        ref, fl = P.step(u, dt)
        assert fl == 0
        g = got[off:off + u.size].reshape(u.shape)
        off += u.size
        err, where = poly_rel_err(g, ref, 1, 2, P.h)
        assert err < TOL[prec], (m, err, where)


def test_weno_orszag_tang_512_full_size_and_adjoint_refusal():
    n = (512, 512)
    u0 = ics.orszag_tang(n)
    P = O.Problem(O.MHD, 2, n, limiter=2)
    dt = P.cfl_dt(u0)[0]
    ref, fl = P.step(u0, dt)
    assert fl == 0
    s = dg.DGSolver("mhd", 2, n, precision="fp32", limiter=2)
    s.set_state(u0)
    s.step(1, dt=dt, sync=True)
    err, where = poly_rel_err(s.get_state(), ref, 1, 2, P.h)
    s.close()
    assert err < TOL["fp32"], (err, where)
    e = dg.DGSolver("euler", 2, (8, 8), limiter=2, ckpt_every=2)
    e.set_state(_euler2d((8, 8)))
    with pytest.raises(dg.DGError):
        e.record(2)
    e.close()
