"""GPU MUSCL-Hancock step (Sec. 2.4, eq. `GalerkUpdate`) against the oracle's, through
the C ABI: one kernel per step, face-centroid (1 point) and Gauss (2 points) face
rules, every tile shape, FP64 within 1e-12 and FP32 within 1e-5 of the variable's
scale (tests/helpers.py), ragged and degenerate grids, the Courant time step
chain over many steps, and the full-size Orszag-Tang 512x512 grid."""
import numpy as np
import pytest

import oracle as O
from paper_1305_5536_gb300 import dg, ics

from helpers import poly_rel_err

pytestmark = pytest.mark.gpu

TOL = {"fp64": 1e-12, "fp32": 1e-5}


def _generic_euler(n, seed=3):
    f = lambda X, Y: (1 + 0.2 * np.sin(2 * np.pi * (X + Y) + 0.31),
                      0.5 + 0.2 * np.sin(2 * np.pi * X + 0.47),
                      -0.3 + 0.2 * np.cos(2 * np.pi * Y + 0.23),
                      1 + 0.1 * np.sin(2 * np.pi * (X - 2 * Y) + 0.11))
    return ics.add_slope_noise(ics.project_2d(f, n), 0, 2, 0.05, np.random.default_rng(seed))


def _mh_one_step(eq, n, u0, prec, fp, limiter=1, box=(1.0, 1.0), frac=0.5):
    P = O.Problem(O.MHD if eq == "mhd" else O.EULER, 2, n, box=box, limiter=limiter)
    dt = frac * P.cfl_dt(u0)[0]
    ref, fl = P.mh_step(u0, dt, face_points=fp)
    assert fl == 0
    s = dg.DGSolver(eq, 2, n, box=box + (1.0,), limiter=limiter, precision=prec,
                    integrator="mh", face_points=fp)
    s.set_state(u0)
    s.step(1, dt=dt, sync=True)
    got = s.get_state()
    name = s.kernel_name()
    s.close()
    assert name.startswith("mh2d_kernel") and name.endswith("%dpt" % fp), name
    return got, ref, P.h


@pytest.mark.parametrize("fp", [1, 2])
@pytest.mark.parametrize("prec", ["fp64", "fp32"])
@pytest.mark.parametrize("n", [(4, 4), (5, 3), (37, 29), (64, 64), (1, 7), (33, 1)])
@pytest.mark.parametrize("limiter", [0, 1])
def test_mh_euler2d_one_step(fp, prec, n, limiter):
    u0 = _generic_euler(n)
    got, ref, h = _mh_one_step("euler", n, u0, prec, fp, limiter=limiter, box=(1.0, 0.9))
    err, where = poly_rel_err(got, ref, 0, 2, h)
    assert err < TOL[prec], (err, where)


@pytest.mark.parametrize("fp", [1, 2])
@pytest.mark.parametrize("prec", ["fp64", "fp32"])
@pytest.mark.parametrize("n", [(24, 20), (64, 64), (17, 5)])
@pytest.mark.parametrize("limiter", [0, 1])
def test_mh_mhd2d_one_step(fp, prec, n, limiter):
    u0 = ics.orszag_tang(n)
    got, ref, h = _mh_one_step("mhd", n, u0, prec, fp, limiter=limiter)
    err, where = poly_rel_err(got, ref, 1, 2, h)
    assert err < TOL[prec], (err, where)


@pytest.mark.parametrize("variant", [0, 1, 2])
@pytest.mark.parametrize("prec", ["fp64", "fp32"])
@pytest.mark.parametrize("eq", ["euler", "mhd"])
def test_mh_every_tile_variant(variant, prec, eq, monkeypatch):
    monkeypatch.setenv("DG_TILE_VARIANT", str(variant))
    n = (72, 40)
    u0 = _generic_euler(n) if eq == "euler" else ics.orszag_tang(n)
    for fp in (1, 2):
        got, ref, h = _mh_one_step(eq, n, u0, prec, fp)
        err, where = poly_rel_err(got, ref, 1 if eq == "mhd" else 0, 2, h)
        assert err < TOL[prec], (fp, err, where)


@pytest.mark.parametrize("fp", [1, 2])
def test_mh_courant_chain_40_steps_fp64(fp):
    """40 steps with the Courant time step computed on the device (fused into the
    step kernel) against the oracle's run: same time steps and final state."""
    n = (48, 40)
    u0 = ics.orszag_tang(n)
    P = O.Problem(O.MHD, 2, n)
    ref, dts, fl = P.mh_run(u0, 40, cfl=0.3, face_points=fp)
    assert fl == 0
    s = dg.DGSolver("mhd", 2, n, precision="fp64", cfl=0.3, integrator="mh", face_points=fp)
    s.set_state(u0)
    t = s.step(40, sync=True)
    assert abs(t - dts.sum()) < 1e-12 * dts.sum()
    err, where = poly_rel_err(s.get_state(), ref, 1, 2, P.h)
    s.close()
    assert err < 1e-10, (err, where)


def test_mh_orszag_tang_512_one_step_full_size():
    """Full-size Orszag-Tang 512x512 (FP64 and FP32), one step, every cell, with the
    paper's face-centroid rule."""
    n = (512, 512)
    u0 = ics.orszag_tang(n)
    P = O.Problem(O.MHD, 2, n)
    dt = P.cfl_dt(u0)[0]
    ref, fl = P.mh_step(u0, dt, face_points=1)
    assert fl == 0
    for prec in ("fp64", "fp32"):
        s = dg.DGSolver("mhd", 2, n, precision=prec, integrator="mh", face_points=1)
        s.set_state(u0)
        s.step(1, dt=dt, sync=True)
        err, where = poly_rel_err(s.get_state(), ref, 1, 2, P.h)
        s.close()
        assert err < TOL[prec], (prec, err, where)


@pytest.mark.parametrize("prec", ["fp64", "fp32"])
def test_mh_conservation_free_stream_and_batch(prec):
    n = (64, 64)
    u0 = ics.orszag_tang(n)
    s = dg.DGSolver("mhd", 2, n, precision=prec, integrator="mh")
    assert s.kernel_name().endswith("1pt")  # the face-centroid rule by default
    s.set_state(u0)
    t0 = s.totals()[0]
    s.step(20, sync=True)
    t1 = s.totals()[0]
    assert np.abs(t1 - t0).max() < (1e-13 if prec == "fp64" else 1e-6) * np.abs(t0).max()
    s.close()
    u = ics.project_2d(lambda X, Y: (1.3, 0.7, -0.4, 2.0, 0.5, -0.8), (16, 12), eq=1)
    s = dg.DGSolver("mhd", 2, (16, 12), precision=prec, integrator="mh")
    s.set_state(u)
    s.step(5, sync=True)
    # FP32: the face solver's and the volume flux's roundings of the same flux
    # differ by ~1e-7 and enter the derivative equations with 3/dx^2
    err, where = poly_rel_err(s.get_state(), u, 1, 2, (1 / 16, 1 / 12))
    assert err < (1e-13 if prec == "fp64" else 1e-5), (err, where)
    s.close()
    # several problems in one context: one launch per problem and step
    sizes = [(40, 40), (24, 32), (17, 9)]
    cfgs = [dg.make_config("mhd", 2, m, precision=prec, integrator="mh") for m in sizes]
    states = [ics.orszag_tang(m) for m in sizes]
    dt = min(O.Problem(O.MHD, 2, m).cfl_dt(u)[0] for m, u in zip(sizes, states)) * 0.5
    b = dg.DGSolver(configs=cfgs)
    b.set_state(np.concatenate([u.ravel() for u in states]))
    b.step(1, dt=dt, sync=True)
    got = b.get_state()
    b.close()
    off = 0
    for m, u in zip(sizes, states):
        P = O.Problem(O.MHD, 2, m)
        ref, _ = P.mh_step(u, dt)
        g = got[off:off + u.size].reshape(u.shape)
        off += u.size
        err, where = poly_rel_err(g, ref, 1, 2, P.h)
        assert err < TOL[prec], (m, err, where)


def _kh_noisy(n, seed=5):
    u = ics.kh3d(n, w0=0.1)
    rng = np.random.default_rng(seed)
    for v in range(5):
        for k in range(1, 4):
            u[v * 4 + k] += 0.02 * rng.standard_normal(u.shape[1:]) * (1 + abs(u[v * 4]))
    return u


@pytest.mark.parametrize("variant", [0, 1])
@pytest.mark.parametrize("fp", [1, 2])
@pytest.mark.parametrize("prec", ["fp64", "fp32"])
@pytest.mark.parametrize("n", [(8, 8, 8), (12, 10, 6), (17, 9, 5), (1, 6, 4)])
@pytest.mark.parametrize("limiter", [0, 1])
def test_mh_euler3d_one_step(variant, fp, prec, n, limiter, monkeypatch):
    monkeypatch.setenv("DG_TILE_VARIANT", str(variant))
    u0 = _kh_noisy(n)
    box = (1.0, 0.9, 1.1)
    P = O.Problem(O.EULER, 3, n, box=box, limiter=limiter)
    dt = 0.5 * P.cfl_dt(u0)[0]
    ref, fl = P.mh_step(u0, dt, face_points=fp)
    assert fl == 0
    s = dg.DGSolver("euler", 3, n, box=box, limiter=limiter, precision=prec, integrator="mh",
                    face_points=fp)
    s.set_state(u0)
    s.step(1, dt=dt, sync=True)
    assert s.kernel_name().startswith("mh3d_kernel")
    err, where = poly_rel_err(s.get_state(), ref, 0, 3, P.h)
    s.close()
    assert err < TOL[prec], (err, where)


def test_mh_kh3d_64_courant_chain_fp64():
    """KH shear layer 64^3, 6 steps with device Courant time steps, against the
    oracle's run."""
    n = (64, 64, 64)
    u0 = ics.kh3d(n)
    P = O.Problem(O.EULER, 3, n)
    ref, dts, fl = P.mh_run(u0, 6, cfl=0.3)
    assert fl == 0
    s = dg.DGSolver("euler", 3, n, precision="fp64", integrator="mh")
    s.set_state(u0)
    t = s.step(6, sync=True)
    assert abs(t - dts.sum()) < 1e-12 * dts.sum()
    err, where = poly_rel_err(s.get_state(), ref, 0, 3, P.h)
    s.close()
    assert err < 1e-11, (err, where)


def test_mh_rejects_what_it_does_not_implement():
    with pytest.raises(dg.DGError):
        dg.DGSolver("euler", 2, (8, 8), integrator="rk2", face_points=1)
    s = dg.DGSolver("euler", 2, (8, 8), integrator="mh", ckpt_every=2)
    s.set_state(_generic_euler((8, 8)))
    with pytest.raises(dg.DGError):
        s.record(2)
    s.close()
