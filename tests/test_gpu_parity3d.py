"""3D Euler GPU stage kernels against the CPU oracle (through the C ABI)."""
import numpy as np
import pytest

import oracle as O
from paper_1305_5536_gb300 import dg, ics

from helpers import poly_rel_err

pytestmark = pytest.mark.gpu

TOL = {"fp64": 1e-12, "fp32": 1e-5}


def _generic3d(n, seed=5):
    """Smooth 3D state in which every primitive varies, plus slope noise."""
    nx, ny, nz = n
    x = (np.arange(nx) + 0.5) / nx
    y = (np.arange(ny) + 0.5) / ny
    z = (np.arange(nz) + 0.5) / nz
    Z, Y, X = np.meshgrid(z, y, x, indexing="ij")
    rho = 1 + 0.2 * np.sin(2 * np.pi * (X + Y + Z) + 0.3)
    v = [0.4 + 0.2 * np.sin(2 * np.pi * X + 0.5), -0.3 + 0.2 * np.cos(2 * np.pi * Y + 0.2),
         0.2 + 0.2 * np.sin(2 * np.pi * Z + 0.7)]
    p = 1 + 0.1 * np.sin(2 * np.pi * (X - Y + 2 * Z) + 0.1)
    E = p / (5 / 3 - 1) + 0.5 * rho * sum(c * c for c in v)
    u = np.zeros((20,) + rho.shape)
    rng = np.random.default_rng(seed)
    for k, f in enumerate([rho, rho * v[0], rho * v[1], rho * v[2], E]):
        u[4 * k] = f
        # smooth gradients + noise
        for d in range(3):
            u[4 * k + 1 + d] = rng.uniform(-0.3, 0.3, rho.shape) * np.abs(f).mean()
    return u


@pytest.mark.parametrize("prec", ["fp64", "fp32"])
@pytest.mark.parametrize("n", [(8, 8, 8), (12, 10, 6), (5, 3, 7), (16, 16, 16)])
@pytest.mark.parametrize("limiter", [0, 1])
def test_euler3d_one_step(prec, n, limiter):
    u0 = _generic3d(n)
    box = (1.0, 0.9, 1.1)
    P = O.Problem(O.EULER, 3, n, box=box, limiter=limiter)
    dt = 0.5 * P.cfl_dt(u0)[0]
    ref, fl = P.step(u0, dt)
    assert fl == 0
    s = dg.DGSolver("euler", 3, n, box=box, limiter=limiter, precision=prec)
    s.set_state(u0)
    s.step(1, dt=dt, sync=True)
    err, where = poly_rel_err(s.get_state(), ref, 0, 3, P.h)
    s.close()
    assert err < TOL[prec], (err, where)


def test_kh3d_small_multi_step_cfl():
    n = (16, 16, 16)
    u0 = ics.kh3d(n, w0=0.1)
    P = O.Problem(O.EULER, 3, n)
    ref, dts, fl = P.run(u0, 5, cfl=0.3)
    assert fl == 0
    s = dg.DGSolver("euler", 3, n, precision="fp64")
    s.set_state(u0)
    t = s.step(5, sync=True)
    assert abs(t - dts.sum()) < 1e-13 * dts.sum()
    err, where = poly_rel_err(s.get_state(), ref, 0, 3, P.h)
    assert err < 1e-11, (err, where)


def test_kh3d_256_full_size_sampled_cells():
    """Full-size 3D Kelvin-Helmholtz 256^3, FP32, one step: sampled cells against
    the oracle run on a periodic 11^3 window around each (the step of a cell only
    depends on cells within Manhattan distance 4)."""
    n = (256, 256, 256)
    u0 = ics.kh3d(n)
    P = O.Problem(O.EULER, 3, n)
    dt, fl = P.cfl_dt(u0)
    assert fl == 0
    s = dg.DGSolver("euler", 3, n, precision="fp32")
    s.set_state(u0)
    tnext = s.times()[1][0]
    assert abs(tnext - dt) < 1e-6 * dt
    s.step(1, dt=dt, sync=True)
    got = s.get_state()
    s.close()
    rng = np.random.default_rng(17)
    # include cells at the shear interfaces (y = 64, 192) and at the periodic seams
    cells = [(0, 63, 0), (255, 64, 255), (17, 191, 128), (128, 192, 3), (255, 255, 255)]
    cells += [tuple(int(c) for c in rng.integers(0, 256, 3)) for _ in range(11)]
    h = 5
    W = O.Problem(O.EULER, 3, (2 * h + 1,) * 3, box=tuple((2 * h + 1) / 256.0 for _ in range(3)))
    worst = 0.0
    for (i, j, k) in cells:
        ix = np.arange(i - h, i + h + 1) % 256
        iy = np.arange(j - h, j + h + 1) % 256
        iz = np.arange(k - h, k + h + 1) % 256
        win = u0[:, iz][:, :, iy][:, :, :, ix]
        out, fl = W.step(np.ascontiguousarray(win), dt)
        assert fl == 0
        ref = out[:, h, h, h]
        g = got[:, k, j, i]
        scale = np.abs(u0[0::4]).reshape(5, -1).max(1)
        scale[1:4] = np.sqrt((u0[4:16:4] ** 2).sum(0)).max()
        for v in range(5):
            d = abs(g[4 * v] - ref[4 * v]) + sum(abs(g[4 * v + 1 + a] - ref[4 * v + 1 + a]) * 0.5 / 256
                                                 for a in range(3))
            worst = max(worst, d / scale[v])
    assert worst < TOL["fp32"], worst
