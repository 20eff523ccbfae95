"""Pins of the oracle's WENO-type limiter (Sec. 2.5, limiter = 2) to things other
than itself (no GPU): invariances it must have by construction, special cases
with a closed-form result, and the convergence and shock behaviour of the scheme
that uses it."""
import math

import numpy as np
import pytest

import oracle as O
from paper_1305_5536_gb300 import ics


def _slope_planes(eq, dim):
    K = dim + 1
    nT = 4 if (dim == 2) else 5
    planes = [v * K + k for v in range(nT) for k in range(1, K)]
    if eq == O.MHD:
        planes += [4 * K + 2, 4 * K + 3, 4 * K + 4]
    return planes


@pytest.mark.parametrize("eq,dim", [(O.EULER, 2), (O.EULER, 3), (O.MHD, 2)])
def test_weno_keeps_linear_data(eq, dim):
    """Linear primitive data (uniform v): the DG gradient and the central
    difference are both the exact gradient, the stencil's min/max factor is 1, so
    every interior cell keeps its coefficients; a linear divergence-free field is
    reproduced by the projection of its stencil gradient."""
    n = (10, 9, 8)[:dim]
    box = (1.0, 0.7, 1.3)[:dim]
    P = O.Problem(eq, dim, n, box=box, limiter=2)
    h = P.h
    u = np.zeros(P.shape)
    grid = np.meshgrid(*[(np.arange(m) + 0.5) * hh for m, hh in zip(n, h)], indexing="ij")
    X = [g.T for g in grid]  # (nz,) ny, nx order
    K = dim + 1
    gr = (0.3, -0.2, 0.15)[:dim]
    gp = (-0.1, 0.25, 0.05)[:dim]
    rho = 1.0 + sum(a * x for a, x in zip(gr, X))
    p = 2.0 + sum(a * x for a, x in zip(gp, X))
    v = (0.4, -0.3, 0.2)[:dim]
    gm = 5.0 / 3.0
    mag = 0.0
    if eq == O.MHD:
        # Bx = 0.5 + 0.2 x + 0.1 y, By = -0.3 + 0.3 x - 0.2 y (divergence free)
        b1 = 0.5 + 0.2 * X[0] + 0.1 * X[1]
        b2 = -0.3 + 0.3 * X[0] - 0.2 * X[1]
        b0 = 4 * K
        u[b0], u[b0 + 1], u[b0 + 2], u[b0 + 3], u[b0 + 4] = b1, b2, 0.1, 0.3, 0.2
        mag = 0.5 * (b1 ** 2 + b2 ** 2)
    # the energy of linear rho, p with uniform v is linear except for the
    # magnetic energy; give the average its exact cell mean and the slopes their
    # centroid derivatives (the limiter only uses centroid values and gradients)
    v2 = sum(a * a for a in v)
    u[0] = rho
    for d in range(dim):
        u[1 + d] = gr[d]
    for a in range(dim):
        u[K * (1 + a)] = rho * v[a]
        for d in range(dim):
            u[K * (1 + a) + 1 + d] = gr[d] * v[a]
    e = K * (1 + dim)
    u[e] = p / (gm - 1) + 0.5 * rho * v2 + mag
    for d in range(dim):
        dB = 0.0
        if eq == O.MHD:
            dB = b1 * (0.2 if d == 0 else 0.1) + b2 * (0.3 if d == 0 else -0.2)
        u[e + 1 + d] = gp[d] / (gm - 1) + 0.5 * gr[d] * v2 + dB
    out, f = P.limit(u)
    assert f == 0
    interior = (slice(None),) + tuple(slice(1, m - 1) for m in reversed(n))
    pl = _slope_planes(eq, dim)
    np.testing.assert_allclose(out[pl][interior], u[pl][interior], rtol=1e-12, atol=1e-13)


def test_weno_removes_the_slope_in_a_flat_neighbourhood():
    """Neighbours equal to the cell (flat averages): the stencil candidate is zero
    with zero oscillation, its weight eps^(-1/2) dominates, and whatever DG slope
    the cell carries is replaced by (almost exactly) zero."""
    n = (8, 8)
    u = ics.project_2d(lambda X, Y: (1.2, 0.3, -0.1, 1.5), n)
    rng = np.random.default_rng(8)
    for pl in (1, 2, 4, 5, 7, 8, 10, 11):
        u[pl] = rng.uniform(-0.5, 0.5, n[::-1])
    P = O.Problem(O.EULER, 2, n, limiter=2)
    out, f = P.limit(u)
    assert f == 0
    # sqrt(eps / o_dg) with o_dg ~ |slope| h: a relative 1e-7 of the slopes
    assert np.abs(out[[1, 2, 4, 5, 7, 8, 10, 11]]).max() < 1e-6


def test_weno_reflection_symmetry():
    """Mirroring the data in x (x -> -x: reversed cells, negated x derivatives and
    x momentum) mirrors the limited state."""
    n = (12, 10)
    f = lambda X, Y: (1 + 0.3 * np.sin(2 * np.pi * X) * np.cos(2 * np.pi * Y) + 0.2 * (X > 0.5),
                      0.4 + 0.2 * np.cos(2 * np.pi * (X + 0.1)), 0.1 * np.sin(2 * np.pi * Y),
                      1 + 0.3 * (X > 0.3))
    u = ics.add_slope_noise(ics.project_2d(f, n), 0, 2, 0.3, np.random.default_rng(2))
    P = O.Problem(O.EULER, 2, n, limiter=2)

    def mirror(a):
        m = a[:, :, ::-1].copy()
        for v in range(4):
            m[3 * v + 1] *= -1  # d/dx
        m[3:6] *= -1           # x momentum: average and derivatives
        return m

    a, _ = P.limit(u)
    b, _ = P.limit(mirror(u))
    np.testing.assert_allclose(mirror(a), b, rtol=1e-12, atol=1e-13)


def test_weno_scale_covariance_of_a_density_limiter():
    """Uniform v and p: only the density's gradient is limited.  Scaling the
    density deviations and slopes by c scales both candidates and every
    oscillation factor by c, so the weights keep their ratio and the limited
    slope scales by c (eps is negligible here)."""
    n = (16, 12)
    rng = np.random.default_rng(4)

    def state(c):
        f = lambda X, Y: (2 + c * np.sin(2 * np.pi * X + 0.2) * np.cos(2 * np.pi * Y), 0.3, -0.2,
                          1.0)
        u = ics.project_2d(f, n)
        return u

    u1, u2 = state(0.1), state(0.3)
    noise = rng.standard_normal((2,) + n[::-1])
    for u, c in ((u1, 0.1), (u2, 0.3)):
        u[1] += c * noise[0]
        u[2] += c * noise[1]
        # momentum and energy slopes follow the density slopes (uniform v, p)
        u[4], u[5] = 0.3 * u[1], 0.3 * u[2]
        u[7], u[8] = -0.2 * u[1], -0.2 * u[2]
        u[10], u[11] = 0.5 * 0.13 * u[1], 0.5 * 0.13 * u[2]
    P = O.Problem(O.EULER, 2, n, limiter=2)
    a, _ = P.limit(u1)
    b, _ = P.limit(u2)
    np.testing.assert_allclose(b[[1, 2]] / 0.3, a[[1, 2]] / 0.1, rtol=1e-10, atol=1e-12)
    assert not np.allclose(a[[1, 2]], u1[[1, 2]])  # the limiter did act


@pytest.mark.parametrize("eq,dim", [(O.EULER, 2), (O.EULER, 3), (O.MHD, 2)])
def test_weno_conservation_and_divergence_free(eq, dim):
    if eq == O.MHD:
        n = (24, 20)
        u = ics.orszag_tang(n)
    elif dim == 2:
        n = (24, 20)
        u = ics.euler2d_wave(n, noise=1e-2)
    else:
        n = (8, 8, 8)
        u = ics.kh3d(n, w0=0.1)
    P = O.Problem(eq, dim, n, limiter=2)
    t0 = P.totals(u)
    out, _, f = P.run(u, 4)
    assert f == 0
    np.testing.assert_allclose(P.totals(out), t0, atol=2e-14 * np.abs(t0).max())
    out2, _, f = P.mh_run(u, 4)
    assert f == 0
    np.testing.assert_allclose(P.totals(out2), t0, atol=2e-14 * np.abs(t0).max())


def _order(errs):
    return [math.log(errs[i] / errs[i + 1], 2) for i in range(len(errs) - 1)]


def test_weno_smooth_wave_second_order():
    """Smooth advected density wave with the WENO-type limiter on: second order
    in L1 (the scheme stays accurate on smooth data)."""
    errs = []
    T = 0.125
    for N in (16, 32, 64):
        u0 = ics.euler2d_wave((N, N), noise=0.0)
        P = O.Problem(O.EULER, 2, (N, N), limiter=2)
        dt0, _ = P.cfl_dt(u0, 0.3)
        ns = int(math.ceil(T / dt0))
        out, _, f = P.run(u0, ns, dt=T / ns)
        assert f == 0
        ex = ics.project_2d(lambda X, Y: (1 + 0.2 * np.sin(2 * np.pi * (X + Y - 2 * T)), 1.0, 1.0,
                                          1.0), (N, N))
        errs.append(np.abs(out[0] - ex[0]).mean())
    assert _order(errs)[-1] > 1.8, errs


def test_weno_sod_first_order_small_overshoot():
    """Sec. 3.2 Sod variant with the WENO-type limiter: first order in L1, and the
    density leaves its initial range by less than 1 % of the jump (the limiter is
    not total-variation diminishing)."""
    g, T, L = 1.4, 5.0, 20.0
    errs = []
    for N in (64, 128, 256):
        nx = 2 * N

        def f(X, Y):
            left = X - L < 0
            return np.where(left, 1.0, 0.25), 0.0, 0.0, np.where(left, 1.0, 0.1795)

        u = ics.project_2d(f, (nx, 1), box=(2 * L, L / N), gamma=g)
        P = O.Problem(O.EULER, 2, (nx, 1), box=(2 * L, L / N), gamma=g, limiter=2)
        t = 0.0
        while t < T - 1e-12:
            dt, _ = P.cfl_dt(u, 0.3)
            dt = min(dt, T - t)
            u, fl = P.step(u, dt)
            assert fl == 0
            t += dt
        dx = L / N
        xs = -L + (np.arange(nx) + 0.5) * dx
        sub = (np.arange(64) + 0.5) / 64 - 0.5
        W, _, _ = O.exact_sample((1.0, 0.0, 1.0), (0.25, 0.0, 0.1795), g,
                                 (xs[:, None] + dx * sub[None, :]).ravel() / T)
        ex = W[:, 0].reshape(nx, 64).mean(1)
        win = np.abs(xs) < 10
        errs.append(np.abs(u[0, 0][win] - ex[win]).mean())
        jump = 1.0 - 0.25
        assert u[0, 0].max() < 1.0 + 0.01 * jump and u[0, 0].min() > 0.25 - 0.01 * jump
    overall = math.log(errs[0] / errs[-1], 2) / (len(errs) - 1)
    assert errs[0] > errs[1] > errs[2] and 0.6 < overall < 1.3, (errs, overall)


def test_weno_limits_the_stencil_candidate():
    """A density step with zero DG slopes.  Next to the step the central
    difference would take the cell below its lower neighbour (0 -> -1/4 of the
    jump at the far face), so its min/max factor is 0 and both candidates are
    zero: the limited slopes stay exactly zero everywhere.  An unlimited stencil
    candidate would leave half of the central difference."""
    n = (16, 1)
    u = ics.project_2d(lambda X, Y: (np.where((X > 0.25) & (X < 0.75), 2.0, 1.0), 0.0, 0.0, 1.0),
                       n, box=(1.0, 1.0 / 16))
    P = O.Problem(O.EULER, 2, n, box=(1.0, 1.0 / 16), limiter=2)
    u[[1, 2, 4, 5, 7, 8, 10, 11]] = 0.0  # the projection leaves rounding there
    out, f = P.limit(u)
    assert f == 0
    assert np.abs(out[[1, 2, 4, 5, 7, 8, 10, 11]]).max() == 0.0
