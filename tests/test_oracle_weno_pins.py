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
        planes += list(range(nT * K + dim, nT * K + (5 if dim == 2 else 11)))
    return planes


# a linear divergence-free 3D field: gradient coefficients a4..a11 of the basis
# Bx = b1 + (a10 + a11) x + a4 y + a5 z, By = b2 + a6 x - a10 y + a7 z,
# Bz = b3 + a8 x + a9 y - a11 z
_A3 = (0.1, -0.05, 0.3, 0.12, -0.07, 0.2, 0.15, -0.1)


def _grad_of(a):
    a4, a5, a6, a7, a8, a9, a10, a11 = a
    return np.array([[a10 + a11, a4, a5], [a6, -a10, a7], [a8, a9, -a11]])


@pytest.mark.parametrize("eq,dim", [(O.EULER, 2), (O.EULER, 3), (O.MHD, 2), (O.MHD, 3)])
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
    if eq == O.MHD and dim == 2:
        # Bx = 0.5 + 0.2 x + 0.1 y, By = -0.3 + 0.3 x - 0.2 y (divergence free)
        b1 = 0.5 + 0.2 * X[0] + 0.1 * X[1]
        b2 = -0.3 + 0.3 * X[0] - 0.2 * X[1]
        b0 = 4 * K
        u[b0], u[b0 + 1], u[b0 + 2], u[b0 + 3], u[b0 + 4] = b1, b2, 0.1, 0.3, 0.2
        mag = 0.5 * (b1 ** 2 + b2 ** 2)
    if eq == O.MHD and dim == 3:
        Gb = _grad_of(_A3)
        Bc = [b + sum(Gb[i][e] * X[e] for e in range(3)) for i, b in enumerate((0.5, -0.3, 0.2))]
        b0 = 5 * K
        for i in range(3):
            u[b0 + i] = Bc[i]
        for k in range(8):
            u[b0 + 3 + k] = _A3[k]
        mag = 0.5 * sum(b ** 2 for b in Bc)
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
        if eq == O.MHD and dim == 2:
            dB = b1 * (0.2 if d == 0 else 0.1) + b2 * (0.3 if d == 0 else -0.2)
        if eq == O.MHD and dim == 3:
            dB = sum(Bc[i] * Gb[i][d] for i in range(3))
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


@pytest.mark.parametrize("eq,dim", [(O.EULER, 2), (O.EULER, 3), (O.MHD, 2), (O.MHD, 3)])
def test_weno_conservation_and_divergence_free(eq, dim):
    if eq == O.MHD and dim == 3:
        n = (8, 8, 8)
        u = ics.orszag_tang_3d(n)
    elif eq == O.MHD:
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


def _field_cell_3d(i, e, g=0.4, box=(1.0, 0.6, 1.7)):
    """5^3 cells, uniform rho, v = 0, p; zero derivative coefficients; the field
    averages B_i = g (x_e - x_c) (centroid coordinate e about the centre cell), so
    that the centre cell's stencil gradient of the field is g in entry (i, e) and
    zero elsewhere.  Returns the centre cell's limited field coefficients a4..a11
    and the cell sizes."""
    n = (5, 5, 5)
    P = O.Problem(O.MHD, 3, n, box=box, limiter=2)
    h = P.h
    u = np.zeros(P.shape)
    grid = np.meshgrid(*[(np.arange(m) - 2) * hh for m, hh in zip(n, h)], indexing="ij")
    X = [a.T for a in grid]
    B = [np.zeros(n[::-1]) + b for b in (0.3, -0.2, 0.25)]
    B[i] = B[i] + g * X[e]
    u[0] = 1.0
    for k in range(3):
        u[20 + k] = B[k]
    u[16] = 1.0 / (5.0 / 3.0 - 1.0) + 0.5 * sum(b ** 2 for b in B)
    out, f = P.limit(u)
    assert f == 0
    return out[23:31, 2, 2, 2], h


@pytest.mark.parametrize("i,e,k", [(0, 1, 0), (0, 2, 1), (1, 0, 2), (1, 2, 3), (2, 0, 4),
                                   (2, 1, 5)])
def test_weno_3d_field_projection_cross_derivatives(i, e, k):
    """The L2 projection onto the divergence-free basis keeps a cross derivative
    dB_i/dx_e (i != e) as its own basis coefficient (a4 = dBx/dy, a5 = dBx/dz,
    a6 = dBy/dx, a7 = dBy/dz, a8 = dBz/dx, a9 = dBz/dy): the limited field of
    a cell whose only field variation is B_i along e has that one coefficient,
    positive, and every other one exactly zero."""
    a, _ = _field_cell_3d(i, e)
    assert a[k] > 0.0
    others = [a[m] for m in range(8) if m != k]
    assert max(abs(x) for x in others) == 0.0, a


@pytest.mark.parametrize("i", [0, 1, 2])
def test_weno_3d_field_projection_diagonal_closed_form(i):
    """A stencil gradient g in the diagonal entry (i, i) alone is not divergence
    free.  Its L2 projection over an h_x x h_y x h_z cell minimises
      h_x^2 (a10 + a11 - G_xx)^2 + h_y^2 (-a10 - G_yy)^2 + h_z^2 (-a11 - G_zz)^2,
    whose minimiser has, with D = h_x^2 h_y^2 + h_x^2 h_z^2 + h_y^2 h_z^2,
      G_xx = g: a10 = g h_x^2 h_z^2 / D, a11 = g h_x^2 h_y^2 / D,
      G_yy = g: a10 = -g h_y^2 (h_x^2 + h_z^2) / D, a11 = g h_x^2 h_y^2 / D,
      G_zz = g: a10 = g h_x^2 h_z^2 / D, a11 = -g h_z^2 (h_x^2 + h_y^2) / D.
    The blend scales the projection by the weight ws/(wd + ws) (the DG candidate
    is zero), so the ratio a10/a11 is the projection's; a4..a9 stay zero."""
    a, h = _field_cell_3d(i, i)
    hx2, hy2, hz2 = h[0] ** 2, h[1] ** 2, h[2] ** 2
    ref = {0: (hx2 * hz2, hx2 * hy2), 1: (-hy2 * (hx2 + hz2), hx2 * hy2),
           2: (hx2 * hz2, -hz2 * (hx2 + hy2))}[i]
    assert np.abs(a[:6]).max() == 0.0
    assert a[6] != 0.0 and a[7] != 0.0
    np.testing.assert_allclose(a[6] / a[7], ref[0] / ref[1], rtol=1e-13)
    assert np.sign(a[6]) == np.sign(ref[0])


def test_weno_3d_mhd_alfven_wave_converges():
    """The circularly polarised Alfven wave along (1, 1, 1) with the WENO-type
    limiter on: the scheme stays close to second order on this smooth exact
    solution (SSP-RK2; about 1.86 between 16^3 and 32^3)."""
    T = 0.05
    errs = []
    for N in (8, 16, 32):
        n = (N, N, N)
        u0 = ics.alfven_cp_3d(n)
        P = O.Problem(O.MHD, 3, n, limiter=2)
        dt0, _ = P.cfl_dt(u0, 0.3)
        ns = int(math.ceil(T / dt0))
        out, _, f = P.run(u0, ns, dt=T / ns)
        assert f == 0
        ex = ics.alfven_cp_3d(n, t=T)
        errs.append(sum(np.abs(out[20 + i] - ex[20 + i]).mean() for i in range(3)))
    o = _order(errs)
    assert o[-1] > 1.7, (errs, o)
