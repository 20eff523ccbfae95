"""Pins of the oracle's MUSCL-Hancock step (Sec. 2.4, eq. `GalerkUpdate`) to things
other than itself (no GPU).

The half-step prediction is checked against the time derivative that the
conservative system itself gives (flux divergence by central differences), the
update against the already pinned Runge-Kutta right-hand side on data where the
primitive and conserved reconstructions coincide, and the whole step against
free streams, conservation, and the convergence orders fixed by the mathematics
of a second-order scheme.
"""
import math

import numpy as np
import pytest

import oracle as O
from paper_1305_5536_gb300 import ics


def _p2c(W, g):
    rho, v, p, B = W[0], W[1:4], W[4], W[5:8]
    E = p / (g - 1) + 0.5 * rho * (v @ v) + 0.5 * (B @ B)
    return np.concatenate([[rho], rho * v, [E], B])


def _c2p(U, g):
    rho, m, E, B = U[0], U[1:4], U[4], U[5:8]
    v = m / rho
    p = (g - 1) * (E - 0.5 * (m @ v) - 0.5 * (B @ B))
    return np.concatenate([[rho], v, [p], B])


def _rates_from_flux_divergence(W, dW, dim, g, eps=1e-6):
    """dW/dt at the centroid of the linear primitive field W + dW.x, from the
    conservative system: dU/dt = -sum_d dF_d/dx_d, then the chain rule through
    the primitive map (both derivatives by central differences)."""
    dUdt = np.zeros(8)
    for d in range(dim):
        e = np.zeros(3)
        e[d] = eps
        Fp = O.phys_flux(_p2c(W + dW @ e, g), d, g)
        Fm = O.phys_flux(_p2c(W - dW @ e, g), d, g)
        dUdt -= (Fp - Fm) / (2 * eps)
    U = _p2c(W, g)
    return (_c2p(U + eps * dUdt, g) - _c2p(U - eps * dUdt, g)) / (2 * eps)


@pytest.mark.parametrize("eq,dim", [(O.EULER, 2), (O.EULER, 3), (O.MHD, 2), (O.MHD, 3)])
def test_prediction_rates_match_flux_divergence(eq, dim):
    """The primitive form used for the half-step prediction is the conservative
    system rewritten: a dropped term, a wrong sign or a transposed index of any
    A_d fails here.  The magnetic gradients are divergence free, as in every cell
    of the scheme."""
    rng = np.random.default_rng(11 + 3 * eq + dim)
    g = 5.0 / 3.0
    for _ in range(6):
        W = np.zeros(8)
        W[0] = rng.uniform(0.5, 2.0)
        W[1:1 + dim] = rng.uniform(-1, 1, dim)
        W[4] = rng.uniform(0.5, 2.0)
        dW = np.zeros((8, 3))
        dW[[0, 1, 2, 4], :dim] = rng.uniform(-1, 1, (4, dim))
        if dim == 3:
            dW[3, :] = rng.uniform(-1, 1, 3)
        if eq == O.MHD:
            W[5:5 + (3 if dim == 3 else 2)] = rng.uniform(-1, 1, 3 if dim == 3 else 2)
            nb = 3 if dim == 3 else 2
            G = rng.uniform(-1, 1, (nb, dim))
            G[nb - 1, nb - 1] = -np.trace(G[:nb - 1, :nb - 1]) if dim == nb else G[nb - 1, nb - 1]
            if dim == 2:
                G[1, 1] = -G[0, 0]
            dW[5:5 + nb, :dim] = G
            assert abs(sum(dW[5 + i, i] for i in range(dim))) < 1e-15
        got = O.prim_rates(W, dW, dim, g)
        ref = _rates_from_flux_divergence(W, dW, dim, g)
        np.testing.assert_allclose(got, ref, atol=1e-7 * (1 + np.abs(ref).max()))


def test_prediction_rates_of_an_advected_density():
    """Uniform v and p, B = 0: only the density changes, at -v.grad rho."""
    W = np.array([1.3, 0.7, -0.4, 0.2, 2.0, 0, 0, 0])
    dW = np.zeros((8, 3))
    dW[0] = (0.3, -0.5, 0.9)
    got = O.prim_rates(W, dW, 3, 1.4)
    ref = np.zeros(8)
    ref[0] = -(0.7 * 0.3 + 0.4 * 0.5 + 0.2 * 0.9)
    np.testing.assert_allclose(got, ref, atol=1e-15)


@pytest.mark.parametrize("fp", [1, 2])
@pytest.mark.parametrize("eq,dim", [(O.EULER, 2), (O.EULER, 3), (O.MHD, 2)])
def test_mh_free_stream(eq, dim, fp):
    n = (6, 5, 4)[:dim]
    P = O.Problem(eq, dim, n, box=(1.0, 0.8, 1.2)[:dim], limiter=1)
    if dim == 2:
        prim = (1.3, 0.7, -0.4, 2.0) + ((0.5, -0.8) if eq == O.MHD else ())
        u = ics.project_2d(lambda X, Y: prim, n, box=(1.0, 0.8), eq=eq)
    else:
        u = np.zeros(P.shape)
        rho, v, p = 1.3, (0.7, -0.4, 0.2), 2.0
        for k, val in enumerate([rho, rho * v[0], rho * v[1], rho * v[2],
                                 p / (5 / 3 - 1) + 0.5 * rho * sum(x * x for x in v)]):
            u[k * 4] = val
    dt, _ = P.cfl_dt(u)
    out, _, f = P.mh_run(u, 3, dt=dt, face_points=fp)
    assert f == 0
    np.testing.assert_allclose(out, u, atol=1e-13 * np.abs(u).max())


@pytest.mark.parametrize("fp", [1, 2])
@pytest.mark.parametrize("eq,dim,lim", [(O.EULER, 2, 1), (O.EULER, 3, 1), (O.MHD, 2, 1),
                                        (O.MHD, 2, 0)])
def test_mh_conservation(eq, dim, lim, fp):
    if eq == O.MHD:
        n = (24, 20)
        u = ics.orszag_tang(n)
    elif dim == 2:
        n = (24, 20)
        u = ics.euler2d_wave(n, noise=1e-2)
    else:
        n = (8, 8, 8)
        u = ics.kh3d(n, w0=0.1)
    P = O.Problem(eq, dim, n, limiter=lim)
    t0 = P.totals(u)
    out, _, f = P.mh_run(u, 4, face_points=fp)
    assert f == 0
    np.testing.assert_allclose(P.totals(out), t0, atol=2e-14 * np.abs(t0).max())


@pytest.mark.parametrize("eq,dim", [(O.EULER, 2), (O.EULER, 3), (O.MHD, 2)])
def test_mh_update_is_the_weak_form_rhs(eq, dim):
    """With uniform v, p and B the primitive reconstruction is the conserved
    polynomial itself, so as dt -> 0 the MUSCL-Hancock update with the Gauss face
    rule tends to dt times the (pinned) right-hand side of the Runge-Kutta step:
    face weights, volume terms and mass matrices of eq. `GalerkUpdate` agree."""
    n = (6, 5, 4)[:dim]
    box = (1.0, 0.8, 1.2)[:dim]
    P = O.Problem(eq, dim, n, box=box, limiter=0)
    rng = np.random.default_rng(5)
    if dim == 2:
        f = lambda X, Y: ((1 + 0.2 * np.sin(2 * np.pi * X + 0.3) * np.cos(2 * np.pi * Y / 0.8)),
                          0.7, -0.4, 2.0) + ((0.5, -0.8) if eq == O.MHD else ())
        u = ics.project_2d(f, n, box=box, eq=eq)
        u[0, :, :] += 0.0
    else:
        u = np.zeros(P.shape)
        rho = 1 + 0.1 * rng.standard_normal(P.shape[1:])
        drho = 0.3 * rng.standard_normal((3,) + P.shape[1:])
        v, p = (0.7, -0.4, 0.2), 2.0
        for k in range(4):
            u[k] = rho if k == 0 else drho[k - 1]
        for a in range(3):
            u[4 * (1 + a)] = rho * v[a]
            for k in range(3):
                u[4 * (1 + a) + 1 + k] = drho[k] * v[a]
        u[16] = p / (5 / 3 - 1) + 0.5 * rho * sum(x * x for x in v)
        for k in range(3):
            u[17 + k] = 0.5 * drho[k] * sum(x * x for x in v)
    L, f0 = P.rhs(u)
    assert f0 == 0
    dt = 1e-7
    out, f1 = P.mh_step(u, dt, face_points=2)
    assert f1 == 0
    np.testing.assert_allclose((out - u) / dt, L, atol=1e-5 * np.abs(L).max())


def test_mh_face_rules_on_one_dimensional_data():
    """y-invariant data (limiter off).  The two Gauss points of an x face see the
    same state, so both face rules give the same averages and x derivatives; with
    the Gauss face rule the y faces' moments and the volume integral of F_y use
    the same x nodes and the y derivatives stay zero.  With the face-centroid rule
    (weight A_f at c_f, eq. `GalerkUpdate`) against the Gauss volume rule they
    cancel only up to the quadrature difference of F_y along x: the increment of
    every y derivative is, in closed form,
        dt * 12/dy^2 * (mean of F_y at x = -+dx/(2 sqrt 3) - F_y at x = 0)
    with F_y the physical flux of the predicted primitive state W_c + dt/2 dW/dt
    + dW/dx x (the y faces carry Riemann problems between equal states)."""
    A = 0.05
    g = 5.0 / 3.0
    f = lambda X, Y: (1 + A * np.sin(2 * np.pi * X), 0.3 + A * np.sin(2 * np.pi * X), 0.2,
                      0.6 + A * np.cos(2 * np.pi * X))
    N = 32
    for eq in (O.EULER, O.MHD):
        fe = f if eq == O.EULER else (lambda X, Y: f(X, Y) + (0.4, 0.7 + 0.1 * np.sin(2 * np.pi * X)))
        u = ics.project_2d(fe, (N, 3), box=(1.0, 3.0 / N), eq=eq)
        P = O.Problem(eq, 2, (N, 3), box=(1.0, 3.0 / N), limiter=0)
        dx, dy = P.h[0], P.h[1]
        dt = 0.3 / N
        a, _ = P.mh_step(u, dt, face_points=1)
        b, _ = P.mh_step(u, dt, face_points=2)
        tvar = [0, 1, 2, 4]
        yplanes = [3 * v + 2 for v in range(4)] + ([14] if eq == O.MHD else [])
        xplanes = [k for k in range(P.nplanes) if k not in yplanes]
        inc = np.abs(b[xplanes] - u[xplanes]).max()
        np.testing.assert_allclose(a[xplanes] - u[xplanes], b[xplanes] - u[xplanes],
                                   atol=1e-10 * inc)
        assert np.abs(b[yplanes]).max() < 1e-10 * inc
        # closed form of the face-centroid rule's y increments, cell by cell
        t = dx / (2 * math.sqrt(3.0))
        exp = np.zeros((len(yplanes), N))
        for i in range(N):
            U = np.zeros(8)
            dU = np.zeros(8)
            for v, q in enumerate(tvar):
                U[q], dU[q] = u[3 * v, 0, i], u[3 * v + 1, 0, i]
            if eq == O.MHD:
                U[5], U[6] = u[12, 0, i], u[13, 0, i]
                dU[5], dU[6] = u[16, 0, i], u[15, 0, i]  # dBx/dx = a3, dBy/dx = a2
            W = _c2p(U, g)
            dW = np.zeros((8, 3))
            dW[0, 0] = dU[0]
            dW[1:4, 0] = (dU[1:4] - W[1:4] * dU[0]) / W[0]
            dW[5:8, 0] = dU[5:8]
            dW[4, 0] = (g - 1) * (dU[4] - 0.5 * (W[1:4] @ W[1:4]) * dU[0]
                                  - W[0] * (W[1:4] @ dW[1:4, 0]) - W[5:8] @ dU[5:8])
            Wp = W + 0.5 * dt * O.prim_rates(W, dW, 2, g)
            Fy = [O.phys_flux(_p2c(Wp + dW[:, 0] * x, g), 1, g) for x in (-t, 0.0, t)]
            rate = 12.0 / dy ** 2 * (0.5 * (Fy[0] + Fy[2]) - Fy[1])
            qs = tvar + ([5] if eq == O.MHD else [])
            exp[:, i] = dt * rate[qs]
        got = a[yplanes][:, 0, :]
        assert np.abs(exp).max() > 1e-4 * inc
        np.testing.assert_allclose(got, exp, atol=1e-9 * np.abs(exp).max())
        np.testing.assert_allclose(a[yplanes][:, 1:, :], np.broadcast_to(got[:, None, :],
                                   (len(yplanes), 2, N)), atol=1e-15)


def _order(errs):
    return [math.log(errs[i] / errs[i + 1], 2) for i in range(len(errs) - 1)]


@pytest.mark.parametrize("fp", [1, 2])
def test_mh_convergence_advected_density_wave_2d(fp):
    """Density wave translated by v = (1, 1): second order in L1 (limiter off)."""
    errs = []
    T = 0.125
    for N in (16, 32, 64):
        u0 = ics.euler2d_wave((N, N), noise=0.0)
        P = O.Problem(O.EULER, 2, (N, N), limiter=0)
        dt0, _ = P.cfl_dt(u0, 0.3)
        ns = int(math.ceil(T / dt0))
        out, _, f = P.mh_run(u0, ns, dt=T / ns, face_points=fp)
        assert f == 0
        ex = ics.project_2d(lambda X, Y: (1 + 0.2 * np.sin(2 * np.pi * (X + Y - 2 * T)), 1.0, 1.0,
                                          1.0), (N, N))
        errs.append(np.abs(out[0] - ex[0]).mean())
    assert _order(errs)[-1] > 1.85, errs


def test_mh_convergence_acoustic_wave():
    """Sec. 3.1 acoustic wave (drho/rho = 1e-6, sound speed 1), one period: second
    order in L1 (limiter off); exercises the velocity-pressure coupling of the
    prediction."""
    errs = []
    for N in (16, 32, 64):
        A = 1e-6

        def f(X, Y):
            s = A * np.sin(2 * np.pi * X)
            return 1 + s, s, 0.0, 0.6 + s

        u0 = ics.project_2d(f, (N, 1), box=(1.0, 1.0 / N))
        P = O.Problem(O.EULER, 2, (N, 1), box=(1.0, 1.0 / N), limiter=0)
        dt0, _ = P.cfl_dt(u0, 0.3)
        ns = int(math.ceil(1.0 / dt0))
        out, _, fl = P.mh_run(u0, ns, dt=1.0 / ns)
        assert fl == 0
        errs.append(np.abs(out[0] - u0[0]).mean())
    assert _order(errs)[-1] > 1.85, errs


def test_mh_convergence_mhd_alfven_wave():
    """Linear Alfven wave along (1, 1) with the field parallel to k; the field
    evolves through the divergence-free basis and the prediction of B: second
    order (limiter off, face-centroid rule)."""
    eps, T = 1e-3, 0.08
    s2 = math.sqrt(2.0)

    def field(X, Y, t):
        s = eps * np.sin(2 * np.pi * (X + Y - s2 * t))
        return 1.0, s / s2, -s / s2, 1.0, 1 / s2 - s / s2, 1 / s2 + s / s2

    errs = []
    for N in (16, 32, 64):
        u0 = ics.project_2d(lambda X, Y: field(X, Y, 0.0), (N, N), eq=O.MHD)
        P = O.Problem(O.MHD, 2, (N, N), limiter=0)
        dt0, _ = P.cfl_dt(u0, 0.3)
        ns = int(math.ceil(T / dt0))
        out, _, fl = P.mh_run(u0, ns, dt=T / ns)
        assert fl == 0
        ex = ics.project_2d(lambda X, Y: field(X, Y, T), (N, N), eq=O.MHD)
        errs.append(np.abs(out[13] - ex[13]).mean() + np.abs(out[12] - ex[12]).mean())
    assert _order(errs)[-1] > 1.8, errs


def test_mh_sod_first_order_convergence():
    """Sec. 3.2 Sod variant, gamma = 1.4, t = 5, limiter on: first order in L1."""
    g, T, L = 1.4, 5.0, 20.0
    errs = []
    for N in (64, 128, 256):
        nx = 2 * N

        def f(X, Y):
            left = X - L < 0
            return np.where(left, 1.0, 0.25), 0.0, 0.0, np.where(left, 1.0, 0.1795)

        u = ics.project_2d(f, (nx, 1), box=(2 * L, L / N), gamma=g)
        P = O.Problem(O.EULER, 2, (nx, 1), box=(2 * L, L / N), gamma=g, limiter=1)
        t = 0.0
        while t < T - 1e-12:
            dt, _ = P.cfl_dt(u, 0.3)
            dt = min(dt, T - t)
            u, fl = P.mh_step(u, dt)
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
    overall = math.log(errs[0] / errs[-1], 2) / (len(errs) - 1)
    assert errs[0] > errs[1] > errs[2] and 0.7 < overall < 1.3, (errs, overall)
