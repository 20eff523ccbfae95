"""Adjoint (vector-Jacobian products) of the 2D Euler and planar MHD DG steps on
the GPU.

Checked against the oracle's FP64 tangent model (dot-product identity
<J^T lam, d> = <lam, J d>), against the full Jacobian built column by column
from the oracle on a tiny grid, and against central finite differences of the
GPU forward map over a checkpointed multi-step rollout with the time steps held
fixed.
"""
import math

import numpy as np
import pytest

import oracle as O
from paper_1305_5536_gb300 import dg, ics

pytestmark = pytest.mark.gpu


def _state(n, seed=3):
    f = lambda X, Y: (1 + 0.2 * np.sin(2 * np.pi * (X + Y) + 0.31),
                      0.5 + 0.2 * np.sin(2 * np.pi * X + 0.47),
                      -0.3 + 0.2 * np.cos(2 * np.pi * Y + 0.23),
                      1 + 0.1 * np.sin(2 * np.pi * (X - 2 * Y) + 0.11))
    return ics.add_slope_noise(ics.project_2d(f, n), 0, 2, 0.05, np.random.default_rng(seed))


def _vjp(n, u, lam, dt, prec, limiter, box=(1.0, 0.9)):
    import torch
    s = dg.DGSolver("euler", 2, n, box=box + (1.0,), precision=prec, limiter=limiter)
    ud = torch.from_numpy(u).cuda()
    ld = torch.from_numpy(lam).cuda()
    out = s.adjoint_step(ld, ud, dt)
    torch.cuda.synchronize()
    s.close()
    return out.cpu().numpy()


@pytest.mark.parametrize("prec,tol", [("fp64", 1e-12), ("fp32", 1e-4)])
@pytest.mark.parametrize("n", [(12, 10), (37, 29), (5, 3)])
@pytest.mark.parametrize("limiter", [0, 1])
def test_adjoint_step_dot_product(prec, tol, n, limiter):
    u = _state(n)
    P = O.Problem(O.EULER, 2, n, box=(1.0, 0.9), limiter=limiter)
    dt = 0.5 * P.cfl_dt(u)[0]
    rng = np.random.default_rng(7)
    lam = rng.standard_normal(u.shape)
    d = rng.standard_normal(u.shape)
    _, Jd, fl = P.tangent_step(u, d, dt)
    assert fl == 0
    JTl = _vjp(n, u, lam, dt, prec, limiter)
    a, b = float((JTl * d).sum()), float((lam * Jd).sum())
    scale = float(np.abs(JTl * d).sum())
    if prec == "fp32" and limiter:
        # The limiter's derivative jumps where its min/max or min(1, psi) switches
        # branch; FP32 rounding of nearly tied neighbour values flips the branch in
        # a few cells, so only rough agreement is expected (FP64 is exact above).
        tol = 0.1
    assert abs(a - b) < tol * scale, (a, b)


@pytest.mark.parametrize("limiter", [0, 1])
def test_adjoint_step_full_jacobian_tiny(limiter):
    n = (4, 4)
    u = _state(n)
    P = O.Problem(O.EULER, 2, n, box=(1.0, 0.9), limiter=limiter)
    dt = 0.5 * P.cfl_dt(u)[0]
    N = u.size
    J = np.zeros((N, N))
    for k in range(N):
        e = np.zeros(N)
        e[k] = 1.0
        _, col, _ = P.tangent_step(u, e.reshape(u.shape), dt)
        J[:, k] = col.ravel()
    rng = np.random.default_rng(8)
    for _ in range(3):
        lam = rng.standard_normal(u.shape)
        ref = (J.T @ lam.ravel()).reshape(u.shape)
        got = _vjp(n, u, lam, dt, "fp64", limiter)
        np.testing.assert_allclose(got, ref, atol=1e-12 * np.abs(ref).max())


def _objective_grad(uT, target, h):
    """J = 1/2 int (rho_h - rho_target)^2 over the box, exact on P1 polynomials:
    V sum [(d avg)^2 + dx^2/12 (d rho_x)^2 + dy^2/12 (d rho_y)^2]; returns (J, dJ/du_T)."""
    V = h[0] * h[1]
    w = np.array([1.0, h[0] ** 2 / 12, h[1] ** 2 / 12])
    d = uT[0:3] - target[0:3]
    J = 0.5 * V * float((w[:, None, None] * d * d).sum())
    g = np.zeros_like(uT)
    g[0:3] = V * w[:, None, None] * d
    return J, g


def _forward_fixed(n, u0, dts, prec, limiter):
    s = dg.DGSolver("euler", 2, n, precision=prec, limiter=limiter)
    s.set_state(u0)
    for dt in dts:
        s.step(1, dt=dt)
    s.sync()
    out = s.get_state()
    s.close()
    return out


def test_adjoint_rollout_vs_central_differences_and_oracle():
    """Smooth random density perturbation (the adjoint workload, reduced to 48x48
    and 12 steps), limiter off as in that workload (its uniform velocity and
    pressure would put every cell on a tie of the limiter's min/max), objective =
    L2 misfit of the final density against a target, checkpoints every 5 steps."""
    limiter = 0
    import torch
    n = (48, 48)
    u0, delta = ics.euler2d_random_density(n, kmax=6)
    h = (1.0 / n[0], 1.0 / n[1])
    nsteps = 12
    s = dg.DGSolver("euler", 2, n, precision="fp64", limiter=limiter, ckpt_every=5)
    s.set_state(u0)
    s.record(nsteps)
    uT = s.get_state()
    target = ics.euler2d_random_density(n, kmax=6, seed=99)[0]
    J0, gT = _objective_grad(uT, target, h)
    g0 = s.adjoint(torch.from_numpy(gT).cuda()).cpu().numpy()
    # the recorded time steps (held fixed), from the oracle's Courant rule
    P = O.Problem(O.EULER, 2, n, limiter=limiter)
    _, dts, _ = P.run(u0, nsteps, cfl=0.3)
    np.testing.assert_allclose(_forward_fixed(n, u0, dts, "fp64", limiter), uT, rtol=0,
                               atol=1e-12 * np.abs(uT).max())
    rng = np.random.default_rng(21)
    d = rng.standard_normal(u0.shape) * 1e-2
    d[1:3] *= 10.0
    gd = float((g0 * d).sum())
    # central differences of the GPU forward map with the same time steps
    eps = 1e-5
    Jp, _ = _objective_grad(_forward_fixed(n, u0 + eps * d, dts, "fp64", limiter), target, h)
    Jm, _ = _objective_grad(_forward_fixed(n, u0 - eps * d, dts, "fp64", limiter), target, h)
    fd = (Jp - Jm) / (2 * eps)
    assert abs(gd - fd) < 1e-6 * abs(fd), (gd, fd)
    # the oracle's own FP64 tangent through the same steps
    u, du = u0.copy(), d.copy()
    for dt in dts:
        u, du, fl = P.tangent_step(u, du, dt)
        assert fl == 0
    ref = float((gT * du).sum())
    assert abs(gd - ref) < 1e-10 * abs(ref), (gd, ref)
    s.close()


def test_adjoint_workload_full_size_vs_central_differences():
    """The adjoint workload at its own size: 2D Euler 256^2, the seeded Gaussian
    random density, 100 SSP-RK2 Courant steps at CFL 0.3 recorded with checkpoints
    every 10, limiter off, FP64.  The checkpointed adjoint's directional derivative
    <dJ/du_0, d> against central differences of the forward map with the recorded
    time steps held fixed, 1e-6 relative (the forward map itself is held to the
    oracle by the forward parity tests)."""
    import torch
    n, nsteps = (256, 256), 100
    u0, _ = ics.euler2d_random_density(n)
    target = ics.euler2d_random_density(n, seed=99)[0]
    h = (1.0 / n[0], 1.0 / n[1])
    # the Courant steps of the recording: the same state and rule, one at a time
    c = dg.DGSolver("euler", 2, n, precision="fp64", limiter=0, cfl=0.3)
    c.set_state(u0)
    dts = []
    for _ in range(nsteps):
        dts.append(float(c.times()[1][0]))
        c.step(1)
    c.sync()
    c.close()
    s = dg.DGSolver("euler", 2, n, precision="fp64", limiter=0, cfl=0.3, ckpt_every=10)
    s.set_state(u0)
    s.record(nsteps)
    uT = s.get_state()
    np.testing.assert_allclose(_forward_fixed(n, u0, dts, "fp64", 0), uT, rtol=0,
                               atol=1e-13 * np.abs(uT).max())
    J0, gT = _objective_grad(uT, target, h)
    g0 = s.adjoint(torch.from_numpy(gT).cuda()).cpu().numpy()
    s.close()
    rng = np.random.default_rng(23)
    d = rng.standard_normal(u0.shape) * 1e-2
    d[1:3] *= 10.0
    gd = float((g0 * d).sum())
    eps = 1e-5
    Jp, _ = _objective_grad(_forward_fixed(n, u0 + eps * d, dts, "fp64", 0), target, h)
    Jm, _ = _objective_grad(_forward_fixed(n, u0 - eps * d, dts, "fp64", 0), target, h)
    fd = (Jp - Jm) / (2 * eps)
    assert abs(gd - fd) < 1e-6 * abs(fd), (gd, fd)


def test_autograd_rollout_fp32_gradient():
    import torch
    n = (32, 32)
    u0, _ = ics.euler2d_random_density(n, kmax=4)
    s = dg.DGSolver("euler", 2, n, precision="fp32", limiter=0, ckpt_every=3)
    x = torch.from_numpy(u0).cuda().requires_grad_(True)
    uT = dg.rollout(x, s, 7)
    loss = (uT[0] ** 2).sum()
    loss.backward()
    g = x.grad.double().cpu().numpy()
    # central differences of the FP64 forward with the recorded time steps
    P = O.Problem(O.EULER, 2, n, limiter=0)
    _, dts, _ = P.run(u0, 7, cfl=0.3)
    rng = np.random.default_rng(5)
    d = rng.standard_normal(u0.shape) * 1e-2
    eps = 1e-4
    f = lambda u: float((_forward_fixed(n, u, dts, "fp64", 0)[0] ** 2).sum())
    fd = (f(u0 + eps * d) - f(u0 - eps * d)) / (2 * eps)
    assert abs(float((g * d).sum()) - fd) < 2e-4 * abs(fd)


def test_step_between_recordings_ends_the_first_one():
    """dg_step between two dg_record calls ends the first recording: dg_adjoint has
    nothing to run back over until the next dg_record, which starts a new recording
    from the state the steps reached -- its gradient is that of a fresh recording
    from that state."""
    import torch
    n = (24, 24)
    u0, _ = ics.euler2d_random_density(n, kmax=4)
    lam = torch.from_numpy(np.random.default_rng(12).standard_normal(u0.shape)).cuda()
    s = dg.DGSolver("euler", 2, n, precision="fp64", limiter=0, ckpt_every=2)
    s.set_state(u0)
    g0 = s.record_generation()
    s.record(3)
    g1 = s.record_generation()
    assert g1 != g0
    s.step(2, sync=True)
    assert s.record_generation() != g1
    with pytest.raises(dg.DGError) as ei:
        s.adjoint(lam)
    assert ei.value.status == dg.DG_ESTATE
    u_mid = s.get_state()
    s.record(4)
    got = s.adjoint(lam).cpu().numpy()
    s.close()
    fresh = dg.DGSolver("euler", 2, n, precision="fp64", limiter=0, ckpt_every=2)
    fresh.set_state(u_mid)
    fresh.record(4)
    ref = fresh.adjoint(lam).cpu().numpy()
    fresh.close()
    np.testing.assert_allclose(got, ref, rtol=0, atol=1e-12 * np.abs(ref).max())


def test_second_rollout_on_one_solver_refuses_the_first_backward():
    """A solver keeps one recording: after a second rollout on it, the first
    rollout's backward pass raises instead of returning the second trajectory's
    gradient; the second backward works."""
    import torch
    n = (16, 16)
    ua, _ = ics.euler2d_random_density(n, kmax=4)
    ub, _ = ics.euler2d_random_density(n, kmax=4, seed=77)
    s = dg.DGSolver("euler", 2, n, precision="fp64", limiter=0, ckpt_every=3)
    xa = torch.from_numpy(ua).cuda().requires_grad_(True)
    xb = torch.from_numpy(ub).cuda().requires_grad_(True)
    ya = dg.rollout(xa, s, 4)
    yb = dg.rollout(xb, s, 4)
    with pytest.raises(RuntimeError, match="recorded trajectory changed"):
        (ya[0] ** 2).sum().backward()
    (yb[0] ** 2).sum().backward()
    assert xb.grad is not None and torch.isfinite(xb.grad).all()
    s.close()


@pytest.mark.parametrize("n", [(37, 29), (64, 48)])
def test_fp32_limited_adjoint_agrees_with_fp64_away_from_branch_flips(n, capsys):
    """FP32 with the limiter on: where the FP32 and FP64 limiters take the same
    branch, the two adjoints agree to FP32 rounding; the limiter's derivative jumps
    where min/max switches, and FP32 rounding of nearly tied neighbour values flips
    the branch in a few cells.  Bound both: at least 95 % of the cells within 1e-4
    of the FP64 adjoint's scale, and the dot-product identity within 10 %."""
    u = _state(n)
    P = O.Problem(O.EULER, 2, n, box=(1.0, 0.9), limiter=1)
    dt = 0.5 * P.cfl_dt(u)[0]
    lam = np.random.default_rng(21).standard_normal(u.shape)
    a64 = _vjp(n, u, lam, dt, "fp64", 1)
    a32 = _vjp(n, u, lam, dt, "fp32", 1)
    scale = np.abs(a64).max()
    cell_err = np.abs(a32 - a64).max(axis=0) / scale
    frac_ok = float((cell_err < 1e-4).mean())
    with capsys.disabled():
        print("\n%s: FP32 vs FP64 limited adjoint, cells within 1e-4: %.4f, median %.2e, "
              "max %.2e" % (n, frac_ok, float(np.median(cell_err)), float(cell_err.max())))
    assert frac_ok >= 0.95, frac_ok
    assert float(np.median(cell_err)) < 1e-5


# ---------------------------------------------------------------------------
# Planar MHD: the face and volume flux Jacobians (HLLD and the physical flux,
# with the divergence-free field basis) in the transposed right-hand side, and
# the transposed min/max limiter with its shared field factor.
# ---------------------------------------------------------------------------
def _mhd_state(n):
    """Orszag-Tang with 1 % noise on the averages and on the Taylor slopes: the
    vortex alone has a uniform density and pressure, so the limiter's min/max
    would sit on exact ties, where its derivative is a choice (an implementation
    may take either neighbour)."""
    rng = np.random.default_rng(5)
    u = ics.orszag_tang(n)
    for v in range(4):
        u[3 * v] *= 1.0 + 0.01 * rng.standard_normal(u.shape[1:])
    return ics.add_slope_noise(u, 0, 2, 0.02, rng)


def _vjp_mhd(n, u, lam, dt, prec, limiter=0, box=(1.0, 0.9)):
    import torch
    s = dg.DGSolver("mhd", 2, n, box=box + (1.0,), precision=prec, limiter=limiter)
    out = s.adjoint_step(torch.from_numpy(lam).cuda(), torch.from_numpy(u).cuda(), dt)
    torch.cuda.synchronize()
    s.close()
    return out.cpu().numpy()


@pytest.mark.parametrize("prec,tol", [("fp64", 1e-12), ("fp32", 1e-4)])
@pytest.mark.parametrize("n", [(12, 10), (37, 29), (5, 3)])
@pytest.mark.parametrize("limiter", [0, 1])
def test_mhd_adjoint_step_dot_product(prec, tol, n, limiter):
    """<J^T lam, d> from the GPU against <lam, J d> from the oracle's FP64 tangent
    of the planar MHD step, every plane of lam and d random."""
    u = _mhd_state(n)
    P = O.Problem(O.MHD, 2, n, box=(1.0, 0.9), limiter=limiter)
    dt = 0.5 * P.cfl_dt(u)[0]
    rng = np.random.default_rng(11)
    lam = rng.standard_normal(u.shape)
    d = rng.standard_normal(u.shape)
    _, Jd, fl = P.tangent_step(u, d, dt)
    assert fl == 0
    JTl = _vjp_mhd(n, u, lam, dt, prec, limiter)
    a, b = float((JTl * d).sum()), float((lam * Jd).sum())
    scale = float(np.abs(JTl * d).sum())
    if prec == "fp32" and limiter:
        tol = 0.1  # branch flips of the limiter under FP32 rounding, as for Euler
    assert abs(a - b) < tol * scale, (a, b)


@pytest.mark.parametrize("limiter", [0, 1])
def test_mhd_adjoint_full_jacobian_tiny(limiter):
    """Every column of the planar MHD step's Jacobian on a 4 x 3 grid: J^T e_i
    from the GPU against the oracle's tangent J e_j, entry by entry."""
    n = (4, 3)
    u = _mhd_state(n)
    P = O.Problem(O.MHD, 2, n, box=(1.0, 0.9), limiter=limiter)
    dt = 0.5 * P.cfl_dt(u)[0]
    m = u.size
    J = np.zeros((m, m))
    for j in range(m):
        e = np.zeros(m)
        e[j] = 1.0
        _, col, fl = P.tangent_step(u, e.reshape(u.shape), dt)
        assert fl == 0
        J[:, j] = col.ravel()
    rng = np.random.default_rng(13)
    for _ in range(3):
        lam = rng.standard_normal(u.shape)
        JTl = _vjp_mhd(n, u, lam, dt, "fp64", limiter)
        np.testing.assert_allclose(JTl.ravel(), J.T @ lam.ravel(), rtol=0,
                                   atol=1e-12 * np.abs(J.T @ lam.ravel()).max())


def _forward_fixed_eq(eq, n, u0, dts, prec, limiter):
    s = dg.DGSolver(eq, 2, n, precision=prec, limiter=limiter)
    s.set_state(u0)
    for dt in dts:
        s.step(1, dt=dt)
    s.sync()
    out = s.get_state()
    s.close()
    return out


def test_mhd_adjoint_rollout_vs_central_differences():
    """A checkpointed planar MHD rollout (24 x 20, 8 Courant steps, checkpoints
    every 3, limiter off), FP64: the adjoint's directional derivative of the
    density misfit against central differences of the forward map with the
    recorded time steps, 1e-6."""
    import torch
    n, nsteps = (24, 20), 8
    u0 = _mhd_state(n)
    h = (1.0 / n[0], 1.0 / n[1])
    c = dg.DGSolver("mhd", 2, n, precision="fp64", limiter=0)
    c.set_state(u0)
    dts = []
    for _ in range(nsteps):
        dts.append(float(c.times()[1][0]))
        c.step(1)
    c.sync()
    c.close()
    s = dg.DGSolver("mhd", 2, n, precision="fp64", limiter=0, ckpt_every=3)
    s.set_state(u0)
    s.record(nsteps)
    uT = s.get_state()
    np.testing.assert_allclose(_forward_fixed_eq("mhd", n, u0, dts, "fp64", 0), uT, rtol=0,
                               atol=1e-13 * np.abs(uT).max())
    target = ics.orszag_tang(n)
    target[0] *= 1.1
    J0, gT = _objective_grad(uT, target, h)
    g0 = s.adjoint(torch.from_numpy(gT).cuda()).cpu().numpy()
    s.close()
    rng = np.random.default_rng(29)
    d = rng.standard_normal(u0.shape) * 1e-2
    eps = 1e-5
    Jp, _ = _objective_grad(_forward_fixed_eq("mhd", n, u0 + eps * d, dts, "fp64", 0), target, h)
    Jm, _ = _objective_grad(_forward_fixed_eq("mhd", n, u0 - eps * d, dts, "fp64", 0), target, h)
    fd = (Jp - Jm) / (2 * eps)
    gd = float((g0 * d).sum())
    assert abs(gd - fd) < 1e-6 * abs(fd), (gd, fd)


def test_mhd_adjoint_with_the_weno_limiter_is_refused():
    import torch
    n = (8, 8)
    s = dg.DGSolver("mhd", 2, n, precision="fp64", limiter=2)
    u = torch.from_numpy(_mhd_state(n)).cuda()
    with pytest.raises(dg.DGError) as err:
        s.adjoint_step(u.clone(), u, 1e-3)
    assert err.value.status == dg.DG_EINVAL
    s.close()


def _mhd_state_generic(n):
    """_mhd_state with noise on the field averages and coefficients as well.  In
    the Orszag-Tang field a cell at an extremum of By along x has a zero By
    gradient, so its limiter factor for By is 0/0 (taken as 1), and the factor
    shared by the whole field (Sec. 2.5) then jumps with the direction of any
    perturbation: the limited step is discontinuous there (in the oracle as on the
    GPU), and central differences across it measure the jump, not a derivative."""
    rng = np.random.default_rng(17)
    u = _mhd_state(n)
    u[12:14] += 0.01 * rng.standard_normal(u[12:14].shape)
    u[14:17] += 0.05 * rng.standard_normal(u[14:17].shape)
    return u


def test_autograd_rollout_mhd_fp64_gradient():
    """torch.autograd through a checkpointed planar MHD rollout (limiter on, FP64):
    the gradient of the sum of squared final averages against central differences
    of the forward map with the recorded time steps held fixed."""
    import torch
    n, nsteps = (20, 16), 6
    u0 = _mhd_state_generic(n)
    c = dg.DGSolver("mhd", 2, n, precision="fp64", limiter=1)
    c.set_state(u0)
    dts = []
    for _ in range(nsteps):
        dts.append(float(c.times()[1][0]))
        c.step(1)
    c.sync()
    c.close()
    s = dg.DGSolver("mhd", 2, n, precision="fp64", limiter=1, ckpt_every=4)
    x = torch.from_numpy(u0).cuda().requires_grad_(True)
    uT = dg.rollout(x, s, nsteps)
    planes = [0, 3, 6, 9, 12, 13]
    loss = (uT[planes] ** 2).sum()
    loss.backward()
    g = x.grad.cpu().numpy()
    s.close()
    rng = np.random.default_rng(31)
    d = rng.standard_normal(u0.shape) * 1e-2
    eps = 1e-6
    f = lambda u: float((_forward_fixed_eq("mhd", n, u, dts, "fp64", 1)[planes] ** 2).sum())
    fd = (f(u0 + eps * d) - f(u0 - eps * d)) / (2 * eps)
    assert abs(float((g * d).sum()) - fd) < 1e-6 * abs(fd), (float((g * d).sum()), fd)
