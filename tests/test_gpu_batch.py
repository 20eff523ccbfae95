"""Batched problems: one persistent cooperative launch per step over the tiles of
many independent 2D MHD problems of different sizes, each with its own time step."""
import os

import numpy as np
import pytest

import oracle as O
from paper_1305_5536_gb300 import dg, ics

from helpers import poly_rel_err

pytestmark = pytest.mark.gpu

SIZES = [32, 48, 17, 40, 64, 23]


def _batch_states(sizes, seed=11):
    rng = np.random.default_rng(seed)
    return [ics.mhd_random_smooth(N, rng=rng) for N in sizes]


def _solver(sizes, prec):
    cfgs = [dg.make_config("mhd", 2, (N, N), precision=prec) for N in sizes]
    return dg.DGSolver(configs=cfgs)


def _split(flat, sizes):
    out, o = [], 0
    for N in sizes:
        k = 17 * N * N
        out.append(flat[o:o + k].reshape(17, N, N))
        o += k
    return out


@pytest.mark.parametrize("prec,tol", [("fp64", 1e-12), ("fp32", 1e-5)])
def test_batch_fixed_dt_matches_oracle_per_problem(prec, tol):
    us = _batch_states(SIZES)
    s = _solver(SIZES, prec)
    s.set_state(np.concatenate([u.ravel() for u in us]))
    dt = 2e-4
    s.step(1, dt=dt, sync=True)
    got = _split(s.get_state(), SIZES)
    for N, u, g in zip(SIZES, us, got):
        P = O.Problem(O.MHD, 2, (N, N))
        ref, fl = P.step(u, dt)
        assert fl == 0
        err, where = poly_rel_err(g, ref, 1, 2, P.h)
        assert err < tol, (N, err, where)


def test_batch_courant_steps_per_problem_fp64():
    us = _batch_states(SIZES)
    s = _solver(SIZES, "fp64")
    s.set_state(np.concatenate([u.ravel() for u in us]))
    s.step(5, sync=True)
    t, dtn = s.times()
    got = _split(s.get_state(), SIZES)
    for k, (N, u, g) in enumerate(zip(SIZES, us, got)):
        P = O.Problem(O.MHD, 2, (N, N))
        ref, dts, fl = P.run(u, 5, cfl=0.3)
        assert fl == 0
        assert abs(t[k] - dts.sum()) < 1e-13 * dts.sum()
        err, where = poly_rel_err(g, ref, 1, 2, P.h)
        assert err < 1e-11, (N, err, where)


def test_batch_equals_single_problem_solvers():
    us = _batch_states(SIZES)
    s = _solver(SIZES, "fp32")
    s.set_state(np.concatenate([u.ravel() for u in us]))
    s.step(4, sync=True)
    got = _split(s.get_state(), SIZES)
    for N, u, g in zip(SIZES, us, got):
        one = dg.DGSolver("mhd", 2, (N, N), precision="fp32")
        one.set_state(u)
        one.step(4, sync=True)
        ref = one.get_state()
        one.close()
        # both kernels run the same tile code (the batched one walks a work list
        # and meets at a grid barrier between the stages), so after 4 steps they
        # may differ by rounding at most
        err, where = poly_rel_err(g, ref, 1, 2, (1.0 / N, 1.0 / N))
        assert err < 1e-6, (N, err, where)


def test_batch_barrier_timeout_is_reported_and_context_stays_usable(monkeypatch):
    """The grid barrier's wait is bounded.  With the test hook the barrier expects
    one CTA more than is launched, so every wait runs out (no hang, no fault) and
    the step reports DG_ETIMEOUT; the context and the GPU stay usable."""
    us = _batch_states(SIZES[:3])
    monkeypatch.setenv("DG_TEST_BARRIER_TIMEOUT", "1")
    s = _solver(SIZES[:3], "fp32")
    monkeypatch.delenv("DG_TEST_BARRIER_TIMEOUT")
    s.set_state(np.concatenate([u.ravel() for u in us]))
    with pytest.raises(dg.DGError) as ei:
        s.step(1, dt=1e-4, sync=True)
    assert ei.value.status == dg.DG_ETIMEOUT
    s.sync()  # error cleared, context usable
    s.close()
    ok = _solver(SIZES[:3], "fp32")
    ok.set_state(np.concatenate([u.ravel() for u in us]))
    ok.step(2, sync=True)
    ok.close()


@pytest.mark.parametrize("prec,tol", [("fp64", 1e-12), ("fp32", 1e-5)])
def test_batch_many_tiles_per_cta_matches_oracle(prec, tol, monkeypatch):
    """The persistent batched kernel with its cooperative grid capped at 5 CTAs
    (test hook DG_TEST_MAX_CTAS): every CTA walks 9-40 tiles across problem
    boundaries, reusing its shared memory and switching problems mid-sweep, in
    both stages and across the grid barrier; one fixed-dt step and a Courant chain
    of 3 steps per problem against the oracle."""
    monkeypatch.setenv("DG_TEST_MAX_CTAS", "5")
    us = _batch_states(SIZES)
    s = _solver(SIZES, prec)
    s.set_state(np.concatenate([u.ravel() for u in us]))
    dt = 2e-4
    s.step(1, dt=dt, sync=True)
    got = _split(s.get_state(), SIZES)
    for N, u, g in zip(SIZES, us, got):
        P = O.Problem(O.MHD, 2, (N, N))
        ref, fl = P.step(u, dt)
        assert fl == 0
        err, where = poly_rel_err(g, ref, 1, 2, P.h)
        assert err < tol, (N, err, where)
    s.set_state(np.concatenate([u.ravel() for u in us]))
    s.step(3, sync=True)
    t, _ = s.times()
    got = _split(s.get_state(), SIZES)
    for k, (N, u, g) in enumerate(zip(SIZES, us, got)):
        P = O.Problem(O.MHD, 2, (N, N))
        ref, dts, fl = P.run(u, 3, cfl=0.3)
        assert fl == 0
        assert abs(t[k] - dts.sum()) < (1e-13 if prec == "fp64" else 1e-5) * dts.sum()
        err, where = poly_rel_err(g, ref, 1, 2, P.h)
        assert err < 3 * tol, (N, err, where)
    s.close()


def test_batch_workload_of_64_problems_one_step():
    """The batched workload itself (64 problems, N log-uniform in [32, 512], 3.39 M
    cells, about 13.5 k tiles: every CTA of the cooperative grid walks many tiles),
    FP32, one step with each problem's own Courant time step; a dozen problems are
    compared whole with the oracle, and every problem's time step with the
    oracle's Courant rule."""
    sizes, us = ics.mhd_batch()
    s = _solver(sizes, "fp32")
    s.set_state(np.concatenate([u.ravel() for u in us]))
    _, dt0 = s.times()
    s.step(1, sync=True)
    t, _ = s.times()
    np.testing.assert_allclose(t, dt0, rtol=1e-15)
    flat = s.get_state()
    s.close()
    offs = np.cumsum([0] + [17 * N * N for N in sizes])
    order = np.argsort(sizes)
    pick = list(order[:6]) + list(order[len(order) // 2:len(order) // 2 + 4]) + list(order[-2:])
    for k in range(len(sizes)):
        N = sizes[k]
        P = O.Problem(O.MHD, 2, (N, N))
        dref = P.cfl_dt(us[k])[0]
        assert abs(dt0[k] - dref) < 1e-6 * dref, (k, N, dt0[k], dref)
        if k not in pick:
            continue
        ref, fl = P.step(us[k], dt0[k])
        assert fl == 0
        g = flat[offs[k]:offs[k + 1]].reshape(17, N, N)
        err, where = poly_rel_err(g, ref, 1, 2, P.h)
        assert err < 1e-5, (k, N, err, where)
