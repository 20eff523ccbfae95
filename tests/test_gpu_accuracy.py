"""Accuracy of the GPU paths over long runs, against the FP64 oracle.

The FP32 path's final-time L1 error and conservation drift, stated against the
FP64 oracle.  Over many steps of a flow with shocks, the min/max
limiter (a discontinuous function of its inputs, Sec. 2.5) amplifies any
difference of rounding: two correct FP64 implementations drift apart.  The tests
therefore also run the oracle on the initial state perturbed by 1e-14 relative
noise, and hold the FP64 GPU path to that self-sensitivity of the problem.

Runs (the oracle's own Courant steps, passed to the GPU as fixed steps, so that
only the arithmetic differs):
  * the smooth density-wave workload, 2D Euler 64^2, limiter on, 50 steps;
  * Orszag-Tang 128^2 with SSP-RK2 for 300 steps (this set-up meets a non-physical
    quadrature state of the method as stated at step 340) and with the paper's
    MUSCL-Hancock step to t = 0.5.
Reported (printed): the L1 error of every average plane relative to the oracle's
mean |average|, and the drift of the conserved totals.
"""
import numpy as np
import pytest

import oracle as O
from paper_1305_5536_gb300 import dg, ics

pytestmark = pytest.mark.gpu


def _l1(a, b, planes):
    return max(float(np.abs(a[q] - b[q]).mean() / np.abs(b[q]).mean()) for q in planes)


def _run(eq, n, u0, integrator, nsteps=None, tend=None):
    P = O.Problem(O.MHD if eq == "mhd" else O.EULER, 2, n)
    tot0 = P.totals(u0)
    rng = np.random.default_rng(17)
    up = u0 * (1.0 + 1e-14 * rng.standard_normal(u0.shape))  # the perturbed oracle run
    sol = {p: dg.DGSolver(eq, 2, n, precision=p, integrator=integrator)
           for p in ("fp64", "fp32")}
    for s in sol.values():
        s.set_state(u0)
    u, t, k = u0, 0.0, 0
    step = (lambda v, dt: P.mh_step(v, dt, face_points=1)) if integrator == "mh" else P.step
    while (nsteps is not None and k < nsteps) or (tend is not None and t < tend - 1e-14):
        dt = P.cfl_dt(u)[0]
        if tend is not None:
            dt = min(dt, tend - t)
        u, fl = step(u, dt)
        assert fl == 0, k
        up, fl = step(up, dt)
        assert fl == 0, k
        for s in sol.values():
            s.step(1, dt=dt)
        t += dt
        k += 1
    planes = [0, 3, 6, 9] + ([12, 13] if eq == "mhd" else [])
    out = {"oracle perturbed 1e-14": (_l1(up, u, planes), None)}
    for p, s in sol.items():
        got = s.get_state()
        tot = s.totals()[0]
        s.close()
        out[p] = (_l1(got, u, planes), float(np.abs(tot - tot0).max() / np.abs(tot0).max()))
    return out, k, t


CASES = {
    "smooth_wave_64_rk2_50": ("euler", (64, 64), "rk2", 50, None),
    "orszag_tang_128_rk2_300": ("mhd", (128, 128), "rk2", 300, None),
    "orszag_tang_128_mh_t0.5": ("mhd", (128, 128), "mh", None, 0.5),
}
# FP32: bounds a few times above the values measured on a GB300 (printed)
FP32_L1 = {"smooth_wave_64_rk2_50": 1e-5, "orszag_tang_128_rk2_300": 2e-2,
           "orszag_tang_128_mh_t0.5": 8e-2}


@pytest.mark.parametrize("case", sorted(CASES))
def test_long_run_against_the_fp64_oracle(case, capsys):
    eq, n, integ, nsteps, tend = CASES[case]
    u0 = ics.euler2d_wave(n) if eq == "euler" else ics.orszag_tang(n)
    out, k, t = _run(eq, n, u0, integ, nsteps, tend)
    with capsys.disabled():
        print("\n%s: %d steps to t = %.4f" % (case, k, t))
        for p, (l1, drift) in out.items():
            print("  %-22s L1 vs oracle %.2e%s" % (
                p, l1, "" if drift is None else "; conservation drift %.2e" % drift))
    sens = out["oracle perturbed 1e-14"][0]
    # the FP64 GPU path is as close to the oracle as the problem's own sensitivity
    # to rounding allows
    assert out["fp64"][0] < max(10 * sens, 1e-11), (out["fp64"][0], sens)
    assert out["fp32"][0] < FP32_L1[case], out["fp32"]
    # FP64 averages on both paths: conservation to rounding
    assert out["fp64"][1] < 1e-14
    assert out["fp32"][1] < 1e-9
