"""Per-phase cycle shares of the SSP-RK2 stage kernels (profiling build).

    python -m paper_1305_5536_gb300.phase_profile --workload kh3d_128 --steps 5

Builds ``libdg_phase.so`` (the library's sources compiled with clock64() stamps
between the phases of the 2D and 3D stage kernels, ``-DDG_PHASE_PROFILE``),
loads it instead of ``libdg.so``, runs the workload's FP32 SSP-RK2 steps with
kernel profiling on, and prints, per stage and phase, the SM cycles summed over
the CTAs, their share of the stage, and the cycles per cell.  The counters are
stamped by thread 0 of each CTA at the end of each phase (after the barrier that
closes it), so shares include the time a phase waits for its slowest warp.
"""
import argparse
import os

import numpy as np

PHASES_2D = ["staging", "primitives", "limiter", "faces", "per-cell rhs + combination",
             "Courant reduction"]
PHASES_3D = ["staging + primitives", "limiter", "volume integral", "x faces", "x gather",
             "y faces", "y gather", "z faces", "z gather", "combination + store",
             "Courant reduction"]


def _state(name):
    from . import ics
    if name == "kh3d_128":
        return "euler", 3, (128, 128, 128), ics.kh3d((128, 128, 128))
    if name == "kh3d_256":
        return "euler", 3, (256, 256, 256), ics.kh3d((256, 256, 256))
    if name == "orszag_tang_512":
        return "mhd", 2, (512, 512), ics.orszag_tang((512, 512))
    if name == "smooth_wave_64":
        return "euler", 2, (64, 64), ics.euler2d_wave((64, 64))
    raise ValueError("unknown workload " + name)


def run(workload, steps=5, warmup=2, precision="fp32"):
    from . import _build
    os.environ["DG_LIBRARY"] = _build.build(phase=True)
    from . import dg
    if os.path.abspath(dg.LIB_PATH) != os.path.abspath(os.environ["DG_LIBRARY"]):
        raise RuntimeError("dg was loaded before the profiling build was selected")
    eq, dim, n, u0 = _state(workload)
    s = dg.DGSolver(eq, dim, n, precision=precision)
    s.set_state(u0)
    s.step(warmup, sync=True)
    s.profile(True)
    for _ in range(steps):
        s.step(1)
    s.sync()
    cyc = s.phase_cycles()
    name = s.kernel_name()
    s.close()
    names = PHASES_3D if dim == 3 else PHASES_2D
    ncell = int(np.prod(n))
    lines = ["%s, %s, %d steps; kernel %s" % (workload, precision, steps, name),
             "| stage | phase | SM cycles (sum over CTAs) | share | cycles per cell |",
             "|---|---|---|---|---|"]
    for st in range(2):
        tot = cyc[st].sum()
        for k, nm in enumerate(names):
            lines.append("| %d | %s | %.4g | %.1f %% | %.1f |" % (
                st + 1, nm, cyc[st, k], 100.0 * cyc[st, k] / tot if tot else 0.0,
                cyc[st, k] / (ncell * steps)))
    return "\n".join(lines)


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--workload", default="kh3d_128")
    ap.add_argument("--steps", type=int, default=5)
    ap.add_argument("--precision", default="fp32")
    a = ap.parse_args()
    print(run(a.workload, a.steps, precision=a.precision))


if __name__ == "__main__":
    main()
