"""Throughput of the GB300 DG step: cell-updates/s and HBM-roofline fraction.

Default workload: 2D ideal MHD Orszag-Tang vortex, 512 x 512 cells, P1 DG with the
locally divergence-free magnetic basis, min/max limiter, HLLD fluxes, CFL 0.3;
FP32 arithmetic with FP64 cell averages (``value``), the FP64 path measured on
the same workload beside it.  One "step" is one SSP-RK2 step of the whole grid.

Timing: W warm-up steps, then K steps timed one by one with CUDA events on the
solver's stream; the L2 cache is flushed (a 512 MiB buffer is written) before
every timed step because the 512^2 state fits in L2.  Every RESTART_STEPS steps
(fewer for workloads whose flow reaches a state the method as stated cannot
step sooner) the solver restarts from the initial state, which stays resident on
the device; the restart lies outside the timed events.  Kernel durations come from
CUDA events the library records around each stage-kernel launch, in K more steps
right after the timed ones (an event between the two stage kernels of a step
serialises them; the timed steps let the second start while the first drains).
End to end (``e2e``): every step the state goes in from page-locked host memory
(dg_set_state), one step, and the state comes back into page-locked host memory
(dg_get_state), with CUDA events; beside it the same loop in two contexts on two
streams driven by two host threads at once (host clock), which shows how much the
host link allows the transfers of one to overlap the other's.  Multi-GPU
(--gpus N under torchrun): independent replicas, one per rank (weak scaling),
barrier + max over ranks.  The default workload's line also carries the adjoint
step time (the checkpointed adjoint of 100 steps of a 2D Euler 256^2 problem,
FP64 and FP32).  ``--impl reference`` times the CPU oracle instead.
"""
import argparse
import hashlib
import json
import math
import os
import subprocess
import sys
import threading
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

L2_FLUSH_BYTES = 512 << 20
# SM clock of the issue ceiling (the GB300's maximum, also the clock the timed runs
# hold: their sampled median is recorded in the line's "clocks")
ISSUE_CLOCK_MHZ = 2070.0
# steps after which the run restarts from the initial state (each workload has run
# at least this far from its initial state without a non-physical state)
RESTART_STEPS = 1000

WORKLOADS = {
    "orszag_tang_512": dict(eq="mhd", dim=2, n=(512, 512), desc=(
        "2D ideal MHD Orszag-Tang vortex 512x512, P1 DG, div-free B basis, HLLD, "
        "min/max limiter, CFL 0.3")),
    "smooth_wave_64": dict(eq="euler", dim=2, n=(64, 64), desc=(
        "2D Euler smooth density wave 64x64 + 1e-3 slope noise, exact Riemann, "
        "limiter, CFL 0.3")),
    "kh3d_256": dict(eq="euler", dim=3, n=(256, 256, 256), desc=(
        "3D Euler Kelvin-Helmholtz shear layer 256^3, exact Riemann, limiter, CFL 0.3")),
    "kh3d_128": dict(eq="euler", dim=3, n=(128, 128, 128), desc=(
        "3D Euler Kelvin-Helmholtz shear layer 128^3 (profiling size), exact Riemann, limiter, "
        "CFL 0.3")),
    "orszag_tang_512_mh": dict(eq="mhd", dim=2, n=(512, 512), integrator="mh", desc=(
        "2D ideal MHD Orszag-Tang vortex 512x512, P1 DG, div-free B basis, HLLD, "
        "min/max limiter, CFL 0.3, MUSCL-Hancock step (Sec. 2.4) with one flux at each "
        "face centroid")),
    "kh3d_256_mh": dict(eq="euler", dim=3, n=(256, 256, 256), integrator="mh", desc=(
        "3D Euler Kelvin-Helmholtz shear layer 256^3, exact Riemann, limiter, CFL 0.3, "
        "MUSCL-Hancock step (Sec. 2.4) with one flux at each face centroid")),
    "kh3d_128_mh": dict(eq="euler", dim=3, n=(128, 128, 128), integrator="mh", desc=(
        "3D Euler Kelvin-Helmholtz shear layer 128^3 (profiling size), exact Riemann, limiter, "
        "CFL 0.3, MUSCL-Hancock step (Sec. 2.4) with one flux at each face centroid")),
    # SSP-RK2 with the min/max limiter meets a non-physical state in step 380
    "ot3d_128": dict(eq="mhd", dim=3, n=(128, 128, 128), restart=250, desc=(
        "3D ideal MHD Orszag-Tang vortex with z-modulated velocity 128^3, P1 DG, 11-function "
        "div-free B basis, HLLD, min/max limiter, CFL 0.3")),
    "ot3d_128_mh": dict(eq="mhd", dim=3, n=(128, 128, 128), integrator="mh", desc=(
        "3D ideal MHD Orszag-Tang vortex with z-modulated velocity 128^3, P1 DG, 11-function "
        "div-free B basis, HLLD, min/max limiter, CFL 0.3, MUSCL-Hancock step (Sec. 2.4) with "
        "one flux at each face centroid")),
    "mhd_batch64": dict(eq="mhd", dim=2, n=None, desc=(
        "64 independent 2D ideal-MHD problems, N log-uniform in [32, 512] (seeded), "
        "random-phase smooth v and div-free B, one persistent launch per step, CFL 0.3")),
}


def _workload_state(W):
    """(initial interchange state, total cells, solver configs or None)."""
    from paper_1305_5536_gb300 import dg, ics
    if W["n"] is None:
        sizes, us = ics.mhd_batch()
        return np.concatenate([u.ravel() for u in us]), sum(N * N for N in sizes), sizes
    if W["eq"] == "mhd" and W["dim"] == 3:
        u0 = ics.orszag_tang_3d(W["n"])
    elif W["eq"] == "mhd":
        u0 = ics.orszag_tang(W["n"])
    elif W["dim"] == 3:
        u0 = ics.kh3d(W["n"])
    else:
        u0 = ics.euler2d_wave(W["n"])
    return u0, int(np.prod(W["n"])), None


def _peaks():
    p = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(p):
        with open(p) as f:
            d = json.load(f)
        return d.get("hbm_gbs", 6800.0), "measured"
    return 6800.0, "fallback"


# Sources each kernel family is compiled from (its ncu figures are void once any
# of them changes).
_FAMILY_SOURCES = {
    "stage2d_kernel": ("dg_stage2d.cuh",),
    "stage2d_tma_kernel": ("dg_stage2d.cuh", "dg_stage2d_tma.cuh", "dg_tma.cuh"),
    "batch2d_kernel": ("dg_stage2d.cuh", "dg_batch.cu", "dg_batch.h"),
    "stage3d_kernel": ("dg_stage3d.cuh",),
    "stage3m_kernel": ("dg_stage3d.cuh", "dg_stage3m.cuh"),
    "mh2d_kernel": ("dg_stage2d.cuh", "dg_mh2d.cuh"),
    "mh3d_kernel": ("dg_stage3d.cuh", "dg_mh3d.cuh"),
    "mh3m_kernel": ("dg_stage3d.cuh", "dg_stage3m.cuh", "dg_mh3d.cuh", "dg_mh3m.cuh"),
}


def _src_sha(kernel):
    h = hashlib.sha256()
    csrc = os.path.join(ROOT, "paper_1305_5536_gb300", "csrc")
    fam = _FAMILY_SOURCES.get(kernel.split()[0], ())
    for f in sorted(fam + ("dg_physics.cuh", "dg_common.cuh", "dg_weno.cuh")):
        h.update(open(os.path.join(csrc, f), "rb").read())
    return h.hexdigest()[:16]


def _ncu_entry(kernel, workload):
    """The committed ncu figures of `kernel` on `workload` (profiles/ncu_traffic.json),
    if they were taken on the current kernel sources; else None."""
    p = os.path.join(ROOT, "profiles", "ncu_traffic.json")
    if not os.path.exists(p):
        return None
    with open(p) as f:
        d = json.load(f)
    e = d.get(workload, {}).get(kernel)
    if not e or e.get("src_sha") != _src_sha(kernel):
        return None
    return e


def _traffic(kernel, workload):
    """Per-launch DRAM bytes of `kernel` from the committed ncu summary, if it was
    taken on the current kernel sources; else None."""
    e = _ncu_entry(kernel, workload)
    return e.get("dram_bytes_per_launch") if e else None


class ClockSampler:
    """nvidia-smi clock / throttle samples while the timed region runs."""

    def __init__(self, gpu):
        self.gpu = gpu
        self.proc = None
        self.lines = []
        self.window = (0.0, float("inf"))

    def __enter__(self):
        q = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
             "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
             "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", "-i", str(self.gpu), "--query-gpu=" + q,
                 "--format=csv,noheader,nounits", "-lms", "50"],
                stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
            self.t = threading.Thread(target=self._read, daemon=True)
            self.t.start()
        except Exception:
            self.proc = None
        return self

    def _read(self):
        for line in self.proc.stdout:
            self.lines.append((time.perf_counter(), line.strip()))

    def __exit__(self, *a):
        if self.proc:
            self.proc.terminate()
            try:
                self.proc.wait(timeout=5)
            except Exception:
                self.proc.kill()

    def summary(self):
        sm, smax, reasons = [], None, set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        t0, t1 = self.window
        for ts, ln in self.lines:
            if not (t0 <= ts <= t1 + 0.06):
                continue
            f = [x.strip() for x in ln.split(",")]
            if len(f) < 9:
                continue
            try:
                sm.append(float(f[1]))
                smax = float(f[2])
            except ValueError:
                continue
            for nm, v in zip(names, f[5:9]):
                if v.lower() == "active":
                    reasons.add(nm)
        return {"sm_mhz": float(np.median(sm)) if sm else None, "sm_max_mhz": smax,
                "reasons": sorted(reasons), "samples": len(sm)}


def _dist():
    ws = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    return ws, rank


def max_over_ranks(x, device="cpu"):
    """Largest value of x over all ranks (the timed region of the slowest replica);
    x itself when torch.distributed is not initialised."""
    import torch
    import torch.distributed as tdist
    if not (tdist.is_available() and tdist.is_initialized()) or tdist.get_world_size() == 1:
        return float(x)
    t = torch.tensor([float(x)], dtype=torch.float64, device=device)
    tdist.all_reduce(t, op=tdist.ReduceOp.MAX)
    return float(t.item())


def run_gpu(args):
    import torch
    import torch.distributed as tdist

    from paper_1305_5536_gb300 import dg, ics

    ws, rank = _dist()
    local = int(os.environ.get("LOCAL_RANK", "0"))
    torch.cuda.set_device(local)
    if ws > 1:
        tdist.init_process_group("nccl")
    flush = torch.empty(L2_FLUSH_BYTES // 4, dtype=torch.float32, device="cuda")
    stream = torch.cuda.current_stream()

    def barrier():
        if ws > 1:
            tdist.barrier()
        torch.cuda.synchronize()

    def measure(wname, prec, K, Wm, with_clock, e2e=True):
        """K timed steps of workload `wname` after Wm warm-up steps (L2 flushed before
        each), with the stage kernels' CUDA-event times; optionally the end-to-end
        loop through the C ABI with page-locked host buffers."""
        W = WORKLOADS[wname]
        u0, ncell, sizes = _workload_state(W)

        def solver(stream=None):
            if sizes is not None:
                return dg.DGSolver(configs=[dg.make_config(W["eq"], 2, (N, N), precision=prec)
                                            for N in sizes], stream=stream)
            return dg.DGSolver(W["eq"], W["dim"], W["n"], precision=prec, cfl=0.3,
                               integrator=W.get("integrator", "rk2"), stream=stream)

        s = solver()
        u0_dev = torch.from_numpy(np.ascontiguousarray(u0)).to("cuda")
        cycle = W.get("restart", RESTART_STEPS)
        s.set_state(u0_dev)
        since = 0

        def restart_if_due():
            nonlocal since
            if since == cycle:
                s.set_state(u0_dev)
                since = 0
            since += 1

        for _ in range(Wm):
            flush.fill_(1.0)
            restart_if_due()
            s.step(1)
        s.sync()
        evs = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True))
               for _ in range(K)]
        barrier()
        sampler = ClockSampler(local) if with_clock else None
        if sampler:
            sampler.__enter__()
            time.sleep(1.0)  # let nvidia-smi start sampling before the timed region
        t_wall = time.perf_counter()
        t_start = t_wall
        for k in range(K):
            flush.fill_(float(k))
            restart_if_due()
            evs[k][0].record(stream)
            s.step(1)
            evs[k][1].record(stream)
        barrier()
        t_wall = time.perf_counter() - t_wall
        # the kernel durations: K more steps with the library's events around each
        # stage-kernel launch (an event between the two stage kernels of a step
        # serialises them, so these steps are not the ones whose time is the value)
        s.profile(True)
        for k in range(K):
            flush.fill_(float(k))
            restart_if_due()
            s.step(1)
        s.sync()
        barrier()
        t_both = time.perf_counter() - t_start
        if sampler:
            sampler.window = (t_start, t_start + t_both)
            time.sleep(0.2)
            sampler.__exit__()
        step_ms = [a.elapsed_time(b) for a, b in evs]
        kms, kn = s.profile_read()
        s.profile(False)
        tot = max_over_ranks(sum(step_ms), "cuda")
        res = dict(ms_total=tot, ms_per_step=tot / K, kernel_ms=kms, kernel_launches=kn,
                   kernel=s.kernel_name(), ncell=ncell, sizes=sizes,
                   bytes=[s.stage_bytes(1), s.stage_bytes(2)], wall_s=t_wall,
                   clocks=sampler.summary() if sampler else None)
        if e2e:
            # end to end through the public API with host buffers (pinned)
            host_in = torch.from_numpy(np.ascontiguousarray(u0)).pin_memory()
            host_out = torch.empty_like(host_in).pin_memory()
            e2e_K = max(3, min(K, 20))
            s.set_state(host_in)
            barrier()
            e0 = torch.cuda.Event(enable_timing=True)
            e1 = torch.cuda.Event(enable_timing=True)
            e0.record(stream)
            for k in range(e2e_K):
                s.set_state(host_in)
                s.step(1)
                s.get_state(host_out)
            e1.record(stream)
            barrier()
            res["e2e_ms_per_step"] = max_over_ranks(e0.elapsed_time(e1), "cuda") / e2e_K
            res["e2e_bytes"] = host_in.numel() * 8
            # the same loop in two contexts, each on a stream of its own and driven by
            # a host thread of its own (the library's calls release the GIL), so that
            # one context's transfers and kernels may overlap the other's: what a
            # caller stepping independent problems held in host memory gets
            ctxs = []
            for _ in range(2):
                st_i = torch.cuda.Stream()
                out_i = torch.empty_like(host_in).pin_memory()
                s_i = solver(stream=st_i.cuda_stream)
                s_i.set_state(host_in)
                s_i.step(1)
                s_i.get_state(out_i)
                ctxs.append((s_i, out_i, st_i))
            errors = []

            def loop(i):
                s_i, out_i, _ = ctxs[i]
                try:
                    for k in range(e2e_K):
                        s_i.set_state(host_in)
                        s_i.step(1)
                        s_i.get_state(out_i)
                except Exception as exc:  # re-raised on the main thread
                    errors.append(exc)

            torch.cuda.synchronize()
            barrier()
            t0 = time.perf_counter()
            threads = [threading.Thread(target=loop, args=(i,)) for i in range(2)]
            for t in threads:
                t.start()
            for t in threads:
                t.join()
            torch.cuda.synchronize()
            t2 = time.perf_counter() - t0
            barrier()
            if errors:
                raise errors[0]
            res["e2e2_ms_per_step"] = max_over_ranks(t2, "cuda") * 1e3 / (2 * e2e_K)
            for s_i, _, _ in ctxs:
                s_i.close()
        s.close()
        return res

    def roofline(wname, r, hbm, peak_kind):
        """HBM roofline of the dominant kernel of a measurement (stage 2 of SSP-RK2,
        the step kernel of MUSCL-Hancock or of a batch)."""
        W = WORKLOADS[wname]
        k = 1 if r["kernel_ms"][1] >= r["kernel_ms"][0] else 0
        avg_ms = r["kernel_ms"][k] / max(r["kernel_launches"][k], 1)
        achieved = r["bytes"][k] / (avg_ms * 1e-3) / 1e9
        if W.get("integrator") == "mh":
            kname = "%s %s, step" % (r["kernel"], W["eq"])
        else:
            kname = "%s %s, stage %s" % (r["kernel"], W["eq"],
                                          "1+2" if r["sizes"] is not None else k + 1)
        out = {"bound": "hbm", "kernel": kname, "achieved": achieved, "peak": hbm,
               "peak_kind": peak_kind, "unit": "GB/s", "frac": achieved / hbm,
               "traffic": _traffic(kname, wname),
               "algorithmic_bytes_per_launch": r["bytes"][k], "avg_launch_ms": avg_ms}
        e = _ncu_entry(kname, wname)
        if e and "issue_active_pct" in e:
            # the kernels are bound by instruction issue, not by DRAM: the ncu
            # figures of the same kernel on the same sources, and the thread-
            # instruction rate of this run against the issue ceiling of the part
            # (152 SMs x 4 schedulers x 32 lanes x the SM clock)
            out["issue"] = {key: e[key] for key in ("issue_active_pct", "pipe_pct",
                                                      "thread_inst_per_cell", "lane_efficiency",
                                                      "captured")
                            if key in e}
            if "thread_inst_per_launch" in e:
                rate = e["thread_inst_per_launch"] / (avg_ms * 1e-3)
                peak = 152 * 4 * 32 * ISSUE_CLOCK_MHZ * 1e6
                out["issue"].update({"achieved_thread_inst_per_s": rate,
                                     "peak_thread_inst_per_s": peak, "frac": rate / peak})
        return kname, out

    def fp32_accuracy():
        """FP32 against FP64 (both on the GPU; the -m gpu tests hold the FP64 path to
        the FP64 oracle and compare FP32 with the oracle directly) on Orszag-Tang
        128^2: SSP-RK2 for 300 Courant steps (the method as stated meets a
        non-physical quadrature state at step 340 at this resolution) and the
        MUSCL-Hancock step to t = 0.5.  L1 of the average planes relative to the
        FP64 state's mean |average|, and the relative drift of the conserved totals
        from the initial state."""
        n = (128, 128)
        u0 = ics.orszag_tang(n)
        out = {"workload": "2D ideal MHD Orszag-Tang 128x128, min/max limiter, CFL 0.3",
               "reference": "FP64 GPU path (held to the FP64 oracle by the -m gpu tests)"}
        names = ["rho", "mx", "my", "E", "b1", "b2"]
        planes = [0, 3, 6, 9, 12, 13]
        for label, integ, nsteps, tend in (("ssprk2_300_steps", "rk2", 300, None),
                                           ("muscl_hancock_t0.5", "mh", None, 0.5)):
            sol = {p: dg.DGSolver("mhd", 2, n, precision=p, integrator=integ)
                   for p in ("fp64", "fp32")}
            tot0 = {}
            for p, s in sol.items():
                s.set_state(u0)
                tot0[p] = s.totals()[0]
            # the FP64 path's Courant steps for both, so that only the arithmetic differs
            t, k = 0.0, 0
            while (nsteps is not None and k < nsteps) or (tend is not None and t < tend - 1e-14):
                dt = sol["fp64"].times()[1][0]
                if tend is not None:
                    dt = min(dt, tend - t)
                for s in sol.values():
                    s.step(1, dt=dt)
                t += dt
                k += 1
            got, drift = {}, {}
            for p, s in sol.items():
                got[p] = s.get_state()
                tot1 = s.totals()[0]
                drift[p] = float(np.abs(tot1 - tot0[p]).max() / np.abs(tot0[p]).max())
                s.close()
            u64, u32 = got["fp64"], got["fp32"]
            l1 = {nm: float(np.abs(u32[q] - u64[q]).mean() / np.abs(u64[q]).mean())
                  for nm, q in zip(names, planes)}
            out[label] = {"steps": k, "t": t, "l1_fp32_vs_fp64": l1,
                          "conservation_drift": drift}
        return out

    r32 = measure(args.workload, "fp32", args.steps, args.warmup, True)
    r64 = measure(args.workload, "fp64", max(3, min(args.steps, 20)), max(3, args.warmup), False,
                  e2e=False)
    W = WORKLOADS[args.workload]
    extra = {}
    if args.workload == "orszag_tang_512" and not args.no_extras:
        # the config the HBM target is judged on (C3: 3D Euler KH 256^3, FP32), its
        # own roofline; and the FP64 path's roofline against the measured FP64 peak
        rk = measure("kh3d_256", "fp32", 20, 3, False, e2e=False)
        extra["kh3d_256"] = rk
        extra["peak_fp64"] = dg.peak_fma("fp64")
        extra["peak_fp32"] = dg.peak_fma("fp32")
        extra["fp32_accuracy"] = fp32_accuracy()
    if rank != 0:
        return
    hbm, peak_kind = _peaks()
    ncell = r32["ncell"]
    value = ws * ncell / (r32["ms_per_step"] * 1e-3)
    kname, roof = roofline(args.workload, r32, hbm, peak_kind)
    v64 = ws * ncell / (r64["ms_per_step"] * 1e-3)
    k64 = 1 if r64["kernel_ms"][1] >= r64["kernel_ms"][0] else 0
    fp64 = {"value": v64, "ms_per_step": r64["ms_per_step"],
            "speedup_fp32_over_fp64": v64 and value / v64,
            "stage_ms_avg": [r64["kernel_ms"][i] / max(r64["kernel_launches"][i], 1)
                             for i in range(2)], "kernel": r64["kernel"]}
    if "peak_fp64" in extra:
        k64name = "%s %s, stage %d" % (r64["kernel"], W["eq"], k64 + 1)
        e = _ncu_entry(k64name, args.workload)
        flops = e.get("fp64_flops_per_launch") if e else None
        avg = fp64["stage_ms_avg"][k64]
        fp64["roofline"] = {
            "bound": "fp64", "kernel": k64name,
            "achieved": flops / (avg * 1e-3) / 1e12 if flops else None,
            "peak": extra["peak_fp64"] / 1e12, "peak_kind": "measured (dg_peak_fma, this run)",
            "unit": "TFLOP/s", "frac": flops / (avg * 1e-3) / extra["peak_fp64"] if flops else None,
            "fp64_flops_per_launch": flops,
            "fp32_fma_peak_tflops": extra["peak_fp32"] / 1e12}
    out = {
        "metric": _metric(W),
        "value": value,
        "unit": "cell-updates/s",
        "n_gpus": ws,
        "steps": args.steps,
        "warmup": args.warmup,
        "ms_per_step": r32["ms_per_step"],
        "higher_is_better": True,
        "scaling": "weak",
        "vs_baseline": None,
        "dtype": "f32",
        "data": "synthetic (analytic initial condition projected onto the P1 bases)",
        "config": {"workload": W["desc"], "grid": list(W["n"]) if W["n"] else r32["sizes"],
                   "precision": "FP32 arithmetic + FP32 derivative coefficients, FP64 averages",
                   "l2": "flushed (512 MiB write) before every timed step",
                   "restart_every": W.get("restart", RESTART_STEPS),
                   "parallelism": "replicas" if ws > 1 else "single GPU"},
        "roofline": roof,
        "kernels": {"stage1_ms_avg": r32["kernel_ms"][0] / max(r32["kernel_launches"][0], 1),
                    "stage2_ms_avg": r32["kernel_ms"][1] / max(r32["kernel_launches"][1], 1),
                    "launches": r32["kernel_launches"]},
        "fp64": fp64,
        "e2e": {"value": ws * ncell / (r32["e2e_ms_per_step"] * 1e-3), "unit": "cell-updates/s",
                "h2d_bytes_per_step": r32["e2e_bytes"], "d2h_bytes_per_step": r32["e2e_bytes"],
                "ms_per_step": r32["e2e_ms_per_step"],
                "method": "dg_set_state from page-locked host memory, dg_step(1), dg_get_state "
                          "into page-locked host memory, every step (CUDA events)",
                "two_contexts": {
                    "value": ws * ncell / (r32["e2e2_ms_per_step"] * 1e-3),
                    "ms_per_step": r32["e2e2_ms_per_step"],
                    "method": "the same loop in two contexts on two streams, driven by two host "
                              "threads at once (host wall clock)"}},
        "gpu_launches": int(sum(r32["kernel_launches"])),
        "clocks": r32["clocks"],
    }
    if "kh3d_256" in extra:
        rk = extra["kh3d_256"]
        _, roof3 = roofline("kh3d_256", rk, hbm, peak_kind)
        out["kh3d_256"] = {
            "workload": WORKLOADS["kh3d_256"]["desc"] + " (FP32; the config the HBM target "
                        "is judged on)",
            "value": rk["ncell"] / (rk["ms_per_step"] * 1e-3), "unit": "cell-updates/s",
            "ms_per_step": rk["ms_per_step"], "steps": 20, "warmup": 3,
            "stage_ms_avg": [rk["kernel_ms"][i] / max(rk["kernel_launches"][i], 1)
                             for i in range(2)],
            "roofline": roof3}
    if "fp32_accuracy" in extra:
        out["fp32_accuracy"] = extra["fp32_accuracy"]
    if args.workload == "orszag_tang_512" and not args.no_adjoint:
        out["adjoint"] = {
            "workload": "2D Euler 256x256, seeded Gaussian random density (rms 0.05, "
                        "correlation length 0.1), 100 SSP-RK2 steps at CFL 0.3, limiter off, "
                        "checkpoint every 10 steps, objective 1/2 int (rho - rho_target)^2",
            "fp64": measure_adjoint(dg, ics, torch, stream, "fp64"),
            "fp32": measure_adjoint(dg, ics, torch, stream, "fp32")}
    if not args.no_cpu_baseline:
        out["cpu_baseline"] = cpu_baseline(args.workload)
    print(json.dumps(out))


def measure_adjoint(dg, ics, torch, stream, prec):
    """The adjoint workload: 2D Euler 256^2, a seeded Gaussian random density on
    the smooth-wave background, 100 SSP-RK2 steps recorded with checkpoints
    every 10 (limiter off), objective 1/2 int (rho_h - rho_target)^2 exact on
    P1; its gradient with respect to the initial coefficients by the
    checkpointed adjoint (recomputation of each segment, reverse sweep).
    Forward and adjoint timed with CUDA events on the solver's stream."""
    n, K = (256, 256), 100
    u0 = torch.from_numpy(ics.euler2d_random_density(n)[0]).cuda()
    tgt = torch.from_numpy(ics.euler2d_random_density(n, seed=99)[0][0:3]).cuda()
    hx, hy = 1.0 / n[0], 1.0 / n[1]
    w = torch.tensor([1.0, hx * hx / 12, hy * hy / 12], dtype=torch.float64,
                     device="cuda").view(3, 1, 1) * (hx * hy)
    s = dg.DGSolver("euler", 2, n, precision=prec, limiter=0, cfl=0.3, ckpt_every=10)
    res = None
    for _ in range(2):  # the first run warms the graphs and the autotuner
        ev = [torch.cuda.Event(enable_timing=True) for _ in range(4)]
        s.set_state(u0)
        ev[0].record(stream)
        s.record(K)
        ev[1].record(stream)
        uT = s.get_state(device="cuda")
        g = torch.zeros_like(uT)
        g[0:3] = w * (uT[0:3] - tgt)
        ev[2].record(stream)
        g0 = s.adjoint(g)
        ev[3].record(stream)
        torch.cuda.synchronize()
        f_ms, a_ms = ev[0].elapsed_time(ev[1]), ev[2].elapsed_time(ev[3])
        res = {"forward_ms": f_ms, "adjoint_ms": a_ms, "adjoint_ms_per_step": a_ms / K,
               "adjoint_over_forward": a_ms / f_ms,
               "adjoint_cell_steps_per_s": K * n[0] * n[1] / (a_ms * 1e-3),
               "grad_norm": float(g0.norm())}
    s.close()
    return res


# Largest grid the oracle steps whole inside the CPU-baseline time budget; bigger
# workloads are sampled on a periodic sub-box of the same cells.
ORACLE_MAX_CELLS = 300_000


def _oracle_sample(workload, u0):
    """[(oracle problem, state)], description, cells per sweep: the bounded CPU
    sample of a workload (whole grid, a periodic sub-box, or a few problems of a
    batch)."""
    import oracle as O
    W = WORKLOADS[workload]
    if W["n"] is None:
        from paper_1305_5536_gb300 import ics
        sizes, us = ics.mhd_batch()
        items, cells = [], 0
        for N, u in zip(sizes, us):
            if cells + N * N > ORACLE_MAX_CELLS:
                continue
            items.append((O.Problem(O.MHD, 2, (N, N)), u))
            cells += N * N
        return items, "%d of the batch's problems (%d cells)" % (len(items), cells), cells
    n = list(W["n"])
    box = [1.0] * W["dim"]
    desc = "whole grid"
    if int(np.prod(n)) > ORACLE_MAX_CELLS:
        m = 64 if W["dim"] == 3 else 512
        sl = tuple(slice(0, min(m, a)) for a in reversed(n))
        box = [min(m, a) / a for a in n]
        n = [min(m, a) for a in n]
        u0 = np.ascontiguousarray(u0[(slice(None),) + sl])
        desc = "periodic %s sub-box of the same cells" % "x".join(map(str, n))
    P = O.Problem(O.MHD if W["eq"] == "mhd" else O.EULER, W["dim"], n, box=box)
    return [(P, u0)], desc, int(np.prod(n))


def _metric(W):
    kind = "MUSCL-Hancock" if W.get("integrator") == "mh" else "SSP-RK2"
    return "DG cell-updates/sec (%s steps x cells / s)" % kind


def _oracle_sweep(items, dts, mh=False):
    if mh:
        return [(P, P.mh_step(u, dt, face_points=1)[0]) for (P, u), dt in zip(items, dts)]
    return [(P, P.step(u, dt)[0]) for (P, u), dt in zip(items, dts)]


def _host_model():
    """CPU model name of this host (lscpu), for the baseline's record."""
    try:
        out = subprocess.run(["lscpu"], capture_output=True, text=True, timeout=10).stdout
        for line in out.splitlines():
            if line.lower().startswith("model name"):
                return line.split(":", 1)[1].strip()
    except Exception:
        pass
    import platform
    return platform.machine()


def _oracle_replica(job):
    """One process of the all-cores oracle run: the workload's CPU sample, `nsteps`
    sweeps after every replica has reached the barrier; returns its (start, end)
    wall-clock times.  Runs in a spawned process (no CUDA)."""
    workload, nsteps, warmup, barrier = job
    W = WORKLOADS[workload]
    u0, _, _ = _workload_state(W)
    items, _, _ = _oracle_sample(workload, u0)
    mh = W.get("integrator") == "mh"
    dts = [P.cfl_dt(u)[0] for P, u in items]
    for _ in range(warmup):
        items = _oracle_sweep(items, dts, mh)
    barrier.wait()
    t0 = time.time()
    for _ in range(nsteps):
        items = _oracle_sweep(items, dts, mh)
    return t0, time.time()


def _oracle_all_cores(workload, nsteps, warmup=0):
    """The oracle, as it stands, on every host core at once: one process per core,
    each stepping the same CPU sample (independent replicas).  Returns (cores,
    wall seconds of the concurrent sweeps)."""
    import multiprocessing as mp
    cores = os.cpu_count() or 1
    ctx = mp.get_context("spawn")
    with ctx.Manager() as m:
        bar = m.Barrier(cores)
        with ctx.Pool(cores) as pool:
            spans = pool.map(_oracle_replica, [(workload, nsteps, warmup, bar)] * cores)
    return cores, max(e for _, e in spans) - min(s for s, _ in spans)


def cpu_baseline(workload, budget_s=10.0, max_steps=50):
    """The CPU oracle, as it stands, on one host core (steps of the same workload,
    or of a bounded part of it, until ~budget_s of CPU time), then on every host
    core at once (one replica of the same sample per core, the same number of
    steps)."""
    u0, _, _ = _workload_state(WORKLOADS[workload])
    items, desc, ncell = _oracle_sample(workload, u0)
    mh = WORKLOADS[workload].get("integrator") == "mh"
    dts = [P.cfl_dt(u)[0] for P, u in items]
    n = 0
    t0 = time.perf_counter()
    while n < max_steps:
        items = _oracle_sweep(items, dts, mh)
        n += 1
        if time.perf_counter() - t0 > budget_s:
            break
    el = time.perf_counter() - t0
    kind = "MUSCL-Hancock" if mh else "SSP-RK2"
    out = {"value": n * ncell / el, "unit": "cell-updates/s", "cores": 1, "kind": "oracle",
           "sample": "%d %s steps, %s (%.1f s)" % (n, kind, desc, el), "host": _host_model()}
    try:
        cores, wall = _oracle_all_cores(workload, n)
        out["all_cores"] = {"value": cores * n * ncell / wall, "unit": "cell-updates/s",
                            "cores": cores,
                            "sample": "%d replicas of the same sample, %d steps each (%.1f s)"
                                      % (cores, n, wall)}
    except Exception as e:  # report, do not fail the bench line
        out["all_cores"] = {"error": str(e)[:200]}
    return out


def run_reference(args):
    """The reference arm: the oracle, as it stands, on every host core (one replica
    of the workload's CPU sample per core); the JSON line of the contract."""
    ws, rank = _dist()
    if rank != 0:
        return
    W = WORKLOADS[args.workload]
    u0, _, _ = _workload_state(W)
    _, desc, ncell = _oracle_sample(args.workload, u0)
    mh = W.get("integrator") == "mh"
    cores, el = _oracle_all_cores(args.workload, args.steps, args.warmup)
    v = cores * args.steps * ncell / el
    print(json.dumps({
        "impl": "reference", "metric": _metric(W),
        "value": v, "unit": "cell-updates/s", "n_gpus": ws, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": el / args.steps * 1e3, "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
        "config": {"workload": W["desc"], "grid": list(W["n"]) if W["n"] else "batch"},
        "cpu_baseline": {"value": v, "unit": "cell-updates/s", "cores": cores, "kind": "oracle",
                         "host": _host_model(),
                         "sample": "%d replicas (one per core) of %d %s steps, %s" % (
                             cores, args.steps, "MUSCL-Hancock" if mh else "SSP-RK2", desc)},
        "e2e": {"value": v, "unit": "cell-updates/s", "h2d_bytes_per_step": 0,
                "d2h_bytes_per_step": 0}}))


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=1000)
    ap.add_argument("--warmup", type=int, default=5)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--workload", default="orszag_tang_512", choices=sorted(WORKLOADS))
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-adjoint", action="store_true",
                    help="skip the adjoint timing of the default workload's line")
    ap.add_argument("--no-extras", action="store_true",
                    help="skip the KH 256^3, FP64-peak and FP32-accuracy objects of the "
                         "default workload's line")
    ap.add_argument("--only-adjoint", choices=["fp32", "fp64"],
                    help="time only the adjoint workload in this precision (for profiling)")
    args = ap.parse_args()
    if args.warmup < 3:
        args.warmup = 3
    if args.only_adjoint:
        import torch
        from paper_1305_5536_gb300 import dg, ics
        print(json.dumps(measure_adjoint(dg, ics, torch, torch.cuda.current_stream(),
                                         args.only_adjoint)))
        return
    if args.impl == "reference":
        run_reference(args)
    else:
        run_gpu(args)


if __name__ == "__main__":
    main()
