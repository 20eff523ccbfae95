"""Python binding of the C ABI in ``include/dg.h`` (ctypes; argument marshalling only).

Every step of the method runs in the CUDA kernels of ``libdg.so``; this module
only converts arguments.  If the library is missing it raises -- there is no
CPU fallback.  PyTorch is used for device memory and streams: torch CUDA tensors
are passed to the library by their data pointers, numpy arrays as host memory.
"""
import ctypes
import os

import numpy as np

PKG = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(PKG, "libdg.so")
# The phase-profiling build of the same sources (phase_profile.py) is loaded
# instead when DG_LIBRARY names it.
LIB_PATH = os.environ.get("DG_LIBRARY") or LIB_PATH
# Tile shapes chosen by the library's autotuner, per (equations, dimension,
# precision, grid): the shipped cache makes runs reproducible; DG_TUNE_CACHE
# names another file.
TUNE_CACHE = os.path.join(PKG, "tune_cache.txt")

DG_OK, DG_EINVAL, DG_ENOMEM, DG_ECUDA, DG_ENONPHYS, DG_ETIMEOUT, DG_ESTATE = range(7)
DG_EULER, DG_MHD = 0, 1
DG_FP64, DG_FP32 = 0, 1
DG_EXACT, DG_HLLD = 0, 1
DG_SSPRK2, DG_MUSCL_HANCOCK = 0, 1
_STATUS = {0: "DG_OK", 1: "DG_EINVAL", 2: "DG_ENOMEM", 3: "DG_ECUDA", 4: "DG_ENONPHYS",
           5: "DG_ETIMEOUT", 6: "DG_ESTATE"}

# every entry point declared in include/dg.h
SYMBOLS = ["dg_num_planes", "dg_init", "dg_init_batch", "dg_destroy", "dg_last_error",
           "dg_set_state", "dg_get_state", "dg_step", "dg_sync", "dg_get_times", "dg_totals",
           "dg_divb", "dg_adjoint_step", "dg_record", "dg_adjoint", "dg_profile",
           "dg_profile_read", "dg_stage_bytes", "dg_totals_noalloc", "dg_kernel_name",
           "dg_record_generation", "dg_peak_fma", "dg_phase_cycles"]


class DGError(RuntimeError):
    def __init__(self, status, msg):
        super().__init__("%s: %s" % (_STATUS.get(status, status), msg))
        self.status = status


class dg_config(ctypes.Structure):
    _fields_ = [("eq", ctypes.c_int), ("dim", ctypes.c_int), ("n", ctypes.c_int * 3),
                ("box", ctypes.c_double * 3), ("gamma", ctypes.c_double),
                ("cfl", ctypes.c_double), ("limiter", ctypes.c_int),
                ("precision", ctypes.c_int), ("riemann", ctypes.c_int),
                ("ckpt_every", ctypes.c_int), ("integrator", ctypes.c_int),
                ("face_points", ctypes.c_int)]


_lib = None


def load():
    """Load libdg.so (building it first if it is missing and nvcc is present)."""
    global _lib
    if _lib is not None:
        return _lib
    if not os.path.exists(LIB_PATH) and not os.environ.get("DG_LIBRARY"):
        from . import _build
        _build.build()
    if not os.path.exists(LIB_PATH):
        raise RuntimeError("libdg.so is missing: the CUDA extension must be built "
                           "(python -c 'import __graft_entry__ as g; g.build()')")
    os.environ.setdefault("DG_TUNE_CACHE", TUNE_CACHE)
    L = ctypes.CDLL(LIB_PATH)
    P, c_int, c_double = ctypes.POINTER, ctypes.c_int, ctypes.c_double
    vp = ctypes.c_void_p
    pcfg = P(dg_config)
    L.dg_num_planes.argtypes = [pcfg]
    L.dg_init.argtypes = [pcfg, vp, P(vp)]
    L.dg_init_batch.argtypes = [pcfg, c_int, vp, P(vp)]
    L.dg_destroy.argtypes = [vp]
    L.dg_destroy.restype = None
    L.dg_last_error.argtypes = [vp]
    L.dg_last_error.restype = ctypes.c_char_p
    L.dg_set_state.argtypes = [vp, vp, c_int]
    L.dg_get_state.argtypes = [vp, vp, c_int]
    L.dg_step.argtypes = [vp, c_int, c_double, P(c_double)]
    L.dg_sync.argtypes = [vp]
    L.dg_get_times.argtypes = [vp, vp, vp]
    L.dg_totals.argtypes = [vp, vp]
    L.dg_divb.argtypes = [vp, vp, c_int]
    L.dg_adjoint_step.argtypes = [vp, vp, vp, vp, c_double]
    L.dg_record.argtypes = [vp, c_int, c_double, P(c_double)]
    L.dg_adjoint.argtypes = [vp, vp, vp]
    L.dg_profile.argtypes = [vp, c_int]
    L.dg_profile_read.argtypes = [vp, P(c_double), P(ctypes.c_longlong)]
    L.dg_stage_bytes.argtypes = [vp, c_int]
    L.dg_stage_bytes.restype = c_double
    L.dg_totals_noalloc.argtypes = [pcfg, vp, vp, c_int, vp]
    L.dg_peak_fma.argtypes = [c_int, P(c_double)]
    L.dg_phase_cycles.argtypes = [vp, P(c_double), c_int]
    L.dg_record_generation.argtypes = [vp]
    L.dg_record_generation.restype = ctypes.c_longlong
    L.dg_kernel_name.argtypes = [vp]
    L.dg_kernel_name.restype = ctypes.c_char_p
    _lib = L
    return L


def _ptr(a):
    """(pointer, on_device) of a numpy array or torch tensor (contiguous float64)."""
    if isinstance(a, np.ndarray):
        assert a.dtype == np.float64 and a.flags.c_contiguous
        return a.ctypes.data_as(ctypes.c_void_p), 0
    import torch
    assert isinstance(a, torch.Tensor) and a.dtype == torch.float64 and a.is_contiguous()
    return ctypes.c_void_p(a.data_ptr()), 1 if a.is_cuda else 0


def _current_stream():
    try:
        import torch
        if torch.cuda.is_available():
            return ctypes.c_void_p(torch.cuda.current_stream().cuda_stream)
    except Exception:
        pass
    return ctypes.c_void_p(0)


def num_totals(eq, dim):
    """Number of conserved totals of a problem: the Taylor variables, then (MHD)
    the field averages b1, b2[, b3]."""
    mhd = eq in ("mhd", DG_MHD)
    return (4 if dim == 2 else 5) + (dim if mhd else 0)


def make_config(eq="euler", dim=2, n=(64, 64), box=(1.0, 1.0, 1.0), gamma=5.0 / 3.0, cfl=0.3,
                limiter=1, precision="fp64", ckpt_every=0, integrator="rk2", face_points=0):
    """integrator: "rk2" (two-stage SSP Runge-Kutta) or "mh" (MUSCL-Hancock, Sec. 2.4);
    face_points: MUSCL-Hancock face rule, 1 (or 0) = face centroid, 2 = Gauss pair."""
    c = dg_config()
    c.eq = DG_MHD if eq in ("mhd", DG_MHD) else DG_EULER
    c.dim = dim
    nn = list(n) + [1] * (3 - len(n))
    bb = list(box) + [1.0] * (3 - len(box))
    for a in range(3):
        c.n[a] = int(nn[a])
        c.box[a] = float(bb[a])
    c.gamma, c.cfl, c.limiter = float(gamma), float(cfl), int(limiter)
    c.precision = DG_FP32 if precision in ("fp32", DG_FP32) else DG_FP64
    c.riemann = DG_HLLD if c.eq == DG_MHD else DG_EXACT
    c.ckpt_every = int(ckpt_every)
    c.integrator = DG_MUSCL_HANCOCK if integrator in ("mh", DG_MUSCL_HANCOCK) else DG_SSPRK2
    c.face_points = int(face_points)
    return c


class DGSolver:
    """One periodic problem (or a batch of problems) stepped by the GPU library."""

    def __init__(self, eq="euler", dim=2, n=(64, 64), box=(1.0, 1.0, 1.0), gamma=5.0 / 3.0,
                 cfl=0.3, limiter=1, precision="fp64", ckpt_every=0, stream=None, configs=None,
                 integrator="rk2", face_points=0):
        L = load()
        self._L = L
        h = ctypes.c_void_p()
        st = _current_stream() if stream is None else ctypes.c_void_p(stream)
        if configs is None:
            cfg = make_config(eq, dim, n, box, gamma, cfl, limiter, precision, ckpt_every,
                              integrator, face_points)
            self.configs = [cfg]
            s = L.dg_init(ctypes.byref(cfg), st, ctypes.byref(h))
        else:
            arr = (dg_config * len(configs))(*configs)
            self.configs = list(configs)
            s = L.dg_init_batch(arr, len(configs), st, ctypes.byref(h))
        if s != DG_OK:
            raise DGError(s, L.dg_last_error(None).decode())
        self._h = h
        c0 = self.configs[0]
        self.eq, self.dim = c0.eq, c0.dim
        self.nplanes = L.dg_num_planes(ctypes.byref(c0))
        self.shapes = []
        for c in self.configs:
            if c.dim == 2:
                self.shapes.append((self.nplanes, c.n[1], c.n[0]))
            else:
                self.shapes.append((self.nplanes, c.n[2], c.n[1], c.n[0]))
        self.size = sum(int(np.prod(s)) for s in self.shapes)

    @property
    def shape(self):
        return self.shapes[0]

    def _check(self, s):
        if s != DG_OK:
            raise DGError(s, self._L.dg_last_error(self._h).decode())

    def close(self):
        if getattr(self, "_h", None):
            self._L.dg_destroy(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def set_state(self, u):
        p, dev = _ptr(u)
        assert u.size == self.size if isinstance(u, np.ndarray) else u.numel() == self.size
        self._check(self._L.dg_set_state(self._h, p, dev))

    def get_state(self, out=None, device=None):
        if out is None:
            if device is not None:
                import torch
                out = torch.empty(self.size if len(self.shapes) > 1 else self.shape,
                                  dtype=torch.float64, device=device)
            else:
                out = np.empty(self.size if len(self.shapes) > 1 else self.shape)
        p, dev = _ptr(out)
        self._check(self._L.dg_get_state(self._h, p, dev))
        return out

    def step(self, nsteps=1, dt=0.0, sync=False):
        t = ctypes.c_double(0.0)
        self._check(self._L.dg_step(self._h, int(nsteps), float(dt),
                                    ctypes.byref(t) if sync else None))
        return t.value if sync else None

    def sync(self):
        self._check(self._L.dg_sync(self._h))

    def times(self):
        n = len(self.configs)
        t, dt = np.zeros(n), np.zeros(n)
        self._check(self._L.dg_get_times(self._h, t.ctypes.data_as(ctypes.c_void_p),
                                         dt.ctypes.data_as(ctypes.c_void_p)))
        return t, dt

    def totals(self):
        nv = num_totals(self.eq, self.dim)
        out = np.zeros(nv * len(self.configs))
        self._check(self._L.dg_totals(self._h, out.ctypes.data_as(ctypes.c_void_p)))
        return out.reshape(len(self.configs), nv)

    def divb(self):
        c = self.configs[0]
        out = np.zeros((c.n[1], c.n[0]))
        self._check(self._L.dg_divb(self._h, out.ctypes.data_as(ctypes.c_void_p), 0))
        return out

    def adjoint_step(self, lam_next, u_n, dt, lam_prev=None):
        import torch
        if lam_prev is None:
            lam_prev = torch.empty_like(lam_next)
        self._check(self._L.dg_adjoint_step(self._h, ctypes.c_void_p(lam_next.data_ptr()),
                                            ctypes.c_void_p(lam_prev.data_ptr()),
                                            ctypes.c_void_p(u_n.data_ptr()), float(dt)))
        return lam_prev

    def record(self, nsteps, dt=0.0):
        t = ctypes.c_double(0.0)
        self._check(self._L.dg_record(self._h, int(nsteps), float(dt), ctypes.byref(t)))
        return t.value

    def record_generation(self):
        """Changes whenever the recorded trajectory does (see dg_record_generation)."""
        return self._L.dg_record_generation(self._h)

    def adjoint(self, lam_N, lam_0=None):
        import torch
        if lam_0 is None:
            lam_0 = torch.empty_like(lam_N)
        self._check(self._L.dg_adjoint(self._h, ctypes.c_void_p(lam_N.data_ptr()),
                                       ctypes.c_void_p(lam_0.data_ptr())))
        return lam_0

    def profile(self, enable=True):
        self._check(self._L.dg_profile(self._h, 1 if enable else 0))

    def profile_read(self):
        ms = (ctypes.c_double * 2)()
        n = (ctypes.c_longlong * 2)()
        self._check(self._L.dg_profile_read(self._h, ms, n))
        return [ms[0], ms[1]], [n[0], n[1]]

    def phase_cycles(self):
        """Per-phase SM cycles of the stage kernels, shape (2 stages, 16 phases)
        (profiling build only; dg_phase_cycles)."""
        out = (ctypes.c_double * 32)()
        self._check(self._L.dg_phase_cycles(self._h, out, 32))
        return np.array(out[:]).reshape(2, 16)

    def kernel_name(self):
        return self._L.dg_kernel_name(self._h).decode()

    def stage_bytes(self, stage):
        return self._L.dg_stage_bytes(self._h, int(stage))


def peak_fma(precision="fp64"):
    """Measured FMA throughput of the current device in flop/s (dg_peak_fma)."""
    L = load()
    out = ctypes.c_double(0.0)
    s = L.dg_peak_fma(DG_FP32 if precision in ("fp32", DG_FP32) else DG_FP64, ctypes.byref(out))
    if s != DG_OK:
        raise DGError(s, L.dg_last_error(None).decode())
    return out.value


def totals_noalloc(u, eq="euler", dim=2, n=(64, 64), box=(1.0, 1.0, 1.0), stream=None):
    """Conservation totals of a caller-held device state (torch CUDA tensor,
    interchange layout) without any device allocation by the library."""
    L = load()
    cfg = make_config(eq, dim, n, box)
    nv = num_totals(cfg.eq, dim)
    out = np.zeros(nv)
    st = _current_stream() if stream is None else ctypes.c_void_p(stream)
    s = L.dg_totals_noalloc(ctypes.byref(cfg), ctypes.c_void_p(u.data_ptr()),
                            out.ctypes.data_as(ctypes.c_void_p), 0, st)
    if s != DG_OK:
        raise DGError(s, L.dg_last_error(None).decode())
    return out


_ROLLOUT = None


def _rollout_fn():
    global _ROLLOUT
    if _ROLLOUT is None:
        import torch

        class DGRollout(torch.autograd.Function):
            """u_T = nsteps GPU DG steps from u_0 (interchange layout, float64 CUDA
            tensor).  The forward pass records the trajectory (checkpoints every
            cfg.ckpt_every steps and the time steps, which are then held fixed);
            the backward pass is the checkpointed adjoint of the library."""

            @staticmethod
            def forward(ctx, u0, solver, nsteps, dt):
                solver.set_state(u0.detach().contiguous())
                solver.record(nsteps, dt)
                ctx.solver = solver
                ctx.generation = solver.record_generation()
                return solver.get_state(device=u0.device)

            @staticmethod
            def backward(ctx, g):
                # the solver keeps one recording: another rollout, a set_state or a
                # step since this forward pass has replaced or ended it
                if ctx.solver.record_generation() != ctx.generation:
                    raise RuntimeError(
                        "the solver's recorded trajectory changed after this rollout's "
                        "forward pass (another rollout, set_state or step on the same "
                        "solver); run backward before reusing the solver, or give each "
                        "rollout its own solver")
                return ctx.solver.adjoint(g.contiguous()), None, None, None

        _ROLLOUT = DGRollout
    return _ROLLOUT


def rollout(u0, solver, nsteps, dt=0.0):
    """Differentiable rollout: gradients of an objective of u_T flow back to u_0."""
    return _rollout_fn().apply(u0, solver, nsteps, dt)


def batch(configs, stream=None):
    return DGSolver(configs=configs, stream=stream)
