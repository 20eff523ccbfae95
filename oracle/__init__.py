"""CPU oracle of the P1 centroidal-Taylor DG step -- TEST INFRASTRUCTURE.

numpy/ctypes front end of ``dg_oracle.cpp``: a plain, slow, float64 statement
of one SSP-RK2 step of the discontinuous Galerkin scheme of Mocz et al. (2013),
Sec. 2 (weak form, Taylor basis, divergence-free magnetic basis, exact/HLLD
Riemann solvers, min/max limiter).  Only ``tests/``, ``__graft_entry__.smoke()``
and the CPU-baseline leg of ``bench.py`` may import this package; the product
path never does and shares no code with it.

Arrays are float64 in the interchange layout ``[plane, nz, ny, nx]`` (2D:
``[plane, ny, nx]``).
"""
import ctypes
import os

import numpy as np

from . import build as _build

EULER, MHD = 0, 1
EXACT, HLLD = 0, 1
FLAG_NONPHYS, FLAG_VACUUM, FLAG_NEWTON, FLAG_UNSUPPORTED = 1, 2, 4, 8


class _Cfg(ctypes.Structure):
    _fields_ = [("eq", ctypes.c_int), ("dim", ctypes.c_int), ("nx", ctypes.c_int),
                ("ny", ctypes.c_int), ("nz", ctypes.c_int), ("limiter", ctypes.c_int),
                ("riemann", ctypes.c_int), ("pad", ctypes.c_int), ("dx", ctypes.c_double),
                ("dy", ctypes.c_double), ("dz", ctypes.c_double), ("gamma", ctypes.c_double)]


_lib = None


def lib():
    global _lib
    if _lib is None:
        path = _build.build()
        L = ctypes.CDLL(path)
        P = ctypes.POINTER
        d, i = ctypes.c_double, ctypes.c_int
        pd = P(d)
        pc = P(_Cfg)
        L.oracle_nplanes.argtypes = [pc]
        L.oracle_limit.argtypes = [pc, pd, pd]
        L.oracle_rhs.argtypes = [pc, pd, pd]
        L.oracle_step.argtypes = [pc, pd, pd, d]
        L.oracle_cfl_dt.argtypes = [pc, pd, d, P(i)]
        L.oracle_cfl_dt.restype = d
        L.oracle_run.argtypes = [pc, pd, pd, i, d, d, pd]
        L.oracle_mh_step.argtypes = [pc, pd, pd, d, i]
        L.oracle_mh_run.argtypes = [pc, pd, pd, i, d, d, i, pd]
        L.oracle_prim_rates.argtypes = [pd, pd, i, d, pd]
        L.oracle_prim_rates.restype = None
        L.oracle_tangent_step.argtypes = [pc, pd, pd, pd, pd, d]
        L.oracle_tangent_rhs.argtypes = [pc, pd, pd, pd, pd]
        L.oracle_tangent_limit.argtypes = [pc, pd, pd, pd, pd]
        L.oracle_riemann.argtypes = [i, pd, pd, i, d, pd]
        L.oracle_exact_sample.argtypes = [pd, pd, d, i, pd, pd, pd]
        L.oracle_phys_flux.argtypes = [pd, i, d, pd]
        L.oracle_phys_flux.restype = None
        L.oracle_eval.argtypes = [pc, pd, ctypes.c_long, pd, pd]
        L.oracle_eval.restype = None
        L.oracle_mass_matrices.argtypes = [pc, pd, pd]
        L.oracle_mass_matrices.restype = None
        L.oracle_totals.argtypes = [pc, pd, pd]
        L.oracle_totals.restype = None
        L.oracle_divb.argtypes = [pc, pd, pd]
        L.oracle_divb.restype = None
        _lib = L
    return _lib


def _p(a):
    return a.ctypes.data_as(ctypes.POINTER(ctypes.c_double))


class Problem:
    """Grid and physics of one periodic box (cell sizes dx, dy[, dz])."""

    def __init__(self, eq, dim, n, box=(1.0, 1.0, 1.0), gamma=5.0 / 3.0, limiter=1,
                 riemann=None):
        self.eq, self.dim = eq, dim
        self.n = tuple(int(v) for v in n) + (1,) * (3 - len(n))
        if dim == 2:
            self.n = (self.n[0], self.n[1], 1)
        self.box = tuple(box) + (1.0,) * (3 - len(box))
        self.gamma = float(gamma)
        self.limiter = int(limiter)
        self.riemann = (HLLD if eq == MHD else EXACT) if riemann is None else riemann
        self.h = tuple(self.box[a] / self.n[a] for a in range(3))
        c = _Cfg()
        c.eq, c.dim = eq, dim
        c.nx, c.ny, c.nz = self.n
        c.limiter, c.riemann = self.limiter, self.riemann
        c.dx, c.dy, c.dz = self.h
        c.gamma = self.gamma
        self._c = c
        self.nplanes = lib().oracle_nplanes(ctypes.byref(c))

    @property
    def shape(self):
        if self.dim == 2:
            return (self.nplanes, self.n[1], self.n[0])
        return (self.nplanes, self.n[2], self.n[1], self.n[0])

    def _chk(self, u):
        u = np.ascontiguousarray(u, dtype=np.float64)
        assert u.shape == self.shape, (u.shape, self.shape)
        return u

    def step(self, u, dt):
        """One SSP-RK2 step with time step dt; returns (u_new, flags)."""
        u = self._chk(u)
        out = np.empty_like(u)
        f = lib().oracle_step(ctypes.byref(self._c), _p(u), _p(out), float(dt))
        return out, f

    def run(self, u, nsteps, cfl=0.3, dt=0.0):
        """nsteps steps (Courant time step unless dt > 0); returns (u, dts, flags)."""
        u = self._chk(u)
        out = np.empty_like(u)
        dts = np.zeros(max(nsteps, 1))
        f = lib().oracle_run(ctypes.byref(self._c), _p(u), _p(out), int(nsteps), float(cfl),
                             float(dt), _p(dts))
        return out, dts[:nsteps], f

    def mh_step(self, u, dt, face_points=1):
        """One MUSCL-Hancock step (Sec. 2.4) with time step dt; face_points 1 = the
        face-centroid flux of eq. `GalerkUpdate`, 2 = the Gauss rule of the RK step."""
        u = self._chk(u)
        out = np.empty_like(u)
        f = lib().oracle_mh_step(ctypes.byref(self._c), _p(u), _p(out), float(dt),
                                 int(face_points))
        return out, f

    def mh_run(self, u, nsteps, cfl=0.3, dt=0.0, face_points=1):
        """nsteps MUSCL-Hancock steps (Courant time step unless dt > 0)."""
        u = self._chk(u)
        out = np.empty_like(u)
        dts = np.zeros(max(nsteps, 1))
        f = lib().oracle_mh_run(ctypes.byref(self._c), _p(u), _p(out), int(nsteps), float(cfl),
                                float(dt), int(face_points), _p(dts))
        return out, dts[:nsteps], f

    def limit(self, u):
        u = self._chk(u)
        out = np.empty_like(u)
        f = lib().oracle_limit(ctypes.byref(self._c), _p(u), _p(out))
        return out, f

    def rhs(self, u):
        u = self._chk(u)
        out = np.empty_like(u)
        f = lib().oracle_rhs(ctypes.byref(self._c), _p(u), _p(out))
        return out, f

    def cfl_dt(self, u, cfl=0.3):
        u = self._chk(u)
        fl = ctypes.c_int(0)
        dt = lib().oracle_cfl_dt(ctypes.byref(self._c), _p(u), float(cfl), ctypes.byref(fl))
        return dt, fl.value

    def tangent_step(self, u, du, dt):
        """(step(u), J du) with the time step held fixed."""
        u = self._chk(u)
        du = self._chk(du)
        out, dout = np.empty_like(u), np.empty_like(u)
        f = lib().oracle_tangent_step(ctypes.byref(self._c), _p(u), _p(du), _p(out), _p(dout),
                                      float(dt))
        return out, dout, f

    def tangent_rhs(self, u, du):
        u = self._chk(u)
        du = self._chk(du)
        out, dout = np.empty_like(u), np.empty_like(u)
        f = lib().oracle_tangent_rhs(ctypes.byref(self._c), _p(u), _p(du), _p(out), _p(dout))
        return out, dout, f

    def tangent_limit(self, u, du):
        u = self._chk(u)
        du = self._chk(du)
        out, dout = np.empty_like(u), np.empty_like(u)
        f = lib().oracle_tangent_limit(ctypes.byref(self._c), _p(u), _p(du), _p(out), _p(dout))
        return out, dout, f

    def eval(self, u, cell, x):
        u = self._chk(u)
        x = np.ascontiguousarray(np.asarray(x, dtype=np.float64).reshape(3))
        U = np.zeros(8)
        lib().oracle_eval(ctypes.byref(self._c), _p(u), int(cell), _p(x), _p(U))
        return U

    def mass_matrices(self):
        """Taylor-basis and magnetic-basis mass matrices (the magnetic one 5x5 in
        2D, 11x11 for 3D MHD)."""
        MT, MB = np.zeros(16), np.zeros(121)
        lib().oracle_mass_matrices(ctypes.byref(self._c), _p(MT), _p(MB))
        k = self.dim + 1
        nb = 11 if (self.eq == MHD and self.dim == 3) else 5
        return MT[: k * k].reshape(k, k), MB[: nb * nb].reshape(nb, nb)

    def totals(self, u):
        u = self._chk(u)
        nv = (4 if self.dim == 2 else 5) + (self.dim if self.eq == MHD else 0)
        out = np.zeros(nv)
        lib().oracle_totals(ctypes.byref(self._c), _p(u), _p(out))
        return out

    def divb(self, u):
        u = self._chk(u)
        out = np.zeros(self.n[0] * self.n[1] * self.n[2])
        lib().oracle_divb(ctypes.byref(self._c), _p(u), _p(out))
        return out.reshape(self.shape[1:])


def riemann(kind, UL, UR, d, gamma):
    UL = np.ascontiguousarray(UL, dtype=np.float64)
    UR = np.ascontiguousarray(UR, dtype=np.float64)
    F = np.zeros(8)
    f = lib().oracle_riemann(int(kind), _p(UL), _p(UR), int(d), float(gamma), _p(F))
    return F, f


def exact_sample(WL, WR, gamma, xi):
    """Exact 1D Euler Riemann solution (rho, u, p) at speeds xi; also (p*, u*)."""
    WL = np.ascontiguousarray(WL, dtype=np.float64)
    WR = np.ascontiguousarray(WR, dtype=np.float64)
    xi = np.ascontiguousarray(np.atleast_1d(xi), dtype=np.float64)
    W = np.zeros((xi.size, 3))
    star = np.zeros(2)
    f = lib().oracle_exact_sample(_p(WL), _p(WR), float(gamma), xi.size, _p(xi), _p(W),
                                  _p(star))
    return W, star, f


def phys_flux(U, d, gamma):
    U = np.ascontiguousarray(U, dtype=np.float64)
    F = np.zeros(8)
    lib().oracle_phys_flux(_p(U), int(d), float(gamma), _p(F))
    return F


def prim_rates(W, dW, dim, gamma):
    """dW/dt = -sum_d A_d(W) dW/dx_d (primitive form used by the MUSCL-Hancock
    prediction); W (8,), dW (8, 3)."""
    W = np.ascontiguousarray(W, dtype=np.float64)
    dW = np.ascontiguousarray(dW, dtype=np.float64).reshape(8, 3)
    out = np.zeros(8)
    lib().oracle_prim_rates(_p(W), _p(dW), int(dim), float(gamma), _p(out))
    return out
