"""FP64 CPU oracle of the radiation step (test infrastructure).

Only tests/, __graft_entry__.smoke() and bench.py's CPU-baseline leg may
import this package.  It shares no code with the CUDA path: rt_oracle.c is
a plain loop nest written from the paper's equations; this module only
marshals numpy arrays into it.  It takes every input from the caller (a
problem object with mesh, angles, gas and cell fields) and imports nothing
from the product package.
"""
import ctypes
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "rt_oracle.c")
_LIB = os.path.join(_HERE, "liboracle.so")
_lock = threading.Lock()
_lib = None

ORC_OK, ORC_ERR_NONCONV, ORC_ERR_NONFINITE = 0, -6, -7


def build(force=False):
    """Compile rt_oracle.c (plain C, OpenMP over cells, no FMA contraction so
    that x86 and Arm hosts give the same bits)."""
    with _lock:
        if force or not os.path.exists(_LIB) or os.path.getmtime(_LIB) < os.path.getmtime(_SRC):
            tmp = _LIB + f".tmp{os.getpid()}"
            subprocess.check_call(["gcc", "-O2", "-std=c11", "-fopenmp", "-ffp-contract=off",
                                   "-shared", "-fPIC", _SRC, "-o", tmp, "-lm"])
            os.replace(tmp, _LIB)
    return _LIB


class _Problem(ctypes.Structure):
    _fields_ = [("n_cells", ctypes.c_int64), ("n_faces", ctypes.c_int64),
                ("n_angles", ctypes.c_int32), ("newton_max_iter", ctypes.c_int32),
                ("cell_volume", ctypes.c_void_p), ("face_cells", ctypes.c_void_p),
                ("face_area", ctypes.c_void_p), ("face_normal", ctypes.c_void_p),
                ("face_w", ctypes.c_void_p), ("cell_face_ptr", ctypes.c_void_p),
                ("cell_face_idx", ctypes.c_void_p), ("dir", ctypes.c_void_p),
                ("wt", ctypes.c_void_p),
                ("cbar", ctypes.c_double), ("c", ctypes.c_double), ("a_rad", ctypes.c_double),
                ("gamma_gas", ctypes.c_double), ("r_gas", ctypes.c_double),
                ("rho", ctypes.c_void_p), ("kappa_P", ctypes.c_void_p),
                ("kappa_J", ctypes.c_void_p), ("kappa_s", ctypes.c_void_p),
                ("kind", ctypes.c_void_p), ("tau", ctypes.c_void_p),
                ("emit_rate", ctypes.c_void_p), ("I_src", ctypes.c_void_p),
                ("bc_row", ctypes.c_void_p), ("I0", ctypes.c_void_p),
                ("face_offset", ctypes.c_void_p), ("boost_all_orders", ctypes.c_int32),
                ("gcl", ctypes.c_int32), ("beta_P", ctypes.c_double), ("beta_J", ctypes.c_double),
                ("T_ref", ctypes.c_double), ("n_groups", ctypes.c_int32),
                ("group_w", ctypes.c_void_p)]


def lib():
    global _lib
    if _lib is None:
        build()
        L = ctypes.CDLL(_LIB)
        P = ctypes.POINTER(_Problem)
        vp, d, i = ctypes.c_void_p, ctypes.c_double, ctypes.c_int
        L.orc_transport.argtypes = [P, d, vp, vp]
        L.orc_newton_power.argtypes = [d, d, d, d, i, ctypes.POINTER(d), ctypes.POINTER(i)]
        L.orc_newton_power.restype = i
        L.orc_gcl_volumes.argtypes = [P, d, vp]
        L.orc_moments.argtypes = [P, vp, vp, vp, vp]
        L.orc_newton.argtypes = [d, d, d, i, ctypes.POINTER(d), ctypes.POINTER(i)]
        L.orc_newton.restype = i
        L.orc_ferrari.argtypes = [d, d, d]
        L.orc_ferrari.restype = d
        L.orc_source.argtypes = [P, d, vp, vp, vp, vp, vp, ctypes.POINTER(i)]
        L.orc_source.restype = i
        L.orc_step.argtypes = [P, d, vp, vp, vp, vp, vp, ctypes.POINTER(i)]
        L.orc_step.restype = i
        L.orc_cfl_dt.argtypes = [P, d]
        L.orc_cfl_dt.restype = d
        L.orc_positivity.argtypes = [P]
        L.orc_positivity.restype = d
        L.orc_totals.argtypes = [P, vp, vp, vp, vp, vp]
        L.orc_step_range.argtypes = [P, d, vp, vp, vp, vp, vp, vp, ctypes.c_int64, ctypes.c_int64]
        L.orc_step_range.restype = i
        L.orc_transport_adjoint.argtypes = [P, d, vp, vp]
        L.orc_adjoint_step.argtypes = [P, d] + [vp] * 12
        L.orc_adjoint_step.restype = i
        L.orc_gradient.argtypes = [P, vp, i, vp]
        L.orc_transport_recon.argtypes = [P, d, vp, vp, vp, vp]
        L.orc_step_vl.argtypes = [P, d, vp, vp, vp, vp, vp, vp, vp, ctypes.POINTER(i)]
        L.orc_step_vl.restype = i
        L.orc_set_threads.argtypes = [i]
        L.orc_set_threads.restype = i
        L.orc_hllc_flux.argtypes = [d, vp, vp, vp, vp]
        L.orc_hllc_flux.restype = i
        L.orc_hydro_dt.argtypes = [P, vp, vp, vp, d]
        L.orc_hydro_dt.restype = d
        L.orc_hydro_step.argtypes = [P, d, i, vp, vp, vp, vp]
        L.orc_hydro_step.restype = i
        _lib = L
    return _lib


def _f64(x, shape=None):
    a = np.ascontiguousarray(np.asarray(x, dtype=np.float64))
    if shape is not None:
        a = a.reshape(shape)
    return a


def newton(alpha, beta, g, max_iter=64):
    """Positive root of alpha T^4 + beta T = g by the oracle's Newton."""
    T, it = ctypes.c_double(), ctypes.c_int()
    st = lib().orc_newton(float(alpha), float(beta), float(g), int(max_iter), ctypes.byref(T),
                          ctypes.byref(it))
    return st, T.value, it.value


def newton_power(alpha, k, beta, g, max_iter=64):
    """Positive root of alpha T^k + beta T = g (k >= 1): (status, T, iterations)."""
    T, it = ctypes.c_double(), ctypes.c_int()
    st = lib().orc_newton_power(float(alpha), float(k), float(beta), float(g), int(max_iter),
                                ctypes.byref(T), ctypes.byref(it))
    return st, T.value, it.value


def set_threads(n):
    """OpenMP threads of the oracle's loops from now on (n > 0); returns the
    number in effect (n <= 0 only queries it)."""
    return int(lib().orc_set_threads(int(n)))


def hllc_flux(gamma, WL, WR, n):
    """HLLC flux per unit area of (rho, m, e) through a face with unit normal
    n, primitive states W = (rho, vx, vy, vz, P) on the two sides."""
    WL, WR, n = _f64(WL), _f64(WR), _f64(n)
    F = np.empty(5)
    st = lib().orc_hllc_flux(float(gamma), WL.ctypes.data, WR.ctypes.data, n.ctypes.data,
                             F.ctypes.data)
    if st != 0:
        raise ValueError("non-positive density or pressure")
    return F


def ferrari(alpha, beta, g):
    return lib().orc_ferrari(float(alpha), float(beta), float(g))


class Oracle:
    """Oracle state for one problem: intensities I[N][A], gas e[N], m[N][3]
    and the boundary / emitter tallies ext[N][4], all float64, in the
    caller's cell numbering."""

    def __init__(self, prob, newton_max_iter=64, threads=None):
        if threads is not None:
            os.environ["OMP_NUM_THREADS"] = str(int(threads))
        m = prob.mesh
        self.prob = prob
        # frequency groups: the oracle's angle set is n_groups copies of the
        # problem's directions, group j weighted by group_w[j] (kappa arrays
        # then hold n_groups values per cell, intensities [N][n_groups * A])
        ng = int(getattr(prob, "n_groups", 1))
        dirs, wts = np.asarray(prob.dirs, np.float64), np.asarray(prob.weights, np.float64)
        if ng > 1:
            gw = np.asarray(prob.group_w, np.float64)
            dirs = np.tile(dirs, (ng, 1))
            wts = (gw[:, None] * wts[None, :]).ravel()
        self.N, self.A = m.n_cells, int(dirs.shape[0])
        keep = self._keep = {}

        def arr(name, x, dt=np.float64):
            a = np.ascontiguousarray(np.asarray(x, dtype=dt))
            keep[name] = a
            return a.ctypes.data

        p = _Problem()
        p.n_cells, p.n_faces, p.n_angles = self.N, m.n_faces, self.A
        p.newton_max_iter = newton_max_iter
        # the oracle's own copy: with the geometric conservation law it evolves
        self.vol = np.array(m.cell_volume, dtype=np.float64, copy=True)
        self._vol_next = np.empty_like(self.vol)
        p.cell_volume = self.vol.ctypes.data
        p.face_cells = arr("fc", m.face_cells, np.int32)
        p.face_area = arr("fa", m.face_area)
        p.face_normal = arr("fn", m.face_normal)
        fw = m.face_w if m.face_w is not None else np.zeros((m.n_faces, 3))
        p.face_w = arr("fw", fw)
        p.cell_face_ptr = arr("ptr", m.cell_face_ptr, np.int64)
        p.cell_face_idx = arr("idx", m.cell_face_idx, np.int32)
        p.dir = arr("dir", dirs)
        p.wt = arr("wt", wts)
        p.cbar, p.c, p.a_rad = prob.cbar, prob.c, prob.a_rad
        p.gamma_gas, p.r_gas = prob.gamma_gas, prob.r_gas
        # the oracle's own copy: it evolves with the hydro step (the radiation reads it)
        self.rho = np.array(prob.rho, dtype=np.float64, copy=True)
        keep["rho"] = self.rho
        p.rho = self.rho.ctypes.data
        p.kappa_P = arr("kP", prob.kappa_P)
        p.kappa_J = arr("kJ", prob.kappa_J)
        p.kappa_s = arr("kS", prob.kappa_s)
        p.kind = arr("kind", prob.kind, np.uint8)
        p.tau = arr("tau", prob.tau)
        p.emit_rate = arr("emit", prob.emit_rate)
        p.I_src = arr("isrc", prob.I_src)
        p.bc_row = arr("bcrow", prob.bc_row, np.int32)
        p.I0 = arr("I0", prob.I0)
        p.face_offset = arr("foff", m.face_offset())
        p.boost_all_orders = int(getattr(prob, "boost", 0))
        p.gcl = int(getattr(prob, "gcl", 0))
        p.beta_P = float(getattr(prob, "beta_P", 0.0))
        p.beta_J = float(getattr(prob, "beta_J", 0.0))
        p.T_ref = float(getattr(prob, "T_ref", 1.0))
        p.n_groups = ng
        p.group_w = arr("gw", prob.group_w) if ng > 1 else None
        self.p = p
        self.integrator = int(getattr(prob, "integrator", 0))
        self.I = _f64(prob.initial_intensity(np.float64))
        self.e = _f64(prob.e).copy()
        self.m = _f64(prob.m).copy()
        self.ext = np.zeros((self.N, 4))
        self.work = np.empty_like(self.I)
        self.last_iters = 0

    # -- single operators ------------------------------------------------
    def transport(self, dt, I=None):
        I = self.I if I is None else _f64(I)
        out = np.empty_like(I)
        lib().orc_transport(ctypes.byref(self.p), float(dt), I.ctypes.data, out.ctypes.data)
        return out

    def source(self, dt, Istar):
        Istar = _f64(Istar)
        out = np.empty_like(Istar)
        it = ctypes.c_int()
        st = lib().orc_source(ctypes.byref(self.p), float(dt), Istar.ctypes.data, out.ctypes.data,
                              self.e.ctypes.data, self.m.ctypes.data, self.ext.ctypes.data,
                              ctypes.byref(it))
        self.last_iters = it.value
        return st, out

    # -- full steps ----------------------------------------------------------
    def step(self, dt):
        """One step with the problem's integrator (first-order upwind, or
        van Leer with limited linear reconstruction)."""
        it = ctypes.c_int()
        if self.integrator == 1 and self.p.gcl:
            raise ValueError("the van Leer step is not built for changing cell volumes")
        if self.integrator == 1:
            if not hasattr(self, "_half"):
                self._half = np.empty_like(self.I)
                self._grad = np.empty((self.N, 3, self.A))
            st = lib().orc_step_vl(ctypes.byref(self.p), float(dt), self.I.ctypes.data,
                                   self.work.ctypes.data, self._half.ctypes.data,
                                   self._grad.ctypes.data, self.e.ctypes.data, self.m.ctypes.data,
                                   self.ext.ctypes.data, ctypes.byref(it))
            self.last_iters = it.value
            return st
        if self.p.gcl:
            lib().orc_gcl_volumes(ctypes.byref(self.p), float(dt), self._vol_next.ctypes.data)
        st = lib().orc_step(ctypes.byref(self.p), float(dt), self.I.ctypes.data,
                            self.work.ctypes.data, self.e.ctypes.data, self.m.ctypes.data,
                            self.ext.ctypes.data, ctypes.byref(it))
        if self.p.gcl:
            self.vol[:] = self._vol_next  # V^{n+1} becomes the volume of the next step
        self.last_iters = it.value
        return st

    def sample_step(self, dt, c0, c1, out=None):
        """Transport + source of cells [c0, c1) only, into `out` (a timing
        sample: the state is left unchanged apart from those cells' gas)."""
        if out is None:
            out = np.empty_like(self.I)
        st = lib().orc_step_range(ctypes.byref(self.p), float(dt), self.I.ctypes.data,
                                  self.work.ctypes.data, out.ctypes.data, self.e.ctypes.data,
                                  self.m.ctypes.data, self.ext.ctypes.data, int(c0), int(c1))
        return st, out

    def run(self, n_steps, dt):
        for _ in range(int(n_steps)):
            st = self.step(dt)
            if st != ORC_OK:
                return st
        return ORC_OK

    # -- hydrodynamics ---------------------------------------------------------
    def hydro_dt(self, cfl=None):
        """Courant step of the gas: cfl * min V^(1/3) / (|v| + sound speed)."""
        cfl = self.prob.cfl if cfl is None else cfl
        return lib().orc_hydro_dt(ctypes.byref(self.p), self.rho.ctypes.data, self.m.ctypes.data,
                                  self.e.ctypes.data, float(cfl))

    def hydro_step(self, dt, order=2):
        """One hydro step of (rho, m, e) in place (HLLC fluxes; order 2: the
        van Leer step with limited linear reconstruction)."""
        if self.p.gcl:
            raise ValueError("the hydro step is built for a static mesh")
        if not hasattr(self, "_hwork"):
            self._hwork = np.empty(36 * self.N + 5 * self.p.n_faces)
        st = lib().orc_hydro_step(ctypes.byref(self.p), float(dt), int(order),
                                  self.rho.ctypes.data, self.m.ctypes.data, self.e.ctypes.data,
                                  self._hwork.ctypes.data)
        if st != 0:
            raise ValueError("the hydro step produced a non-positive density or pressure")

    def radhydro_step(self, dt, n_sub=1, order=2):
        """One radiation-hydrodynamics step: the hydro step over dt, then n_sub
        radiation steps (transport + implicit source with the updated gas) of
        dt / n_sub each."""
        self.hydro_step(dt, order)
        for _ in range(int(n_sub)):
            st = self.step(dt / n_sub)
            if st != ORC_OK:
                return st
        return ORC_OK

    # -- diagnostics -----------------------------------------------------------
    def gradient(self, I=None, limit=True):
        """[N, 3, A] least-squares gradients of I (Barth-Jespersen limited)."""
        I = self.I if I is None else _f64(I)
        g = np.empty((self.N, 3, self.A))
        lib().orc_gradient(ctypes.byref(self.p), I.ctypes.data, int(bool(limit)), g.ctypes.data)
        return g

    def transport_recon(self, dt, I, Ih, grad):
        """Transport of I over dt with upwind face values reconstructed from
        (Ih, grad)."""
        I, Ih, grad = _f64(I), _f64(Ih), _f64(grad)
        out = np.empty_like(I)
        lib().orc_transport_recon(ctypes.byref(self.p), float(dt), I.ctypes.data, Ih.ctypes.data,
                                  grad.ctypes.data, out.ctypes.data)
        return out

    def moments(self, I=None):
        I = self.I if I is None else _f64(I)
        E = np.empty(self.N)
        F = np.empty((self.N, 3))
        P = np.empty((self.N, 6))
        lib().orc_moments(ctypes.byref(self.p), I.ctypes.data, E.ctypes.data, F.ctypes.data,
                          P.ctypes.data)
        return E, F, P

    def totals(self):
        out = np.empty(16)
        lib().orc_totals(ctypes.byref(self.p), self.I.ctypes.data, self.e.ctypes.data,
                         self.m.ctypes.data, self.ext.ctypes.data, out.ctypes.data)
        return out

    def cfl_dt(self, cfl=None):
        cfl = self.prob.cfl if cfl is None else cfl
        return lib().orc_cfl_dt(ctypes.byref(self.p), float(cfl))

    def positivity(self):
        return lib().orc_positivity(ctypes.byref(self.p))

    def transport_adjoint(self, dt, lam):
        lam = _f64(lam)
        out = np.empty_like(lam)
        lib().orc_transport_adjoint(ctypes.byref(self.p), float(dt), lam.ctypes.data,
                                    out.ctypes.data)
        return out

    def adjoint_step(self, dt, I, e, m, lI1, le1, lm1, gP, gJ):
        """Cotangents of the step's inputs (I, e, m) from those of its
        outputs; gP, gJ (float64 [N]) accumulate dL/dkappa_P, dL/dkappa_J."""
        I, e, m = _f64(I), _f64(e), _f64(m)
        lI1, le1, lm1 = _f64(lI1), _f64(le1), _f64(lm1)
        lI, le, lm = np.empty_like(I), np.empty_like(e), np.empty_like(m)
        work = np.empty(2 * I.size)
        st = lib().orc_adjoint_step(ctypes.byref(self.p), float(dt), I.ctypes.data, e.ctypes.data,
                                    m.ctypes.data, lI1.ctypes.data, le1.ctypes.data,
                                    lm1.ctypes.data, lI.ctypes.data, le.ctypes.data,
                                    lm.ctypes.data, gP.ctypes.data, gJ.ctypes.data,
                                    work.ctypes.data)
        if st != ORC_OK:
            raise ValueError("the oracle's adjoint reverses the grey first-order transformation "
                             "on fixed cell volumes with constant opacities only")
        return lI, le, lm

    def temperature(self):
        """Gas temperature from the conserved gas state."""
        pr = self.prob
        kin = 0.5 * np.sum(self.m ** 2, axis=1) / pr.rho
        return (self.e - kin) * (pr.gamma_gas - 1.0) / (pr.rho * pr.r_gas)
