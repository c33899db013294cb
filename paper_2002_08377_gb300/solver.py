"""Python handle on one radiation state of the C ABI (include/rt.h).

Argument marshalling only: every step of the method runs in the CUDA
library.  PyTorch supplies the CUDA stream and device tensors for the
on-device I/O paths; numpy arrays go through the host paths.
"""
import ctypes

import numpy as np

from . import capi

try:  # torch is optional for the host-buffer paths
    import torch
except Exception:  # pragma: no cover
    torch = None


def _c(a, dt):
    return np.ascontiguousarray(np.asarray(a, dtype=dt))


class RTSolver:
    """One mesh + angle set + gas state on the current CUDA device.

    precision: "fp32" (float intensities/transport, double quartic and
    exchange) or "fp64".  float_quartic: 1 makes an fp32 state solve the
    temperature quartic in float instead (faster, float-rounded T).  hydro: 1
    lets the state evolve the gas dynamics too (hydro_step, radhydro_step).
    integrator: 0 first-order upwind step, 1 van Leer step with limited
    linear reconstruction (needs mesh.face_offset()).  plain_launches: 1
    turns off the CUDA-graph replay of run() / launch() (same kernels, same
    results; see rt_run in include/rt.h).
    """

    def __init__(self, mesh, dirs, weights, *, cbar, c, a_rad=1.0, gamma_gas=5.0 / 3.0,
                 r_gas=1.0, cfl=0.3, precision="fp32", newton_max_iter=64, integrator=0, boost=0, gcl=0,
                 beta_P=0.0, beta_J=0.0, T_ref=1.0, n_groups=1, group_w=None,
                 plain_launches=0, float_quartic=0, hydro=0, stream=None):
        if torch is None or not torch.cuda.is_available():
            raise RuntimeError("RTSolver needs a CUDA device (no CPU fallback exists)")
        self.lib = capi.load()
        self.precision = precision
        self.dtype = np.float32 if precision == "fp32" else np.float64
        self.tdtype = torch.float32 if precision == "fp32" else torch.float64
        # with frequency groups the intensities are [N][n_groups * A]
        self.N = int(mesh.n_cells)
        self.A = int(np.asarray(dirs).shape[0]) * max(1, int(n_groups))
        self.stream = stream if stream is not None else torch.cuda.current_stream()
        keep = self._keep = []

        def ptr(a, dt):
            if a is None:
                return None
            a = _c(a, dt)
            keep.append(a)
            return a.ctypes.data

        md = capi.MeshDesc()
        md.n_cells, md.n_faces = self.N, int(mesh.n_faces)
        md.n_angles = int(np.asarray(dirs).shape[0])
        md.n_groups = int(n_groups)
        md.group_w = ptr(group_w, np.float64) if int(n_groups) > 1 else None
        md.cell_volume = ptr(mesh.cell_volume, np.float64)
        md.cell_centroid = ptr(mesh.cell_centroid, np.float64)
        md.face_cells = ptr(mesh.face_cells, np.int32)
        md.face_area = ptr(mesh.face_area, np.float64)
        md.face_normal = ptr(mesh.face_normal, np.float64)
        md.face_centroid = ptr(mesh.face_centroid, np.float64)
        fw = getattr(mesh, "face_w", None)
        md.face_w = ptr(fw, np.float64) if fw is not None and np.any(fw) else None
        md.cell_face_ptr = ptr(mesh.cell_face_ptr, np.int64)
        md.cell_face_idx = ptr(mesh.cell_face_idx, np.int32)
        md.angle_dir = ptr(dirs, np.float64)
        md.angle_w = ptr(weights, np.float64)
        if integrator == capi.RT_VAN_LEER or hydro:
            md.face_offset = ptr(mesh.face_offset(), np.float64)
        pr = capi.Params(cbar, c, a_rad, gamma_gas, r_gas, cfl,
                         capi.RT_FP32 if precision == "fp32" else capi.RT_FP64, newton_max_iter,
                         int(integrator), int(boost), int(gcl), int(plain_launches), float(beta_P),
                         float(beta_J), float(T_ref), int(float_quartic), int(hydro))
        st = ctypes.c_void_p()
        code = self.lib.rt_create(ctypes.byref(md), ctypes.byref(pr),
                                  ctypes.c_void_p(self.stream.cuda_stream), ctypes.byref(st))
        self._keep = []
        if code != capi.RT_OK:
            raise capi.RTError(code, "rt_create failed (details on stderr)")
        self.state = st

    @classmethod
    def from_problem(cls, prob, precision="fp32", **kw):
        kw.setdefault("integrator", getattr(prob, "integrator", 0))
        kw.setdefault("boost", getattr(prob, "boost", 0))
        kw.setdefault("gcl", getattr(prob, "gcl", 0))
        for k, d in (("beta_P", 0.0), ("beta_J", 0.0), ("T_ref", 1.0), ("n_groups", 1),
                     ("group_w", None)):
            kw.setdefault(k, getattr(prob, k, d))
        s = cls(prob.mesh, prob.dirs, prob.weights, cbar=prob.cbar, c=prob.c, a_rad=prob.a_rad,
                gamma_gas=prob.gamma_gas, r_gas=prob.r_gas, cfl=prob.cfl, precision=precision, **kw)
        s.set_gas(prob.rho, prob.e, prob.m, prob.kappa_P, prob.kappa_J, prob.kappa_s)
        s.set_cells(prob.kind, prob.tau, prob.emit_rate, prob.I_src, prob.bc_row, prob.I0)
        s.set_intensity(prob.initial_intensity(s.dtype))
        return s

    # -------------------------------------------------------------- inputs
    def _check(self, code):
        return capi.check(self.state, code)

    def set_gas(self, rho, e, m, kappa_P, kappa_J, kappa_s):
        arrs = [_c(x, np.float64) for x in (rho, e, m, kappa_P, kappa_J, kappa_s)]
        self._check(self.lib.rt_set_gas(self.state, *[a.ctypes.data for a in arrs]))

    def set_cells(self, kind=None, tau=None, emit_rate=None, I_src=None, bc_row=None, I0=None):
        if kind is None:
            self._check(self.lib.rt_set_cells(self.state, None, None, None, None, None, 0, None))
            return
        k = _c(kind, np.uint8)
        t, er, isrc = (_c(x, np.float64) for x in (tau, emit_rate, I_src))
        br = _c(bc_row, np.int32)
        i0 = _c(I0, np.float64).reshape(-1, self.A)
        self._check(self.lib.rt_set_cells(self.state, k.ctypes.data, t.ctypes.data, er.ctypes.data,
                                          isrc.ctypes.data, br.ctypes.data, i0.shape[0],
                                          i0.ctypes.data))

    def set_intensity(self, I):
        if torch is not None and isinstance(I, torch.Tensor) and I.is_cuda:
            I = I.to(self.tdtype).contiguous()
            assert I.numel() == self.N * self.A
            self._check(self.lib.rt_set_intensity(self.state, ctypes.c_void_p(I.data_ptr()), 1))
        else:
            a = _c(I, self.dtype).reshape(self.N, self.A)
            self._check(self.lib.rt_set_intensity(self.state, a.ctypes.data, 0))

    # -------------------------------------------------------------- stepping
    def dt_limits(self):
        a, b = ctypes.c_double(), ctypes.c_double()
        self._check(self.lib.rt_dt_limits(self.state, ctypes.byref(a), ctypes.byref(b)))
        return a.value, b.value

    def step(self, dt=0.0):
        used = ctypes.c_double()
        self._check(self.lib.rt_step(self.state, float(dt), ctypes.byref(used)))
        return used.value

    def run(self, n_steps, dt=0.0):
        used = ctypes.c_double()
        self._check(self.lib.rt_run(self.state, int(n_steps), float(dt), ctypes.byref(used)))
        return used.value

    def launch(self, n_steps, dt=0.0):
        """Queue n_steps steps on the stream without waiting (see sync())."""
        used = ctypes.c_double()
        self._check(self.lib.rt_launch(self.state, int(n_steps), float(dt), ctypes.byref(used)))
        return used.value

    def sync(self):
        self._check(self.lib.rt_sync(self.state))

    def step_io(self, host_in, host_out, dt=0.0):
        """Queue one step that reads its intensities from the page-locked host
        tensor host_in and writes the result to the page-locked host tensor
        host_out (both [N][A] in the state's precision; rt_step_io).  Leave
        both untouched until sync()."""
        for t in (host_in, host_out):
            if (tuple(t.shape) != (self.N, self.A) or t.dtype != self.tdtype or not t.is_pinned()
                    or not t.is_contiguous()):
                raise ValueError("step_io wants page-locked host tensors of shape (N, A) "
                                 "in the state's precision")
        self._check(self.lib.rt_step_io(self.state, float(dt), ctypes.c_void_p(host_in.data_ptr()),
                                        ctypes.c_void_p(host_out.data_ptr())))

    # -------------------------------------------------------------- outputs
    def get_intensity(self, device=False):
        if device:
            out = torch.empty((self.N, self.A), dtype=self.tdtype, device="cuda")
            self._check(self.lib.rt_get_intensity(self.state, ctypes.c_void_p(out.data_ptr()), 1))
            return out
        out = np.empty((self.N, self.A), self.dtype)
        self._check(self.lib.rt_get_intensity(self.state, out.ctypes.data, 0))
        return out

    def gas(self):
        e, m, x = np.empty(self.N), np.empty((self.N, 3)), np.empty((self.N, 4))
        self._check(self.lib.rt_get_gas(self.state, e.ctypes.data, m.ctypes.data, x.ctypes.data, 0))
        return e, m, x

    def moments(self, device=False):
        if device:
            E = torch.empty(self.N, dtype=torch.float64, device="cuda")
            F = torch.empty((self.N, 3), dtype=torch.float64, device="cuda")
            P = torch.empty((self.N, 6), dtype=torch.float64, device="cuda")
            self._check(self.lib.rt_moments(self.state, ctypes.c_void_p(E.data_ptr()),
                                            ctypes.c_void_p(F.data_ptr()),
                                            ctypes.c_void_p(P.data_ptr()), 1))
            return E, F, P
        E, F, P = np.empty(self.N), np.empty((self.N, 3)), np.empty((self.N, 6))
        self._check(self.lib.rt_moments(self.state, E.ctypes.data, F.ctypes.data, P.ctypes.data, 0))
        return E, F, P

    def set_gas_energy(self, e, m):
        """Replace only the evolving gas (e[N], m[N][3], caller order): CUDA
        tensors stay on the device, anything else goes through the host."""
        if torch.is_tensor(e) and e.is_cuda:
            e = e.to(torch.float64).contiguous()
            m = m.to(torch.float64).contiguous()
            self._check(self.lib.rt_set_gas_energy(self.state, ctypes.c_void_p(e.data_ptr()),
                                                   ctypes.c_void_p(m.data_ptr()), 1))
            return
        e, m = _c(e, np.float64), _c(m, np.float64)
        self._check(self.lib.rt_set_gas_energy(self.state, e.ctypes.data, m.ctypes.data, 0))

    # -------------------------------------------------------------- gas dynamics
    def hydro_dt(self, cfl=0.3):
        dt = ctypes.c_double()
        self._check(self.lib.rt_hydro_dt(self.state, float(cfl), ctypes.byref(dt)))
        return dt.value

    def hydro_step(self, dt, order=2):
        self._check(self.lib.rt_hydro_step(self.state, float(dt), int(order)))

    def radhydro_step(self, dt, n_sub=1, order=2):
        """The hydro step over dt, then n_sub radiation steps of dt / n_sub."""
        used = ctypes.c_double()
        self._check(self.lib.rt_radhydro_step(self.state, float(dt), int(n_sub), int(order),
                                              ctypes.byref(used)))
        return used.value

    def density(self):
        rho = np.empty(self.N)
        self._check(self.lib.rt_get_density(self.state, rho.ctypes.data, 0))
        return rho

    def gas_device(self):
        """(e[N], m[N][3]) as float64 CUDA tensors, caller order."""
        e = torch.empty(self.N, dtype=torch.float64, device="cuda")
        m = torch.empty((self.N, 3), dtype=torch.float64, device="cuda")
        self._check(self.lib.rt_get_gas(self.state, ctypes.c_void_p(e.data_ptr()),
                                        ctypes.c_void_p(m.data_ptr()), None, 1))
        return e, m

    def adjoint_step(self, dt, I, e, m, lam_I1, lam_e1, lam_m1, grad_kP, grad_kJ):
        """Reverse of one step on CUDA tensors (caller order).  I, lam_I1 in
        the state precision; e, m, cotangents and gradients float64.  Returns
        (lam_I, lam_e, lam_m); grad_kP, grad_kJ are accumulated in place."""
        def dev(x, dt_):
            return x.to(device="cuda", dtype=dt_).contiguous()
        I, lam_I1 = dev(I, self.tdtype), dev(lam_I1, self.tdtype)
        e, m = dev(e, torch.float64), dev(m, torch.float64)
        lam_e1, lam_m1 = dev(lam_e1, torch.float64), dev(lam_m1, torch.float64)
        lam_I = torch.empty_like(I)
        lam_e, lam_m = torch.empty_like(e), torch.empty_like(m)
        assert grad_kP.is_cuda and grad_kP.dtype == torch.float64 and grad_kP.is_contiguous()
        assert grad_kJ.is_cuda and grad_kJ.dtype == torch.float64 and grad_kJ.is_contiguous()
        p = lambda t: ctypes.c_void_p(t.data_ptr())
        self._check(self.lib.rt_adjoint_step(self.state, float(dt), p(I), p(e), p(m), p(lam_I1),
                                             p(lam_e1), p(lam_m1), p(lam_I), p(lam_e), p(lam_m),
                                             p(grad_kP), p(grad_kJ), 1))
        return lam_I, lam_e, lam_m

    def totals(self):
        out = np.empty(16)
        self._check(self.lib.rt_totals(self.state, out.ctypes.data))
        return out

    def get_state(self):
        n = ctypes.c_size_t()
        self._check(self.lib.rt_get_state(self.state, None, ctypes.byref(n)))
        buf = np.empty(n.value, np.uint8)
        self._check(self.lib.rt_get_state(self.state, buf.ctypes.data, ctypes.byref(n)))
        return buf

    def set_state(self, buf):
        buf = np.ascontiguousarray(buf, np.uint8)
        self._check(self.lib.rt_set_state(self.state, buf.ctypes.data, buf.size))

    def device_bytes(self):
        n = ctypes.c_size_t()
        self._check(self.lib.rt_device_bytes(self.state, ctypes.byref(n)))
        return n.value

    def launch_count(self):
        return int(self.lib.rt_launch_count(self.state))

    def close(self):
        if getattr(self, "state", None):
            self.lib.rt_destroy(self.state)
            self.state = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass
