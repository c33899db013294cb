"""Differentiable radiation runs: torch.autograd around the C ABI's forward
step and its hand-written adjoint (rt_step / rt_adjoint_step).

RTRun maps (initial intensities I0, per-cell absorption opacity kappa_a) to
the intensities after n_steps steps, with kappa_P = kappa_J = kappa_a and the
rest of the gas state fixed by the solver's problem.  The forward pass keeps
a checkpoint (I, e, m) every `every` steps; the backward pass recomputes each
segment from its checkpoint, storing the segment's step inputs on the device,
and runs the adjoint steps in reverse.  Gradients come back for I0 and
kappa_a.  All arithmetic runs in the CUDA library; this module moves tensors.
"""
import numpy as np
import torch


class RTRun(torch.autograd.Function):
    @staticmethod
    def forward(ctx, I0, kappa, solver, gas, n_steps, dt, every):
        """gas: dict of host float64 arrays rho, e, m, kappa_s (caller order)."""
        k = kappa.detach().to("cpu", torch.float64).numpy()
        solver.set_gas(gas["rho"], gas["e"], gas["m"], k, k, gas["kappa_s"])
        solver.set_intensity(I0.detach().to("cuda", solver.tdtype).contiguous())
        checkpoints = []
        for n in range(n_steps):
            if n % every == 0:
                e, m = solver.gas_device()
                checkpoints.append((n, solver.get_intensity(device=True), e, m))
            solver.step(dt)
        out = solver.get_intensity(device=True)
        ctx.solver, ctx.gas, ctx.k, ctx.n_steps, ctx.dt, ctx.every = solver, gas, k, n_steps, dt, every
        ctx.checkpoints = checkpoints
        ctx.kappa_device, ctx.kappa_dtype = kappa.device, kappa.dtype
        ctx.I0_device, ctx.I0_dtype = I0.device, I0.dtype
        ctx.final = (out.clone(),) + solver.gas_device()
        return out

    @staticmethod
    def backward(ctx, grad_out):
        s, gas, k = ctx.solver, ctx.gas, ctx.k
        N = s.N
        lam_I = grad_out.to("cuda", s.tdtype).contiguous()
        lam_e = torch.zeros(N, dtype=torch.float64, device="cuda")
        lam_m = torch.zeros((N, 3), dtype=torch.float64, device="cuda")
        gP = torch.zeros(N, dtype=torch.float64, device="cuda")
        gJ = torch.zeros(N, dtype=torch.float64, device="cuda")
        for n0, I, e, m in reversed(ctx.checkpoints):
            n1 = min(n0 + ctx.every, ctx.n_steps)
            s.set_gas_energy(e, m)  # the checkpoint, on the device
            s.set_intensity(I)
            inputs = []
            for _ in range(n0, n1):
                ee, mm = s.gas_device()
                inputs.append((s.get_intensity(device=True), ee, mm))
                s.step(ctx.dt)
            for I_n, e_n, m_n in reversed(inputs):
                lam_I, lam_e, lam_m = s.adjoint_step(ctx.dt, I_n, e_n, m_n, lam_I, lam_e, lam_m,
                                                     gP, gJ)
        # leave the solver in the state the forward pass ended in
        I_f, e_f, m_f = ctx.final
        s.set_gas_energy(e_f, m_f)
        s.set_intensity(I_f)
        grad_I0 = lam_I.to(ctx.I0_device, ctx.I0_dtype)
        grad_kappa = (gP + gJ).to(ctx.kappa_device, ctx.kappa_dtype)
        return grad_I0, grad_kappa, None, None, None, None, None


def run(solver, I0, kappa, gas, n_steps, dt, every=8):
    """Differentiable n_steps run; see RTRun."""
    return RTRun.apply(I0, kappa, solver, gas, int(n_steps), float(dt), int(every))


def outflow_weights(prob, axis=0):
    """dL/dI of the outgoing flux through the upper face of `axis`: for every
    face from an interior cell into a boundary-layer cell of that face,
    A_f 4 pi w_a cbar max(n_a . n_f, 0).  Returns [N][A] float64."""
    m = prob.mesh
    ix = m.lattice_index()[axis]
    bnd = (prob.kind == 1) & (ix == m.n[axis] - 1)
    i, j = m.face_cells[:, 0], m.face_cells[:, 1]
    g = np.zeros((prob.n_cells, prob.n_angles))
    mu = m.face_normal @ prob.dirs.T  # [Nf][A], i -> j
    base = m.face_area[:, None] * 4 * np.pi * prob.weights[None, :] * prob.cbar
    sel = (prob.kind[i] != 1) & bnd[j]
    np.add.at(g, i[sel], base[sel] * np.maximum(mu[sel], 0.0))
    sel = (prob.kind[j] != 1) & bnd[i]
    np.add.at(g, j[sel], base[sel] * np.maximum(-mu[sel], 0.0))
    return g
