"""Small hand-made problems for the oracle pins and the GPU parity tests.

Built only from the input module (meshes, angle sets, Problem records);
no arithmetic of the radiation method lives here.
"""
import numpy as np

from paper_2002_08377_gb300.inputs import Problem, build_mesh, level_symmetric


def make(n=(4, 4, 4), order=6, jitter=0.25, seed=7, cbar=10.0, c=10.0, a_rad=1.0,
         gamma_gas=5.0 / 3.0, r_gas=1.0, cfl=0.3, rho=1.0, T=1.0, v=(0.0, 0.0, 0.0),
         kP=1.0, kJ=1.0, kS=0.0, J0=None, q0=None, w=None, steps=10):
    mesh = build_mesh(n, jitter=jitter, seed=seed)
    if w is not None:
        mesh.face_w = np.ascontiguousarray(np.broadcast_to(np.asarray(w, float), (mesh.n_faces, 3)))
    dirs, wt = level_symmetric(order)
    N, A = mesh.n_cells, dirs.shape[0]

    def full(x):
        x = np.asarray(x, float)
        return np.ascontiguousarray(np.broadcast_to(x, (N,)).copy()) if x.ndim == 0 else x.copy()

    rho = full(rho)
    T = full(T)
    vv = np.ascontiguousarray(np.broadcast_to(np.asarray(v, float), (N, 3)).copy())
    m = rho[:, None] * vv
    e = rho * r_gas * T / (gamma_gas - 1.0) + 0.5 * np.sum(m * m, axis=1) / rho
    J0 = full(a_rad * T ** 4 / (4 * np.pi) if J0 is None else J0)
    q0 = np.ones(A) if q0 is None else np.asarray(q0, float)
    return Problem("custom", mesh, dirs, wt, cbar, c, a_rad, gamma_gas, r_gas, cfl, steps,
                   rho, e, m, full(kP), full(kJ), full(kS), np.zeros(N, np.uint8), np.zeros(N),
                   np.zeros(N), np.zeros(N), np.full(N, -1, np.int32), np.zeros((1, A)), J0, q0)


def randomise(prob, seed=11, v_scale=0.05, aniso=0.5, kinds=True):
    """Random opacities, velocities, anisotropic intensities and a few
    boundary / emitter cells, for conservation and parity tests."""
    rng = np.random.default_rng(seed)
    N, A = prob.n_cells, prob.n_angles
    prob.kappa_P = np.exp(rng.uniform(np.log(0.1), np.log(10.0), N))
    prob.kappa_J = prob.kappa_P * rng.uniform(0.5, 2.0, N)
    prob.kappa_s = np.exp(rng.uniform(np.log(0.01), np.log(5.0), N))
    v = rng.uniform(-1, 1, (N, 3)) * v_scale * prob.c
    T = rng.uniform(0.5, 2.0, N)
    prob.m = np.ascontiguousarray(prob.rho[:, None] * v)
    prob.e = prob.rho * prob.r_gas * T / (prob.gamma_gas - 1.0) + 0.5 * np.sum(prob.m ** 2, 1) / prob.rho
    I = prob.a_rad * rng.uniform(0.2, 3.0, (N, 1)) / (4 * np.pi) * (1 + aniso * rng.uniform(-1, 1, (N, A)))
    # store I exactly as J0 x q0 is impossible for a random field: keep it in extra
    prob.extra["I_init"] = np.ascontiguousarray(I)
    prob.initial_intensity = lambda dtype=np.float64, _I=I: np.ascontiguousarray(_I.astype(dtype))
    if kinds:
        kind = np.zeros(N, np.uint8)
        cells = rng.permutation(N)
        nb = max(1, N // 10)
        bc = cells[:nb]
        em = cells[nb:nb + max(1, N // 20)]
        kind[bc] = 1
        kind[em] = 2
        prob.kind = kind
        prob.tau = np.where(rng.uniform(size=N) < 0.5, 0.0, rng.uniform(0.0, 1.0, N))
        prob.I0 = rng.uniform(0.0, 1.0, (3, A))
        prob.bc_row = np.where(kind == 1, rng.integers(0, 3, N), -1).astype(np.int32)
        prob.emit_rate = np.where(kind == 2, rng.uniform(1.0, 20.0, N), 0.0)
        prob.I_src = np.where(kind == 2, rng.uniform(0.5, 2.0, N), 0.0)
    return prob


def grouped(prob, group_w, scale_P=None, scale_J=None, scale_S=None, I_group=None):
    """The problem with len(group_w) frequency groups: group j's opacities are
    the cell's times scale_*[j] (1 if None), its initial intensities the
    problem's times I_group[j] (1 if None), its boundary rows the problem's."""
    G = len(group_w)
    N, A = prob.n_cells, prob.n_angles
    one = np.ones(G)
    sP, sJ, sS = (np.asarray(x if x is not None else one, float) for x in (scale_P, scale_J, scale_S))
    prob.n_groups = G
    prob.group_w = np.asarray(group_w, float)
    prob.kappa_P = np.ascontiguousarray(prob.kappa_P[:, None] * sP[None, :])
    prob.kappa_J = np.ascontiguousarray(prob.kappa_J[:, None] * sJ[None, :])
    prob.kappa_s = np.ascontiguousarray(prob.kappa_s[:, None] * sS[None, :])
    I = prob.initial_intensity()
    ig = np.asarray(I_group if I_group is not None else one, float)
    Ig = np.ascontiguousarray(np.concatenate([I * ig[j] for j in range(G)], axis=1))
    prob.initial_intensity = lambda dtype=np.float64, _I=Ig: np.ascontiguousarray(_I.astype(dtype))
    prob.I0 = np.ascontiguousarray(np.tile(prob.I0, (1, G)))
    return prob
