"""CPU pins of the oracle's limited linear reconstruction and van Leer step.

Sec. 2 integrates with a van Leer half step and Sec. 2.2 reconstructs the
face state linearly with a limiter; the paper defers the gradient estimate
and the limiter to its hydrodynamics code, so the oracle takes a
least-squares gradient and a Barth-Jespersen limiter (readings).  These tests
check them against geometry identities, exactness on linear fields, the
limiter's bound, conservation, and the orders of accuracy a second-order
scheme must show.
"""
import numpy as np

import oracle
from paper_2002_08377_gb300.inputs import Problem, build_mesh, level_symmetric
from tests._problems import make, randomise


def _quasi1d(N, jitter=0.1, seed=5):
    h = 1.0 / N
    return build_mesh((N, 3, 3), box=(1.0, 3 * h, 3 * h), jitter=jitter, seed=seed)


def _free_problem(mesh, order=2, integrator=0, I=None):
    """No opacity, gas at rest: the source step is the identity."""
    dirs, wt = level_symmetric(order)
    n, A = mesh.n_cells, dirs.shape[0]
    z = np.zeros(n)
    rho = np.ones(n)
    prob = Problem("free", mesh, dirs, wt, 1.0, 1.0, 1.0, 5.0 / 3.0, 1.0, 0.3, 0, rho, rho * 1.5,
                   np.zeros((n, 3)), z.copy(), z.copy(), z.copy(), np.zeros(n, np.uint8), z.copy(),
                   z.copy(), z.copy(), np.full(n, -1, np.int32), np.zeros((1, A)), np.ones(n),
                   np.ones(A), integrator=integrator)
    if I is not None:
        prob.initial_intensity = lambda dtype=np.float64, _I=I: np.ascontiguousarray(_I.astype(dtype))
    return prob


def test_face_offsets_satisfy_the_divergence_identity():
    """For a polyhedron with planar faces, sum_f A_f n_f (x_f - x_c)^T = V_c I
    (Gauss' theorem applied to grad x); every cell, from both sides of every
    face, including faces across the periodic boundary."""
    m = build_mesh((5, 4, 6), jitter=0.25, seed=3)
    off = m.face_offset()
    S = np.zeros((m.n_cells, 3, 3))
    for f in range(m.n_faces):
        i, j = m.face_cells[f]
        an = m.face_area[f] * m.face_normal[f]
        S[i] += np.outer(an, off[f, 0])
        S[j] -= np.outer(an, off[f, 1])
    target = m.cell_volume[:, None, None] * np.eye(3)
    assert np.abs(S - target).max() < 1e-12 * m.cell_volume.max()


def test_gradient_is_exact_for_linear_fields():
    """Unlimited least-squares gradients of I_a = alpha_a + beta_a . x are
    beta_a in every cell none of whose faces crosses the periodic boundary."""
    m = build_mesh((7, 6, 8), jitter=0.25, seed=4)
    prob = _free_problem(m, order=4)
    A = prob.n_angles
    rng = np.random.default_rng(0)
    beta = rng.standard_normal((A, 3))
    I = rng.standard_normal(A)[None, :] + m.cell_centroid @ beta.T
    g = oracle.Oracle(prob).gradient(I, limit=False)
    crosses = np.zeros(m.n_cells, bool)
    per = np.any(m.face_shift != 0, axis=1)
    crosses[m.face_cells[per, 0]] = True
    crosses[m.face_cells[per, 1]] = True
    inner = ~crosses
    assert inner.sum() > 50
    err = np.abs(g[inner] - beta.T[None, :, :]).max()
    assert err < 1e-11 * np.abs(beta).max(), err


def test_limited_face_values_stay_within_the_neighbour_range():
    """Barth-Jespersen: I_c + g . (x_f - x_c) lies within [min, max] of I_c
    and its face neighbours on every face (random field)."""
    m = build_mesh((6, 5, 7), jitter=0.25, seed=6)
    prob = _free_problem(m, order=4)
    rng = np.random.default_rng(1)
    I = rng.uniform(0.5, 2.0, (m.n_cells, prob.n_angles))
    g = oracle.Oracle(prob).gradient(I, limit=True)
    off = m.face_offset()
    lo, hi = I.copy(), I.copy()
    for f in range(m.n_faces):
        i, j = m.face_cells[f]
        lo[i] = np.minimum(lo[i], I[j]); hi[i] = np.maximum(hi[i], I[j])
        lo[j] = np.minimum(lo[j], I[i]); hi[j] = np.maximum(hi[j], I[i])
    tol = 1e-12
    for f in range(m.n_faces):
        i, j = m.face_cells[f]
        for c, d in ((i, off[f, 0]), (j, off[f, 1])):
            v = I[c] + d @ g[c]
            assert np.all(v <= hi[c] + tol) and np.all(v >= lo[c] - tol)
    # the limiter is active somewhere and leaves gradients unchanged elsewhere
    g0 = oracle.Oracle(prob).gradient(I, limit=False)
    scale = np.linalg.norm(g, axis=1) / np.maximum(np.linalg.norm(g0, axis=1), 1e-300)
    assert scale.min() < 0.5 and np.isclose(scale.max(), 1.0)


def test_reconstructed_transport_is_conservative_and_reduces_to_upwind():
    prob = randomise(make(n=(5, 4, 6), order=4, w=(0.2, -0.1, 0.0)), seed=3)
    o = oracle.Oracle(prob)
    dt = 0.5 / o.positivity()
    rng = np.random.default_rng(2)
    I = o.I
    Ih = I * rng.uniform(0.9, 1.1, I.shape)
    # zero gradients: piecewise-constant upwinding of Ih, applied to I
    zero = np.zeros((prob.n_cells, 3, prob.n_angles))
    pc = o.transport(dt, Ih) - Ih + I
    assert np.abs(o.transport_recon(dt, I, Ih, zero) - pc).max() < 1e-13 * np.abs(I).max()
    # any gradients: every face flux leaves one cell and enters the other
    g = rng.standard_normal(zero.shape) * np.abs(I).mean()
    Is = o.transport_recon(dt, I, Ih, g)
    V = prob.mesh.cell_volume
    assert abs(np.sum(V[:, None] * (Is - I))) < 1e-13 * np.sum(V[:, None] * np.abs(I))


def _advection_error(N, integrator, t_end=0.25):
    m = _quasi1d(N)
    x = m.cell_centroid[:, 0]
    dirs, _ = level_symmetric(2)
    I0 = 1 + 0.5 * np.sin(2 * np.pi * x)[:, None] * np.ones(len(dirs))
    o = oracle.Oracle(_free_problem(m, integrator=integrator, I=I0))
    steps = int(np.ceil(t_end / o.cfl_dt()))
    assert o.run(steps, t_end / steps) == 0
    exact = 1 + 0.5 * np.sin(2 * np.pi * (x[:, None] - dirs[None, :, 0] * t_end))
    return np.mean(np.abs(o.I - exact))


def test_van_leer_is_higher_order_on_smooth_advection():
    """A sine wave carried along x by every ordinate (no opacity) on a quasi-
    1-D jittered Voronoi mesh: the first-order step converges at order 1, the
    van Leer step with limited reconstruction at order > 1.3 (the limiter
    clips the extrema) and far below the first-order error."""
    Ns = (32, 64, 128)
    pc = np.array([_advection_error(N, 0) for N in Ns])
    vl = np.array([_advection_error(N, 1) for N in Ns])
    o_pc = np.log2(pc[:-1] / pc[1:])
    o_vl = np.log2(vl[:-1] / vl[1:])
    assert np.all((o_pc > 0.9) & (o_pc < 1.1)), pc
    assert np.all(o_vl > 1.3), vl
    assert np.all(vl < pc / 8), (pc, vl)


def test_van_leer_passes_the_diffusion_gaussian():
    """Sec. 3.3: the paper passes the dynamic diffusion test with its van
    Leer integration.  With reconstruction the Gaussian of the optically
    thick scattering box matches Eq. (diff analytic) to below 1 % at 128
    cells across, ten times closer than the first-order step."""
    from tests.test_oracle_pins import _diffusion_gaussian_error

    def err(integrator):
        return _diffusion_gaussian_error(128, 0.0, integrator=integrator)
    e_pc, e_vl = err(0), err(1)
    assert e_vl < 0.01 and e_vl < e_pc / 10, (e_pc, e_vl)


def test_van_leer_conserves_energy_and_momentum():
    """Sec. 2.3.1 totals with the van Leer step: reconstructed fluxes are
    antisymmetric across faces and the source step is the conservative one,
    so E_gas + (c/cbar) E_r and rho v + F_r/(c cbar) stay constant to
    round-off (moving mesh and gas, scattering, boundary and emitter cells)."""
    prob = randomise(make(n=(4, 3, 5), order=6, cbar=10.0, c=100.0, w=(0.3, 0.1, 0.0)), seed=9)
    prob.integrator = 1
    o = oracle.Oracle(prob)
    dt = 0.5 / o.positivity()
    t0 = o.totals()
    assert o.run(20, dt) == 0
    t1 = o.totals()
    assert abs(t1[12] - t0[12]) < 1e-13 * abs(t0[12])
    scale = np.abs(t0[3:12]).sum() + np.abs(t1[3:12]).sum()
    assert np.abs(t1[13:16] - t0[13:16]).max() < 1e-13 * scale
