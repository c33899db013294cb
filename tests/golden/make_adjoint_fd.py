"""Writes tests/golden/adjoint_fd_64.json: central differences of the FP64
oracle's loss on the full-size adjoint workload, per cell and per initial
intensity entry, for the GPU gradient test.

Workload: the 64^3 jittered box (S6, log-normal kappa_a, absorbing +-x
layers, one emitter), 64 Courant steps; loss L = sum_{c,a} g_ca I_ca after
the last step, with g the outgoing flux through the +x boundary layer
(A_f 4 pi w_a cbar max(n_a . n_f, 0) over faces from interior cells into
that layer).  Entries:
  * 32 seeded random interior cells c: dL/dkappa_a[c] (kappa_P = kappa_J =
    kappa_a moved together) by the central difference (L(kappa + h kappa_c
    e_c) - L(kappa - h kappa_c e_c)) / (2 h kappa_c), h = 1e-3; the
    difference of the two losses is summed as sum g (I+ - I-), so that its
    rounding is relative to the difference, not to L (intensities the
    perturbation does not reach cancel exactly);
  * 16 seeded random (cell, angle) entries: dL/dI0[c, a] likewise.
Entries are drawn among those whose derivative (by the oracle's discrete
adjoint) is at least 1e-3 of the largest, so that the differences resolve
them; the oracle's adjoint values are stored beside the differences and
must agree with them to 1e-5 (checked here).

Calls only oracle/ and the input generators.  Takes about an hour on
eight cores:  python tests/golden/make_adjoint_fd.py
"""
import json
import os
import sys
import time

import numpy as np

ROOT = os.path.dirname(os.path.dirname(os.path.dirname(os.path.abspath(__file__))))
sys.path.insert(0, ROOT)

import oracle  # noqa: E402
from paper_2002_08377_gb300.inputs import adjoint  # noqa: E402

OUT = os.path.join(os.path.dirname(os.path.abspath(__file__)), "adjoint_fd_64.json")
K, H, SEED = 64, 1e-3, 2024


def outflow_weights(prob):
    """g[c, a] = sum over faces f from interior cell c into a cell of the
    +x boundary layer of A_f 4 pi w_a cbar max(n_a . n_f(out of c), 0)."""
    m = prob.mesh
    layer = (prob.kind == 1) & (m.lattice_index()[0] == m.n[0] - 1)
    g = np.zeros((prob.n_cells, prob.n_angles))
    for f in range(m.n_faces):
        i, j = m.face_cells[f]
        for c, other, sign in ((i, j, 1.0), (j, i, -1.0)):
            if prob.kind[c] != 1 and layer[other]:
                mu = sign * (prob.dirs @ m.face_normal[f])
                g[c] += m.face_area[f] * 4 * np.pi * prob.weights * prob.cbar * np.maximum(mu, 0.0)
    return g


def final_intensity(prob, dt, kappa=None, I0=None):
    p = prob
    if kappa is not None or I0 is not None:
        import copy
        p = copy.copy(prob)
        if kappa is not None:
            p.kappa_P, p.kappa_J = kappa.copy(), kappa.copy()
        if I0 is not None:
            p.initial_intensity = lambda dtype=np.float64, _I=I0: _I.astype(dtype)
    o = oracle.Oracle(p)
    for _ in range(K):
        assert o.step(dt) == oracle.ORC_OK
    return o.I


def main():
    t0 = time.time()
    prob = adjoint(n=64, steps=K)
    dt = prob.cfl_dt()
    g = outflow_weights(prob)
    # the oracle's discrete adjoint, to choose entries the differences resolve
    o = oracle.Oracle(prob)
    states = []
    for _ in range(K):
        states.append((o.I.copy(), o.e.copy(), o.m.copy()))
        assert o.step(dt) == oracle.ORC_OK
    L0 = float(np.sum(g * o.I))
    N = prob.n_cells
    lI, le, lm = g.copy(), np.zeros(N), np.zeros((N, 3))
    gP, gJ = np.zeros(N), np.zeros(N)
    for n in reversed(range(K)):
        I, e, m = states[n]
        lI, le, lm = o.adjoint_step(dt, I, e, m, lI, le, lm, gP, gJ)
    del states
    gk, gI = gP + gJ, lI
    rng = np.random.default_rng(SEED)
    interior = np.nonzero(prob.kind == 0)[0]
    cand = interior[np.abs(gk[interior]) >= 1e-3 * np.abs(gk).max()]
    cells = np.sort(rng.choice(cand, size=32, replace=False))
    mask = (np.abs(gI) >= 1e-3 * np.abs(gI).max()) & (prob.kind == 0)[:, None]
    ci, ai = np.nonzero(mask)
    pick = rng.choice(len(ci), size=16, replace=False)
    entries = sorted(zip(ci[pick].tolist(), ai[pick].tolist()))
    print(f"base run and adjoint: {time.time() - t0:.0f} s", flush=True)

    def central(run, x0):
        dx = H * x0
        return float(np.sum(g * (run(+dx) - run(-dx)))) / (2 * dx)

    kap = prob.kappa_P.copy()
    out_k, bad = [], []
    for c in cells.tolist():
        def run(dx, c=c):
            k = kap.copy()
            k[c] += dx
            return final_intensity(prob, dt, kappa=k)
        fd = central(run, kap[c])
        if abs(fd - gk[c]) > 1e-5 * max(abs(fd), 1e-3 * np.abs(gk).max()):
            bad.append(("kappa", c, fd, float(gk[c])))
        out_k.append({"cell": c, "fd": fd, "oracle_adjoint": float(gk[c])})
        print(f"kappa cell {c}: fd {fd:.12e} adjoint {gk[c]:.12e} ({time.time() - t0:.0f} s)",
              flush=True)
    I0 = prob.initial_intensity()
    out_i = []
    for c, a in entries:
        def run(dx, c=c, a=a):
            x = I0.copy()
            x[c, a] += dx
            return final_intensity(prob, dt, I0=x)
        fd = central(run, I0[c, a])
        if abs(fd - gI[c, a]) > 1e-5 * max(abs(fd), 1e-3 * np.abs(gI).max()):
            bad.append(("I0", c, a, fd, float(gI[c, a])))
        out_i.append({"cell": c, "angle": a, "fd": fd, "oracle_adjoint": float(gI[c, a])})
        print(f"I0 entry ({c}, {a}): fd {fd:.12e} adjoint {gI[c, a]:.12e} "
              f"({time.time() - t0:.0f} s)", flush=True)
    rec = {"what": "central differences of the FP64 oracle's outflow loss, adjoint workload",
           "workload": "adjoint", "n": 64, "steps": K, "dt": dt, "h": H, "seed": SEED,
           "loss": L0, "max_abs_dL_dkappa": float(np.abs(gk).max()),
           "max_abs_dL_dI0": float(np.abs(gI).max()), "kappa": out_k, "I0": out_i,
           "script": "tests/golden/make_adjoint_fd.py"}
    with open(OUT, "w") as f:
        json.dump(rec, f, indent=1)
    print(f"wrote {OUT} in {time.time() - t0:.0f} s")
    assert not bad, bad  # the oracle's adjoint agrees with its differences


if __name__ == "__main__":
    main()
