"""Discrete-ordinate angle sets (an input of the radiation step).

The transport state is one intensity per cell per direction n_hat_a with
solid-angle weight w_a, sum_a w_a = 1 (Sec. 2, moment quadrature; Sec. 2.3,
comoving weights normalised to one).  The paper uses 80 angles for its beam
tests and one angle per octant for the diffusion and wave tests, without
naming the quadrature.  These sets are level-symmetric S_N sets with equal
weights 1/A:

    mu_i^2 = mu_1^2 + (i - 1) * 2 (1 - 3 mu_1^2) / (N - 2),   i = 1..N/2
    directions (+-mu_i, +-mu_j, +-mu_k) with i + j + k = N/2 + 2

which gives A = N (N + 2) directions: S2 = 8 (one per octant), S6 = 48,
S8 = 80.  The sets are closed under axis permutations and reflections, so
sum_a w_a n_a = 0 and sum_a w_a n_a n_a = I/3 exactly in real arithmetic.

Ordering: the first A/2 directions have n_z > 0 and direction a + A/2 is the
exact negative of direction a.  The CUDA path relies on this pairing.
"""
import numpy as np

# mu_1 of the classic level-symmetric sets
_MU1 = {2: 1.0 / np.sqrt(3.0), 4: 0.3500212, 6: 0.2666355, 8: 0.2182179}


def level_symmetric(order: int):
    """Return (dirs[A,3] float64, weights[A] float64) for S_order."""
    if order not in _MU1:
        raise ValueError("supported orders: 2, 4, 6, 8")
    n = order
    half = n // 2
    mu1 = _MU1[n]
    if n == 2:
        mus = np.array([mu1])
    else:
        mus = np.sqrt(mu1 ** 2 + np.arange(half) * 2.0 * (1.0 - 3.0 * mu1 ** 2) / (n - 2))
    base = []
    for i in range(1, half + 1):
        for j in range(1, half + 1):
            k = half + 2 - i - j
            if 1 <= k <= half:
                base.append((mus[i - 1], mus[j - 1], mus[k - 1]))
    base = np.array(base, dtype=np.float64)
    # renormalise to unit length (the tabulated mu_1 carry 7 digits)
    base /= np.linalg.norm(base, axis=1, keepdims=True)
    upper = []
    for sx in (1.0, -1.0):
        for sy in (1.0, -1.0):
            for d in base:
                upper.append((sx * d[0], sy * d[1], d[2]))
    upper = np.array(upper, dtype=np.float64)
    dirs = np.concatenate([upper, -upper], axis=0)
    a = dirs.shape[0]
    w = np.full(a, 1.0 / a, dtype=np.float64)
    return np.ascontiguousarray(dirs), w


def n_angles(order: int) -> int:
    return order * (order + 2)
