"""Independent McMurchie-Davidson nuclear-attraction integral in plain Python.

Test-only cross-check of the oracle's Obara-Saika recurrences: a different
algorithm (Hermite expansion of the Gaussian product, Helgaker, Joergensen &
Olsen, Molecular Electronic-Structure Theory, Sec. 9.5 and 9.9) with the Boys
function taken from SciPy's regularised incomplete gamma function,
    F_n(T) = Gamma(n+1/2) P(n+1/2, T) / (2 T^{n+1/2}).
Small cases only.
"""
import math
from functools import lru_cache

import numpy as np
from scipy.special import gamma, gammainc


def boys_scipy(n: int, T: float) -> float:
    if T < 1e-14:
        return 1.0 / (2 * n + 1) - T / (2 * n + 3)
    a = n + 0.5
    return float(gamma(a) * gammainc(a, T) / (2.0 * T ** a))


def hermite_E(i, j, t, Qx, a, b):
    """E^{ij}_t for one Cartesian direction; Qx = A_x - B_x; includes exp(-mu Qx^2)."""
    p = a + b
    q = a * b / p
    if t < 0 or t > i + j:
        return 0.0
    if i == 0 and j == 0 and t == 0:
        return math.exp(-q * Qx * Qx)
    if j == 0:
        return (hermite_E(i - 1, j, t - 1, Qx, a, b) / (2 * p)
                - (q * Qx / a) * hermite_E(i - 1, j, t, Qx, a, b)
                + (t + 1) * hermite_E(i - 1, j, t + 1, Qx, a, b))
    return (hermite_E(i, j - 1, t - 1, Qx, a, b) / (2 * p)
            + (q * Qx / b) * hermite_E(i, j - 1, t, Qx, a, b)
            + (t + 1) * hermite_E(i, j - 1, t + 1, Qx, a, b))


def hermite_R(t, u, v, p, PC):
    """R_tuv(p, P-C) by the McMurchie-Davidson recursion."""
    T = p * float(np.dot(PC, PC))

    @lru_cache(maxsize=None)
    def R(t, u, v, n):
        if t < 0 or u < 0 or v < 0:
            return 0.0
        if t == 0 and u == 0 and v == 0:
            return (-2.0 * p) ** n * boys_scipy(n, T)
        if t == 0 and u == 0:
            return (v - 1) * R(t, u, v - 2, n + 1) + PC[2] * R(t, u, v - 1, n + 1)
        if t == 0:
            return (u - 1) * R(t, u - 2, v, n + 1) + PC[1] * R(t, u - 1, v, n + 1)
        return (t - 1) * R(t - 2, u, v, n + 1) + PC[0] * R(t - 1, u, v, n + 1)

    return R(t, u, v, 0)


def md_pair_potential(A, a, la, B, b, lb, C) -> float:
    A, B, C = (np.asarray(x, dtype=np.float64) for x in (A, B, C))
    p = a + b
    P = (a * A + b * B) / p
    PC = P - C
    total = 0.0
    for t in range(la[0] + lb[0] + 1):
        Ex = hermite_E(la[0], lb[0], t, A[0] - B[0], a, b)
        for u in range(la[1] + lb[1] + 1):
            Ey = hermite_E(la[1], lb[1], u, A[1] - B[1], a, b)
            for v in range(la[2] + lb[2] + 1):
                Ez = hermite_E(la[2], lb[2], v, A[2] - B[2], a, b)
                total += Ex * Ey * Ez * hermite_R(t, u, v, p, PC)
    return 2.0 * math.pi / p * total
