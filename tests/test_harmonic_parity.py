"""The reading behind offset mirroring in the pair-packed M2L, checked with
scipy's associated Legendre functions (independent of the library and of
the oracle).

The irregular solid harmonic Th_n^m(r) = (n-m)! P_n^m(cos t) e^{i m f} /
|r|^{n+1} (Sec. 2.3.1) is even or odd in r with its degree n: r -> -r sends
cos t -> -cos t and f -> f + pi, and P_n^m(-x) = (-1)^(n+m) P_n^m(x).  Every
term of the M2L entry (l, j) of Eq. FMM_local holds a harmonic of degree
j + l, so T_{-o} = (-1)^(j+l) T_o, which lets the pairs of offset -o use the
operator of o with the odd-degree coefficients negated on the way in and out.
"""
import math

import numpy as np
from scipy.special import lpmv


def irregular(n, m, v):
    x, y, z = v
    r = math.sqrt(x * x + y * y + z * z)
    ct = z / r
    f = math.atan2(y, x)
    return math.factorial(n - m) * lpmv(m, n, ct) * np.exp(1j * m * f) / r ** (n + 1)


def m2l_entry(l, h, j, k, o):
    """The coefficient of M_j^k in L_l^h (Eq. FMM_local, complex form)."""
    if abs(k + h) > j + l:
        return 0.0
    mm = k + h
    th = irregular(j + l, abs(mm), o)
    if mm < 0:  # X_n^{-m} = (-1)^m conj(X_n^m)
        th = (-1) ** (-mm) * np.conj(th)
    return (-1) ** l * th


def test_irregular_harmonics_have_the_parity_of_their_degree():
    rng = np.random.default_rng(3)
    for _ in range(20):
        o = rng.integers(-3, 4, size=3).astype(float)
        if np.max(np.abs(o)) <= 1:
            continue
        for n in range(17):
            a = np.array([irregular(n, m, o) for m in range(n + 1)])
            b = np.array([irregular(n, m, -o) for m in range(n + 1)])
            # relative to the degree's largest harmonic (exact zeros of
            # P_n^m(0) come back as rounding noise)
            assert np.max(np.abs(b - (-1) ** n * a)) <= 1e-12 * np.max(np.abs(a))


def test_m2l_operator_of_minus_o_is_the_sign_pattern_of_o():
    p = 6
    o = np.array([3.0, -2.0, 1.0])
    for l in range(p + 1):
        for h in range(-l, l + 1):
            for j in range(p + 1):
                for k in range(-j, j + 1):
                    a, b = m2l_entry(l, h, j, k, o), m2l_entry(l, h, j, k, -o)
                    scale = abs(irregular(j + l, 0, o)) + abs(a)
                    assert abs(b - (-1) ** (j + l) * a) <= 1e-12 * scale
