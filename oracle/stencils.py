"""Finite-difference coefficients and circulant first rows (oracle; test
infrastructure only).

Sec. 2.1, eq. yee:D0D1: the second-order Yee matrices D1 (backward
difference divided by h) and D0 (two-point average) are circulant.
Sec. 2.5, eqs. kc:highord:stencil and kc:high:coef: a 2m-th order stencil
replaces their first rows by

    (d phi/dx)_{j-1/2} ~ (1/h) sum_s c1_s (phi_{j+s-1} - phi_{j-s})
    phi_{j-1/2}        ~       sum_s c0_s (phi_{j+s-1} + phi_{j-s})

with coefficients solving  sum_t ((2t-1)/2)^(2s+k-2) c_t^(k) = delta_{s1}/2
for s = 1..m (k = 1 derivative, k = 0 interpolation).
"""
from __future__ import annotations

from fractions import Fraction

import numpy as np


def fd_coefficients(m: int, kind: int) -> list:
    """Exact rational coefficients c_1..c_m of the 2m-th order stencil of
    Sec. 2.5 (eq. kc:high:coef): Gaussian elimination over Fractions.
    kind = 1: staggered derivative; kind = 0: staggered interpolation."""
    if m < 1 or kind not in (0, 1):
        raise ValueError("m >= 1 and kind in {0, 1}")
    a = [[Fraction(2 * t - 1, 2) ** (2 * s + kind - 2) for t in range(1, m + 1)]
         for s in range(1, m + 1)]
    rhs = [Fraction(1, 2)] + [Fraction(0)] * (m - 1)
    # augmented elimination with partial pivoting on exact rationals
    for col in range(m):
        piv = next(r for r in range(col, m) if a[r][col] != 0)
        a[col], a[piv] = a[piv], a[col]
        rhs[col], rhs[piv] = rhs[piv], rhs[col]
        for r in range(m):
            if r != col and a[r][col] != 0:
                f = a[r][col] / a[col][col]
                a[r] = [x - f * y for x, y in zip(a[r], a[col])]
                rhs[r] -= f * rhs[col]
    return [rhs[i] / a[i][i] for i in range(m)]


def stencil_offsets(m: int, kind: int, h: float):
    """Offsets and FP64 weights of the staggered operator acting as
    (D phi)_i = sum_a w_a phi_{i+a}  (periodic).  kind=1: D1, kind=0: D0."""
    c = fd_coefficients(m, kind)
    terms = {}
    for s in range(1, m + 1):
        w = float(c[s - 1])
        if kind == 1:
            w /= h
            terms[s - 1] = terms.get(s - 1, 0.0) + w
            terms[-s] = terms.get(-s, 0.0) - w
        else:
            terms[s - 1] = terms.get(s - 1, 0.0) + w
            terms[-s] = terms.get(-s, 0.0) + w
    return sorted(terms.items())


def circulant_first_row(n: int, m: int, kind: int) -> np.ndarray:
    """First row (c_1..c_N) of the N x N circulant D1 (kind=1, h = 1/N) or
    D0 (kind=0), in the convention of Lemma 2.1: C_ij = c_{(j-i) mod N}."""
    if n < 2 * m:
        raise ValueError("grid too small for the stencil")
    row = np.zeros(n, dtype=np.float64)
    for off, w in stencil_offsets(m, kind, 1.0 / n):
        row[off % n] += w
    return row


def circulant(first_row: np.ndarray) -> np.ndarray:
    """Dense circulant matrix with C_ij = c_{(j-i) mod N} (Lemma 2.1)."""
    n = len(first_row)
    i = np.arange(n)
    return first_row[(i[None, :] - i[:, None]) % n]
