"""Pins of the oracle's stencils, circulant symbols and DFT (CPU only)."""
import os
from fractions import Fraction

import numpy as np
import pytest

from oracle import fourier, stencils

GOLDEN = os.path.join(os.path.dirname(__file__), "golden", "fd_coefficients.txt")


def _golden_rows():
    rows = []
    with open(GOLDEN) as fh:
        for line in fh:
            line = line.split("#")[0].strip()
            if not line:
                continue
            parts = line.split()
            rows.append((int(parts[0]), int(parts[1]), int(parts[2]), Fraction(parts[3]), "typo" in parts[4:]))
    return rows


def test_printed_table_matches_moment_system():
    """Sec. 2.5, Table tab:kc:fd1d: every printed coefficient equals the
    exact solution of eq. kc:high:coef, except the flagged m=3 typo."""
    rows = _golden_rows()
    assert len(rows) == 30
    for m, kind, s, val, typo in rows:
        got = stencils.fd_coefficients(m, kind)[s - 1]
        if typo:
            assert got != val and got == Fraction(75, 64)
        else:
            assert got == val, (m, kind, s)


@pytest.mark.parametrize("m", [1, 2, 3, 4, 5])
def test_stencils_exact_on_polynomials(m):
    """A 2m-th order staggered stencil reproduces d/dx and point values at
    the half point exactly on every polynomial of degree < 2m (Taylor
    argument of Sec. 2.5); checked with exact rationals on monomials around
    x_{j-1/2} = 0, i.e. phi_{j+s-1} = x^q at x = (2s-1)/2, phi_{j-s} at -(2s-1)/2."""
    c1 = stencils.fd_coefficients(m, 1)
    c0 = stencils.fd_coefficients(m, 0)
    for q in range(2 * m):
        d = sum(c1[s - 1] * (Fraction(2 * s - 1, 2) ** q - Fraction(-(2 * s - 1), 2) ** q) for s in range(1, m + 1))
        v = sum(c0[s - 1] * (Fraction(2 * s - 1, 2) ** q + Fraction(-(2 * s - 1), 2) ** q) for s in range(1, m + 1))
        assert d == (1 if q == 1 else 0), (m, q)
        assert v == (1 if q == 0 else 0), (m, q)
    # and not on degree 2m (the order is exactly 2m)
    q = 2 * m + 1
    d = sum(c1[s - 1] * (Fraction(2 * s - 1, 2) ** q - Fraction(-(2 * s - 1), 2) ** q) for s in range(1, m + 1))
    assert d != 0


def test_yee_matrices_second_order():
    """Sec. 2.1 eq. yee:D0D1: first rows (1,0,..,0,-1)/h and (1,0,..,0,1)/2."""
    n = 7
    d1 = stencils.circulant(stencils.circulant_first_row(n, 1, 1))
    d0 = stencils.circulant(stencils.circulant_first_row(n, 1, 0))
    e = np.eye(n)
    shift = np.roll(e, -1, axis=1)       # row i has a 1 in column i-1
    np.testing.assert_allclose(d1, n * (e - shift))
    np.testing.assert_allclose(d0, 0.5 * (e + shift))
    assert d1[0, -1] == -n and d1[1, 0] == -n


@pytest.mark.parametrize("n,m", [(8, 1), (9, 2), (16, 5)])
def test_circulant_lemma(n, m):
    """Lemma 2.1: C = F diag(lambda) F^H with F unitary; the eigenvalues are
    checked against LAPACK independently (as a multiset)."""
    f = fourier.dft_matrix(n)
    np.testing.assert_allclose(f @ f.conj().T, np.eye(n), atol=1e-13)
    for kind in (0, 1):
        row = stencils.circulant_first_row(n, m, kind)
        c = stencils.circulant(row)
        lam = fourier.circulant_symbol(row)
        np.testing.assert_allclose(f @ np.diag(lam) @ f.conj().T, c, atol=1e-12 * max(1, np.abs(c).max()))
        ev = np.linalg.eigvals(c)
        np.testing.assert_allclose(np.sort_complex(np.round(ev, 9)), np.sort_complex(np.round(lam, 9)), atol=1e-8 * n)


def test_second_order_symbols_closed_form():
    """For m = 1 the symbols are Lambda_1(p) = (1 - e^{-2 pi i p/N})/h and
    Lambda_0(p) = (1 + e^{-2 pi i p/N})/2 (direct evaluation of Lemma 2.1
    on the first rows of eq. yee:D0D1)."""
    n = 12
    lam1, lam0 = fourier.lambda_tables(n, 1)
    z = np.exp(-2j * np.pi * np.arange(n) / n)
    np.testing.assert_allclose(lam1, n * (1 - z), atol=1e-12)
    np.testing.assert_allclose(lam0, 0.5 * (1 + z), atol=1e-14)


@pytest.mark.parametrize("n", [4, 6, 8])
def test_fft_route_equals_dft_matrix(n):
    """The numpy FFT route of F3 / F3^H equals the Kronecker product of the
    Lemma 2.1 DFT matrices (Sec. 2.4)."""
    rng = np.random.default_rng(1)
    u = rng.standard_normal((2, 3, n, n, n)) + 1j * rng.standard_normal((2, 3, n, n, n))
    np.testing.assert_allclose(fourier.f3(u), fourier.f3(u, explicit=True), atol=1e-12)
    np.testing.assert_allclose(fourier.f3h(u), fourier.f3h(u, explicit=True), atol=1e-12)
    f = fourier.dft_matrix(n)
    big = np.kron(np.kron(f, f), f)
    np.testing.assert_allclose(fourier.f3(u)[1, 2].ravel(), big @ u[1, 2].ravel(), atol=1e-12)
