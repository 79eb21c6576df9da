"""The oracle alone against the paper's printed high-order convergence
table (Sec. 4.2, eq. display:num:testsmooth, table
tab:num:convergence_highord): SC cell, eps(x, y, z) = 8.9 sin(2 pi (x + y +
z)) + 13, k = (pi, pi, pi), the 10th-order stencils (m = 5) of Sec. 2.5,
M_Trivial sampling 1/eps at the edge DoFs.  The oracle's LOBPCG at 16^3 and
32^3 gives the eight lowest eigenvalues lambda = omega^2; the printed h = 1/32
column is |omega_h - omega_2h| / (2 pi), the difference of the normalised
frequency between N = 32 and N = 16, and the oracle must reproduce it to 1%
(a dropped stencil term, a shifted sample point or a wrong symbol moves it
by orders of magnitude).  CPU only, about 40 s."""
import os

import numpy as np

from oracle import eig, fourier, learned, penalty

K = np.array([np.pi, np.pi, np.pi])
GOLDEN = os.path.join(os.path.dirname(__file__), "golden", "highorder_smooth_eps.txt")


def _inv_eps_blocks(n):
    """Per-cell blocks diag(1/eps(E1), 1/eps(E2), 1/eps(E3)) at the edge DoFs
    ((i - 1/2) h, j h, k h), (i h, (j - 1/2) h, k h), (i h, j h, (k - 1/2) h)."""
    h = 1.0 / n
    idx = np.arange(1, n + 1, dtype=np.float64)
    z, y, x = np.meshgrid(idx, idx, idx, indexing="ij")
    blocks = np.zeros((n, n, n, 3, 3), dtype=np.complex128)
    for c in range(3):
        shift = [0.0, 0.0, 0.0]
        shift[c] = 0.5
        s = ((x - shift[0]) + (y - shift[1]) + (z - shift[2])) * h
        blocks[..., c, c] = 1.0 / (8.9 * np.sin(2 * np.pi * s) + 13.0)
    return blocks


def _eigs(n):
    blocks = _inv_eps_blocks(n)
    kap = fourier.kappa(n, np.eye(3), K, 5)
    g = penalty.gamma_practical(K)

    def apply_m(e):
        return np.einsum("zyxij,...jzyx->...izyx", blocks, e)

    rng = np.random.default_rng(1)
    x0 = rng.standard_normal((12, 3, n, n, n)) + 1j * rng.standard_normal((12, 3, n, n, n))
    th, _, res, _ = eig.lobpcg(lambda X: fourier.apply_symbols(X, kap, apply_m, g),
                               lambda R: learned.sandwich_precondition(R, kap, blocks, g), x0, 8, tol=1e-9,
                               maxit=300)
    assert np.max(res) <= 1e-9
    return np.asarray(th)


def test_oracle_reproduces_the_printed_h32_column():
    printed = np.array([list(map(float, l.split())) for l in open(GOLDEN) if l.strip() and not l.startswith("#")])
    p32 = printed[:, 1]
    e16, e32 = _eigs(16), _eigs(32)
    d32 = np.abs(np.sqrt(e32) - np.sqrt(e16)) / (2 * np.pi)
    np.testing.assert_allclose(d32, p32, rtol=1e-2)
