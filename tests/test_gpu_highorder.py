"""High-order stencils (2m = 10) on the paper's smooth-permittivity study.

Sec. 4.2 (eq. display:num:testsmooth, table tab:num:convergence_highord)
solves the SC unit cell with the smooth scalar permittivity
eps(x, y, z) = 8.9 sin(2 pi (x + y + z)) + 13 at k = (pi, pi, pi) with the
m = 5 stencils of Sec. 2.5 and prints, under the heading
|omega_h^2 - omega_2h^2|, the differences between grid levels for the
first eight eigenvalues.  The printed values are differences of the
normalised frequency omega / (2 pi) (omega a / 2 pi c, a = 1), where
omega^2 is the eigenvalue: |sqrt(lambda_h) - sqrt(lambda_2h)| / (2 pi)
reproduces every printed h = 1/32 entry (N = 32 against N = 16) to 0.2%,
and the eigenvalue differences themselves are 16-18 times the printed
numbers, the factor 4 pi sqrt(lambda) with lambda = 1.68 and 2.15.  Here
the GPU solver (FP64, cell blocks passed in through the dense-block path of
pcx_setup) is checked three ways:

- against the oracle's LOBPCG on the same discretisation at 16^3;
- the frequency differences at h = 1/32 equal the printed ones to 1%;
- the convergence rate between h = 1/32 and 1/64 is the stencils' tenth
  order, as printed (log2 of the printed ratio is 9.8).  The h = 1/64
  differences (near 1e-10 in the eigenvalue) sit at the FP64 rounding of
  the Rayleigh quotients (eps_mach times ||Op||, with gamma |kappa|^2 up to
  ~1e6 at 64^3), so they agree with the printed column only to a factor 2.

For an isotropic eps the M_Trivial block of a cell is diag(1/eps(E1),
1/eps(E2), 1/eps(E3)), sampled at the edge DoFs of Sec. 2.1,
((i - 1/2) h, j h, k h), (i h, (j - 1/2) h, k h), (i h, j h, (k - 1/2) h) with
1-based i, j, k.
"""
import os

import numpy as np
import pytest

torch = pytest.importorskip("torch")

pytestmark = pytest.mark.gpu

GOLDEN = os.path.join(os.path.dirname(__file__), "golden", "highorder_smooth_eps.txt")
K = np.array([np.pi, np.pi, np.pi])


@pytest.fixture(scope="module")
def pcx():
    if not torch.cuda.is_available():
        pytest.skip("needs a GPU")
    from paper_2511_17107_gb300 import build, pcx as _pcx
    build.build()
    return _pcx


def _printed():
    rows = [list(map(float, line.split())) for line in open(GOLDEN) if line.strip() and not line.startswith("#")]
    a = np.array(rows)
    return a[:, 1], a[:, 2]   # h = 1/32, h = 1/64


def _inv_eps_diag(n):
    """(3, N^3): 1/eps at the E1, E2, E3 edge points, cells in z, y, x order."""
    h = 1.0 / n
    idx = np.arange(1, n + 1, dtype=np.float64)
    z, y, x = np.meshgrid(idx, idx, idx, indexing="ij")
    out = np.zeros((3, n ** 3))
    for c in range(3):
        shift = [0.0, 0.0, 0.0]
        shift[c] = 0.5
        s = ((x - shift[0]) + (y - shift[1]) + (z - shift[2])) * h
        out[c] = (1.0 / (8.9 * np.sin(2 * np.pi * s) + 13.0)).reshape(-1)
    return out


def _gpu_eigs(pcx, n):
    blocks = np.zeros((n ** 3, 9))
    blocks[:, :3] = _inv_eps_diag(n).T
    ctx = pcx.pcx_setup(n, stencil_m=5, cell_blocks=blocks)
    # Res <= 1e-8 puts the eigenvalue error near Res^2 / gap, far below the
    # differences (the FP64 rounding of Op x, about 1e-16 ||Op||, keeps Res
    # above 1e-10 at 64^3 with these stencils and gamma).  The curl-sandwich
    # preconditioner carries eps; K_P^{-1} ignores it and converges slowly at
    # eps ~ 13.
    ev, res, its, st = pcx.pcx_solve(ctx, [K], 8, 1e-8, block=12, precision=pcx.PCX_FP64, raise_on_noconv=False,
                                     precond_kind=1)
    assert st == pcx.PCX_OK, (n, st, res)
    return ev[0]


def _oracle_eigs(n):
    from oracle import eig, fourier, learned, penalty
    d = _inv_eps_diag(n)
    blocks = np.zeros((n, n, n, 3, 3), dtype=np.complex128)
    for c in range(3):
        blocks[..., c, c] = d[c].reshape(n, n, n)
    kap = fourier.kappa(n, np.eye(3), K, 5)
    g = penalty.gamma_practical(K)

    def apply_m(e):
        return np.einsum("zyxij,...jzyx->...izyx", blocks, e)

    rng = np.random.default_rng(1)
    x0 = rng.standard_normal((12, 3, n, n, n)) + 1j * rng.standard_normal((12, 3, n, n, n))
    th, _, res, _ = eig.lobpcg(lambda X: fourier.apply_symbols(X, kap, apply_m, g),
                               lambda R: learned.sandwich_precondition(R, kap, blocks, g), x0, 8, tol=1e-9, maxit=300)
    assert np.max(res) <= 1e-9
    return np.asarray(th)


def test_tenth_order_convergence_on_the_smooth_permittivity(pcx, capsys):
    e16, e32, e64 = (_gpu_eigs(pcx, n) for n in (16, 32, 64))
    o16 = _oracle_eigs(16)
    # normalised frequency omega / (2 pi) with omega^2 the eigenvalue
    f16, f32, f64 = (np.sqrt(e) / (2 * np.pi) for e in (e16, e32, e64))
    d32, d64 = np.abs(f32 - f16), np.abs(f64 - f32)
    p32, p64 = _printed()
    order = np.log2(np.abs(e32 - e16) / np.abs(e64 - e32))
    with capsys.disabled():
        print("\nomega^2 at 64^3:", e64)
        print("|d omega/2pi| h=1/32:", d32, "\n|d omega/2pi| h=1/64:", d64, "\norder:", order)
        print("ratio to the printed differences:", d32 / p32, d64 / p64)
    # GPU solver and oracle on the same discretisation, to the FP64
    # eigenvalue tolerance (1e-10 relative)
    np.testing.assert_allclose(e16, o16, rtol=1e-10)
    # the printed constants at h = 1/32
    np.testing.assert_allclose(d32, p32, rtol=1e-2)
    # tenth order between h = 1/32 and 1/64, like the printed table (9.8);
    # the h = 1/64 column to the FP64 noise of the eigenvalues
    assert np.all(order > 8.5) and np.all(order < 11.0), order
    assert np.all(d64 / p64 > 0.4) and np.all(d64 / p64 < 2.0), d64 / p64
