"""Pins of the per-mode penalty form gamma_p = 4 pi^2 max(1, |kappa_p|^-2)
(the rule of Remark 2.6 applied to each Fourier mode with that mode's B
eigenvalue |kappa_p|^2, Lemma kc_ABblock) in the oracle."""
import math

import numpy as np
import pytest

import workloads as wl
from oracle import eig, fourier, learned, penalty, permittivity, yee

FOUR_PI2 = 4.0 * math.pi ** 2


def _eigh(mat):
    return np.linalg.eigvalsh(0.5 * (mat + mat.conj().T))


def test_gamma_per_mode_values():
    """gamma_p |kappa_p|^2 = 4 pi^2 max(1, |kappa_p|^2) on every mode with
    kappa_p != 0; near Gamma the p = 0 mode carries the scalar rule's value
    4 pi^2 / |kappa_0|^2 and the others 4 pi^2."""
    n = 8
    k = np.array([0.05, -0.08, 0.03])
    kap = fourier.kappa(n, wl.SC, k)
    g = penalty.gamma_per_mode(kap)
    k2 = np.sum(np.abs(kap) ** 2, axis=0)
    np.testing.assert_allclose(g * k2, FOUR_PI2 * np.maximum(1.0, k2), rtol=1e-14)
    assert g[0, 0, 0] == pytest.approx(FOUR_PI2 / k2[0, 0, 0], rel=1e-14)
    # the p = 0 symbol is the Yee symbol of k: close to |k|^2, so gamma_0 is
    # close to the scalar rule's gamma
    assert g[0, 0, 0] == pytest.approx(penalty.gamma_practical(k), rel=1e-2)
    others = np.ones_like(k2, dtype=bool)
    others[0, 0, 0] = False
    assert np.all(g[others] == FOUR_PI2)


@pytest.mark.parametrize("lattice,kvec", [("SC", (0.05, -0.08, 0.03)), ("FCC", (0.3, 0.2, -0.1)),
                                          ("SC", (2 * math.pi - 0.1, 0.0, 0.0))])
def test_per_mode_spectrum_is_physical_union_closed_form(lattice, kvec):
    """The per-mode operator K_A F3^H M F3 K_A^H + diag(gamma_p K_B(p)) has
    the spectrum {nonzero eigenvalues of A M A^H} u {gamma_p |kappa_p|^2}:
    the first from the real-space stencils (dense), the second in closed
    form.  The last case lies outside the first zone, where the scalar rule's
    4 pi^2 leaves a penalty eigenvalue 4 pi^2 |kappa|^2 ~ 0.4 among the
    physical ones; the per-mode rule keeps every penalty eigenvalue >= 4 pi^2."""
    n = 6
    lat = getattr(wl, lattice)
    k = np.array(kvec)
    s = wl.sc_gyro_sphere() if lattice == "SC" else wl.fcc_air_spheres()
    blocks = permittivity.cell_blocks(s, n)
    ops = yee.YeeOperators(n, lat, k, 1)
    am = lambda e: permittivity.apply_m(blocks, e)
    dim = 3 * n ** 3
    shape = (3, n, n, n)
    amah = eig.dense_matrix(lambda c: ops.curl(am(ops.curl_adj(c.reshape((-1,) + shape)))).reshape(c.shape[0], -1),
                            dim)
    ev_a = _eigh(amah)
    phys = ev_a[np.abs(ev_a) > 1e-9 * ev_a.max()]
    kap = fourier.kappa(n, lat, k)
    g = penalty.gamma_per_mode(kap)
    k2 = np.sum(np.abs(kap) ** 2, axis=0)
    pen = (g * k2)[k2 > 0]
    op = eig.dense_matrix(
        lambda c: fourier.apply_symbols(c.reshape((-1,) + shape), kap, am, g).reshape(c.shape[0], -1), dim)
    ev = _eigh(op)
    expect = np.sort(np.concatenate([phys, pen, np.zeros(int(np.sum(k2 == 0)))]))
    np.testing.assert_allclose(ev, expect, atol=1e-9 * expect.max())
    assert pen.min() >= FOUR_PI2 * (1 - 1e-12)
    assert ev.max() <= ev_a.max() + FOUR_PI2 * max(1.0, k2.max()) * (1 + 1e-12)


def test_per_mode_and_scalar_forms_share_the_lowest_eigenvalues():
    """Near Gamma both forms satisfy Prop. 2.5's condition, so their lowest
    eigenvalues (the physical ones) coincide, while the scalar form's top of
    the spectrum is about gamma / 4 pi^2 times higher."""
    n = 6
    k = np.array([0.05, -0.08, 0.03])
    s = wl.sc_gyro_sphere()
    blocks = permittivity.cell_blocks(s, n)
    am = lambda e: permittivity.apply_m(blocks, e)
    kap = fourier.kappa(n, wl.SC, k)
    shape, dim = (3, n, n, n), 3 * n ** 3
    mk = lambda gam: _eigh(eig.dense_matrix(
        lambda c: fourier.apply_symbols(c.reshape((-1,) + shape), kap, am, gam).reshape(c.shape[0], -1), dim))
    gs = penalty.gamma_practical(k)
    ev_s, ev_m = mk(gs), mk(penalty.gamma_per_mode(kap))
    # dense eigensolvers resolve eigenvalues to ~1e-16 ||Op||, which the
    # scalar form makes large: compare on that scale
    np.testing.assert_allclose(ev_m[:12], ev_s[:12], rtol=0, atol=1e-13 * ev_s.max())
    assert ev_s.max() > 0.5 * gs / FOUR_PI2 * ev_m.max()


def test_per_mode_preconditioner_inverts_the_vacuum_operator():
    """K_P = K_A K_A^H + gamma_p K_B is the per-mode operator with M = I, so
    K_P^{-1} undoes apply_symbols (FFT route, M = identity) on every mode
    with kappa != 0."""
    rng = np.random.default_rng(5)
    n = 8
    k = np.array([0.07, 0.02, -0.05])
    kap = fourier.kappa(n, wl.SC, k)
    g = penalty.gamma_per_mode(kap)
    x = rng.standard_normal((2, 3, n, n, n)) + 1j * rng.standard_normal((2, 3, n, n, n))
    y = fourier.apply_symbols(x, kap, lambda e: e, g)
    np.testing.assert_allclose(fourier.precondition(y, kap, g), x, atol=1e-10 * np.abs(x).max())


def test_per_mode_sandwich_is_exact_for_a_homogeneous_isotropic_medium():
    """T0 (curl sandwich) with the per-mode penalty inverts the per-mode
    operator exactly for M = m0 I: K_A K_A^H + K_B = |kappa|^2 I per mode,
    and the longitudinal part conj(kappa) (kappa . r) / (gamma_p |kappa|^4)
    undoes gamma_p K_B."""
    rng = np.random.default_rng(6)
    n, m0 = 8, 0.37
    k = np.array([0.04, -0.06, 0.09])
    blocks = np.broadcast_to(m0 * np.eye(3), (n, n, n, 3, 3)).astype(np.complex128)
    kap = fourier.kappa(n, wl.FCC, k)
    g = penalty.gamma_per_mode(kap)
    x = rng.standard_normal((2, 3, n, n, n)) + 1j * rng.standard_normal((2, 3, n, n, n))
    y = fourier.apply_symbols(x, kap, lambda e: permittivity.apply_m(blocks, e), g)
    np.testing.assert_allclose(learned.sandwich_precondition(y, kap, blocks, g), x, atol=1e-9 * np.abs(x).max())


@pytest.mark.parametrize("lattice,kvec", [("SC", (0.05, -0.08, 0.03)), ("FCC", (1.3, 0.2, -0.7))])
def test_projector_spectrum_is_physical_union_constant(lattice, kvec):
    """Projector form gamma_p = gamma / |kappa_p|^2: the spectrum is the
    nonzero spectrum of A M A^H (dense real-space stencils) and the value
    gamma (16 pi^2 by default) once per mode with kappa_p != 0; the largest
    eigenvalue is that of A M A^H or gamma, far below the rule's
    4 pi^2 max|kappa|^2."""
    n = 6
    lat = getattr(wl, lattice)
    k = np.array(kvec)
    s = wl.sc_gyro_sphere() if lattice == "SC" else wl.fcc_air_spheres()
    blocks = permittivity.cell_blocks(s, n)
    ops = yee.YeeOperators(n, lat, k, 1)
    am = lambda e: permittivity.apply_m(blocks, e)
    dim, shape = 3 * n ** 3, (3, n, n, n)
    ev_a = _eigh(eig.dense_matrix(
        lambda c: ops.curl(am(ops.curl_adj(c.reshape((-1,) + shape)))).reshape(c.shape[0], -1), dim))
    phys = ev_a[np.abs(ev_a) > 1e-9 * ev_a.max()]
    kap = fourier.kappa(n, lat, k)
    k2 = np.sum(np.abs(kap) ** 2, axis=0)
    ev = _eigh(eig.dense_matrix(
        lambda c: fourier.apply_symbols(c.reshape((-1,) + shape), kap, am, penalty.gamma_projector(kap))
        .reshape(c.shape[0], -1), dim))
    gam = 4 * FOUR_PI2
    expect = np.sort(np.concatenate([phys, np.full(int(np.sum(k2 > 0)), gam), np.zeros(int(np.sum(k2 == 0)))]))
    np.testing.assert_allclose(ev, expect, atol=1e-10 * expect.max())
    assert ev.max() <= max(ev_a.max(), gam) * (1 + 1e-12)


def test_projector_preconditioner_and_sandwich_invert():
    """K_P^{-1} undoes the projector-form vacuum operator and T0 the
    projector-form operator of M = m0 I, on every mode with kappa != 0."""
    rng = np.random.default_rng(7)
    n, m0 = 8, 0.37
    k = np.array([0.07, 0.02, -0.05])
    kap = fourier.kappa(n, wl.FCC, k)
    g = penalty.gamma_projector(kap)
    x = rng.standard_normal((2, 3, n, n, n)) + 1j * rng.standard_normal((2, 3, n, n, n))
    y = fourier.apply_symbols(x, kap, lambda e: e, g)
    np.testing.assert_allclose(fourier.precondition(y, kap, g), x, atol=1e-10 * np.abs(x).max())
    blocks = np.broadcast_to(m0 * np.eye(3), (n, n, n, 3, 3)).astype(np.complex128)
    y = fourier.apply_symbols(x, kap, lambda e: permittivity.apply_m(blocks, e), g)
    np.testing.assert_allclose(learned.sandwich_precondition(y, kap, blocks, g), x, atol=1e-9 * np.abs(x).max())
