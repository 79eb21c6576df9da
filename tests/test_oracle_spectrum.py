"""Pins of the oracle's spectra, penalty rule, preconditioner and LOBPCG."""
import math

import numpy as np
import pytest

import workloads as wl
from oracle import eig, fourier, penalty, permittivity, yee


def _dense_ops(structure, n, k, lattice=None, m=1):
    lat = structure.lattice if lattice is None else lattice
    blocks = permittivity.cell_blocks(structure, n)
    ops = yee.YeeOperators(n, lat, k, m)
    am = lambda e: permittivity.apply_m(blocks, e)
    dim = 3 * n ** 3
    shape = (3, n, n, n)

    def mk(fn):
        return eig.dense_matrix(lambda c: fn(c.reshape((-1,) + shape)).reshape(c.shape[0], -1), dim)

    amah = mk(lambda h: ops.curl(am(ops.curl_adj(h))))
    bhb = mk(lambda h: ops.div_adj(ops.div(h)))
    return blocks, ops, am, amah, bhb


def _eigh(mat):
    return np.linalg.eigvalsh(0.5 * (mat + mat.conj().T))


@pytest.mark.parametrize("lattice", ["SC", "FCC"])
def test_homogeneous_dense_equals_mode_blocks(lattice):
    """A homogeneous anisotropic medium: the dense spectrum of the
    real-space operator equals the union of the per-mode 3x3 block spectra."""
    rng = np.random.default_rng(11)
    n = 6
    lat = getattr(wl, lattice)
    s = wl.homogeneous(wl.hermitian_pd(rng, 2.0, 7.0), lat)
    k = np.array([0.9, -0.3, 1.7])
    g = penalty.gamma_practical(k)
    _, _, _, amah, bhb = _dense_ops(s, n, k)
    dense = _eigh(amah + g * bhb)
    modes = eig.homogeneous_spectrum(fourier.kappa(n, lat, k), permittivity.inverse_permittivity(s)[0], g)
    np.testing.assert_allclose(dense, modes, atol=1e-11 * modes.max())


def test_isotropic_mode_spectrum_closed_form():
    """For P = c I the block K_A P K_A^H + gamma K_B has eigenvalues
    {c|kappa|^2, c|kappa|^2, gamma|kappa|^2}: K_A K_A^H = |kappa|^2 I -
    conj(kappa) kappa^T and K_B conj(kappa) = |kappa|^2 conj(kappa)."""
    n = 8
    k = np.array([0.5, 1.0, -0.25])
    c, g = 1.0 / 12.0, penalty.gamma_practical(k)
    kap = fourier.kappa(n, wl.SC, k)
    spec = eig.homogeneous_spectrum(kap, c * np.eye(3), g)
    k2 = np.sum(np.abs(kap) ** 2, axis=0).ravel()
    closed = np.sort(np.concatenate([c * k2, c * k2, g * k2]))
    np.testing.assert_allclose(spec, closed, atol=1e-10 * closed.max())


@pytest.mark.parametrize("kvec,zeros_op,extra", [((0.0, 0.0, 0.0), 3, 2), ((0.6, -1.2, 0.4), 0, 0)])
def test_null_space_dimensions(kvec, zeros_op, extra):
    """Prop. 2.5 (1): dim H = 3 at k = 0 (constant fields) and 0 otherwise;
    A M A^H (M HPD) has the null space ker A^H of dimension N^3 (k != 0) or
    N^3 + 2 (k = 0)."""
    n = 6
    k = np.array(kvec)
    g = penalty.gamma_practical(k)
    _, _, _, amah, bhb = _dense_ops(wl.sc_gyro_sphere(), n, k)
    ev = _eigh(amah + g * bhb)
    tol = 1e-9 * ev.max()
    assert int(np.sum(np.abs(ev) < tol)) == zeros_op
    ev_a = _eigh(amah)
    assert int(np.sum(np.abs(ev_a) < 1e-9 * ev_a.max())) == n ** 3 + extra


def test_penalised_spectrum_is_the_union():
    """Prop. 2.3: the nonzero spectrum of A M A^H + gamma B^H B is the union
    of the nonzero spectrum of A M A^H and gamma times that of B^H B."""
    n = 6
    k = np.array([0.8, 0.3, -1.1])
    g = penalty.gamma_practical(k)
    _, _, _, amah, bhb = _dense_ops(wl.sc_gyro_sphere(), n, k)
    ev = _eigh(amah + g * bhb)
    ea, eb = _eigh(amah), _eigh(bhb)
    ea = ea[np.abs(ea) > 1e-9 * ea.max()]
    eb = eb[np.abs(eb) > 1e-9 * eb.max()]
    union = np.sort(np.concatenate([ea, g * eb]))
    np.testing.assert_allclose(ev, union, atol=1e-9 * ev.max())


def test_gamma_rule():
    """Remark 2.6 eq. kc_settingofgamma1 and Prop. 2.5 eq. kc_settingofgamma."""
    fp = 4 * math.pi ** 2
    assert penalty.gamma_practical([0, 0, 0]) == fp
    assert penalty.gamma_practical([2.0, 0, 0]) == fp
    assert abs(penalty.gamma_practical([0.5, 0, 0]) - fp / 0.25) < 1e-12
    assert abs(penalty.gamma_practical([1.0, 0, 0]) - fp) < 1e-12
    assert abs(penalty.gamma_practical([1 - 1e-12, 0, 0]) - fp) < 1e-9
    assert penalty.gamma_sufficient([0.5, 0, 0], 3.0) == 12.0
    assert penalty.gamma_sufficient([0, 0, 0], 0.5) == 1.0
    # with lambda_m^A = 4 pi^2 the sufficient rule reduces to the practical one
    for kv in ([0.3, 0.2, 0.1], [1.5, 0, 0], [0, 0, 0]):
        assert abs(penalty.gamma_sufficient(kv, fp) - penalty.gamma_practical(kv)) < 1e-9


@pytest.mark.parametrize("kvec", [(0.0, 0.0, 0.0), (0.4, 2.2, -0.9)])
def test_preconditioned_rayleigh_quotient_bounds(kvec):
    """Prop. 2.9: x^H Op x / x^H K_P x lies in [min(lambda_min(M), 1),
    max(lambda_max(M), 1)]; and the preconditioner inverts K_P on every
    non-null mode."""
    rng = np.random.default_rng(12)
    n = 8
    k = np.array(kvec)
    g = penalty.gamma_practical(k)
    blocks = permittivity.cell_blocks(wl.sc_gyro_sphere(), n)
    lam = np.linalg.eigvalsh(blocks)
    lo, hi = min(lam.min(), 1.0), max(lam.max(), 1.0)
    kap = fourier.kappa(n, wl.SC, k)
    am = lambda e: permittivity.apply_m(blocks, e)
    kp = fourier.kp_matrix(kap, g)
    for _ in range(5):
        x = rng.standard_normal((1, 3, n, n, n)) + 1j * rng.standard_normal((1, 3, n, n, n))
        x[:, :, 0, 0, 0] = 0.0 if np.all(k == 0) else x[:, :, 0, 0, 0]
        num = np.vdot(x, fourier.apply_symbols(x, kap, am, g)).real
        den = np.vdot(x, np.einsum("zyxij,...jzyx->...izyx", kp, x)).real
        assert lo - 1e-12 <= num / den <= hi + 1e-12
        back = fourier.precondition(np.einsum("zyxij,...jzyx->...izyx", kp, x), kap, g)
        np.testing.assert_allclose(back, x, atol=1e-10 * np.abs(x).max())


def _solve_dense(structure, n, k, nev):
    g = penalty.gamma_practical(k)
    _, _, _, amah, bhb = _dense_ops(structure, n, k)
    ev = _eigh(amah + g * bhb)
    return ev[ev > 1e-9 * ev.max()][:nev]


@pytest.mark.parametrize("kvec", [(0.0, 0.0, 0.0), (0.6, 1.3, -0.5)])
def test_lobpcg_matches_dense(kvec):
    """The textbook LOBPCG (soft locking, K_P^{-1} preconditioner, p = 0
    deflation at k = 0) finds the smallest positive eigenvalues of the
    dense operator."""
    n = 6
    nev, nblk = 5, 8
    k = np.array(kvec)
    s = wl.sc_gyro_sphere()
    want = _solve_dense(s, n, k, nev)
    g = penalty.gamma_practical(k)
    blocks = permittivity.cell_blocks(s, n)
    ops = yee.YeeOperators(n, s.lattice, k)
    am = lambda e: permittivity.apply_m(blocks, e)
    kap = fourier.kappa(n, s.lattice, k)
    x0 = wl.random_block(nblk, n, seed=3)
    theta, _, res, it = eig.lobpcg(lambda x: fourier.apply_definition(x, ops, am, g),
                                   lambda r: fourier.precondition(r, kap, g), x0, nev,
                                   tol=1e-9, maxit=500, deflate=bool(np.all(k == 0)))
    assert np.all(res <= 1e-9) and it < 500
    np.testing.assert_allclose(theta, want, rtol=1e-10)


def test_continuum_limit_of_the_bands():
    """Homogeneous isotropic medium eps, continuous problem (Sec. 1 eq.
    intro_magneticshifted): transverse plane waves have w^2 = |k + G|^2 / eps.
    The two lowest discrete eigenvalues (mode p = 0) equal |k|^2 / eps
    exactly (Lambda_1(0) = 0, Lambda_0(0) = 1), and the next pair tends to
    min_{G != 0} |k + G|^2 / eps with an O(h^2) error."""
    eps = 4.0
    k = np.array([0.3, 0.5, -0.2])
    g = penalty.gamma_practical(k)
    gs = [2 * np.pi * np.array(v) for v in np.ndindex(3, 3, 3)]
    gs = [v - 2 * np.pi for v in gs if np.any(v != 2 * np.pi)]
    cont = min(np.sum((k + v) ** 2) for v in gs) / eps
    errs = []
    for n in (16, 32, 64):
        spec = eig.homogeneous_spectrum(fourier.kappa(n, wl.SC, k), np.eye(3) / eps, g)
        assert abs(spec[0] - k @ k / eps) < 1e-13 and abs(spec[1] - k @ k / eps) < 1e-13
        assert abs(spec[2] - spec[3]) < 1e-10
        errs.append(abs(spec[2] - cont))
    assert errs[0] < 0.02 * cont
    assert 3.5 < errs[0] / errs[1] < 4.6 and 3.5 < errs[1] / errs[2] < 4.6, errs
