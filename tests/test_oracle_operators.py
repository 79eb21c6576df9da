"""Pins of the oracle's Yee operators and Fourier-basis operator (CPU only)."""
import math

import numpy as np
import pytest

import workloads as wl
from oracle import fourier, penalty, permittivity, yee


def _rand(rng, shape):
    return rng.standard_normal(shape) + 1j * rng.standard_normal(shape)


def _vdot(a, b):
    return np.vdot(a.ravel(), b.ravel())


@pytest.mark.parametrize("lattice", ["SC", "FCC", "BCC"])
@pytest.mark.parametrize("m", [1, 3])
@pytest.mark.parametrize("reading", ["summed", "literal"])
def test_div_curl_is_zero(lattice, m, reading):
    """Prop. 2.2: B A = 0 for every lattice (all hat D_i commute)."""
    rng = np.random.default_rng(2)
    n = 8
    ops = yee.YeeOperators(n, getattr(wl, lattice), rng.standard_normal(3) * 2, m, reading)
    e = _rand(rng, (3, n, n, n))
    scale = np.abs(ops.curl(e)).max() * n
    assert np.abs(ops.div(ops.curl(e))).max() <= 1e-13 * scale


@pytest.mark.parametrize("m", [1, 2])
def test_curl_curl_plus_grad_div_is_block_laplacian(m):
    """Lemma 2.4 (1), A = I: A A^H + B^H B = diag(L, L, L), L = B B^H."""
    rng = np.random.default_rng(3)
    n = 8
    ops = yee.YeeOperators(n, wl.SC, rng.standard_normal(3), m)
    h = _rand(rng, (3, n, n, n))
    lhs = ops.curl(ops.curl_adj(h)) + ops.div_adj(ops.div(h))
    rhs = np.stack([ops.div(ops.div_adj(h[i])) for i in range(3)])
    np.testing.assert_allclose(lhs, rhs, atol=1e-11 * np.abs(rhs).max())


@pytest.mark.parametrize("lattice", ["SC", "FCC"])
def test_adjoints(lattice):
    """<A E, H> = <E, A^H H> and <B H, psi> = <H, B^H psi>."""
    rng = np.random.default_rng(4)
    n = 6
    ops = yee.YeeOperators(n, getattr(wl, lattice), rng.standard_normal(3), 2)
    e, h, psi = _rand(rng, (3, n, n, n)), _rand(rng, (3, n, n, n)), _rand(rng, (n, n, n))
    a = _vdot(ops.curl(e), h)
    assert abs(a - _vdot(e, ops.curl_adj(h))) <= 1e-12 * abs(a) * n
    b = _vdot(ops.div(h), psi)
    assert abs(b - _vdot(h, ops.div_adj(psi))) <= 1e-12 * abs(b) * n


@pytest.mark.parametrize("n", [8, 16, 33])
def test_khk_spectrum_closed_form(n):
    """Lemma 2.4 (2), eqs. kc_lapblockeigs and kc_minKeigen: the eigenvalues
    |Lambda_1 + i k Lambda_0|^2 of K^H K are
    (2/h^2 + k^2/2)(1 - cos(phi + 2 pi j h)), tan phi = 4kh/(4 - k^2h^2),
    and their minimum is k^2 when |k| <= pi and h < 1/pi."""
    h = 1.0 / n
    lam1, lam0 = fourier.lambda_tables(n, 1)
    for k in (0.3, -1.7, math.pi, 2.9):
        mu = np.sort(np.abs(lam1 + 1j * k * lam0) ** 2)
        phi = math.atan2(4 * k * h, 4 - k * k * h * h)
        j = np.arange(1, n + 1)
        closed = np.sort((2 / h ** 2 + k ** 2 / 2) * (1 - np.cos(phi + 2 * j * math.pi * h)))
        np.testing.assert_allclose(mu, closed, rtol=1e-10, atol=1e-9)
        assert abs(mu[0] - k * k) <= 1e-9 * max(1, k * k)


@pytest.mark.parametrize("lattice", ["SC", "FCC", "BCC"])
@pytest.mark.parametrize("m", [1, 2])
def test_symbol_form_equals_stencil_form(lattice, m):
    """Prop. 2.8: K_A F3^H M F3 K_A^H + gamma K_B equals F3^H (A M A^H +
    gamma B^H B) F3 built from the real-space stencils, for an
    inhomogeneous anisotropic M."""
    rng = np.random.default_rng(5)
    n = 8
    lat = getattr(wl, lattice)
    k = rng.standard_normal(3) * 3
    blocks = permittivity.cell_blocks(wl.sc_gyro_sphere(), n)
    am = lambda e: permittivity.apply_m(blocks, e)
    ops = yee.YeeOperators(n, lat, k, m)
    x = _rand(rng, (2, 3, n, n, n))
    g = penalty.gamma_practical(k)
    a = fourier.apply_definition(x, ops, am, g)
    b = fourier.apply_symbols(x, fourier.kappa(n, lat, k, m), am, g)
    np.testing.assert_allclose(a, b, atol=1e-12 * np.abs(a).max())


def test_operator_is_hermitian():
    rng = np.random.default_rng(6)
    n = 8
    k = np.array([0.4, -1.1, 2.0])
    blocks = permittivity.cell_blocks(wl.fcc_air_spheres(), n)
    am = lambda e: permittivity.apply_m(blocks, e)
    ops = yee.YeeOperators(n, wl.FCC, k)
    x, y = _rand(rng, (1, 3, n, n, n)), _rand(rng, (1, 3, n, n, n))
    g = penalty.gamma_practical(k)
    lhs = _vdot(y, fourier.apply_definition(x, ops, am, g))
    rhs = _vdot(fourier.apply_definition(y, ops, am, g), x)
    assert abs(lhs - rhs) <= 1e-13 * abs(lhs) * n ** 2


@pytest.mark.parametrize("lattice", ["SC", "FCC", "BCC"])
def test_symbols_have_the_continuum_limit(lattice):
    """The Fourier symbol of hat D tends to the continuum symbol of
    grad_{A,k} = A^{-T} grad_{x'} + i k (Sec. 2.2 eq. ct_newnabla): for the
    plane wave exp(2 pi i p.x') of mode p (p in (-N/2, N/2]) that symbol is
    q = i (A^{-T} 2 pi p + k).  The staggered differences carry a half-cell
    phase exp(-i pi p_j / N) per axis, so the phase-free quantity |kappa|^2
    is compared with |q|^2 for every lattice (O(h^2)), and for the simple
    cubic lattice each component, with its phase removed, is compared with
    q_i (O(h^2))."""
    lat = getattr(wl, lattice)
    k = np.array([0.7, -0.4, 1.3])
    p = np.array([1, -2, 1])                      # (p1, p2, p3)
    cont = 1j * (np.linalg.inv(lat).T @ (2 * np.pi * p) + k)
    errs, comp_errs = [], []
    for n in (16, 32, 64):
        kap = fourier.kappa(n, lat, k)
        idx = tuple(int(v) % n for v in p[::-1])      # array index (p3, p2, p1)
        kv = kap[(slice(None),) + idx]
        errs.append(abs(np.sum(np.abs(kv) ** 2) - np.sum(np.abs(cont) ** 2)))
        if lattice == "SC":
            comp_errs.append(np.abs(kv * np.exp(1j * np.pi * p / n) - cont).max())
    for e in (errs, comp_errs) if lattice == "SC" else (errs,):
        assert 3.5 < e[0] / e[1] < 4.5 and 3.5 < e[1] / e[2] < 4.5, e
    assert errs[-1] < 0.02 * np.sum(np.abs(cont) ** 2)


def test_homogeneous_m_is_the_constitutive_map():
    """Filled with one material, M applied to a uniform field is
    multiplication by epsilon_1 = eps^{-1} (Sec. 1 eq. intro_permittivity,
    Sec. 3.2.1 eq. trivial_trivial with I_i = I_V = I)."""
    rng = np.random.default_rng(7)
    eps = wl.hermitian_pd(rng, 2.0, 9.0)
    s = wl.homogeneous(eps)
    n = 4
    blocks = permittivity.cell_blocks(s, n)
    v = _rand(rng, 3)
    e = np.broadcast_to(v[:, None, None, None], (3, n, n, n))
    out = permittivity.apply_m(blocks, e)
    want = np.linalg.solve(eps, v)
    np.testing.assert_allclose(out[:, 1, 2, 3], want, rtol=1e-13)
