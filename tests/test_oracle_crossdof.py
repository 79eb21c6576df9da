"""Pins of the oracle's M_CrossDoF (Sec. 3.2.2, eqs. crossdof_xytemplate,
crossdof_Tmat, crossdof_herm): Hermiticity, reduction to M_Trivial for a
diagonal permittivity, constant fields in a homogeneous medium, the
geometry of the four-point transfer, and the per-mode closed form of a
homogeneous anisotropic medium."""
import numpy as np
import pytest

import workloads as wl
from oracle import crossdof, permittivity


def _rand(rng, shape):
    return rng.standard_normal(shape) + 1j * rng.standard_normal(shape)


def test_hermitian_on_an_anisotropic_structure():
    s = wl.sc_gyro_sphere()
    m = crossdof.CrossDofM(s, 8)
    rng = np.random.default_rng(0)
    x, y = _rand(rng, (3, 8, 8, 8)), _rand(rng, (3, 8, 8, 8))
    lhs = np.vdot(y, m.apply(x))
    rhs = np.vdot(m.apply(y), x)
    assert abs(lhs - rhs) <= 1e-13 * abs(lhs)


def test_diagonal_permittivity_reduces_to_m_trivial():
    rng = np.random.default_rng(1)
    eps = np.stack([wl.VACUUM, np.diag([9.0, 11.0, 13.0]).astype(np.complex128)])
    s = wl.Structure("diag", wl.SC.copy(), eps, 0, [wl.Shape(wl.SHAPE_SPHERE, 1, (0.5, 0.5, 0.5, 0.3))])
    x = _rand(rng, (2, 3, 8, 8, 8))
    got = crossdof.CrossDofM(s, 8).apply(x)
    want = permittivity.apply_m(permittivity.cell_blocks(s, 8), x)
    assert np.array_equal(got, want)


def test_constant_field_in_a_homogeneous_medium():
    rng = np.random.default_rng(2)
    eps = wl.hermitian_pd(rng, 2.0, 9.0)
    s = wl.homogeneous(eps, wl.SC)
    c = _rand(rng, 3)
    e = np.broadcast_to(c[:, None, None, None], (3, 6, 6, 6))
    got = crossdof.CrossDofM(s, 6).apply(e)
    want = (np.linalg.inv(eps) @ c)[:, None, None, None]
    assert np.abs(got - want).max() <= 1e-14 * np.abs(want).max()


@pytest.mark.parametrize("i,j", [(0, 1), (0, 2), (1, 2)])
def test_transfer_averages_the_four_nearest_dofs(i, j):
    """T_ij carries E^j to each E^i point as the mean of the four E^j points
    nearest to it (at distance h / sqrt 2), checked point by point against
    the staggered coordinates of Sec. 2.1."""
    n = 6
    names = ("E1", "E2", "E3")
    pi = permittivity.fractional_points(n, names[i]).reshape(-1, 3)
    pj = permittivity.fractional_points(n, names[j]).reshape(-1, 3)
    n3 = n ** 3
    eye = np.eye(n3).reshape(n3, n, n, n)
    t = crossdof.transfer(i, j, eye).reshape(n3, n3).T   # t[a, b]: weight of E^j point b at E^i point a
    for a in range(0, n3, 7):
        d = pj - pi[a]
        d -= np.round(d)                                # periodic
        dist = np.linalg.norm(d, axis=1)
        near = np.sort(np.flatnonzero(np.abs(dist - np.sqrt(0.5) / n) < 1e-12))
        assert len(near) == 4
        assert np.array_equal(np.sort(np.flatnonzero(t[a])), near)
        assert np.allclose(t[a, near], 0.25)
    # and the transpose is the adjoint
    tt = crossdof.transfer_t(i, j, eye).reshape(n3, n3).T
    assert np.array_equal(tt, t.T)


def test_homogeneous_spectrum_is_the_union_of_mode_blocks():
    """For a homogeneous anisotropic eps_1, D0 has the symbol
    (1 + exp(-2 pi i p / N)) / 2 and D0^T its conjugate, so M_CrossDoF has
    one 3 x 3 block per Fourier mode; its eigenvalues are the union of
    theirs."""
    n = 4
    rng = np.random.default_rng(3)
    eps = wl.hermitian_pd(rng, 2.0, 9.0)
    e1 = np.linalg.inv(eps)
    m = crossdof.CrossDofM(wl.homogeneous(eps, wl.SC), n).dense()
    assert np.abs(m - m.conj().T).max() <= 1e-15
    d0 = 0.5 * (1 + np.exp(-2j * np.pi * np.arange(n) / n))
    sym = {0: d0, 1: d0, 2: d0}   # along x, y, z (indices p1, p2, p3)
    want = []
    for p3 in range(n):
        for p2 in range(n):
            for p1 in range(n):
                p = (p1, p2, p3)
                t = {(0, 1): sym[0][p1] * np.conj(sym[1][p2]),
                     (0, 2): sym[0][p1] * np.conj(sym[2][p3]),
                     (1, 2): sym[1][p2] * np.conj(sym[2][p3])}
                b = np.diag(np.diag(e1).real).astype(np.complex128)
                for (a, c), v in t.items():
                    b[a, c] = e1[a, c] * v
                    b[c, a] = np.conj(e1[a, c] * v)
                want.extend(np.linalg.eigvalsh(b))
    got = np.linalg.eigvalsh(m)
    assert np.abs(np.sort(got) - np.sort(want)).max() <= 1e-13 * np.abs(want).max()


def test_hpd_under_the_papers_assumptions():
    """Sec. 3.3: M_CrossDoF is HPD when the eigenvalues of eps_1 lie in
    (0, 1] and eps_1 is strictly diagonally dominant or has a zero
    off-diagonal.  The paper's anisotropic eps_1 (eq. display:exp_permittivity,
    beta = 0.875, eps_lattice = 16) satisfies all three; a gyroid of it on
    the BCC lattice gives a dense M_CrossDoF with a positive spectrum."""
    eps = wl.paper_anisotropic(16.0)
    e1 = np.linalg.inv(eps)
    lam = np.linalg.eigvalsh(e1)
    assert lam.min() > 0 and lam.max() <= 1
    assert np.all(np.diag(e1).real > np.sum(np.abs(e1), axis=1) - np.abs(np.diag(e1)))
    s = wl.Structure("g", wl.BCC.copy(), np.stack([wl.VACUUM, eps]), 0, [wl.Shape(wl.SHAPE_GYROID, 1, (1.1, 0))])
    m = crossdof.CrossDofM(s, 6).dense()
    ev = np.linalg.eigvalsh(0.5 * (m + m.conj().T))
    assert ev.min() > 0
