"""GPU parity of the per-mode penalty form (PCX_PENALTY_PER_MODE: gamma_p =
4 pi^2 max(1, |kappa_p|^-2), the rule of Remark 2.6 applied mode by mode)
against the oracle, through the C ABI: the apply (five-pass FP64, three- and
five-pass FP32, M_CrossDoF, k-batched), K_P^{-1}, the T0 sandwich, the
penalty quadratic form, and solves near Gamma.  Tolerances: 1e-12 of the
largest entry (FP64 apply), 2e-5 (complex64 apply); eigenvalues 1e-10
(FP64) and 1e-6 (mixed) relative."""
import math

import numpy as np
import pytest

import workloads as wl
from oracle import crossdof, eig, fourier, learned, penalty, permittivity

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

FOUR_PI2 = 4.0 * math.pi ** 2
K_NEAR_GAMMA = np.array([0.06, -0.07, 0.03])


@pytest.fixture(scope="module")
def pcx():
    from paper_2511_17107_gb300 import build, pcx as binding
    build.build()
    assert torch.cuda.is_available(), "GPU tests need a CUDA device"
    return binding


def _err(got, want):
    return np.abs(got - want).max() / np.abs(want).max()


def _oracle_apply(s, n, k, x, m_kind="trivial"):
    kap = fourier.kappa(n, s.lattice, k)
    if m_kind == "crossdof":
        am = crossdof.CrossDofM(s, n).apply
    else:
        blocks = permittivity.cell_blocks(s, n)
        am = lambda e: permittivity.apply_m(blocks, e)
    return fourier.apply_symbols(x, kap, am, penalty.gamma_per_mode(kap))


def _per_mode_ctx(pcx, s, n, **kw):
    ctx = pcx.setup_structure(s, n, **kw)
    assert pcx.pcx_get_penalty_form(ctx) == pcx.PCX_PENALTY_SCALAR
    pcx.pcx_set_penalty_form(ctx, pcx.PCX_PENALTY_PER_MODE)
    assert pcx.pcx_get_penalty_form(ctx) == pcx.PCX_PENALTY_PER_MODE
    return ctx


def test_penalty_form_rejects_other_values(pcx):
    ctx = pcx.setup_structure(wl.sc_gyro_sphere(), 8)
    with pytest.raises(pcx.PcxError):
        pcx.pcx_set_penalty_form(ctx, 3)
    assert pcx.pcx_get_penalty_form(ctx) == pcx.PCX_PENALTY_SCALAR


@pytest.mark.parametrize("n,k", [(16, K_NEAR_GAMMA), (32, np.array([0.3, 0.9, -0.2])), (16, np.zeros(3))])
def test_per_mode_apply_fp64(pcx, n, k):
    s = wl.sc_gyro_sphere()
    x = wl.random_block(3, n, seed=41)
    want = _oracle_apply(s, n, k, x)
    ctx = _per_mode_ctx(pcx, s, n)
    X = torch.from_numpy(x).cuda()
    Y = torch.empty_like(X)
    pcx.pcx_apply(ctx, k, X, Y)
    torch.cuda.synchronize()
    assert _err(Y.cpu().numpy(), want) <= 1e-12


@pytest.mark.parametrize("path", ["three", "five"])
def test_per_mode_apply_fp32(pcx, path):
    n = 32
    s = wl.fcc_air_spheres()
    k = K_NEAR_GAMMA
    x = wl.random_block(3, n, seed=42).astype(np.complex64)
    want = _oracle_apply(s, n, k, x.astype(np.complex128))
    ctx = _per_mode_ctx(pcx, s, n)
    pcx.pcx_set_apply_path(ctx, pcx.PCX_APPLY_THREE_PASS if path == "three" else pcx.PCX_APPLY_FIVE_PASS)
    X = torch.from_numpy(x).cuda()
    Y = torch.empty_like(X)
    pcx.pcx_apply(ctx, k, X, Y)
    torch.cuda.synchronize()
    assert _err(Y.cpu().numpy(), want) <= 2e-5


def test_per_mode_apply_crossdof(pcx):
    n = 16
    s = wl.sc_gyro_sphere()
    k = K_NEAR_GAMMA
    x = wl.random_block(2, n, seed=43)
    want = _oracle_apply(s, n, k, x, "crossdof")
    ctx = _per_mode_ctx(pcx, s, n, m_kind=pcx.PCX_M_CROSSDOF)
    X = torch.from_numpy(x).cuda()
    Y = torch.empty_like(X)
    pcx.pcx_apply(ctx, k, X, Y)
    torch.cuda.synchronize()
    assert _err(Y.cpu().numpy(), want) <= 1e-12


def test_per_mode_apply_kbatch(pcx):
    n = 16
    s = wl.fcc_air_spheres()
    kpts = np.array([K_NEAR_GAMMA, [0.0, 0.0, 0.0], [1.1, 0.4, -0.7]])
    x = wl.random_block(3 * 2, n, seed=44).reshape(3, 2, 3, n, n, n)
    ctx = _per_mode_ctx(pcx, s, n)
    X = torch.from_numpy(x).cuda()
    Y = torch.empty_like(X)
    pcx.pcx_apply_kbatch(ctx, kpts, X, Y)
    torch.cuda.synchronize()
    got = Y.cpu().numpy()
    for i, k in enumerate(kpts):
        assert _err(got[i], _oracle_apply(s, n, k, x[i])) <= 1e-12


@pytest.mark.parametrize("prec", [0, 1])
def test_per_mode_preconditioners(pcx, prec):
    """K_P^{-1} and the T0 sandwich with gamma_p, FP64 and complex64."""
    n = 16
    s = wl.fcc_air_spheres()
    k = K_NEAR_GAMMA
    kap = fourier.kappa(n, s.lattice, k)
    g = penalty.gamma_per_mode(kap)
    blocks = permittivity.cell_blocks(s, n)
    r = wl.random_block(2, n, seed=45)
    dt = np.complex128 if prec == 0 else np.complex64
    tol = 1e-12 if prec == 0 else 2e-5
    ctx = _per_mode_ctx(pcx, s, n)
    R = torch.from_numpy(r.astype(dt)).cuda()
    W = torch.empty_like(R)
    pcx.pcx_precond(ctx, k, R, W)
    torch.cuda.synchronize()
    assert _err(W.cpu().numpy(), fourier.precondition(r, kap, g)) <= tol
    pcx.pcx_sandwich_precond(ctx, k, R, W)
    torch.cuda.synchronize()
    assert _err(W.cpu().numpy(), learned.sandwich_precondition(r, kap, blocks, g)) <= tol


def test_per_mode_penalty_quadratic_form(pcx):
    """pcx_div_norms weighs each mode by gamma_p / gamma: out[j] times gamma
    is x_j^H (gamma_p K_B) x_j."""
    n = 16
    s = wl.sc_gyro_sphere()
    k = K_NEAR_GAMMA
    kap = fourier.kappa(n, s.lattice, k)
    g = penalty.gamma_per_mode(kap)
    x = wl.random_block(3, n, seed=46)
    kbx = fourier._per_mode(fourier.kb_matrix(kap), x)
    want = np.real(np.sum(np.conj(x) * g * kbx, axis=(1, 2, 3, 4))) / FOUR_PI2
    ctx = _per_mode_ctx(pcx, s, n)
    X = torch.from_numpy(x).cuda()
    out = torch.zeros(6, dtype=torch.float64, device="cuda")
    pcx.pcx_div_norms(ctx, k, X, out)
    torch.cuda.synchronize()
    got = out.cpu().numpy()
    np.testing.assert_allclose(got[:3], want, rtol=1e-11)
    np.testing.assert_allclose(got[3:], np.sum(np.abs(x) ** 2, axis=(1, 2, 3, 4)), rtol=1e-12)


def _dense_lowest_per_mode(s, n, k, nev):
    kap = fourier.kappa(n, s.lattice, k)
    blocks = permittivity.cell_blocks(s, n)
    am = lambda e: permittivity.apply_m(blocks, e)
    g = penalty.gamma_per_mode(kap)
    shape = (3, n, n, n)
    mat = eig.dense_matrix(
        lambda c: fourier.apply_symbols(c.reshape((-1,) + shape), kap, am, g).reshape(c.shape[0], -1), 3 * n ** 3)
    ev = np.linalg.eigvalsh(0.5 * (mat + mat.conj().T))
    return ev[ev > 1e-9 * ev.max()][:nev]


@pytest.mark.parametrize("prec,rtol", [(0, 1e-10), (1, 1e-6)])
def test_per_mode_solve_matches_dense_8(pcx, prec, rtol):
    n, nev = 8, 6
    s = wl.sc_gyro_sphere()
    k = np.array([0.3, -0.25, 0.2])
    want = _dense_lowest_per_mode(s, n, k, nev)
    ctx = _per_mode_ctx(pcx, s, n)
    ev, res, its, st = pcx.pcx_solve(ctx, [k], nev, 1e-10, block=nev + 4, precision=prec)
    assert st == pcx.PCX_OK and np.all(res <= 1e-10)
    np.testing.assert_allclose(ev[0], want, rtol=rtol)


def test_per_mode_solve_near_gamma_reaches_1e8_at_64(pcx):
    """FCC air spheres at 64^3, |k| = 0.1: the scalar rule's gamma ~ 3950
    lifts the top of the spectrum to ~12 N^2 gamma ~ 2e8 (FP64 residual
    floor ~1e-8); the per-mode form keeps it at ~12 N^2 4 pi^2, and the
    solve reaches Res_j <= 1e-8 in FP64 and mixed precision with the same
    eigenvalues as the scalar form solved to 1e-6."""
    n, nev = 64, 6
    s = wl.fcc_air_spheres()
    k = np.array([0.1, 0.0, 0.0])
    ctx_s = pcx.setup_structure(s, n)
    ev_s, res_s, _, _ = pcx.pcx_solve(ctx_s, [k], nev, 1e-6, block=nev + 4, precision=1, raise_on_noconv=False)
    assert np.all(res_s <= 1e-6)
    ctx = _per_mode_ctx(pcx, s, n)
    for prec in (0, 1):
        ev, res, its, st = pcx.pcx_solve(ctx, [k], nev, 1e-8, block=nev + 4, precision=prec, maxit=400)
        assert st == pcx.PCX_OK and np.all(res <= 1e-8), (prec, res)
        np.testing.assert_allclose(ev[0], ev_s[0], rtol=2e-6)


def _projector_ctx(pcx, s, n, **kw):
    ctx = pcx.setup_structure(s, n, **kw)
    pcx.pcx_set_penalty_form(ctx, pcx.PCX_PENALTY_PROJECTOR)
    assert pcx.pcx_get_penalty_form(ctx) == pcx.PCX_PENALTY_PROJECTOR
    return ctx


@pytest.mark.parametrize("dtype,path,tol", [(np.complex128, None, 1e-12), (np.complex64, "three", 2e-5),
                                            (np.complex64, "five", 2e-5)])
def test_projector_apply_and_preconditioners(pcx, dtype, path, tol):
    """The projector form gamma_p = 16 pi^2 / |kappa_p|^2 against the oracle:
    the apply (both pass structures in complex64), K_P^{-1} and T0."""
    n = 32
    s = wl.fcc_air_spheres()
    k = np.array([0.4, -1.1, 0.7])
    kap = fourier.kappa(n, s.lattice, k)
    g = penalty.gamma_projector(kap)
    blocks = permittivity.cell_blocks(s, n)
    x = wl.random_block(2, n, seed=47)
    want = fourier.apply_symbols(x, kap, lambda e: permittivity.apply_m(blocks, e), g)
    ctx = _projector_ctx(pcx, s, n)
    if path is not None:
        pcx.pcx_set_apply_path(ctx, pcx.PCX_APPLY_THREE_PASS if path == "three" else pcx.PCX_APPLY_FIVE_PASS)
    X = torch.from_numpy(x.astype(dtype)).cuda()
    Y = torch.empty_like(X)
    pcx.pcx_apply(ctx, k, X, Y)
    torch.cuda.synchronize()
    assert _err(Y.cpu().numpy(), want) <= tol
    W = torch.empty_like(X)
    pcx.pcx_precond(ctx, k, X, W)
    torch.cuda.synchronize()
    assert _err(W.cpu().numpy(), fourier.precondition(x, kap, g)) <= tol
    pcx.pcx_sandwich_precond(ctx, k, X, W)
    torch.cuda.synchronize()
    assert _err(W.cpu().numpy(), learned.sandwich_precondition(x, kap, blocks, g)) <= tol


@pytest.mark.parametrize("prec,rtol", [(0, 1e-10), (1, 1e-6)])
def test_projector_solve_matches_scalar_form(pcx, prec, rtol):
    """The projector form keeps the physical eigenpairs: the 8^3 solve
    returns the lowest eigenvalues of the scalar form's dense operator."""
    n, nev = 8, 6
    s = wl.sc_gyro_sphere()
    k = np.array([0.6, 1.3, -0.5])
    kap = fourier.kappa(n, s.lattice, k)
    blocks = permittivity.cell_blocks(s, n)
    am = lambda e: permittivity.apply_m(blocks, e)
    shape = (3, n, n, n)
    mat = eig.dense_matrix(lambda c: fourier.apply_symbols(c.reshape((-1,) + shape), kap, am,
                                                           penalty.gamma_practical(k)).reshape(c.shape[0], -1),
                           3 * n ** 3)
    ev_d = np.linalg.eigvalsh(0.5 * (mat + mat.conj().T))
    want = ev_d[ev_d > 1e-9 * ev_d.max()][:nev]
    ctx = _projector_ctx(pcx, s, n)
    ev, res, its, st = pcx.pcx_solve(ctx, [k], nev, 1e-10, block=nev + 4, precision=prec)
    assert st == pcx.PCX_OK and np.all(res <= 1e-10)
    np.testing.assert_allclose(ev[0], want, rtol=rtol)
