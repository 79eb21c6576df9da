"""GPU parity of the operator apply, the preconditioner and the block
kernels against the CPU oracle (element by element), through the C ABI.

Tolerances: every output is compared as |y_gpu - y_oracle| <= tol *
max|y_oracle|.  Each 1D transform stage adds at most a few units in the last
place relative to the largest entry, over log2 N^3 <= 24 stages plus the
pointwise products (the symbols reach |kappa| <= 2 sqrt 3 / h, absorbed by
normalising with max|y|): tol = 1e-12 for FP64, and 24 * 4u * 3 ~ 2e-5 with
u = 6e-8 for FP32 storage and arithmetic.
"""
import numpy as np
import pytest

import workloads as wl
from oracle import fourier, penalty, permittivity, yee

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

TOL = {np.complex128: 1e-12, np.complex64: 2e-5}


@pytest.fixture(scope="module")
def pcx():
    from paper_2511_17107_gb300 import build, pcx as binding
    build.build()
    assert torch.cuda.is_available(), "GPU tests need a CUDA device"
    return binding


def _oracle_apply(structure, n, k, x, m=1, reading="summed"):
    blocks = permittivity.cell_blocks(structure, n)
    ops = yee.YeeOperators(n, structure.lattice, k, m, reading)
    g = penalty.gamma_practical(k)
    return fourier.apply_definition(x, ops, lambda e: permittivity.apply_m(blocks, e), g)


def _close(got, want, dtype):
    err = np.abs(got - want).max() / np.abs(want).max()
    assert err <= TOL[dtype], err
    return err


CASES = [
    # name, structure maker, N, dtype, nvec, stencil m, reading
    ("sc8-f64", wl.sc_gyro_sphere, 8, np.complex128, 3, 1, "summed"),
    ("sc16-f64", wl.sc_gyro_sphere, 16, np.complex128, 2, 1, "summed"),
    ("fcc16-f64", wl.fcc_air_spheres, 16, np.complex128, 2, 1, "summed"),
    ("diamond32-f64", wl.diamond_rods, 32, np.complex128, 1, 1, "summed"),
    ("sc32-f32", wl.sc_gyro_sphere, 32, np.complex64, 3, 1, "summed"),
    ("fcc32-f32", wl.fcc_air_spheres, 32, np.complex64, 2, 1, "summed"),
    ("woodpile16-m3-f64", wl.woodpile, 16, np.complex128, 2, 3, "summed"),
    ("sc16-m5-f64", wl.sc_gyro_sphere, 16, np.complex128, 1, 5, "summed"),
    ("fcc16-m4-f32", wl.fcc_air_spheres, 16, np.complex64, 1, 4, "summed"),
    ("fcc16-literal-f64", wl.fcc_air_spheres, 16, np.complex128, 1, 1, "literal"),
    ("random64-f32", lambda: wl.random_inclusions(3), 64, np.complex64, 1, 2, "summed"),
]


@pytest.mark.parametrize("name,maker,n,dtype,nvec,m,reading", CASES, ids=[c[0] for c in CASES])
def test_apply_matches_oracle(pcx, name, maker, n, dtype, nvec, m, reading):
    s = maker()
    k = wl.config_k(s.name)[min(3, len(wl.config_k(s.name)) - 1)] if not s.name.startswith("random") else \
        np.array([np.pi, np.pi, np.pi])
    x = wl.random_block(nvec, n, seed=11).astype(dtype)
    want = _oracle_apply(s, n, k, x.astype(np.complex128), m, reading)
    ctx = pcx.setup_structure(s, n, stencil_m=m, ct_reading=pcx.PCX_CT_LITERAL if reading == "literal" else 0)
    X = torch.from_numpy(x).cuda()
    Y = torch.empty_like(X)
    pcx.pcx_apply(ctx, k, X, Y)
    torch.cuda.synchronize()
    _close(Y.cpu().numpy(), want, dtype)


@pytest.mark.parametrize("dtype", [np.complex64, np.complex128])
def test_apply_at_k_zero_and_host_entry(pcx, dtype):
    """k = 0 (mode p = 0 maps to 0) and the host-buffer entry point."""
    n = 16
    s = wl.sc_gyro_sphere()
    k = np.zeros(3)
    x = wl.random_block(2, n, seed=5).astype(dtype)
    want = _oracle_apply(s, n, k, x.astype(np.complex128))
    ctx = pcx.setup_structure(s, n)
    y = np.zeros_like(x)
    pcx.pcx_apply_host(ctx, k, x, y)
    _close(y, want, dtype)
    assert np.abs(y[:, :, 0, 0, 0]).max() <= TOL[dtype] * np.abs(want).max()


@pytest.mark.parametrize("nvec,pinned", [(7, False), (10, True), (17, True)])
def test_apply_host_pipelined_chunks(pcx, nvec, pinned):
    """pcx_apply_host moves the block in chunks through two staging slots on
    three streams; every chunking (1, 2 and 3 vectors, ragged tails, slot
    reuse) gives the device entry's result bit for bit, from pageable and
    pinned host memory."""
    n = 32
    s = wl.fcc_air_spheres()
    k = wl.config_k(s.name)[3]
    x = wl.random_block(nvec, n, seed=40 + nvec).astype(np.complex64)
    ctx = pcx.setup_structure(s, n)
    X = torch.from_numpy(x).cuda()
    Y = torch.empty_like(X)
    pcx.pcx_apply(ctx, k, X, Y)
    torch.cuda.synchronize()
    want = Y.cpu().numpy()
    xh = torch.from_numpy(x)
    yh = torch.zeros_like(xh)
    if pinned:
        xh, yh = xh.pin_memory(), yh.pin_memory()
    for _ in range(2):   # the second call reuses the staging slots and events
        yh.zero_()
        pcx.pcx_apply_host(ctx, k, xh, yh)
        assert np.array_equal(yh.numpy(), want)


@pytest.mark.parametrize("vpk,xs,ys,pinned", [(6, 6, 6, True), (5, 5, 0, False), (3, 0, 3, True), (8, 9, 8, True)])
def test_apply_kbatch_host(pcx, vpk, xs, ys, pinned):
    """pcx_apply_kbatch_host: three Bloch vectors, vec_per_k vectors each,
    input and output groups at the given strides (0: one block reused).
    Every group's images equal the device k-batched entry's bit for bit
    (for output stride 0, the last k's)."""
    n, nk = 32, 3
    s = wl.fcc_air_spheres()
    ks = wl.config_k(s.name)[2:2 + nk]
    nx = (nk - 1) * xs + vpk
    x = wl.random_block(nx, n, seed=60 + vpk).astype(np.complex64)
    ctx = pcx.setup_structure(s, n)
    xg = np.stack([x[i * xs:i * xs + vpk] for i in range(nk)])
    X = torch.from_numpy(xg).cuda()
    Y = torch.empty_like(X)
    pcx.pcx_apply_kbatch(ctx, ks, X, Y)
    torch.cuda.synchronize()
    want = Y.cpu().numpy()
    xh = torch.from_numpy(x)
    yh = torch.zeros(((nk - 1) * ys + vpk,) + x.shape[1:], dtype=torch.complex64)
    if pinned:
        xh, yh = xh.pin_memory(), yh.pin_memory()
    pcx.pcx_apply_kbatch_host(ctx, ks, xh, yh, vpk, x_stride=xs, y_stride=ys)
    got = yh.numpy()
    if ys == 0:
        assert np.array_equal(got, want[-1])
    else:
        for i in range(nk):
            assert np.array_equal(got[i * ys:i * ys + vpk], want[i]), i
    with pytest.raises(pcx.PcxError):
        pcx.pcx_apply_kbatch_host(ctx, ks, xh, yh, vpk, x_stride=-1, y_stride=ys)


@pytest.mark.parametrize("name,maker,n,dtype,nvec,chunk", [
    ("sc16-f64", wl.sc_gyro_sphere, 16, np.complex128, 3, 0),
    ("sc16-f64-chunk1", wl.sc_gyro_sphere, 16, np.complex128, 3, 1),
    ("fcc16-f64", wl.fcc_air_spheres, 16, np.complex128, 2, 0),
    ("sc32-f32", wl.sc_gyro_sphere, 32, np.complex64, 2, 0),
], ids=lambda v: v if isinstance(v, str) else None)
def test_apply_crossdof_matches_oracle(pcx, name, maker, n, dtype, nvec, chunk):
    """M_CrossDoF (Sec. 3.2.2): the seven-pass apply (z sandwich split into
    transforms around the real-space cross-DoF stencil) against the oracle's
    operator on the oracle's M_CrossDoF; chunked launches and the k-batched
    entry give the same bits as one launch per k."""
    from oracle import crossdof, penalty
    s = maker()
    k = wl.config_k(s.name)[min(3, len(wl.config_k(s.name)) - 1)]
    x = wl.random_block(nvec, n, seed=31).astype(dtype)
    ops = yee.YeeOperators(n, s.lattice, k)
    want = fourier.apply_definition(x.astype(np.complex128), ops, crossdof.CrossDofM(s, n).apply,
                                    penalty.gamma_practical(k))
    ctx = pcx.setup_structure(s, n, m_kind=pcx.PCX_M_CROSSDOF)
    if chunk:
        pcx.pcx_set_apply_chunk(ctx, chunk)
    X = torch.from_numpy(x).cuda()
    Y = torch.empty_like(X)
    pcx.pcx_apply(ctx, k, X, Y)
    torch.cuda.synchronize()
    _close(Y.cpu().numpy(), want, dtype)
    Yb = torch.empty((2,) + tuple(X.shape), dtype=X.dtype, device="cuda")
    pcx.pcx_apply_kbatch(ctx, np.stack([k, k]), torch.stack([X, X]), Yb)
    torch.cuda.synchronize()
    assert torch.equal(Yb[0], Y) and torch.equal(Yb[1], Y)


def test_apply_full_size_bench_workload(pcx):
    """The benchmark's workload: 128^3 diamond rods, complex64, checked on a
    full vector against the oracle (2 vectors of the timed launch shape)."""
    n = 128
    s = wl.diamond_rods()
    k = wl.config_k(s.name)[5]
    x = wl.random_block(2, n, seed=20251117).astype(np.complex64)
    ctx = pcx.setup_structure(s, n)
    X = torch.from_numpy(x).cuda()
    Y = torch.empty_like(X)
    pcx.pcx_apply(ctx, k, X, Y)
    torch.cuda.synchronize()
    got = Y.cpu().numpy()
    want = _oracle_apply(s, n, k, x[1:2].astype(np.complex128))
    _close(got[1:2], want, np.complex64)


@pytest.mark.parametrize("dtype", [np.complex64, np.complex128])
def test_apply_dense_cell_blocks_and_chunking(pcx, dtype):
    """Caller-supplied cell blocks (the dense M path) agree with the oracle
    and with the material-id path, for several chunk sizes (1, 2, default)."""
    n = 32
    s = wl.fcc_air_spheres()
    k = wl.config_k(s.name)[7]
    ob = permittivity.cell_blocks(s, n).reshape(-1, 3, 3)
    packed = np.stack([ob[:, 0, 0].real, ob[:, 1, 1].real, ob[:, 2, 2].real, ob[:, 0, 1].real, ob[:, 0, 1].imag,
                       ob[:, 0, 2].real, ob[:, 0, 2].imag, ob[:, 1, 2].real, ob[:, 1, 2].imag], axis=1)
    dense = pcx.pcx_setup(n, s.lattice, cell_blocks=packed)
    ids = pcx.setup_structure(s, n)
    x = wl.random_block(3, n, seed=2).astype(dtype)
    want = _oracle_apply(s, n, k, x.astype(np.complex128))
    X = torch.from_numpy(x).cuda()
    for ctx in (dense, ids):
        for chunk in (1, 2, 0):
            pcx.pcx_set_apply_chunk(ctx, chunk)
            Y = torch.empty_like(X)
            pcx.pcx_apply(ctx, k, X, Y)
            _close(Y.cpu().numpy(), want, dtype)


def test_apply_rejects_bad_arguments(pcx):
    n = 8
    ctx = pcx.setup_structure(wl.sc_gyro_sphere(), n)
    X = torch.zeros((1, 3, n, n, n), dtype=torch.complex64, device="cuda")
    with pytest.raises(pcx.PcxError) as e:
        pcx.pcx_apply(ctx, [0.1, 0.2, 0.3], X, X)
    assert e.value.status == pcx.PCX_EINVAL
    with pytest.raises(pcx.PcxError):
        pcx.pcx_setup(12, wl.SC, np.stack([wl.VACUUM]), 0, [])


@pytest.mark.parametrize("dtype,lat,kvec", [(np.complex128, "SC", (0.3, -1.2, 2.0)), (np.complex64, "FCC", (1.0, 0.5, 3.0)),
                                            (np.complex128, "SC", (0.0, 0.0, 0.0))])
def test_precond_matches_oracle(pcx, dtype, lat, kvec):
    n = 16
    lattice = getattr(wl, lat)
    s = wl.homogeneous(wl.VACUUM, lattice)
    k = np.array(kvec)
    g = penalty.gamma_practical(k)
    r = wl.random_block(3, n, seed=9).astype(dtype)
    want = fourier.precondition(r.astype(np.complex128), fourier.kappa(n, lattice, k), g)
    ctx = pcx.setup_structure(s, n)
    R = torch.from_numpy(r).cuda()
    W = torch.empty_like(R)
    pcx.pcx_precond(ctx, k, R, W)
    _close(W.cpu().numpy(), want, dtype)
    pcx.pcx_precond(ctx, k, R, R)          # in place
    _close(R.cpu().numpy(), want, dtype)


@pytest.mark.parametrize("dtype", [np.complex64, np.complex128])
@pytest.mark.parametrize("na,nb,L", [(5, 7, 1000), (48, 48, 3 * 16 ** 3), (33, 17, 12345)])
def test_gram_combine_residual(pcx, dtype, na, nb, L):
    rng = np.random.default_rng(na + nb)
    a = (rng.standard_normal((na, L)) + 1j * rng.standard_normal((na, L))).astype(dtype)
    b = (rng.standard_normal((nb, L)) + 1j * rng.standard_normal((nb, L))).astype(dtype)
    A, B = torch.from_numpy(a).cuda(), torch.from_numpy(b).cuda()
    G = torch.empty((na, nb), dtype=torch.complex128, device="cuda")
    pcx.pcx_gram(A, B, G)
    want = a.astype(np.complex128).conj() @ b.astype(np.complex128).T
    tol = 1e-12 if dtype == np.complex128 else 1e-5
    assert np.abs(G.cpu().numpy() - want).max() <= tol * np.abs(want).max() * 10
    c = rng.standard_normal((na, nb)) + 1j * rng.standard_normal((na, nb))
    Y = torch.from_numpy(b.copy()).cuda()
    pcx.pcx_combine(A, torch.from_numpy(c).cuda(), Y, beta=0.5)
    wantc = c.T @ a.astype(np.complex128) + 0.5 * b
    assert np.abs(Y.cpu().numpy() - wantc).max() <= TOL[dtype] * 10 * np.abs(wantc).max()
    th = rng.uniform(0, 5, size=nb)
    R = torch.empty_like(B)
    norms = torch.zeros(2 * nb, dtype=torch.float64, device="cuda")
    pcx.pcx_residual(B, Y, torch.from_numpy(th).cuda(), R, norms)
    wr = Y.cpu().numpy().astype(np.complex128) - th[:, None] * b
    assert np.abs(R.cpu().numpy() - wr).max() <= TOL[dtype] * 10 * np.abs(wr).max()
    nr = norms.cpu().numpy()
    np.testing.assert_allclose(nr[:nb], np.sum(np.abs(R.cpu().numpy().astype(np.complex128)) ** 2, axis=1), rtol=1e-5)
    np.testing.assert_allclose(nr[nb:], np.sum(np.abs(b.astype(np.complex128)) ** 2, axis=1), rtol=1e-5)


@pytest.mark.parametrize("same", [True, False])
@pytest.mark.parametrize("na,nb", [(48, 48), (64, 16), (1, 1)])
def test_gram_tensor_cores_long_blocks(pcx, same, na, nb):
    """complex64 Gram products run on the tensor cores (TF32 with error
    compensation, FP64 sums across CTAs); checked against FP64 products of
    the same FP32 data over L = 3 * 64^3 rows."""
    if same:
        nb = na
    L = 3 * 64 ** 3
    rng = np.random.default_rng(na * 7 + nb)
    a = (rng.standard_normal((na, L)) + 1j * rng.standard_normal((na, L))).astype(np.complex64)
    b = a if same else (rng.standard_normal((nb, L)) + 1j * rng.standard_normal((nb, L))).astype(np.complex64)
    A = torch.from_numpy(a).cuda()
    B = A if same else torch.from_numpy(b).cuda()
    G = torch.empty((na, nb), dtype=torch.complex128, device="cuda")
    pcx.pcx_gram(A, B, G)
    want = a.astype(np.complex128).conj() @ b.astype(np.complex128).T
    err = np.abs(G.cpu().numpy() - want).max() / np.abs(want).max()
    assert err <= 1e-5, err


@pytest.mark.parametrize("path", ["tensor", "fp32"])
@pytest.mark.parametrize("same,na,nb,L", [(False, 16, 16, 3 * 64 ** 3), (True, 48, 48, 3 * 64 ** 3),
                                          (False, 48, 48, 3 * 32 ** 3 + 2), (False, 13, 29, 1234),
                                          (True, 29, 29, 3 * 16 ** 3), (False, 64, 7, 66), (True, 1, 1, 2),
                                          (False, 3, 5, 200002)])
def test_gram_paths_agree_with_fp64(pcx, path, same, na, nb, L):
    """Both complex64 Gram kernels (tensor cores, FP32 pipes), selected with
    pcx_set_gram_path, against FP64 products of the same FP32 data: shapes
    of the eigensolver's blocks, ragged column counts, row counts that end
    inside a stage, A^H A (upper triangle mirrored) and a column block that
    starts inside a larger allocation."""
    rng = np.random.default_rng(na * 31 + nb + L % 97)
    a = (rng.standard_normal((na + 2, L)) + 1j * rng.standard_normal((na + 2, L))).astype(np.complex64)
    b = a[2:] if same else (rng.standard_normal((nb, L)) + 1j * rng.standard_normal((nb, L))).astype(np.complex64)
    Afull = torch.from_numpy(a).cuda()
    A = Afull[2:]                       # starts two columns into the allocation
    B = A if same else torch.from_numpy(b).cuda()
    G = torch.empty((na, nb), dtype=torch.complex128, device="cuda")
    pcx.pcx_set_gram_path(pcx.PCX_GRAM_TENSOR if path == "tensor" else pcx.PCX_GRAM_FP32)
    try:
        pcx.pcx_gram(A, B, G)
    finally:
        pcx.pcx_set_gram_path(pcx.PCX_GRAM_AUTO)
    a64 = a[2:].astype(np.complex128)
    want = a64.conj() @ b.astype(np.complex128).T
    err = np.abs(G.cpu().numpy() - want).max() / np.abs(want).max()
    assert err <= 1e-5, err
    if same and path == "fp32":   # the lower triangle mirrors the upper one, bit for bit
        g = G.cpu().numpy()
        assert np.array_equal(g, g.conj().T)


@pytest.mark.parametrize("same", [True, False])
def test_gram_fp64_on_fp32_pipes(pcx, same):
    """complex128 Gram products by split FP32 hi/lo products and double-float
    accumulation, against numpy FP64 products (relative 1e-12 of max|G|)."""
    na = nb = 48
    L = 3 * 64 ** 3
    rng = np.random.default_rng(5 + same)
    a = rng.standard_normal((na, L)) + 1j * rng.standard_normal((na, L))
    b = a if same else rng.standard_normal((nb, L)) + 1j * rng.standard_normal((nb, L))
    A = torch.from_numpy(a).cuda()
    B = A if same else torch.from_numpy(b).cuda()
    G = torch.empty((na, nb), dtype=torch.complex128, device="cuda")
    pcx.pcx_gram(A, B, G)
    want = a.conj() @ b.T
    err = np.abs(G.cpu().numpy() - want).max() / np.abs(want).max()
    assert err <= 1e-12, err


@pytest.mark.parametrize("na,nb,L", [(33, 5, 3 * 17 ** 3), (32, 32, 3 * 64 ** 3), (1, 40, 1), (7, 1, 31)])
def test_gram_mixed_fp64_fp32(pcx, na, nb, L):
    """pcx_gram_mixed: complex128 rows against complex64 columns, with the
    columns of B orthogonalised against A before rounding to FP32 so that
    G is ~1e-7 of the norms (the cancelling case of the mixed Rayleigh-Ritz
    rows).  Entries of A span twelve decades and include exact zeros.
    Absolute error <= 1e-13 of max ||a_i|| ||b_j|| against numpy FP64."""
    rng = np.random.default_rng(na * 131 + nb + L)
    scale = 10.0 ** rng.uniform(-8, 4, size=(na, L))
    a = (rng.standard_normal((na, L)) + 1j * rng.standard_normal((na, L))) * scale
    a[:, 1::97] = 0.0
    b = rng.standard_normal((nb, L)) + 1j * rng.standard_normal((nb, L))
    if na < L:
        q, _ = np.linalg.qr(a.T)
        b = b - (b @ q.conj()) @ q.T
    b32 = b.astype(np.complex64)
    A = torch.from_numpy(a).cuda()
    B = torch.from_numpy(b32).cuda()
    G = torch.empty((na, nb), dtype=torch.complex128, device="cuda")
    pcx.pcx_gram_mixed(A, B, G)
    want = a.conj() @ b32.astype(np.complex128).T
    norm = np.linalg.norm(a, axis=1).max() * np.linalg.norm(b32.astype(np.complex128), axis=1).max()
    err = np.abs(G.cpu().numpy() - want).max() / norm
    assert err <= 1e-13, err


DIV_CASES = [
    ("fcc16-f64", wl.fcc_air_spheres, 16, np.complex128, 1, "summed"),
    ("woodpile16-m3-f64", wl.woodpile, 16, np.complex128, 3, "summed"),
    ("fcc8-literal-f64", wl.fcc_air_spheres, 8, np.complex128, 1, "literal"),
    ("sc32-f32", wl.sc_gyro_sphere, 32, np.complex64, 2, "summed"),
]


@pytest.mark.parametrize("name,maker,n,dtype,m,reading", DIV_CASES, ids=[c[0] for c in DIV_CASES])
def test_div_norms_match_real_space_divergence(pcx, name, maker, n, dtype, m, reading):
    """pcx_div_norms: x^H K_B x equals ||B h||^2 of the real-space field
    h = F3_3 x, with B built from the oracle's stencils (Sec. 2.2) rather than
    from the Fourier symbols; also ||x||^2."""
    s = maker()
    k = np.array([0.9, -1.7, 2.3])
    x = wl.random_block(3, n, seed=21).astype(dtype)
    ops = yee.YeeOperators(n, s.lattice, k, m, reading)
    h = fourier.f3(x.astype(np.complex128))
    want_b = np.array([np.sum(np.abs(ops.div(h[j])) ** 2) for j in range(3)])
    want_x = np.sum(np.abs(x.astype(np.complex128)) ** 2, axis=(1, 2, 3, 4))
    ctx = pcx.setup_structure(s, n, stencil_m=m, ct_reading=pcx.PCX_CT_LITERAL if reading == "literal" else 0)
    out = torch.zeros(6, dtype=torch.float64, device="cuda")
    pcx.pcx_div_norms(ctx, k, torch.from_numpy(x).cuda(), out)
    got = out.cpu().numpy()
    rtol = 1e-12 if dtype == np.complex128 else 1e-5
    np.testing.assert_allclose(got[:3], want_b, rtol=rtol)
    np.testing.assert_allclose(got[3:], want_x, rtol=rtol)
