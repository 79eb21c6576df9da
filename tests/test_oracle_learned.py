"""Pins of the learned-correction oracle (oracle/learned.py) against
definitions outside it: scipy's periodic correlation, the circular
correlation theorem through numpy FFTs, the adjoint identity, central finite
differences of the loss, the exact inverse of a homogeneous isotropic medium,
Hermitian symmetry, a dense-solve reconstruction of Op^{-1} r, and the limit
in which T reduces to the curl-sandwich base T0."""
import numpy as np
import pytest

import workloads as wl
from oracle import fourier, learned, permittivity

ndimage = pytest.importorskip("scipy.ndimage")


def _rand_params(rng, c, scale=0.3):
    p = {name: rng.standard_normal(shape) * scale for name, shape in learned.param_shapes(c)}
    return p


def test_conv_matches_scipy_periodic_correlation():
    rng = np.random.default_rng(0)
    x = rng.standard_normal((2, 5, 6, 7))
    w = rng.standard_normal((3, 2, 3, 3, 3))
    got = learned.conv(x, w)
    want = np.zeros_like(got)
    for o in range(3):
        for i in range(2):
            want[o] += ndimage.correlate(x[i], w[o, i], mode="wrap")
    np.testing.assert_allclose(got, want, rtol=1e-12, atol=1e-12)


def test_conv_matches_correlation_theorem():
    """conv(x, w)[o] = sum_i IFFT(FFT(x_i) * conj(FFT(k_oi))) with k the taps
    placed at the periodic offsets: an evaluation that shares nothing with
    the shifted sums of the oracle."""
    rng = np.random.default_rng(1)
    n = 6
    x = rng.standard_normal((2, n, n, n))
    w = rng.standard_normal((4, 2, 3, 3, 3))
    want = np.zeros((4, n, n, n))
    for o in range(4):
        for i in range(2):
            k = np.zeros((n, n, n))
            for dz, dy, dx in learned.OFFSETS:
                k[dz % n, dy % n, dx % n] = w[o, i, dz + 1, dy + 1, dx + 1]
            want[o] += np.real(np.fft.ifftn(np.fft.fftn(x[i]) * np.conj(np.fft.fftn(k))))
    np.testing.assert_allclose(learned.conv(x, w), want, rtol=1e-11, atol=1e-11)


def test_conv_adjoint_and_weight_gradient_identities():
    rng = np.random.default_rng(2)
    x = rng.standard_normal((3, 4, 5, 6))
    w = rng.standard_normal((2, 3, 3, 3, 3))
    dy = rng.standard_normal((2, 4, 5, 6))
    lhs = np.sum(dy * learned.conv(x, w))
    np.testing.assert_allclose(np.sum(learned.conv_adjoint(dy, w) * x), lhs, rtol=1e-12)
    np.testing.assert_allclose(np.sum(learned.conv_weight_grad(dy, x) * w), lhs, rtol=1e-12)


def test_loss_gradient_matches_finite_differences():
    rng = np.random.default_rng(3)
    c, n, nv = 2, 4, 2
    p = _rand_params(rng, c)
    f = rng.uniform(0.05, 1.0, size=(9, n, n, n))
    U = rng.standard_normal((nv, 3, n, n, n)) + 1j * rng.standard_normal((nv, 3, n, n, n))
    T = rng.standard_normal((nv, 3, n, n, n)) + 1j * rng.standard_normal((nv, 3, n, n, n))
    w = np.array([0.7, 1.3])
    _, grads = learned.loss_and_grad(p, f, U, T, w)
    flat = learned.pack(p, c)
    gflat = learned.pack(grads, c)
    idx = rng.choice(flat.size, size=60, replace=False)
    h = 1e-6
    for j in idx:
        fp = flat.copy()
        fm = flat.copy()
        fp[j] += h
        fm[j] -= h
        lp, _ = learned.loss_and_grad(learned.unpack(fp, c), f, U, T, w)
        lm, _ = learned.loss_and_grad(learned.unpack(fm, c), f, U, T, w)
        fd = (lp - lm) / (2 * h)
        assert abs(fd - gflat[j]) <= 1e-6 * max(1.0, abs(fd)), (j, fd, gflat[j])


def _small_case(n=8, seed=7):
    s = wl.random_inclusions(seed)
    blocks = permittivity.cell_blocks(s, n)
    k = np.array([0.4, -0.9, 1.7])
    kap = fourier.kappa(n, s.lattice, k)
    return learned.features(blocks), blocks, kap, 4 * np.pi ** 2


def _op(blocks, kap, gam):
    return lambda x: fourier.apply_symbols(x, kap, lambda e: permittivity.apply_m(blocks, e), gam)


def test_sandwich_inverts_the_operator_of_a_homogeneous_isotropic_medium():
    """M = m0 I: T0 Op r = r, the identity K_A K_A^H + K_B = |k|^2 I at work."""
    n, m0, gam = 6, 0.37, 4 * np.pi ** 2
    for lat in (wl.SC, wl.FCC):
        kap = fourier.kappa(n, lat, np.array([0.7, -1.3, 2.1]))
        blocks = np.broadcast_to(m0 * np.eye(3), (n, n, n, 3, 3)).astype(np.complex128)
        r = wl.random_block(2, n, seed=3)
        got = learned.sandwich_precondition(_op(blocks, kap, gam)(r), kap, blocks, gam)
        np.testing.assert_allclose(got, r, rtol=0, atol=1e-12 * np.abs(r).max())


def test_sandwich_is_hermitian_positive():
    f, blocks, kap, gam = _small_case()
    n = f.shape[-1]
    x = wl.random_block(1, n, seed=4)[0]
    y = wl.random_block(1, n, seed=5)[0]
    lhs = np.vdot(x, learned.sandwich_precondition(y, kap, blocks, gam))
    rhs = np.conj(np.vdot(y, learned.sandwich_precondition(x, kap, blocks, gam)))
    assert abs(lhs - rhs) <= 1e-12 * abs(lhs)
    assert np.vdot(x, learned.sandwich_precondition(x, kap, blocks, gam)).real > 0


def test_preconditioner_is_complex_linear_and_reduces_to_the_sandwich():
    rng = np.random.default_rng(4)
    f, blocks, kap, gam = _small_case()
    n = f.shape[-1]
    p = _rand_params(rng, learned.HIDDEN, 0.2)
    r1 = wl.random_block(1, n, seed=8)[0]
    r2 = wl.random_block(1, n, seed=9)[0]
    a, b = 0.3 - 1.1j, -2.0 + 0.5j
    lhs = learned.precondition(p, f, a * r1 + b * r2, kap, gam, blocks)
    rhs = a * learned.precondition(p, f, r1, kap, gam, blocks) + b * learned.precondition(p, f, r2, kap, gam, blocks)
    np.testing.assert_allclose(lhs, rhs, rtol=1e-11, atol=1e-11 * np.abs(rhs).max())
    p["W3"][:] = 0.0
    np.testing.assert_allclose(learned.precondition(p, f, r1, kap, gam, blocks),
                               learned.sandwich_precondition(r1, kap, blocks, gam), rtol=1e-13, atol=0)


def test_exact_training_pair_reconstructs_the_inverse():
    """With e = Op^{-1} r from a dense solve (N = 4), T0 r + K_A F3^H T / |k|^2
    built from the training pair equals e: the target carries exactly the
    part of the error that the correction can reach."""
    n = 4
    s = wl.random_inclusions(3)
    blocks = permittivity.cell_blocks(s, n)
    kap = fourier.kappa(n, s.lattice, np.array([0.9, -0.4, 1.3]))
    gam = 4 * np.pi ** 2
    op = _op(blocks, kap, gam)
    dim = 3 * n ** 3
    mat = np.stack([op(np.eye(dim)[j].reshape(3, n, n, n)).ravel() for j in range(dim)], axis=1)
    r = wl.random_block(1, n, seed=2)[0]
    e = np.linalg.solve(mat, r.ravel()).reshape(r.shape)
    U, T, en2 = learned.training_pair(r[None], e[None], kap, gam, blocks)
    rec = learned.sandwich_precondition(r, kap, blocks, gam) + learned.curl_scaled(fourier.f3h(T[0]), kap)
    np.testing.assert_allclose(rec, e, rtol=0, atol=1e-10 * np.abs(e).max())
    np.testing.assert_allclose(U[0], fourier.f3(learned.curl_h_scaled(r, kap)), rtol=1e-14)


def test_open_gates_reduce_to_plain_convolutions():
    """With V = 0 and large biases the gates are 1 and g is three plain
    convolutions, evaluated here through the correlation theorem."""
    rng = np.random.default_rng(6)
    c, n = 3, 5
    p = _rand_params(rng, c)
    p["V1"][:] = 0
    p["V2"][:] = 0
    p["c1"][:] = 60.0
    p["c2"][:] = 60.0
    f = rng.uniform(0, 1, size=(9, n, n, n))
    u = rng.standard_normal((3, n, n, n))

    def fftconv(x, w):
        out = np.zeros((w.shape[0], n, n, n))
        for o in range(w.shape[0]):
            for i in range(w.shape[1]):
                k = np.zeros((n, n, n))
                for dz, dy, dx in learned.OFFSETS:
                    k[dz % n, dy % n, dx % n] = w[o, i, dz + 1, dy + 1, dx + 1]
                out[o] += np.real(np.fft.ifftn(np.fft.fftn(x[i]) * np.conj(np.fft.fftn(k))))
        return out

    want = fftconv(fftconv(fftconv(u, p["W1"]), p["W2"]), p["W3"])
    got, _ = learned.forward_real(p, f, u)
    np.testing.assert_allclose(got, want, rtol=1e-10, atol=1e-10 * np.abs(want).max())


def test_features_layout():
    rng = np.random.default_rng(7)
    b = rng.standard_normal((2, 3, 4, 3, 3)) + 1j * rng.standard_normal((2, 3, 4, 3, 3))
    f = learned.features(b)
    assert f.shape == (9, 2, 3, 4)
    np.testing.assert_array_equal(f[0], b[..., 0, 0].real)
    np.testing.assert_array_equal(f[4], b[..., 0, 1].imag)
    np.testing.assert_array_equal(f[8], b[..., 1, 2].imag)
    assert learned.param_count(8) == 8 * 3 * 27 + 64 * 27 + 3 * 8 * 27 + 2 * (8 * 9 * 27 + 8)


def test_symmetric_form_gradient_matches_finite_differences():
    rng = np.random.default_rng(13)
    c, n, nv = 2, 4, 2
    p = _rand_params(rng, c)
    f = rng.uniform(0.05, 1.0, size=(9, n, n, n))
    U = rng.standard_normal((nv, 3, n, n, n)) + 1j * rng.standard_normal((nv, 3, n, n, n))
    T = rng.standard_normal((nv, 3, n, n, n)) + 1j * rng.standard_normal((nv, 3, n, n, n))
    w = np.array([0.9, 1.1])
    _, grads = learned.loss_and_grad(p, f, U, T, w, symmetric=True)
    flat = learned.pack(p, c)
    gflat = learned.pack(grads, c)
    h = 1e-4   # the loss is quadratic in each weight entry; 1e-4 keeps the FD rounding small
    for j in rng.choice(flat.size, size=60, replace=False):
        fp, fm = flat.copy(), flat.copy()
        fp[j] += h
        fm[j] -= h
        lp, _ = learned.loss_and_grad(learned.unpack(fp, c), f, U, T, w, symmetric=True)
        lm, _ = learned.loss_and_grad(learned.unpack(fm, c), f, U, T, w, symmetric=True)
        fd = (lp - lm) / (2 * h)
        assert abs(fd - gflat[j]) <= 1e-6 * max(1.0, abs(fd)), (j, fd, gflat[j])


def test_symmetric_form_is_symmetric_and_the_preconditioner_hermitian():
    """<v, g_s u> = <g_s v, u> for real fields (while g itself is not
    symmetric), and T(r) built on g_s is Hermitian: <x, T y> = conj <y, T x>."""
    rng = np.random.default_rng(14)
    c, n = 3, 5
    p = _rand_params(rng, c)
    f = rng.uniform(0.05, 1.0, size=(9, n, n, n))
    u = rng.standard_normal((3, n, n, n))
    v = rng.standard_normal((3, n, n, n))
    gs = lambda x: learned.forward(p, f, x[None].astype(complex), symmetric=True)[0].real
    g = lambda x: learned.forward_real(p, f, x)[0]
    assert abs(np.sum(v * gs(u)) - np.sum(gs(v) * u)) <= 1e-12 * abs(np.sum(v * gs(u)))
    assert abs(np.sum(v * g(u)) - np.sum(g(v) * u)) > 1e-3 * abs(np.sum(v * g(u)))
    fs, blocks, kap, gam = _small_case()
    nn = fs.shape[-1]
    ps = _rand_params(rng, learned.HIDDEN, 0.2)
    x = wl.random_block(1, nn, seed=21)[0]
    y = wl.random_block(1, nn, seed=22)[0]
    lhs = np.vdot(x, learned.precondition(ps, fs, y, kap, gam, blocks, symmetric=True))
    rhs = np.conj(np.vdot(y, learned.precondition(ps, fs, x, kap, gam, blocks, symmetric=True)))
    assert abs(lhs - rhs) <= 1e-11 * abs(lhs)


def test_bf16_rounding():
    """Round to nearest even at 7 fraction bits, checked on exact binary
    values and against torch's float32 -> bfloat16 conversion."""
    vals = np.array([1.0, 1 + 2 ** -7, 1 + 2 ** -8, 1 + 3 * 2 ** -8, 1 + 2 ** -8 + 2 ** -20, -3.140625, 0.0])
    want = np.array([1.0, 1 + 2 ** -7, 1.0, 1 + 2 ** -6, 1 + 2 ** -7, -3.140625, 0.0])
    np.testing.assert_array_equal(learned.to_bf16(vals), want)
    torch = pytest.importorskip("torch")
    rng = np.random.default_rng(31)
    x = (rng.standard_normal(10000) * 10.0 ** rng.uniform(-6, 6, 10000)).astype(np.float32)
    ref = torch.from_numpy(x).to(torch.bfloat16).to(torch.float64).numpy()
    np.testing.assert_array_equal(learned.to_bf16(x), ref)
