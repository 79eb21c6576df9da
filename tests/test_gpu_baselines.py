"""The cuFFT / cuBLAS baselines that the benchmark times beside libpcx
compute the same operator and Gram products: checked against pcx_apply and
numpy on small cases.  Tolerances as for the apply (2e-5 of max|y| for
complex64, 1e-12 for complex128); the cuBLAS complex64 Gram sums in FP32,
so it gets 1e-4 of max|G|."""
import numpy as np
import pytest

import workloads as wl

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def pcx():
    from paper_2511_17107_gb300 import build, pcx as binding
    build.build()
    assert torch.cuda.is_available(), "GPU tests need a CUDA device"
    return binding


@pytest.mark.parametrize("dtype,tol", [(torch.complex64, 2e-5), (torch.complex128, 1e-12)])
def test_cufft_apply_equals_pcx_apply(pcx, dtype, tol):
    from paper_2511_17107_gb300 import baselines
    n = 32
    s = wl.diamond_rods()
    k = wl.config_k(s.name)[6]
    ctx = pcx.setup_structure(s, n)
    X = torch.from_numpy(wl.random_block(4, n, seed=12)).to(dtype).cuda()
    ref = torch.empty_like(X)
    pcx.pcx_apply(ctx, k, X, ref)
    prec = pcx.PCX_FP32 if dtype == torch.complex64 else pcx.PCX_FP64
    base = baselines.CufftApply(pcx, ctx, k, prec, chunk=2)
    Y = torch.empty_like(X)
    base(X, Y)
    torch.cuda.synchronize()
    err = float((Y - ref).abs().max() / ref.abs().max())
    assert err <= tol, err
    base.close()


@pytest.mark.parametrize("dtype,tol", [(torch.complex64, 1e-4), (torch.complex128, 1e-12)])
def test_cublas_gram_equals_numpy(pcx, dtype, tol):
    from paper_2511_17107_gb300 import baselines
    rng = np.random.default_rng(3)
    na, nb, L = 16, 48, 3 * 16 ** 3
    a = rng.standard_normal((na, L)) + 1j * rng.standard_normal((na, L))
    b = rng.standard_normal((nb, L)) + 1j * rng.standard_normal((nb, L))
    A = torch.from_numpy(a).to(dtype).cuda()
    B = torch.from_numpy(b).to(dtype).cuda()
    G = torch.empty((nb, na), dtype=dtype, device="cuda")   # column-major (na, nb)
    baselines.cublas_gram(A, B, G)
    torch.cuda.synchronize()
    got = G.cpu().numpy().T
    want = A.cpu().numpy().astype(np.complex128).conj() @ B.cpu().numpy().astype(np.complex128).T
    assert np.abs(got - want).max() <= tol * np.abs(want).max()
