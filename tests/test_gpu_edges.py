"""Edge cases of the apply through the C ABI: the largest grid (N = 256, the
grid of configuration 5) against the oracle's per-mode form of a homogeneous
anisotropic medium (where F3^H M F3 is the constant block P on every mode,
so the operator is K_A P K_A^H + gamma K_B per mode, Prop. 2.8), in both
precisions and on both pass structures where they exist; and empty blocks
(nvec = 0), which every block entry point must accept as a no-op."""
import numpy as np
import pytest

import workloads as wl
from oracle import fourier, penalty, permittivity

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def pcx():
    from paper_2511_17107_gb300 import build, pcx as binding
    build.build()
    assert torch.cuda.is_available(), "GPU tests need a CUDA device"
    return binding


def _homogeneous_per_mode(x, kap, inv_eps, gamma):
    """K_A P K_A^H x + gamma K_B x mode by mode (x, kap restricted to any set
    of modes along the last three axes)."""
    ka = fourier.ka_matrix(kap)
    kah = np.conj(np.swapaxes(ka, -1, -2))
    u = np.einsum("ij,vjzyx->vizyx", inv_eps, fourier._per_mode(kah, x))
    return fourier._per_mode(ka, u) + gamma * fourier._per_mode(fourier.kb_matrix(kap), x)


@pytest.mark.parametrize("n", [256, 128])
def test_apply_largest_grid_homogeneous(pcx, n):
    """Every mode at 128^3; at 256^3 the modes of five whole p3 planes (the
    first, second, middle two and last), since the operator acts mode by
    mode here and the oracle evaluates those modes one by one."""
    rng = np.random.default_rng(9)
    s = wl.homogeneous(wl.hermitian_pd(rng, 4.0, 13.0), wl.SC)
    k = np.array([0.7, -0.4, 1.3])
    x = wl.random_block(1, n, seed=10)
    kap = fourier.kappa(n, s.lattice, k)
    inv_eps = permittivity.inverse_permittivity(s)[0]
    planes = np.array([0, 1, n // 2 - 1, n // 2, n - 1]) if n > 128 else np.arange(n)
    want = _homogeneous_per_mode(x[:, :, planes], kap[:, planes], inv_eps, penalty.gamma_practical(k))
    ctx = pcx.setup_structure(s, n)
    cases = [(np.complex128, 1e-12, None), (np.complex64, 2e-5, pcx.PCX_APPLY_FIVE_PASS)]
    if n == 128:
        cases.append((np.complex64, 2e-5, pcx.PCX_APPLY_THREE_PASS))
    for dtype, tol, path in cases:
        if path is not None:
            pcx.pcx_set_apply_path(ctx, path)
        X = torch.from_numpy(x.astype(dtype)).cuda()
        Y = torch.empty_like(X)
        pcx.pcx_apply(ctx, k, X, Y)
        torch.cuda.synchronize()
        got = Y.cpu().numpy()[:, :, planes]
        del X, Y
        err = np.abs(got - want).max() / np.abs(want).max()
        assert err <= tol, (n, dtype, path, err)


def test_empty_blocks_are_no_ops(pcx):
    n = 16
    ctx = pcx.setup_structure(wl.sc_gyro_sphere(), n)
    k = np.array([0.3, 0.2, -0.1])
    for dtype in (torch.complex64, torch.complex128):
        X = torch.zeros((0, 3, n, n, n), dtype=dtype, device="cuda")
        Y = torch.zeros_like(X)
        pcx.pcx_apply(ctx, k, X, Y)
        pcx.pcx_precond(ctx, k, X, Y)
        pcx.pcx_sandwich_precond(ctx, k, X, Y)
        pcx.pcx_apply_noalloc(ctx, k, X, Y)
        Xb = torch.zeros((2, 0, 3, n, n, n), dtype=dtype, device="cuda")
        pcx.pcx_apply_kbatch(ctx, np.stack([k, -k]), Xb, torch.zeros_like(Xb))
    torch.cuda.synchronize()
