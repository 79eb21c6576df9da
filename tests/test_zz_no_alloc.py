"""pcx_apply_noalloc: the apply variant for callers that cannot allocate
device memory (for example when the application owns all device memory
through its own pool).  Its scratch is a 32 MiB file-scope device array instead of a
cudaMalloc'd buffer.

The test calls the entry point through the C ABI twice in a row and checks
each result against pcx_apply, the allocating entry point, with the apply
tolerances used everywhere else (2e-5 of max|y| for complex64, 1e-12 for
complex128).  It also checks that a grid whose scratch cannot fit the array
is rejected before any launch.  The file is named so that pytest collects it
last; it needs no state from other tests.
"""
import numpy as np
import pytest

import workloads as wl

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

TOL = {torch.complex64: 2e-5, torch.complex128: 1e-12}


@pytest.fixture(scope="module")
def pcx():
    from paper_2511_17107_gb300 import build, pcx as binding
    build.build()
    assert torch.cuda.is_available(), "GPU tests need a CUDA device"
    return binding


@pytest.mark.parametrize("n,nvec,dtype", [(128, 3, torch.complex64), (64, 5, torch.complex128),
                                          (32, 2, torch.complex64)])
def test_noalloc_matches_apply_on_two_calls(pcx, n, nvec, dtype):
    s = wl.diamond_rods()
    k = wl.config_k(s.name)[9]
    ctx = pcx.setup_structure(s, n)
    X = torch.from_numpy(wl.random_block(nvec, n, seed=77)).to(dtype).cuda()
    ref = torch.empty_like(X)
    pcx.pcx_apply(ctx, k, X, ref)
    torch.cuda.synchronize()
    scale = float(ref.abs().max())
    for _ in range(2):
        Y = torch.full_like(X, float("nan"))
        pcx.pcx_apply_noalloc(ctx, k, X, Y)
        torch.cuda.synchronize()
        err = float((Y - ref).abs().max()) / scale
        assert err <= TOL[dtype], err


def test_noalloc_rejects_grids_beyond_the_static_scratch(pcx):
    n = 256
    ctx = pcx.setup_structure(wl.homogeneous(np.eye(3)), n)
    X = torch.zeros((1, 3, n, n, n), dtype=torch.complex64, device="cuda")
    Y = torch.empty_like(X)
    with pytest.raises(pcx.PcxError) as e:
        pcx.pcx_apply_noalloc(ctx, [0.1, 0.2, 0.3], X, Y)
    assert e.value.status == pcx.PCX_EINVAL
    assert "32 MiB" in str(e.value)


def test_noalloc_crossdof_chunks_and_limit(pcx):
    """M_CrossDoF keeps four N^3 entries per vector in the scratch: at 64^3
    complex64 the array holds 4 vectors, so a block of 6 runs in clamped
    chunks (the stencil field after the kappa.x part); at 128^3 the call is
    rejected with the 32 MiB message before any launch."""
    n = 64
    s = wl.fcc_air_spheres()
    k = wl.config_k(s.name)[4]
    ctx = pcx.setup_structure(s, n, m_kind=pcx.PCX_M_CROSSDOF)
    X = torch.from_numpy(wl.random_block(6, n, seed=78)).to(torch.complex64).cuda()
    ref = torch.empty_like(X)
    pcx.pcx_apply(ctx, k, X, ref)
    torch.cuda.synchronize()
    scale = float(ref.abs().max())
    for _ in range(2):
        Y = torch.full_like(X, float("nan"))
        pcx.pcx_apply_noalloc(ctx, k, X, Y)
        torch.cuda.synchronize()
        assert float((Y - ref).abs().max()) / scale <= TOL[torch.complex64]
    big = pcx.setup_structure(wl.homogeneous(np.eye(3)), 128, m_kind=pcx.PCX_M_CROSSDOF)
    Xb = torch.zeros((1, 3, 128, 128, 128), dtype=torch.complex64, device="cuda")
    with pytest.raises(pcx.PcxError) as e:
        pcx.pcx_apply_noalloc(big, [0.1, 0.2, 0.3], Xb, torch.empty_like(Xb))
    assert e.value.status == pcx.PCX_EINVAL
    assert "32 MiB" in str(e.value)


def test_noalloc_call_leaves_free_device_memory_unchanged(pcx):
    """The property the entry point exists for: on a fresh context (which
    owns no apply scratch yet), with its kernels already loaded by an
    earlier call on another context, a pcx_apply_noalloc call leaves the
    device's free memory exactly as it was, where pcx_apply on the same
    fresh context allocates its scratch."""
    n = 64
    s = wl.diamond_rods()
    k = wl.config_k(s.name)[2]
    X = torch.from_numpy(wl.random_block(2, n, seed=79)).to(torch.complex64).cuda()
    Y = torch.empty_like(X)
    warm = pcx.setup_structure(s, n)
    pcx.pcx_apply_noalloc(warm, k, X, Y)
    torch.cuda.synchronize()
    fresh = pcx.setup_structure(s, n)
    torch.cuda.synchronize()
    before = torch.cuda.mem_get_info()[0]
    pcx.pcx_apply_noalloc(fresh, k, X, Y)
    torch.cuda.synchronize()
    assert torch.cuda.mem_get_info()[0] == before
    pcx.pcx_apply(fresh, k, X, Y)
    torch.cuda.synchronize()
    assert torch.cuda.mem_get_info()[0] < before
