"""GPU parity of the three-pass apply (the y transforms split four-step and
folded into the x and z passes) against the CPU oracle, through the C ABI,
next to the five-pass chain on the same inputs.  complex64 arithmetic:
|y_gpu - y_oracle| <= 2e-5 max|y_oracle| (the five-pass bound; the split
transform has the same number of rounding stages per axis)."""
import numpy as np
import pytest

import workloads as wl
from oracle import fourier, learned, penalty, permittivity, yee

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

TOL = 2e-5


@pytest.fixture(scope="module")
def pcx():
    from paper_2511_17107_gb300 import build, pcx as binding
    build.build()
    assert torch.cuda.is_available(), "GPU tests need a CUDA device"
    return binding


def _oracle_apply(structure, n, k, x):
    blocks = permittivity.cell_blocks(structure, n)
    ops = yee.YeeOperators(n, structure.lattice, k)
    return fourier.apply_definition(x, ops, lambda e: permittivity.apply_m(blocks, e), penalty.gamma_practical(k))


def _err(got, want):
    return np.abs(got - want).max() / np.abs(want).max()


CASES = [
    # name, structure, N, vectors, chunk (0: default)
    ("sc32", wl.sc_gyro_sphere, 32, 3, 0),
    ("fcc32-chunk2", wl.fcc_air_spheres, 32, 5, 2),
    ("diamond64", wl.diamond_rods, 64, 2, 0),
    ("random64-chunk1", lambda: wl.random_inclusions(3), 64, 3, 1),
    ("woodpile32", wl.woodpile, 32, 2, 0),
]


@pytest.mark.parametrize("name,maker,n,nvec,chunk", CASES, ids=[c[0] for c in CASES])
def test_three_pass_apply_matches_oracle(pcx, name, maker, n, nvec, chunk):
    s = maker()
    ks = wl.config_k(s.name)
    k = ks[min(3, len(ks) - 1)]
    x = wl.random_block(nvec, n, seed=17).astype(np.complex64)
    want = _oracle_apply(s, n, k, x.astype(np.complex128))
    ctx = pcx.setup_structure(s, n)
    if chunk:
        pcx.pcx_set_apply_chunk(ctx, chunk)
    X = torch.from_numpy(x).cuda()
    got = {}
    for path in (pcx.PCX_APPLY_THREE_PASS, pcx.PCX_APPLY_FIVE_PASS):
        pcx.pcx_set_apply_path(ctx, path)
        Y = torch.empty_like(X)
        pcx.pcx_apply(ctx, k, X, Y)
        torch.cuda.synchronize()
        got[path] = Y.cpu().numpy()
        assert _err(got[path], want) <= TOL, (path, _err(got[path], want))
    # the two pass structures round differently but agree to FP32 accuracy
    assert _err(got[pcx.PCX_APPLY_THREE_PASS], got[pcx.PCX_APPLY_FIVE_PASS]) <= TOL


def test_three_pass_full_size_bench_workload(pcx):
    """128^3 diamond rods (the benchmark's workload), one full vector of a
    two-vector launch against the oracle, and the k = 0 mode."""
    n = 128
    s = wl.diamond_rods()
    k = wl.config_k(s.name)[5]
    x = wl.random_block(2, n, seed=20251117).astype(np.complex64)
    ctx = pcx.setup_structure(s, n)
    pcx.pcx_set_apply_path(ctx, pcx.PCX_APPLY_THREE_PASS)
    X = torch.from_numpy(x).cuda()
    Y = torch.empty_like(X)
    pcx.pcx_apply(ctx, k, X, Y)
    torch.cuda.synchronize()
    want = _oracle_apply(s, n, k, x[0:1].astype(np.complex128))
    assert _err(Y.cpu().numpy()[0:1], want) <= TOL


def test_bench_launch_configuration_sampled_against_oracle(pcx):
    """The benchmark's launch as timed: 40 Bloch vectors of the diamond-rod
    path x 16 vectors at 128^3 in one pcx_apply_kbatch (complex64, three-pass
    chain, 16 vectors per launch, the default kernel variants), inputs seeded
    on the device; three sampled (k, vector) outputs, the first, a middle and
    the last, against the oracle's operator one by one."""
    n, nk, vpk = 128, 40, 16
    s = wl.diamond_rods()
    ks = wl.config_k(s.name)[:nk]
    ctx = pcx.setup_structure(s, n)
    pcx.pcx_set_apply_path(ctx, pcx.PCX_APPLY_THREE_PASS)
    pcx.pcx_set_apply_chunk(ctx, 16)
    g = torch.Generator(device="cuda").manual_seed(20251117)
    X = torch.randn((nk, vpk, 3, n, n, n), dtype=torch.complex64, device="cuda", generator=g)
    Y = torch.empty_like(X)
    pcx.pcx_apply_kbatch(ctx, ks, X, Y)
    torch.cuda.synchronize()
    blocks = permittivity.cell_blocks(s, n)
    for i, j in ((0, 0), (17, 9), (39, 15)):
        x = X[i, j:j + 1].cpu().numpy().astype(np.complex128)
        ops = yee.YeeOperators(n, s.lattice, ks[i])
        want = fourier.apply_definition(x, ops, lambda e: permittivity.apply_m(blocks, e),
                                        penalty.gamma_practical(ks[i]))
        assert _err(Y[i, j:j + 1].cpu().numpy(), want) <= TOL, (i, j)
    del X, Y


def test_three_pass_at_k_zero(pcx):
    n = 32
    s = wl.fcc_air_spheres()
    k = np.zeros(3)
    x = wl.random_block(2, n, seed=8).astype(np.complex64)
    want = _oracle_apply(s, n, k, x.astype(np.complex128))
    ctx = pcx.setup_structure(s, n)
    pcx.pcx_set_apply_path(ctx, pcx.PCX_APPLY_THREE_PASS)
    X = torch.from_numpy(x).cuda()
    Y = torch.empty_like(X)
    pcx.pcx_apply(ctx, k, X, Y)
    y = Y.cpu().numpy()
    assert _err(y, want) <= TOL
    assert np.abs(y[:, :, 0, 0, 0]).max() <= TOL * np.abs(want).max()


@pytest.mark.parametrize("n", [32, 128])
def test_three_pass_kbatch_equals_per_k(pcx, n):
    """The k-batched sweep (per-vector k table in the x passes) gives the
    per-k applies' bits on the three-pass chain."""
    s = wl.diamond_rods()
    ks = wl.config_k(s.name)[:3]
    vpk = 2 if n < 128 else 1
    ctx = pcx.setup_structure(s, n)
    pcx.pcx_set_apply_path(ctx, pcx.PCX_APPLY_THREE_PASS)
    x = wl.random_block(3 * vpk, n, seed=6).astype(np.complex64).reshape(3, vpk, 3, n, n, n)
    X = torch.from_numpy(x).cuda()
    Y = torch.empty_like(X)
    pcx.pcx_apply_kbatch(ctx, ks, X, Y)
    for i in range(3):
        Yi = torch.empty_like(X[i])
        pcx.pcx_apply(ctx, ks[i], X[i].contiguous(), Yi)
        assert torch.equal(Yi, Y[i]), i


@pytest.mark.parametrize("n", [32, 64])
def test_three_pass_sandwich_preconditioner(pcx, n):
    """The curl-sandwich T0 runs on the same three-pass chain; checked
    against the oracle's T0, out of place and in place."""
    s = wl.random_inclusions(8)
    blocks = permittivity.cell_blocks(s, n)
    k = np.array([-0.8, 1.9, 0.3])
    g = penalty.gamma_practical(k)
    kap = fourier.kappa(n, s.lattice, k)
    ctx = pcx.setup_structure(s, n)
    pcx.pcx_set_apply_path(ctx, pcx.PCX_APPLY_THREE_PASS)
    r = wl.random_block(2, n, seed=40).astype(np.complex64)
    want = learned.sandwich_precondition(r.astype(np.complex128), kap, blocks, g)
    R = torch.from_numpy(r).cuda()
    W = torch.empty_like(R)
    pcx.pcx_sandwich_precond(ctx, k, R, W)
    assert _err(W.cpu().numpy(), want) <= TOL
    pcx.pcx_sandwich_precond(ctx, k, R, R)
    assert _err(R.cpu().numpy(), want) <= TOL


def test_apply_path_rejects_unknown_value(pcx):
    ctx = pcx.setup_structure(wl.sc_gyro_sphere(), 8)
    with pytest.raises(pcx.PcxError) as e:
        pcx.pcx_set_apply_path(ctx, 7)
    assert e.value.status == pcx.PCX_EINVAL


@pytest.mark.parametrize("n", [32, 64, 128])
def test_kernel_variants_give_identical_results(pcx, n):
    """Every x / z kernel variant of the three-pass chain runs the same
    arithmetic in the same order: outputs bit-identical to the default's,
    for the apply and for T0; out-of-range variants are refused."""
    s = wl.diamond_rods()
    k = wl.config_k(s.name)[5]
    x = wl.random_block(3, n, seed=21).astype(np.complex64)
    ctx = pcx.setup_structure(s, n)
    pcx.pcx_set_apply_path(ctx, pcx.PCX_APPLY_THREE_PASS)
    pcx.pcx_set_apply_chunk(ctx, 2)   # a ragged last chunk of one vector
    X = torch.from_numpy(x).cuda()
    ref = {}
    for xv in range(4):
        for zv in range(2):
            pcx.pcx_set_apply_variant(ctx, xv, zv)
            assert pcx.pcx_get_apply_variant(ctx) == (xv, zv)
            Y = torch.empty_like(X)
            W = torch.empty_like(X)
            pcx.pcx_apply(ctx, k, X, Y)
            pcx.pcx_sandwich_precond(ctx, k, X, W)
            torch.cuda.synchronize()
            got = (Y.cpu().numpy(), W.cpu().numpy())
            if not ref:
                ref = {"y": got[0], "w": got[1]}
            assert np.array_equal(got[0], ref["y"]) and np.array_equal(got[1], ref["w"]), (xv, zv)
    pcx.pcx_set_apply_variant(ctx, -1, -1)
    assert pcx.pcx_get_apply_variant(ctx) == (3, 0)
    for bad in ((4, 0), (0, 2), (-2, 0)):
        with pytest.raises(pcx.PcxError) as e:
            pcx.pcx_set_apply_variant(ctx, *bad)
        assert e.value.status == pcx.PCX_EINVAL


def test_autotune_picks_the_variants(pcx):
    """At 32^3 (three-pass chain available) the tuner times the kernel
    variants and leaves the chosen pair in the context; the result is valid
    and the apply with it matches the oracle."""
    n = 32
    s = wl.fcc_air_spheres()
    k = wl.config_k(s.name)[3]
    ctx = pcx.setup_structure(s, n)
    r = pcx.pcx_autotune(ctx, pcx.PCX_FP32, 3, stream=torch.cuda.Stream())
    if r["path"] == pcx.PCX_APPLY_THREE_PASS:
        assert 0 <= r["x_variant"] < 4 and 0 <= r["z_variant"] < 2
        assert pcx.pcx_get_apply_variant(ctx) == (r["x_variant"], r["z_variant"])
        if not r["from_cache"]:
            assert r["candidates"] >= 6
    else:
        assert (r["x_variant"], r["z_variant"]) == (-1, -1)
    x = wl.random_block(2, n, seed=22).astype(np.complex64)
    want = _oracle_apply(s, n, k, x.astype(np.complex128))
    X = torch.from_numpy(x).cuda()
    Y = torch.empty_like(X)
    pcx.pcx_apply(ctx, k, X, Y)
    torch.cuda.synchronize()
    assert _err(Y.cpu().numpy(), want) <= TOL
