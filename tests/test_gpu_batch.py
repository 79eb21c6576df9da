"""k-batched apply, CUDA-graph replay of the apply chain and the launch
autotuner, through the C ABI.  The batched and replayed applies run the same
kernels with the same parameters as pcx_apply, so their results must be
bit-identical to it; pcx_apply itself is checked against the oracle in
test_gpu_apply.py."""
import os

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


@pytest.mark.parametrize("n,dtype", [(32, np.complex64), (16, np.complex128), (128, np.complex64)])
def test_apply_kbatch_matches_per_k_applies(pcx, n, dtype):
    s = wl.diamond_rods()
    ks = wl.config_k(s.name)[:3]
    vpk = 2 if n < 128 else 1
    ctx = pcx.setup_structure(s, n)
    x = wl.random_block(3 * vpk, n, seed=6).astype(dtype).reshape(3, vpk, 3, n, n, n)
    X = torch.from_numpy(x).cuda()
    Y = torch.empty_like(X)
    pcx.pcx_apply_kbatch(ctx, ks, X, Y)
    for i in range(3):
        Yi = torch.empty_like(X[i])
        pcx.pcx_apply(ctx, ks[i], X[i].contiguous(), Yi)
        assert torch.equal(Yi, Y[i]), i


def test_graph_replay_matches_eager(pcx):
    n = 32
    s = wl.fcc_air_spheres()
    k = wl.config_k(s.name)[2]
    ctx = pcx.setup_structure(s, n)
    X = torch.from_numpy(wl.random_block(3, n, seed=2).astype(np.complex64)).cuda()
    ref = torch.empty_like(X)
    pcx.pcx_apply(ctx, k, X, ref)
    stream = torch.cuda.Stream()
    pcx.pcx_set_apply_graphs(ctx, 1)
    Y = torch.empty_like(X)
    with torch.cuda.stream(stream):
        for _ in range(3):   # eager, capture, replay
            Y.zero_()
            pcx.pcx_apply(ctx, k, X, Y)
    stream.synchronize()
    assert torch.equal(Y, ref)
    # new data in the same buffers: the replay reads it
    X2 = torch.from_numpy(wl.random_block(3, n, seed=9).astype(np.complex64)).cuda()
    ref2 = torch.empty_like(X)
    pcx.pcx_set_apply_graphs(ctx, 0)
    pcx.pcx_apply(ctx, k, X2, ref2)
    pcx.pcx_set_apply_graphs(ctx, 1)
    with torch.cuda.stream(stream):
        for _ in range(2):
            pcx.pcx_apply(ctx, k, X, Y)   # replays of the cached key
        X.copy_(X2)
        pcx.pcx_apply(ctx, k, X, Y)
    stream.synchronize()
    assert torch.equal(Y, ref2)


def test_autotune_chooses_and_caches(pcx, tmp_path):
    n, nvec = 32, 8
    s = wl.sc_gyro_sphere()
    k = wl.config_k(s.name)[0]
    ctx = pcx.setup_structure(s, n)
    stream = torch.cuda.Stream()
    os.environ["PCX_TUNE_CACHE"] = str(tmp_path / "tune.txt")
    try:
        r = pcx.pcx_autotune(ctx, pcx.PCX_FP32, nvec, stream=stream)
        assert r["from_cache"] == 0 and r["candidates"] >= 4
        assert r["chunk"] in (1, 2, 4, 8) and r["graphs"] in (0, 1) and r["us_per_vector"] > 0
        assert pcx.pcx_get_apply_chunk(ctx, pcx.PCX_FP32) == r["chunk"]
        # complex64 at 32^3 has both pass structures; the tuner timed both
        assert r["path"] in (pcx.PCX_APPLY_FIVE_PASS, pcx.PCX_APPLY_THREE_PASS)
        assert pcx.pcx_get_apply_path(ctx, pcx.PCX_FP32) == r["path"]
        line = (tmp_path / "tune.txt").read_text().strip().split()
        assert line[1:3] == [str(r["chunk"]), str(r["graphs"])] and line[4] == str(r["path"])
        ctx2 = pcx.setup_structure(s, n)
        r2 = pcx.pcx_autotune(ctx2, pcx.PCX_FP32, nvec, stream=stream)
        assert r2["from_cache"] == 1 and r2["chunk"] == r["chunk"] and r2["path"] == r["path"]
    finally:
        del os.environ["PCX_TUNE_CACHE"]
    # the tuned context still computes the same apply
    X = torch.from_numpy(wl.random_block(nvec, n, seed=4).astype(np.complex64)).cuda()
    Y = torch.empty_like(X)
    ref = torch.empty_like(X)
    with torch.cuda.stream(stream):
        for _ in range(3):
            pcx.pcx_apply(ctx, k, X, Y)
    stream.synchronize()
    ctx3 = pcx.setup_structure(s, n)
    pcx.pcx_set_apply_path(ctx3, r["path"])
    pcx.pcx_apply(ctx3, k, X, ref)
    assert torch.equal(Y, ref)
