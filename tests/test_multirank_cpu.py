"""The N > 1 host path of bench.py on CPU (gloo, world size 2): the
k-points of the band path shard over ranks with no data-path collective,
so the only exchange is the max-over-ranks step time, and only rank 0 runs
and prints the reference arm."""
import os
import socket
import sys

import pytest
import torch.distributed as td
import torch.multiprocessing as mp

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank_main(rank, world, port, out):
    sys.path.insert(0, ROOT)
    import bench
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    td.init_process_group("gloo", rank=rank, world_size=world)
    try:
        # rank r took 10 (r + 1) ms for 2 steps of 640 vector applies
        ms, value = bench.whole_job_rate(10.0 * (rank + 1), 640, 2, world, "cpu")
        out.put((rank, ms, value))
    finally:
        td.destroy_process_group()


def test_whole_job_rate_takes_the_slowest_rank():
    world, port = 2, _free_port()
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    procs = [ctx.Process(target=_rank_main, args=(r, world, port, q)) for r in range(world)]
    for p in procs:
        p.start()
    res = sorted(q.get(timeout=120) for _ in range(world))
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    for rank, ms, value in res:
        assert ms == 20.0                               # the slower rank's time
        assert value == pytest.approx(2 * 640 * 2 / 0.020)   # both ranks' units over that time


def test_single_rank_rate():
    sys.path.insert(0, ROOT)
    import bench
    ms, value = bench.whole_job_rate(5.0, 16, 4, 1)
    assert ms == 5.0 and value == pytest.approx(16 * 4 / 0.005)


def test_reference_arm_runs_on_rank_zero_only(capsys, monkeypatch):
    sys.path.insert(0, ROOT)
    import bench

    class Args:
        gpus, steps, warmup = 2, 1, 0

    monkeypatch.setenv("RANK", "1")
    assert bench.run_reference(Args) == 0
    assert capsys.readouterr().out == ""



def _shard_main(rank, world, port, out):
    sys.path.insert(0, ROOT)
    import bench
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    td.init_process_group("gloo", rank=rank, world_size=world)
    try:
        import torch
        ks = torch.from_numpy(bench.rank_k_points(40, rank, world))
        parts = [torch.zeros_like(ks) for _ in range(world)]
        td.all_gather(parts, ks)
        out.put((rank, [p.numpy() for p in parts]))
    finally:
        td.destroy_process_group()


def test_ranks_take_disjoint_parts_of_the_band_path():
    """Weak scaling over k: each of 2 ranks gets 40 k-points, no k-point
    twice, and together they are the path X-U-L-G-X-W-K sampled at 80
    points (the one-GPU job is its 40-point sampling)."""
    import numpy as np

    import workloads as wl
    world, port = 2, _free_port()
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    procs = [ctx.Process(target=_shard_main, args=(r, world, port, q)) for r in range(world)]
    for p in procs:
        p.start()
    res = sorted(q.get(timeout=120) for _ in range(world))
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    parts = res[0][1]
    assert all(len(p) == 40 for p in parts)
    allk = np.concatenate(parts)
    assert len(np.unique(np.round(allk, 12), axis=0)) == 80
    full = wl.k_path(wl.FCC_POINTS, ["X", "U", "L", "G", "X", "W", "K"], 80)
    np.testing.assert_allclose(np.sort(allk, axis=0), np.sort(full, axis=0))
    sys.path.insert(0, ROOT)
    import bench
    np.testing.assert_allclose(bench.rank_k_points(40, 0, 1), np.stack(bench.k_list(wl.config_k("diamond-rods"), 40)))
