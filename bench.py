"""Benchmark: compensated-operator applies per second at 128^3.

Workload (one step): the compensated operator A M A^H + gamma B^H B applied
in the Fourier basis to one block of 16 vectors on the 128^3 diamond-rod
structure (FCC lattice, four seeded anisotropic rod tensors, air), complex64,
through the C ABI call pcx_apply.  value = vectors applied per second over
the whole job.  Inputs (805 MB per block) are larger than the 129 MB L2, so
no flush is needed between steps.

  python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference]

The line also carries "solve": the per-k solve time to Res_j <= 1e-8
(12 bands, block 16, pcx_solve) on the same structure and k, mixed precision
(FP32 apply and directions, FP64 X and Rayleigh-Ritz) against the plain FP64
solve, wall-clock around the synchronising call (--no-solve skips it).

--impl reference times the CPU oracle (the FP64 numpy definition
F3^H (A M A^H + gamma B^H B) F3 x) on the same workload, one vector per step.
"""
from __future__ import annotations

import argparse
import json
import os
import statistics
import subprocess
import sys
import threading
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

N = 128
BLOCK = 16
K_INDEX = 5
WORKLOAD = "diamond-rods 128^3 FCC, block of 16 vectors, complex64 apply (pcx_apply)"
METRIC = "compensated-operator applies/s at 128^3"
# DRAM bytes of one vector through the five pass kernels (sum over the five
# launches of one chunk), from the ncu capture summarised in
# profiles/apply_pass_kernels_diamond128_c64.md; None once the kernels change.
TRAFFIC_BYTES_PER_VECTOR_128_C64 = 292.67e6
UNIT = "vector-applies/s"


def algorithmic_bytes(n, nvec, elem_bytes, m_bytes):
    """read X + write Y (3 N^3 complex per vector) + the cell blocks once."""
    return 2 * nvec * 3 * n ** 3 * elem_bytes + 9 * n ** 3 * m_bytes


def peaks():
    path = os.path.join(ROOT, "MEASURED_PEAKS.json")
    try:
        with open(path) as fh:
            d = json.load(fh)
        return float(d["hbm_gbs"]), "measured"
    except Exception:
        return 6800.0, "fallback"


class ClockSampler:
    """nvidia-smi clocks and throttle reasons sampled during the timed region."""

    FIELDS = ("clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.hw_slowdown,"
              "clocks_event_reasons.hw_thermal_slowdown,clocks_event_reasons.sw_thermal_slowdown,"
              "clocks_event_reasons.sw_power_cap")

    def __init__(self, index=0):
        self.index = index
        self.samples = []
        self.proc = None
        self.thread = None

    def start(self):
        try:
            self.proc = subprocess.Popen(["nvidia-smi", "-i", str(self.index), "--query-gpu=" + self.FIELDS,
                                          "--format=csv,noheader,nounits", "-lms", "200"],
                                         stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
        except Exception:
            self.proc = None
            return
        self.thread = threading.Thread(target=self._read, daemon=True)
        self.thread.start()

    def _read(self):
        for line in self.proc.stdout:
            self.samples.append([x.strip() for x in line.split(",")])

    def stop(self):
        if self.proc:
            self.proc.terminate()
            try:
                self.proc.wait(timeout=5)
            except Exception:
                self.proc.kill()
        if self.thread:
            self.thread.join(timeout=2)
        sm = [float(s[0]) for s in self.samples if len(s) >= 7 and s[0].replace(".", "").isdigit()]
        mx = [float(s[1]) for s in self.samples if len(s) >= 7 and s[1].replace(".", "").isdigit()]
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        reasons = sorted({names[i] for s in self.samples if len(s) >= 7 for i in range(4)
                          if s[3 + i].lower() == "active"})
        return {"sm_mhz": statistics.median(sm) if sm else None, "sm_max_mhz": max(mx) if mx else None,
                "reasons": reasons, "samples": len(self.samples)}


def cpu_oracle_applies(n, seconds_budget=20.0, max_vectors=3):
    """Time the oracle's apply on whole vectors of the workload (1 thread)."""
    import numpy as np

    import workloads as wl
    from oracle import fourier, penalty, permittivity, yee
    s = wl.diamond_rods()
    k = wl.config_k(s.name)[K_INDEX]
    blocks = permittivity.cell_blocks(s, n)
    ops = yee.YeeOperators(n, s.lattice, k)
    g = penalty.gamma_practical(k)
    am = lambda e: permittivity.apply_m(blocks, e)
    x = wl.random_block(1, n, seed=20251117)
    done, t0 = 0, time.perf_counter()
    while done < max_vectors:
        fourier.apply_definition(x, ops, am, g)
        done += 1
        if time.perf_counter() - t0 > seconds_budget:
            break
    dt = time.perf_counter() - t0
    return done / dt, done, dt


def cpu_baseline_subprocess():
    """Run the oracle timing single-threaded in a child process."""
    env = dict(os.environ, OMP_NUM_THREADS="1", OPENBLAS_NUM_THREADS="1", MKL_NUM_THREADS="1")
    code = ("import sys, json; sys.path.insert(0, %r); import bench; "
            "r = bench.cpu_oracle_applies(%d); print(json.dumps(r))" % (ROOT, N))
    out = subprocess.run([sys.executable, "-c", code], capture_output=True, text=True, env=env, timeout=900)
    if out.returncode != 0:
        return None
    v, done, dt = json.loads(out.stdout.strip().splitlines()[-1])
    return {"value": v, "unit": UNIT, "cores": 1, "kind": "oracle",
            "sample": f"{done} whole-vector applies of the 128^3 workload in FP64 numpy ({dt:.1f} s)"}


def run_reference(args):
    rank = int(os.environ.get("RANK", "0"))
    if rank != 0:
        return 0
    import numpy as np  # noqa: F401
    # warmup and timed steps: one whole-vector oracle apply per step
    import workloads as wl
    from oracle import fourier, penalty, permittivity, yee
    s = wl.diamond_rods()
    k = wl.config_k(s.name)[K_INDEX]
    blocks = permittivity.cell_blocks(s, N)
    ops = yee.YeeOperators(N, s.lattice, k)
    g = penalty.gamma_practical(k)
    am = lambda e: permittivity.apply_m(blocks, e)
    x = wl.random_block(1, N, seed=20251117)
    for _ in range(args.warmup):
        fourier.apply_definition(x, ops, am, g)
    t0 = time.perf_counter()
    for _ in range(args.steps):
        fourier.apply_definition(x, ops, am, g)
    dt = time.perf_counter() - t0
    value = args.steps / dt
    line = {"impl": "reference", "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": args.gpus,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1e3 * dt / args.steps,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
            "data": "synthetic", "config": {"workload": WORKLOAD.replace("block of 16", "1 vector per step"),
                                            "N": N, "vectors_per_step": 1},
            "cpu_baseline": {"value": value, "unit": UNIT, "cores": 1, "kind": "oracle",
                             "sample": f"{args.steps} whole-vector FP64 oracle applies at 128^3"},
            "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line))
    return 0


def solve_legs(pcx, ctx, kpath, nk, n, nev=12, block=16, tol=1e-8):
    """Per-k time to Res_j <= tol, mixed precision vs plain FP64 (pcx_solve)."""
    import numpy as np
    ks = [kpath[(K_INDEX + i) % len(kpath)] for i in range(nk)]
    out = {"tol": tol, "nev": nev, "block": block, "k_points": nk, "k_first_index": K_INDEX,
           "timer": "host wall-clock around pcx_solve (synchronises its stream)"}
    eigs = {}
    for name, prec in (("mixed", pcx.PCX_FP32), ("fp64", pcx.PCX_FP64)):
        stats = pcx.pcx_solve_stats()
        t0 = time.perf_counter()
        ev, res, its, st = pcx.pcx_solve(ctx, ks, nev, tol, block=block, precision=prec, stats=stats,
                                         raise_on_noconv=False)
        dt = time.perf_counter() - t0
        eigs[name] = ev
        d = stats.as_dict()
        out[name] = {"s_per_k": dt / nk, "status": int(st), "max_res": float(np.max(res)),
                     "iters_per_k": float(np.mean(its)), "iters_fp32": d["iters_fp32"], "iters_fp64": d["iters_fp64"],
                     "applies_fp32": d["applies_fp32"], "applies_fp64": d["applies_fp64"],
                     "ms_apply": d["ms_apply"], "ms_gram": d["ms_gram"], "ms_rr": d["ms_rr"],
                     "ms_other": d["ms_other"], "gamma_raises": d["gamma_raises"]}
    out["speedup_mixed_vs_fp64"] = out["fp64"]["s_per_k"] / out["mixed"]["s_per_k"]
    out["max_rel_eig_diff"] = float(np.max(np.abs(eigs["mixed"] - eigs["fp64"]) / np.abs(eigs["fp64"])))
    return out


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=20)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-e2e", action="store_true", help="skip the host-buffer leg (profiling runs)")
    ap.add_argument("--n", type=int, default=N, help="grid size (profiling runs use the default)")
    ap.add_argument("--block", type=int, default=BLOCK, help="vectors per step (profiling runs)")
    ap.add_argument("--precision", default="f32", choices=["f32", "f64"])
    ap.add_argument("--no-solve", action="store_true", help="skip the per-k solve-time legs")
    ap.add_argument("--solve-nk", type=int, default=1, help="k-points of the solve legs (from index k_index)")
    args = ap.parse_args()
    if args.warmup < 3:
        args.warmup = 3
    if args.impl == "reference":
        return run_reference(args)

    import numpy as np
    import torch

    import workloads as wl
    from paper_2511_17107_gb300 import build as _build
    from paper_2511_17107_gb300 import pcx

    rank = int(os.environ.get("RANK", "0"))
    world = int(os.environ.get("WORLD_SIZE", "1"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    dist = world > 1
    if dist:
        import torch.distributed as td
        td.init_process_group("nccl")
    torch.cuda.set_device(local)
    if rank == 0 or not dist:
        _build.build()
    if dist:
        td.barrier()
    n, block = args.n, args.block
    cdt, es = (np.complex64, 8) if args.precision == "f32" else (np.complex128, 16)
    s = wl.diamond_rods()
    k = wl.config_k(s.name)[K_INDEX]
    ctx = pcx.setup_structure(s, n)
    x = wl.random_block(block, n, seed=20251117 + rank).astype(cdt)
    X = torch.from_numpy(x).cuda()
    Y = torch.empty_like(X)
    stream = torch.cuda.current_stream()

    def step():
        pcx.pcx_apply(ctx, k, X, Y)

    for _ in range(args.warmup):
        step()
    torch.cuda.synchronize()
    # per-launch timing of the apply (events on the launching stream)
    ev0 = [torch.cuda.Event(enable_timing=True) for _ in range(args.steps)]
    ev1 = [torch.cuda.Event(enable_timing=True) for _ in range(args.steps)]
    clocks = ClockSampler(local)
    clocks.start()
    time.sleep(0.3)
    if dist:
        td.barrier()
    torch.cuda.synchronize()
    start = torch.cuda.Event(enable_timing=True)
    end = torch.cuda.Event(enable_timing=True)
    start.record(stream)
    for i in range(args.steps):
        ev0[i].record(stream)
        step()
        ev1[i].record(stream)
    end.record(stream)
    torch.cuda.synchronize()
    if dist:
        td.barrier()
    ck = clocks.stop()
    ms = start.elapsed_time(end)
    if dist:
        t = torch.tensor([ms], device="cuda")
        td.all_reduce(t, op=td.ReduceOp.MAX)
        ms = float(t.item())
    per_launch_ms = sum(a.elapsed_time(b) for a, b in zip(ev0, ev1)) / args.steps
    value = world * block * args.steps / (ms / 1e3)

    # end-to-end: host buffers through pcx_apply_host (copies inside the timed region)
    e2e = None
    if not args.no_e2e:
        xh = torch.from_numpy(x).pin_memory()
        yh = torch.empty_like(xh).pin_memory()
        pcx.pcx_apply_host(ctx, k, xh, yh)
        e2e_steps = max(3, min(args.steps, 10))
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        for _ in range(e2e_steps):
            pcx.pcx_apply_host(ctx, k, xh, yh)
        e2e_dt = time.perf_counter() - t0
        e2e = {"value": world * block * e2e_steps / e2e_dt, "unit": UNIT,
               "h2d_bytes_per_step": int(xh.numel() * es), "d2h_bytes_per_step": int(yh.numel() * es)}

    peak, peak_kind = peaks()
    abytes = algorithmic_bytes(n, block, es, 4)
    achieved = abytes / (per_launch_ms / 1e3) / 1e9
    line = {
        "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": ms / args.steps, "higher_is_better": True, "scaling": "weak",
        "vs_baseline": None, "dtype": args.precision, "data": "synthetic",
        "config": {"workload": WORKLOAD if (n, block, es) == (N, BLOCK, 8) else
                   f"diamond-rods {n}^3 FCC, block of {block} vectors, {args.precision} apply (pcx_apply)",
                   "N": n, "block": block, "k_index": K_INDEX,
                   "l2": "inputs larger than L2 (805 MB per block)", "parallelism": f"replicas x{world}"},
        "roofline": {"bound": "hbm", "achieved": achieved, "peak": peak, "unit": "GB/s",
                     "frac": achieved / peak,
                     "traffic": (TRAFFIC_BYTES_PER_VECTOR_128_C64 * block
                                 if (n, es) == (N, 8) and TRAFFIC_BYTES_PER_VECTOR_128_C64 else None),
                     "kernel": "pcx_apply pass chain (5 pass kernels per chunk of vectors)",
                     "peak_kind": peak_kind + " (burst HBM copy)",
                     "algorithmic_bytes_per_launch": abytes},
        "e2e": e2e,
        "gpu_launches": 5 * -(-block // pcx.pcx_get_apply_chunk(ctx, pcx.PCX_FP32 if es == 8 else pcx.PCX_FP64))
                        * args.steps,
        "clocks": ck,
    }
    if rank == 0 and not args.no_solve:
        line["solve"] = solve_legs(pcx, ctx, wl.config_k(s.name), args.solve_nk, n)
    if rank == 0 and not args.no_cpu_baseline:
        line["cpu_baseline"] = cpu_baseline_subprocess()
    if rank == 0:
        print(json.dumps(line))
    if dist:
        td.destroy_process_group()
    return 0


if __name__ == "__main__":
    sys.exit(main())
