"""Benchmark: compensated-operator applies per second at 128^3, and the
per-k solve time to a 1e-8 residual.

Workload (one step): the compensated operator A M A^H + gamma B^H B applied
in the Fourier basis on the 128^3 diamond-rod structure (FCC lattice, four
seeded anisotropic rod tensors, air), complex64, to 40 Bloch vectors x a
block of 16 vectors in one k-batched call (pcx_apply_kbatch: one launch per
pass sweeps every (k, vector) pair).  The launch configuration comes from
pcx_autotune on the timing stream.  value = vectors applied per second over
the whole job.  Inputs (32 GB per step) are far larger than the 129 MB L2,
so no flush is needed between steps.  e2e: pcx_apply_kbatch_host on host
buffers, the same 40 Bloch vectors x 16 vectors per step (one pinned host
block sent for every k), copies inside the timed region.

The line also carries "solve": the per-k time to Res_j <= 1e-8 (12 bands,
block 16, pcx_solve) on the same structure, in mixed precision with the
FFT-diagonal K_P^{-1}, with the curl-sandwich T0, with the learned
correction (trained in the run on random structures at the same N, time
reported), and plain FP64 with K_P^{-1}; wall-clock around the synchronising
call (--no-solve skips it).

  python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference]

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
NK = 40
K_INDEX = 5
WORKLOAD = ("diamond-rods 128^3 FCC, 40 Bloch vectors x block of 16, complex64, "
            "one k-batched call per step (pcx_apply_kbatch)")
METRIC = "compensated-operator applies/s at 128^3"
# DRAM bytes of one vector through the pass kernels at 16 vectors per
# launch: dram__bytes_read.sum + dram__bytes_write.sum of the launches of one
# chunk in an ncu capture of this benchmark, divided by 16; keyed by the pass
# structure and, for the three-pass chain, pass B's kernel variant (one tile
# per CTA, or the warp-specialised one); the x-pass variants move the same
# bytes.  Used only when the run uses that chunk, structure and variant.
TRAFFIC_BYTES_PER_VECTOR_128_C64 = {(5, None): 8.8128e9 / 16, (3, 0): 5.321861e9 / 16, (3, 1): 5.304722e9 / 16}
TRAFFIC_CHUNK = 16
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


def cpu_oracle_solve16():
    """The oracle's textbook LOBPCG (FP64 numpy, K_P^{-1}) on configuration 1:
    16^3 gyrotropic sphere, 10 bands, block 14, to Res <= 1e-8 (1 thread)."""
    import numpy as np

    import workloads as wl
    from oracle import eig, fourier, penalty, permittivity
    n, nev = 16, 10
    s = wl.sc_gyro_sphere()
    k = wl.config_k(s.name)[0]
    g = penalty.gamma_practical(k)
    blocks = permittivity.cell_blocks(s, n)
    kap = fourier.kappa(n, s.lattice, k)
    t0 = time.perf_counter()
    th, _, res, its = eig.lobpcg(lambda x: fourier.apply_symbols(x, kap, lambda e: permittivity.apply_m(blocks, e), g),
                                 lambda r: fourier.precondition(r, kap, g), wl.random_block(nev + 4, n, seed=1), nev,
                                 tol=1e-8, maxit=600)
    return time.perf_counter() - t0, int(its), float(np.max(res))


def cpu_oracle_solve(name, n, ik, nev=12, block=16, tol=1e-8, maxit=600):
    """The oracle's textbook LOBPCG (FP64 numpy, K_P^{-1}, one thread) on
    structure `name` at n^3, Bloch vector ik of its path, nev bands to
    Res <= tol: (seconds, iterations, max residual)."""
    import numpy as np

    import workloads as wl
    from oracle import eig, fourier, penalty, permittivity
    s = {"fcc-air-spheres": wl.fcc_air_spheres, "diamond-rods": wl.diamond_rods}[name]()
    k = wl.config_k(s.name)[ik]
    g = penalty.gamma_practical(k)
    blocks = permittivity.cell_blocks(s, n)
    kap = fourier.kappa(n, s.lattice, k)
    t0 = time.perf_counter()
    th, _, res, its = eig.lobpcg(lambda x: fourier.apply_symbols(x, kap, lambda e: permittivity.apply_m(blocks, e), g),
                                 lambda r: fourier.precondition(r, kap, g), wl.random_block(block, n, seed=1), nev,
                                 tol=tol, maxit=maxit)
    return time.perf_counter() - t0, int(its), float(np.max(res))


def study_cpu_solve(k64=(1, 2, 3), k128=(K_INDEX,), it128=5):
    """CPU solve-time baselines: the oracle's LOBPCG (FP64 numpy, K_P^{-1},
    12 bands, block 16, Res <= 1e-8) on configuration 2 (64^3 FCC air
    spheres, three Bloch vectors of its path after Gamma, which the
    textbook LOBPCG does not deflate; one single-threaded child process per
    k, all running at once) and configuration 3 (128^3 diamond rods, one
    Bloch vector, one child, it128 iterations: the time per iteration, with
    the whole solve projected to the 87 iterations the FP64 GPU solve takes
    on that k).  Host cores only, no GPU."""
    env = dict(os.environ, OMP_NUM_THREADS="1", OPENBLAS_NUM_THREADS="1", MKL_NUM_THREADS="1")
    model, ncores = cpu_model()

    def spawn(name, n, ik, maxit):
        code = ("import sys, json; sys.path.insert(0, %r); import bench; "
                "print(json.dumps(bench.cpu_oracle_solve(%r, %d, %d, maxit=%d)))" % (ROOT, name, n, ik, maxit))
        return subprocess.Popen([sys.executable, "-c", code], stdout=subprocess.PIPE, stderr=subprocess.PIPE,
                                env=env, text=True)

    out = {"study": "cpu-solve", "kind": "oracle", "cpu_model": model, "nproc": ncores,
           "solver": "oracle LOBPCG, FP64 numpy, K_P^-1, 12 bands, block 16, Res <= 1e-8, one thread per k"}
    t0 = time.perf_counter()
    jobs = [("config2_64", ik, spawn("fcc-air-spheres", 64, ik, 600)) for ik in k64]
    jobs += [("config3_128", ik, spawn("diamond-rods", 128, ik, it128)) for ik in k128]
    for label, ik, p in jobs:
        o, e = p.communicate()
        entry = out.setdefault(label, {"runs": [], "concurrent_processes": len(jobs)})
        if p.returncode != 0:
            entry["runs"].append({"k_index": ik, "error": e.strip().splitlines()[-1] if e.strip() else "failed"})
            continue
        sec, its, mres = json.loads(o.strip().splitlines()[-1])
        run = {"k_index": ik, "s": sec, "iterations": its, "max_res": mres}
        if label == "config3_128":
            run["s_per_iteration"] = sec / max(its, 1)
            run["projected_s_87_iterations"] = 87 * sec / max(its, 1)
        entry["runs"].append(run)
    ok = [r["s"] for r in out.get("config2_64", {}).get("runs", []) if "s" in r]
    if ok:
        out["config2_64"]["mean_s_per_k"] = sum(ok) / len(ok)
    out["wall_s"] = time.perf_counter() - t0
    print(json.dumps(out), flush=True)
    return 0


def cpu_model():
    """The host CPU's model name and core count (lscpu, else the platform)."""
    import platform
    model = platform.processor() or platform.machine()
    try:
        out = subprocess.run(["lscpu"], capture_output=True, text=True, timeout=10).stdout
        for line in out.splitlines():
            if line.lower().startswith("model name"):
                model = line.split(":", 1)[1].strip()
    except Exception:
        pass
    return model, os.cpu_count()


def cpu_baseline_subprocess():
    """The oracle timed on the host: its whole-vector apply single-threaded in
    a child process (the line's value), the same apply in one child process
    per core at once (aggregate rate on all cores), and its LOBPCG solve of
    configuration 1 (16^3) to Res <= 1e-8."""
    env = dict(os.environ, OMP_NUM_THREADS="1", OPENBLAS_NUM_THREADS="1", MKL_NUM_THREADS="1")
    code = ("import sys, json; sys.path.insert(0, %r); import bench; "
            "r = bench.cpu_oracle_applies(%d); print(json.dumps(r))" % (ROOT, N))
    out = subprocess.run([sys.executable, "-c", code], capture_output=True, text=True, env=env, timeout=900)
    if out.returncode != 0:
        return None
    v, done, dt = json.loads(out.stdout.strip().splitlines()[-1])
    model, ncores = cpu_model()
    res = {"value": v, "unit": UNIT, "cores": 1, "kind": "oracle",
           "sample": f"{done} whole-vector applies of the 128^3 workload in FP64 numpy ({dt:.1f} s)",
           "cpu_model": model, "nproc": ncores}
    # all cores: one single-threaded child per core, one whole vector each
    one = ("import sys, json; sys.path.insert(0, %r); import bench; "
           "r = bench.cpu_oracle_applies(%d, seconds_budget=0.0, max_vectors=1); print(json.dumps(r))" % (ROOT, N))
    procs = [subprocess.Popen([sys.executable, "-c", one], stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, env=env,
                              text=True) for _ in range(ncores or 1)]
    rates = []
    for p in procs:
        o, _ = p.communicate(timeout=900)
        if p.returncode == 0:
            rates.append(json.loads(o.strip().splitlines()[-1])[0])
    res["all_cores"] = {"value": sum(rates), "unit": UNIT, "cores": len(procs),
                        "sample": f"{len(rates)} single-threaded children, one per core, each timing one "
                                  "whole-vector apply while the others run; their rates summed"}
    code = ("import sys, json; sys.path.insert(0, %r); import bench; "
            "print(json.dumps(bench.cpu_oracle_solve16()))" % ROOT)
    out = subprocess.run([sys.executable, "-c", code], capture_output=True, text=True, env=env, timeout=900)
    if out.returncode == 0:
        sec, its, mres = json.loads(out.stdout.strip().splitlines()[-1])
        res["solve_config1"] = {"s": sec, "iterations": its, "max_res": mres, "cores": 1,
                                "sample": "oracle LOBPCG, 16^3 gyrotropic sphere, 10 bands, Res <= 1e-8"}
    return res


def blockops_table(n, reps=5):
    """CUDA-event timings (median of reps, L2 flushed before each) of the
    eigensolver's block operations at grid n: the complex64 Gram products on
    both paths (tensor cores, FP32 pipes) for the shapes LOBPCG uses, and the
    complex64 combinations.  One JSON line per shape."""
    import numpy as np
    import torch

    from paper_2511_17107_gb300 import build as _build
    from paper_2511_17107_gb300 import pcx
    _build.build()
    L = 3 * n ** 3
    g = torch.Generator(device="cuda").manual_seed(7)

    def block(m):
        return torch.complex(torch.randn(m, L, device="cuda", generator=g),
                             torch.randn(m, L, device="cuda", generator=g))

    S, AS = block(48), block(48)
    flush = torch.empty(64 << 20, dtype=torch.float32, device="cuda")

    def timeit(fn):
        fn()
        ts = []
        for _ in range(reps):
            flush.fill_(1.0)
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            e0.record()
            fn()
            e1.record()
            torch.cuda.synchronize()
            ts.append(e0.elapsed_time(e1))
        return float(np.median(ts))

    for na, nb, herm in ((16, 16, False), (16, 16, True), (16, 32, False), (32, 32, True), (16, 48, False),
                         (32, 48, False), (48, 48, True), (48, 48, False)):
        A = S[:na]
        B = A if herm else AS[:nb]
        G = torch.empty((na, nb), dtype=torch.complex128, device="cuda")
        row = {"op": "gram", "na": na, "nb": nb, "hermitian": herm, "L": L}
        for path, name in ((pcx.PCX_GRAM_TENSOR, "tensor"), (pcx.PCX_GRAM_FP32, "fp32"), (pcx.PCX_GRAM_AUTO, "auto")):
            pcx.pcx_set_gram_path(path)
            ms = timeit(lambda: pcx.pcx_gram(A, B, G))
            row[name + "_ms"] = round(ms, 4)
            row[name + "_gbs"] = round((na if herm else na + nb) * L * 8 / ms / 1e6, 1)
        pcx.pcx_set_gram_path(pcx.PCX_GRAM_AUTO)
        print(json.dumps(row), flush=True)
    for ns, ny in ((16, 16), (32, 16), (48, 16), (48, 32)):
        C = torch.complex(torch.randn(ns, ny, dtype=torch.float64, device="cuda", generator=g),
                          torch.randn(ns, ny, dtype=torch.float64, device="cuda", generator=g))
        Y = torch.empty((ny, L), dtype=torch.complex64, device="cuda")
        ms = timeit(lambda: pcx.pcx_combine(S[:ns], C, Y))
        print(json.dumps({"op": "combine", "ns": ns, "ny": ny, "L": L, "ms": round(ms, 4),
                          "gbs": round((ns + ny) * L * 8 / ms / 1e6, 1)}), flush=True)
    return 0


def apply_sizes_table(n, reps=5):
    """CUDA-event timings of pcx_apply (one Bloch vector, the diamond-rod
    workload) at n vectors per call for n in {1, 16, 48}, complex64 and
    complex128, each after pcx_autotune for that shape, with the L2 flushed
    before each call.  complex128 also
    reports its FP64 rate against a measured FP64 GEMM peak (torch float64
    matmul, best of 3), since the FP64 pipes bound it.  One JSON line each."""
    import numpy as np
    import torch

    import workloads as wl
    from paper_2511_17107_gb300 import build as _build
    from paper_2511_17107_gb300 import pcx
    _build.build()
    s = wl.diamond_rods()
    k = wl.config_k(s.name)[K_INDEX]
    ctx = pcx.setup_structure(s, n)
    flush = torch.empty(64 << 20, dtype=torch.float32, device="cuda")
    a = torch.randn(4096, 4096, dtype=torch.float64, device="cuda")
    best = 1e30
    for _ in range(3):
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record()
        torch.matmul(a, a)
        e1.record()
        torch.cuda.synchronize()
        best = min(best, e0.elapsed_time(e1))
    fp64_tflops = 2 * 4096 ** 3 / (best / 1e3) / 1e12
    del a
    # FFT flop convention 5 N log2 N per complex transform of N points:
    # 6 transforms of N^3 points per vector, plus about 200 flops per cell
    flops = 6 * 5 * n ** 3 * np.log2(n ** 3) + 200 * n ** 3
    for dt, es in ((torch.complex64, 8), (torch.complex128, 16)):
        for nv in (1, 16, 48):
            x = torch.complex(torch.randn(nv, 3, n, n, n, device="cuda", dtype=torch.float64),
                              torch.randn(nv, 3, n, n, n, device="cuda", dtype=torch.float64)).to(dt)
            y = torch.empty_like(x)
            tune = pcx.pcx_autotune(ctx, pcx.PCX_FP32 if es == 8 else pcx.PCX_FP64, nv)
            pcx.pcx_apply(ctx, k, x, y)
            ts = []
            for _ in range(reps):
                flush.fill_(1.0)
                e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
                e0.record()
                pcx.pcx_apply(ctx, k, x, y)
                e1.record()
                torch.cuda.synchronize()
                ts.append(e0.elapsed_time(e1))
            ms = float(np.median(ts))
            row = {"op": "apply", "N": n, "dtype": "c64" if es == 8 else "c128", "vectors": nv,
                   "us_per_vector": round(1e3 * ms / nv, 2), "applies_per_s": round(nv / (ms / 1e3), 1),
                   "algorithmic_gbs": round(2 * nv * 3 * n ** 3 * es / (ms / 1e3) / 1e9, 1),
                   "chunk": tune["chunk"] if isinstance(tune, dict) else None}
            if es == 16:
                row["fp64_tflops"] = round(nv * flops / (ms / 1e3) / 1e12, 3)
                row["fp64_gemm_peak_tflops"] = round(fp64_tflops, 3)
            print(json.dumps(row), flush=True)
            del x, y
    # M_CrossDoF (Sec. 3.2.2): the seven-pass chain with the real-space
    # cross-DoF stencil pass, on the same workload and k at 16 vectors (the
    # diamond materials fail the sufficient HPD conditions of Sec. 3.3, so
    # the context is built without that proof; the timing does not depend
    # on it)
    cctx = pcx.setup_structure(s, n, m_kind=pcx.PCX_M_CROSSDOF, crossdof_unchecked=True)
    for dt, es in ((torch.complex64, 8), (torch.complex128, 16)):
        nv = 16
        x = torch.complex(torch.randn(nv, 3, n, n, n, device="cuda", dtype=torch.float64),
                          torch.randn(nv, 3, n, n, n, device="cuda", dtype=torch.float64)).to(dt)
        y = torch.empty_like(x)
        tune = pcx.pcx_autotune(cctx, pcx.PCX_FP32 if es == 8 else pcx.PCX_FP64, nv)
        pcx.pcx_apply(cctx, k, x, y)
        ts = []
        for _ in range(reps):
            flush.fill_(1.0)
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            e0.record()
            pcx.pcx_apply(cctx, k, x, y)
            e1.record()
            torch.cuda.synchronize()
            ts.append(e0.elapsed_time(e1))
        ms = float(np.median(ts))
        print(json.dumps({"op": "apply", "m_kind": "crossdof", "N": n, "dtype": "c64" if es == 8 else "c128",
                          "vectors": nv, "us_per_vector": round(1e3 * ms / nv, 2),
                          "applies_per_s": round(nv / (ms / 1e3), 1),
                          "algorithmic_gbs": round(2 * nv * 3 * n ** 3 * es / (ms / 1e3) / 1e9, 1),
                          "chunk": tune["chunk"] if isinstance(tune, dict) else None}), flush=True)
        del x, y
    return 0


def library_baselines(pcx, ctx, k, n, block=16, reps=5):
    """The cuFFT / cuBLAS versions of the apply and of the Gram products
    (libpcx_baselines.so, timed only) next to libpcx on the same inputs:
    CUDA events on one stream, L2 flushed before each call, median of reps."""
    import numpy as np
    import torch

    from paper_2511_17107_gb300 import baselines
    st = torch.cuda.Stream()
    flush = torch.empty(64 << 20, dtype=torch.float32, device="cuda")

    def timeit(fn):
        with torch.cuda.stream(st):
            fn()
            fn()
            ts = []
            for _ in range(reps):
                flush.fill_(1.0)
                e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
                e0.record(st)
                fn()
                e1.record(st)
                st.synchronize()
                ts.append(e0.elapsed_time(e1))
        return float(np.median(ts))

    out = {"workload": f"diamond rods {n}^3, one Bloch vector x {block} vectors; Gram at L = 3 N^3",
           "timer": "CUDA events, L2 flushed, median of 5"}
    for dt, prec, name, chunk in ((torch.complex64, pcx.PCX_FP32, "c64", block),
                                  (torch.complex128, pcx.PCX_FP64, "c128", block // 2)):
        x = torch.complex(torch.randn(block, 3, n, n, n, device="cuda", dtype=torch.float64),
                          torch.randn(block, 3, n, n, n, device="cuda", dtype=torch.float64)).to(dt)
        y = torch.empty_like(x)
        base = baselines.CufftApply(pcx, ctx, k, prec, chunk)
        ms_b = timeit(lambda: base(x, y, st))
        ms_o = timeit(lambda: pcx.pcx_apply(ctx, k, x, y, stream=st))
        out["apply_" + name] = {"cufft_us_per_vector": round(1e3 * ms_b / block, 2),
                                "pcx_us_per_vector": round(1e3 * ms_o / block, 2),
                                "pcx_over_cufft": round(ms_b / ms_o, 3)}
        base.close()
        del x, y
    L = 3 * n ** 3
    g = torch.Generator(device="cuda").manual_seed(5)
    for dt, name in ((torch.complex64, "c64"), (torch.complex128, "c128")):
        A = torch.complex(torch.randn(48, L, device="cuda", generator=g, dtype=torch.float64),
                          torch.randn(48, L, device="cuda", generator=g, dtype=torch.float64)).to(dt)
        B = torch.complex(torch.randn(48, L, device="cuda", generator=g, dtype=torch.float64),
                          torch.randn(48, L, device="cuda", generator=g, dtype=torch.float64)).to(dt)
        rows = []
        for na, nb in ((16, 16), (16, 48), (48, 48)):
            G = torch.empty((na, nb), dtype=torch.complex128, device="cuda")
            Gb = torch.empty((nb, na), dtype=dt, device="cuda")
            ms_b = timeit(lambda: baselines.cublas_gram(A[:na], B[:nb], Gb, st))
            ms_o = timeit(lambda: pcx.pcx_gram(A[:na], B[:nb], G, stream=st))
            rows.append({"na": na, "nb": nb, "cublas_ms": round(ms_b, 4), "pcx_ms": round(ms_o, 4),
                         "pcx_over_cublas": round(ms_b / ms_o, 3)})
        out["gram_" + name] = rows
        del A, B
    return out


def study_bcc_convergence(pcx, grids=(16, 32, 64, 128), nev=8, tol=1e-7):
    """Sec. 4.2, tables tab:num:convergence_type1 / type2: BCC-SG in the
    anisotropic medium at k = (pi, pi, pi), 10th-order stencils (m = 5),
    M_Trivial and M_CrossDoF, the first eight eigenvalues at N = 16 ... 128;
    differences between grid levels of the normalised frequency omega/(2 pi)
    next to the printed ones.  Mixed precision with the curl-sandwich
    preconditioner; one JSON line."""
    import numpy as np

    import workloads as wl
    printed = {"trivial": [[2.58e-02, 7.70e-03, 2.64e-03], [3.09e-02, 1.10e-02, 3.43e-03], [1.65e-02, 1.89e-02, 8.63e-03],
                           [9.54e-03, 1.62e-02, 1.02e-02], [4.71e-02, 1.45e-02, 4.85e-03], [3.15e-02, 2.10e-02, 7.67e-03],
                           [3.85e-02, 2.06e-02, 6.66e-03], [5.69e-02, 2.10e-02, 5.73e-03]],
               "crossdof": [[2.90e-02, 8.21e-03, 2.90e-03], [3.31e-02, 1.21e-02, 3.81e-03], [1.91e-02, 2.30e-02, 1.08e-02],
                            [1.39e-02, 1.58e-02, 1.27e-02], [5.01e-02, 2.16e-02, 6.28e-03], [4.01e-02, 2.59e-02, 9.60e-03],
                            [5.10e-02, 2.43e-02, 8.81e-03], [7.02e-02, 2.55e-02, 6.14e-03]]}
    s = wl.bcc_gyroid()
    k = np.array([np.pi, np.pi, np.pi])
    out = {"study": "bcc-sg-convergence", "structure": s.name, "k": "(pi, pi, pi)", "stencil_m": 5, "nev": nev,
           "tol": tol, "grids": list(grids)}
    for name, mk in (("trivial", pcx.PCX_M_TRIVIAL), ("crossdof", pcx.PCX_M_CROSSDOF)):
        lam = []
        t0 = time.perf_counter()
        for n in grids:
            ctx = pcx.setup_structure(s, n, stencil_m=5, m_kind=mk)
            ev, res, its, st = pcx.pcx_solve(ctx, [k], nev, tol, block=nev + 4, precision=pcx.PCX_FP32,
                                             precond_kind=1, raise_on_noconv=False)
            lam.append(ev[0])
        lam = np.array(lam)
        f = np.sqrt(lam) / (2 * np.pi)
        d = np.abs(np.diff(f, axis=0)).T          # [eigenvalue][level]
        p = np.array(printed[name])
        out[name] = {"omega2": lam.tolist(), "diff_freq": d.tolist(), "printed": p.tolist(),
                     "ratio_to_printed": (d / p).tolist(), "s": time.perf_counter() - t0}
    print(json.dumps(out), flush=True)
    return 0


def study_frequency_difference(pcx, n=128, nk=30, nev=10, tol=1e-6, m=1, k_concurrency=4):
    """Sec. 4.1, table tab:frequency_difference: the relative difference of
    the band frequencies computed with M_Trivial and M_CrossDoF over the
    band path (max and mean over k and the first nev bands) for BCC-SG and
    BCC-DG in the anisotropic medium.  The paper uses N = 120; the grid here
    is a power of two (N = 128).  Path H'-Gamma-P-N-H through the BCC points
    in the order the paper lists them, nk points uniform in arc length."""
    import numpy as np

    import workloads as wl
    printed = {"bcc-sg": (4.71e-3, 1.47e-3), "bcc-dg": (4.72e-3, 1.08e-3)}
    path = wl.k_path(wl.BCC_POINTS, ["H'", "G", "P", "N", "H"], nk)
    out = {"study": "frequency-difference", "N": n, "k_points": nk, "nev": nev, "stencil_m": m, "tol": tol}
    for dbl in (False, True):
        s = wl.bcc_gyroid(double=dbl)
        key = "bcc-dg" if dbl else "bcc-sg"
        omega = {}
        t0 = time.perf_counter()
        for name, mk in (("trivial", pcx.PCX_M_TRIVIAL), ("crossdof", pcx.PCX_M_CROSSDOF)):
            ctx = pcx.setup_structure(s, n, stencil_m=m, m_kind=mk)
            ev, res, its, st = pcx.pcx_solve(ctx, path, nev, tol, block=nev + 4, precision=pcx.PCX_FP32,
                                             precond_kind=1, raise_on_noconv=False, k_concurrency=k_concurrency)
            omega[name] = np.sqrt(np.maximum(ev, 0.0))
        rel = np.abs(omega["trivial"] - omega["crossdof"]) / np.abs(omega["crossdof"])
        out[key] = {"d_omega_max": float(rel.max()), "d_omega_mean": float(rel.mean()),
                    "printed_max": printed[key][0], "printed_mean": printed[key][1], "s": time.perf_counter() - t0}
    print(json.dumps(out), flush=True)
    return 0


def study_configs_1_2(pcx, tol=1e-8, k_concurrency=4):
    """Configurations 1 and 2 on the GPU, time to Res_j <= tol per k.
    Configuration 1: 16^3 gyrotropic sphere (SC), one k, 10 bands.
    Configuration 2: 64^3 FCC air spheres in the anisotropic background, 30 k
    on Gamma-X-W-L, 12 bands.  Legs: FP64 with K_P^{-1}, mixed precision with
    K_P^{-1}, mixed with T0; k_concurrency k-points in flight.  Per leg: total
    and per-k wall time, iterations, status, the k-points that missed tol and
    the largest relative eigenvalue difference against the FP64 leg.  One
    JSON line."""
    import numpy as np

    import workloads as wl
    out = {"study": "configurations-1-2", "tol": tol, "k_concurrency": k_concurrency,
           "timer": "host wall-clock around pcx_solve (synchronises its stream)"}
    for key, maker, n, nev in (("config1", wl.sc_gyro_sphere, 16, 10), ("config2", wl.fcc_air_spheres, 64, 12)):
        s = maker()
        ks = wl.config_k(s.name)
        ctx = pcx.setup_structure(s, n)
        res_c = {"N": n, "k_points": len(ks), "nev": nev, "block": nev + 4}
        eig = {}
        for leg, prec, kind in (("fp64", pcx.PCX_FP64, 0), ("mixed", pcx.PCX_FP32, 0), ("mixed_t0", pcx.PCX_FP32, 1)):
            pcx.pcx_solve(ctx, ks[:1], nev, 1e-4, block=nev + 4, precision=prec, precond_kind=kind,
                          raise_on_noconv=False)   # warm-up: module load, scratch
            t0 = time.perf_counter()
            ev, r, its, st = pcx.pcx_solve(ctx, ks, nev, tol, block=nev + 4, precision=prec, precond_kind=kind,
                                           raise_on_noconv=False, k_concurrency=k_concurrency)
            dt = time.perf_counter() - t0
            eig[leg] = ev
            res_c[leg] = {"s_total": dt, "s_per_k": dt / len(ks), "iters_mean": float(np.mean(its)),
                          "iters_max": int(np.max(its)), "status": int(st), "max_res": float(np.max(r)),
                          "k_not_converged": [int(i) for i in np.nonzero(np.max(r, axis=1) > tol)[0]]}
            if leg != "fp64":
                res_c[leg]["max_rel_eig_diff_vs_fp64"] = float(np.max(np.abs(ev - eig["fp64"]) / np.abs(eig["fp64"])))
                res_c[leg]["speedup_vs_fp64"] = res_c["fp64"]["s_total"] / dt
        out[key] = res_c
    print(json.dumps(out), flush=True)
    return 0


def study_ill_conditioned(pcx, grids=(32, 64), nev=8, tol=1e-8, maxit=600, long_maxit=4000):
    """Sec. 4.4 (row f4): the ill-conditioned inverse permittivity
    U diag(1e-1, 1e-3, 1e-5) U^H in a sphere of the SC cell at
    k = (1/7, 3/5, 4/13) pi, 8 bands, with M_Trivial and M_CrossDoF (the
    latter built without the Sec. 3.3 proof, which this material does not
    meet, as in the paper): per grid and M kind, FP64 and mixed precision
    with K_P^{-1} and mixed precision with T0 (maxit iterations), and
    M_CrossDoF again with long_maxit; per run the worst wanted residual of
    every iteration (every 10th kept), its mean decrease per iteration (log10
    per iteration, least squares over the history), the final residual and
    the lowest Ritz values.  One JSON line."""
    import numpy as np

    import workloads as wl
    s = wl.ill_conditioned_sphere()
    k = wl.config_k(s.name)[0]
    out = {"study": "ill-conditioned", "structure": s.name, "k": "(1/7, 3/5, 4/13) pi", "nev": nev, "tol": tol,
           "maxit": maxit}
    for n in grids:
        for mname, mk in (("trivial", pcx.PCX_M_TRIVIAL), ("crossdof", pcx.PCX_M_CROSSDOF)):
            ctx = pcx.setup_structure(s, n, m_kind=mk, crossdof_unchecked=True)
            legs = [("fp64", pcx.PCX_FP64, 0, maxit), ("mixed", pcx.PCX_FP32, 0, maxit),
                    ("mixed_t0", pcx.PCX_FP32, 1, maxit)]
            if mk == pcx.PCX_M_CROSSDOF:
                legs += [("fp64_long", pcx.PCX_FP64, 0, long_maxit), ("mixed_long", pcx.PCX_FP32, 0, long_maxit)]
            for leg, prec, kind, cap in legs:
                hist = np.zeros(4 * cap + 64)
                stats = pcx.pcx_solve_stats()
                t0 = time.perf_counter()
                ev, res, its, st = pcx.pcx_solve(ctx, [k], nev, tol, block=nev + 4, maxit=cap, precision=prec,
                                                 precond_kind=kind, raise_on_noconv=False, stats=stats,
                                                 res_history=hist, penalty_tol=-1.0)
                h = hist[:stats.history_len]
                good = h[np.isfinite(h) & (h > 0)]
                slope = float(np.polyfit(np.arange(good.size), np.log10(good), 1)[0]) if good.size > 2 else None
                out[f"N{n}_{mname}_{leg}"] = {
                    "status": int(st), "iters": int(its[0]), "s": time.perf_counter() - t0,
                    "max_res": float(np.max(res)), "log10_res_per_iter": slope,
                    "res_history_every10": [float(v) for v in h[::10]][:200], "omega2": ev[0].tolist()}
    print(json.dumps(out), flush=True)
    return 0


def study_woodpile(pcx, n=256, nev=20, tol=1e-8):
    """Configuration 5: the 256^3 simple cubic woodpile of anisotropic rods at
    k = 2 pi (0.1, 0.2, 0.3), 20 bands, mixed precision with the
    curl-sandwich preconditioner and the FP64 refinement, to Res <= 1e-8.
    The block is sized to the free device memory: each block column costs
    13 complex64 and 5 complex128 vectors of 3 N^3 entries (805 MB at
    256^3), capped at 32 and at least nev + 4.  One JSON line."""
    import numpy as np
    import torch

    import workloads as wl
    s = wl.woodpile()
    k = wl.config_k(s.name)[0]
    ctx = pcx.setup_structure(s, n)
    free, total = torch.cuda.mem_get_info()
    per_col = 3 * n ** 3 * (13 * 8 + 5 * 16)
    block = int(min(32, max(nev + 4, (0.85 * free) // per_col)))
    stats = pcx.pcx_solve_stats()
    t0 = time.perf_counter()
    ev, res, its, st = pcx.pcx_solve(ctx, [k], nev, tol, block=block, precision=pcx.PCX_FP32, precond_kind=1,
                                     stats=stats, raise_on_noconv=False)
    dt = time.perf_counter() - t0
    d = stats.as_dict()
    print(json.dumps({"study": "woodpile-256", "N": n, "nev": nev, "block": block, "tol": tol, "status": int(st),
                      "s": dt, "iters": int(its[0]), "iters_fp32": d["iters_fp32"], "iters_fp64": d["iters_fp64"],
                      "max_res": float(np.max(res)), "omega2": ev[0].tolist(),
                      "free_gb_before": free / 1e9, "ms_apply": d["ms_apply"], "ms_gram": d["ms_gram"],
                      "ms_precond": d["ms_precond"], "ms_other": d["ms_other"]}), flush=True)
    return 0


def study_learned(pcx, n=64, n_train=200, n_eval=50, pairs=8, steps=800, nev=12, tol=1e-8):
    """Configuration 4: the learned correction (Hermitian form, BF16 weights,
    FP32 accumulation) trained on the GPU on residual/error pairs that the
    solver dumps on n_train seeded random structures at 64^3 (1-4 spheres or
    rods, tensors with eigenvalues in [2, 16]), then evaluated on n_eval
    held-out structures at 12 bands to Res <= 1e-8 in mixed precision:
    iterations and wall time with K_P^{-1} (the plain preconditioner), with
    T0 (the learned correction's base) and with the learned T.  Structures
    whose M_Trivial blocks are not HPD are skipped.  One JSON line."""
    import numpy as np

    import workloads as wl
    from paper_2511_17107_gb300 import learned as lrn
    rng = np.random.default_rng(4)
    t0 = time.perf_counter()
    samples, seed = [], 100
    while len(samples) < n_train and seed < 100 + 4 * n_train:
        s = wl.random_inclusions(seed)
        seed += 1
        try:
            ctx = pcx.setup_structure(s, n)
        except pcx.PcxError:
            continue
        smp = lrn.collect(ctx, rng.uniform(-np.pi, np.pi, 3), n_pairs=pairs, seed=seed)
        if smp is not None:
            samples.append(smp)
    t_collect = time.perf_counter() - t0
    P, losses = lrn.train(samples, steps=steps, lr=3e-3)
    t_train = time.perf_counter() - t0 - t_collect
    import torch
    P0 = torch.empty_like(P)
    pcx.pcx_cnn_init(1, P0)
    res = {"K_P": {"iters": [], "s": []}, "T0": {"iters": [], "s": []}, "learned": {"iters": [], "s": []}}
    worst_rel = 0.0
    seed = 5000
    while len(res["K_P"]["iters"]) < n_eval and seed < 5000 + 4 * n_eval:
        s = wl.random_inclusions(seed)
        seed += 1
        try:
            ctx = pcx.setup_structure(s, n)
        except pcx.PcxError:
            continue
        pcx.pcx_set_cnn_form(ctx, lrn.FORM)
        k = rng.uniform(-np.pi, np.pi, 3)
        ev = {}
        for name, cp, kind in (("K_P", None, 0), ("T0", None, 1), ("learned", P, 1)):
            a = time.perf_counter()
            e, r, it, st = pcx.pcx_solve(ctx, [k], nev, tol, block=nev + 4, precision=pcx.PCX_FP32, cnn_params=cp,
                                         precond_kind=kind, raise_on_noconv=False)
            res[name]["s"].append(time.perf_counter() - a)
            res[name]["iters"].append(int(it[0]))
            ev[name] = e[0]
        worst_rel = max(worst_rel, float(np.max(np.abs(ev["learned"] - ev["K_P"]) / np.abs(ev["K_P"]))))
    out = {"study": "learned-64", "N": n, "train_structures": len(samples), "pairs_per_structure": pairs,
           "steps": steps, "form": "hermitian, bf16 weights, fp32 accumulation", "collect_s": t_collect,
           "train_s": t_train, "loss_start": float(losses[0]), "loss_end": float(np.mean(losses[-20:])),
           "relative_error_T0": lrn.relative_error(samples[:20], P0),
           "relative_error_trained": lrn.relative_error(samples[:20], P),
           "eval_structures": len(res["K_P"]["iters"]), "max_rel_eig_diff_learned_vs_K_P": worst_rel}
    for name, d in res.items():
        out[name] = {"iters_mean": float(np.mean(d["iters"])), "s_mean": float(np.mean(d["s"])),
                     "iters": d["iters"]}
    print(json.dumps(out), flush=True)
    return 0


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
            "data": "synthetic", "config": {"workload": WORKLOAD, "N": N, "vectors_per_step": 1,
                                            "sample_per_step": "one whole vector of the workload (Bloch vector "
                                                               f"{K_INDEX} of the path) through the oracle's FP64 "
                                                               "operator, numpy, one thread"},
            "cpu_baseline": {"value": value, "unit": UNIT, "cores": 1, "kind": "oracle",
                             "sample": f"{args.steps} whole-vector FP64 oracle applies at 128^3"},
            "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line))
    return 0


def whole_job_rate(ms_local, units_per_rank, steps, world, device=None):
    """Max-over-ranks step time and the whole-job rate.  Every rank processes
    units_per_rank units per step (weak scaling); with world > 1 the local
    times are reduced with MAX over the initialised process group, so every
    rank returns the same pair."""
    ms = ms_local
    if world > 1:
        import torch
        import torch.distributed as td
        t = torch.tensor([ms], dtype=torch.float64, device=device)
        td.all_reduce(t, op=td.ReduceOp.MAX)
        ms = float(t.item())
    return ms, world * units_per_rank * steps / (ms / 1e3)


def k_list(kpath, nk):
    return [kpath[(K_INDEX + i) % len(kpath)] for i in range(nk)]


def rank_k_points(nk, rank, world):
    """The Bloch vectors of one rank.  One GPU: nk points of the
    configuration's 40-point path (from K_INDEX).  N GPUs (weak scaling):
    the whole job is the same polyline X-U-L-G-X-W-K sampled at nk N points,
    and rank r takes every N-th of them (r, r + N, ...), so the ranks' k-points
    are distinct, each rank has nk of them, and together they are the path."""
    import numpy as np

    import workloads as wl
    if world == 1:
        return np.stack(k_list(wl.config_k("diamond-rods"), nk))
    full = wl.k_path(wl.FCC_POINTS, ["X", "U", "L", "G", "X", "W", "K"], nk * world)
    return full[rank::world]


def train_learned(pcx, n, n_struct=3, n_pairs=8, steps=120):
    """The learned correction trained on random structures at grid n."""
    import numpy as np

    import workloads as wl
    from paper_2511_17107_gb300 import learned
    rng = np.random.default_rng(11)
    t0 = time.perf_counter()
    samples, seed = [], 300
    while len(samples) < n_struct and seed < 340:
        s = wl.random_inclusions(seed)
        seed += 1
        try:
            ctx = pcx.setup_structure(s, n)
        except pcx.PcxError:
            continue
        smp = learned.collect(ctx, rng.uniform(-np.pi, np.pi, 3), n_pairs=n_pairs, seed=seed)
        if smp is not None:
            samples.append(smp)
    import torch
    P0 = torch.empty(pcx.PCX_CNN_NPARAMS, dtype=torch.float32, device="cuda")
    pcx.pcx_cnn_init(1, P0)   # the initial correction is zero: T = T0
    P, losses = learned.train(samples, steps=steps, lr=3e-3)
    return P, {"structures": len(samples), "pairs_per_structure": n_pairs, "steps": steps,
               "loss_T0": learned.relative_error(samples, P0), "loss_trained": learned.relative_error(samples, P),
               "s": time.perf_counter() - t0}


def solve_legs(pcx, ctx, kpath, nk, n, nev=12, block=16, tol=1e-8, learned_steps=120, only="", batched_nk=0,
               k_concurrency=4):
    """Per-k time to Res_j <= tol: mixed (K_P^{-1}, T0, learned) vs plain FP64;
    with batched_nk, also the mixed T0 solve of batched_nk k-points of the
    path with k_concurrency of them in flight (total and mean per k)."""
    import numpy as np
    ks = k_list(kpath, nk)
    out = {"tol": tol, "nev": nev, "block": block, "k_points": nk, "k_first_index": K_INDEX,
           "timer": "host wall-clock around pcx_solve (synchronises its stream)"}
    want = set(x for x in only.split(",") if x)
    P = None
    if learned_steps > 0 and (not want or "mixed_learned" in want):
        P, out["learned_training"] = train_learned(pcx, n, steps=learned_steps)
    scalar, projector = pcx.PCX_PENALTY_SCALAR, pcx.PCX_PENALTY_PROJECTOR
    legs = [("mixed", pcx.PCX_FP32, 0, None, scalar), ("mixed_sandwich", pcx.PCX_FP32, 1, None, scalar)]
    if P is not None:
        from paper_2511_17107_gb300 import learned as lrn
        pcx.pcx_set_cnn_form(ctx, lrn.FORM)   # the form the correction was trained in
        legs.append(("mixed_learned", pcx.PCX_FP32, 1, P, scalar))
    legs.append(("fp64", pcx.PCX_FP64, 0, None, scalar))
    legs.append(("fp64_sandwich", pcx.PCX_FP64, 1, None, scalar))
    # the projector penalty form (the same physical eigenpairs, every
    # penalty eigenvalue 16 pi^2): a lower FP32 rounding floor
    legs.append(("mixed_sandwich_projector", pcx.PCX_FP32, 1, None, projector))
    if want:
        legs = [leg for leg in legs if leg[0] in want]
    eigs = {}
    for name, prec, kind, params, form in legs:
        stats = pcx.pcx_solve_stats()
        pcx.pcx_set_penalty_form(ctx, form)
        t0 = time.perf_counter()
        ev, res, its, st = pcx.pcx_solve(ctx, ks, nev, tol, block=block, precision=prec, stats=stats,
                                         raise_on_noconv=False, precond_kind=kind, cnn_params=params)
        dt = time.perf_counter() - t0
        pcx.pcx_set_penalty_form(ctx, scalar)
        eigs[name] = ev
        d = stats.as_dict()
        out[name] = {"s_per_k": dt / nk, "status": int(st), "max_res": float(np.max(res)),
                     "iters_per_k": float(np.mean(its)), "iters_fp32": d["iters_fp32"], "iters_fp64": d["iters_fp64"],
                     "applies_fp32": d["applies_fp32"], "applies_fp64": d["applies_fp64"],
                     "ms_apply": d["ms_apply"], "ms_precond": d["ms_precond"], "ms_gram": d["ms_gram"],
                     "ms_rr": d["ms_rr"], "ms_other": d["ms_other"], "gamma_raises": d["gamma_raises"],
                     "learned_fallbacks": d["learned_fallbacks"]}
    if batched_nk > 0 and (not want or "mixed_sandwich_all_k" in want):
        # the whole band path: every k of the path, several in flight
        # The path passes close to Gamma, where the scalar rule's gamma =
        # 4 pi^2 / |k|^2 lifts the top of the spectrum to ~12 N^2 gamma and
        # the FP64 residual floor (~1e-16 of it) above 1e-8 at N = 128; the
        # per-mode penalty keeps the same physical eigenpairs with the top at
        # ~12 N^2 4 pi^2.
        kall = k_list(kpath, batched_nk)
        pcx.pcx_set_penalty_form(ctx, pcx.PCX_PENALTY_PER_MODE)
        stats = pcx.pcx_solve_stats()
        t0 = time.perf_counter()
        ev, res, its, st = pcx.pcx_solve(ctx, kall, nev, tol, block=block, precision=pcx.PCX_FP32, stats=stats,
                                         raise_on_noconv=False, precond_kind=1, k_concurrency=k_concurrency)
        dt = time.perf_counter() - t0
        pcx.pcx_set_penalty_form(ctx, pcx.PCX_PENALTY_SCALAR)
        out["mixed_sandwich_all_k"] = {"k_points": batched_nk, "k_concurrency": k_concurrency, "s_total": dt,
                                       "s_per_k": dt / batched_nk, "status": int(st), "max_res": float(np.max(res)),
                                       "iters_per_k": float(np.mean(its)), "iters_max": int(np.max(its)),
                                       "penalty_form": "per-mode",
                                       "k_not_converged": [int(i) for i in np.nonzero(np.max(res, axis=1) > tol)[0]]}
        if "mixed_sandwich" in out and nk >= 1:
            out["mixed_sandwich_all_k"]["max_rel_eig_diff_vs_per_k_leg"] = float(
                np.max(np.abs(ev[:nk] - eigs["mixed_sandwich"]) / np.abs(eigs["mixed_sandwich"])))
    for name in eigs:
        if name != "fp64" and name in out and "fp64" in out:
            out[name]["speedup_vs_fp64"] = out["fp64"]["s_per_k"] / out[name]["s_per_k"]
            out[name]["max_rel_eig_diff_vs_fp64"] = float(np.max(np.abs(eigs[name] - eigs["fp64"])
                                                                 / np.abs(eigs["fp64"])))
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
    ap.add_argument("--nk", type=int, default=NK, help="Bloch vectors per k-batched step")
    ap.add_argument("--no-solve", action="store_true", help="skip the per-k solve-time legs")
    ap.add_argument("--no-baselines", action="store_true", help="skip the cuFFT / cuBLAS baseline timings")
    ap.add_argument("--solve-nk", type=int, default=1, help="k-points of the solve legs (from index k_index)")
    ap.add_argument("--solve-all-k", type=int, default=NK,
                    help="k-points of the batched mixed T0 leg over the band path (0: skip)")
    ap.add_argument("--k-concurrency", type=int, default=4, help="k-points in flight in the batched leg")
    ap.add_argument("--learned-steps", type=int, default=120, help="training steps of the learned leg (0: skip)")
    ap.add_argument("--solve-legs", default="", help="comma list of solve legs to run (default: all)")
    ap.add_argument("--no-tune", action="store_true", help="keep the default launch configuration")
    ap.add_argument("--chunk", type=int, default=0, help="vectors per launch chunk (implies --no-tune)")
    ap.add_argument("--apply-path", default="auto", choices=["auto", "five", "three"],
                    help="pass structure of the apply (pcx_set_apply_path)")
    ap.add_argument("--apply-variant", default="",
                    help="X,Z: the three-pass chain's kernel variants (pcx_set_apply_variant; overrides the tuner's)")
    ap.add_argument("--blockops", action="store_true",
                    help="print timings of the eigensolver's Gram products and combinations instead")
    ap.add_argument("--sizes", action="store_true",
                    help="print pcx_apply timings at 1, 16 and 48 vectors per call, complex64 and complex128, instead")
    ap.add_argument("--study", default="",
                    choices=["", "bcc-convergence", "frequency-difference", "woodpile-256", "learned-64",
                             "configs-1-2", "ill-conditioned", "cpu-solve"],
                    help="run one of the paper's studies or configuration 5 instead of the benchmark (one JSON line)")
    args = ap.parse_args()
    if args.study == "cpu-solve":
        return study_cpu_solve()
    if args.study:
        from paper_2511_17107_gb300 import build as _build
        from paper_2511_17107_gb300 import pcx
        _build.build()
        return {"bcc-convergence": study_bcc_convergence, "frequency-difference": study_frequency_difference,
                "woodpile-256": study_woodpile, "learned-64": study_learned,
                "configs-1-2": study_configs_1_2, "ill-conditioned": study_ill_conditioned}[args.study](pcx)
    if args.warmup < 3:
        args.warmup = 3
    if args.blockops:
        return blockops_table(args.n)
    if args.sizes:
        return apply_sizes_table(args.n)
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
    n, block, nk = args.n, args.block, args.nk
    cdt, es = (np.complex64, 8) if args.precision == "f32" else (np.complex128, 16)
    prec = pcx.PCX_FP32 if es == 8 else pcx.PCX_FP64
    s = wl.diamond_rods()
    kpath = wl.config_k(s.name)
    ks = rank_k_points(nk, rank, world)
    ctx = pcx.setup_structure(s, n)
    stream = torch.cuda.Stream()
    if args.chunk > 0:
        args.no_tune = True
        pcx.pcx_set_apply_chunk(ctx, args.chunk)
    tune = None if args.no_tune else pcx.pcx_autotune(ctx, prec, block, stream=stream)
    if args.apply_path != "auto":   # an explicit pass structure overrides the tuner's choice
        pcx.pcx_set_apply_path(ctx, {"five": pcx.PCX_APPLY_FIVE_PASS, "three": pcx.PCX_APPLY_THREE_PASS}[args.apply_path])
    if args.apply_variant:
        xv, zv = (int(t) for t in args.apply_variant.split(","))
        pcx.pcx_set_apply_variant(ctx, xv, zv)
    x = wl.random_block(block, n, seed=20251117 + rank).astype(cdt)
    X = torch.empty((nk, block, 3, n, n, n), dtype=torch.complex64 if es == 8 else torch.complex128, device="cuda")
    X.copy_(torch.from_numpy(x).cuda().unsqueeze(0).expand_as(X))
    Y = torch.empty_like(X)
    vecs = nk * block

    def step():
        pcx.pcx_apply_kbatch(ctx, ks, X, Y, stream=stream)

    with torch.cuda.stream(stream):
        for _ in range(args.warmup):
            step()
    stream.synchronize()
    # per-call timing of the k-batched apply (events on the launching stream)
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
    ms, value = whole_job_rate(start.elapsed_time(end), vecs, args.steps, world, "cuda")
    per_launch_ms = sum(a.elapsed_time(b) for a, b in zip(ev0, ev1)) / args.steps

    # end-to-end: the same step (every Bloch vector of the batch x the block)
    # from pinned host buffers through pcx_apply_kbatch_host, copies inside
    # the timed region: for every k the block goes host -> device and its
    # image comes back into one pinned host buffer (each k's result
    # overwrites the previous one), in one pipeline per step
    e2e = None
    if not args.no_e2e:
        xh = torch.from_numpy(x).pin_memory()
        yh = torch.empty_like(xh).pin_memory()
        pcx.pcx_apply_kbatch_host(ctx, ks[:1], xh, yh, block, x_stride=0, y_stride=0)
        e2e_steps = max(1, min(args.steps, 3))
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        for _ in range(e2e_steps):
            pcx.pcx_apply_kbatch_host(ctx, ks, xh, yh, block, x_stride=0, y_stride=0)
        e2e_dt = time.perf_counter() - t0
        e2e_ms, e2e_rate = whole_job_rate(e2e_dt * 1e3, len(ks) * block, e2e_steps, world, "cuda")
        e2e = {"value": e2e_rate, "unit": UNIT,
               "h2d_bytes_per_step": int(len(ks) * xh.numel() * es), "d2h_bytes_per_step": int(len(ks) * yh.numel() * es),
               "step": f"{len(ks)} Bloch vectors x {block} vectors from pinned host buffers, one "
                       "pcx_apply_kbatch_host call per step (one host block, stride 0, sent for every k)"}

    peak, peak_kind = peaks()
    abytes = algorithmic_bytes(n, vecs, es, 4)
    achieved = abytes / (per_launch_ms / 1e3) / 1e9
    chunk = pcx.pcx_get_apply_chunk(ctx, prec)
    passes = pcx.pcx_get_apply_path(ctx, prec)
    passes = 3 if passes == pcx.PCX_APPLY_THREE_PASS else (5 if passes == pcx.PCX_APPLY_FIVE_PASS else passes)
    tkey = (passes, pcx.pcx_get_apply_variant(ctx)[1] if passes == 3 else None)
    traffic = TRAFFIC_BYTES_PER_VECTOR_128_C64[tkey] * vecs \
        if (n, es) == (N, 8) and tkey in TRAFFIC_BYTES_PER_VECTOR_128_C64 and chunk == TRAFFIC_CHUNK else None
    line = {
        "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": ms / args.steps, "higher_is_better": True, "scaling": "weak",
        "vs_baseline": None, "dtype": args.precision, "data": "synthetic",
        "config": {"workload": WORKLOAD if (n, block, nk, es) == (N, BLOCK, NK, 8) else
                   f"diamond-rods {n}^3 FCC, {nk} Bloch vectors x block of {block}, {args.precision}, "
                   "one k-batched call per step (pcx_apply_kbatch)",
                   "N": n, "block": block, "k_points": nk, "k_first_index": K_INDEX,
                   "l2": f"inputs larger than L2 ({vecs * 3 * n ** 3 * es / 1e9:.1f} GB per step)",
                   "parallelism": f"replicas x{world}", "autotune": tune},
        "roofline": {"bound": "hbm", "achieved": achieved, "peak": peak, "unit": "GB/s",
                     "frac": achieved / peak,
                     "traffic": traffic,
                     # DRAM bytes the pass chain moves (ncu) over the same launch time
                     "traffic_gbs": traffic / (per_launch_ms / 1e3) / 1e9 if traffic else None,
                     "traffic_frac": traffic / (per_launch_ms / 1e3) / 1e9 / peak if traffic else None,
                     "kernel": f"pcx_apply pass chain ({passes} pass kernels per chunk of vectors"
                               + (", kernel variants x %d z %d)" % pcx.pcx_get_apply_variant(ctx) if passes == 3 else ")"),
                     "peak_kind": peak_kind + " (burst HBM copy)",
                     "algorithmic_bytes_per_launch": abytes},
        "e2e": e2e,
        "gpu_launches": passes * -(-vecs // chunk) * args.steps,
        "clocks": ck,
    }
    if rank == 0 and not args.no_baselines:
        del X, Y
        torch.cuda.empty_cache()
        line["baselines"] = library_baselines(pcx, ctx, ks[0], n)
    if rank == 0 and not args.no_solve:
        line["solve"] = solve_legs(pcx, ctx, kpath, args.solve_nk, n, learned_steps=args.learned_steps,
                                   only=args.solve_legs, batched_nk=args.solve_all_k,
                                   k_concurrency=args.k_concurrency)
    if rank == 0 and not args.no_cpu_baseline:
        line["cpu_baseline"] = cpu_baseline_subprocess()
    if rank == 0:
        print(json.dumps(line))
    if dist:
        td.destroy_process_group()
    return 0


if __name__ == "__main__":
    sys.exit(main())
