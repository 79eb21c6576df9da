"""In-tree build of libpcx.so for sm_103a with nvcc.

Every translation unit under csrc/ is compiled in parallel into
_build/*.o and linked into paper_2511_17107_gb300/libpcx.so.  Rebuilds only
what changed (source or header newer than its object).
"""
from __future__ import annotations

import concurrent.futures as cf
import os
import shutil
import subprocess
import sys

HERE = os.path.dirname(os.path.abspath(__file__))
CSRC = os.path.join(HERE, "csrc")
BUILD = os.path.join(HERE, "_build")
LIB = os.path.join(HERE, "libpcx.so")
ROOT = os.path.dirname(HERE)

ARCH = ["-gencode", "arch=compute_103a,code=sm_103a"]
COMMON = ["-O3", "-std=c++17", "-lineinfo", "-Xcompiler", "-fPIC", "-Xcompiler", "-fopenmp",
          "-I" + os.path.join(ROOT, "include")]
# extra nvcc flags for tuning builds (e.g. "-DPCX_E32=8"); a change of this
# variable needs a clean _build directory
COMMON += os.environ.get("PCX_NVCC_FLAGS", "").split()


def nvcc() -> str:
    for cand in (os.environ.get("NVCC"), shutil.which("nvcc"), "/usr/local/cuda/bin/nvcc"):
        if cand and os.path.exists(cand):
            return cand
    raise RuntimeError("nvcc not found")


def _sources():
    return sorted(f for f in os.listdir(CSRC) if f.endswith((".cu", ".cpp")))


def _headers_mtime():
    hs = [os.path.join(CSRC, f) for f in os.listdir(CSRC) if f.endswith((".h", ".cuh"))]
    hs.append(os.path.join(ROOT, "include", "pcx.h"))
    return max(os.path.getmtime(h) for h in hs)


def _compile(src: str, verbose: bool) -> str:
    obj = os.path.join(BUILD, src + ".o")
    path = os.path.join(CSRC, src)
    if os.path.exists(obj) and os.path.getmtime(obj) >= max(os.path.getmtime(path), _headers_mtime()):
        return obj
    flags = list(COMMON)
    if src == "setup.cpp":
        flags += ["-Xcompiler", "-ffp-contract=off"]
    if src in ("linalg.cpp", "solver.cpp"):
        # plain complex products and quotients (no Inf/NaN recovery calls)
        flags += ["-Xcompiler", "-fcx-limited-range"]
    cmd = [nvcc()] + ARCH + flags + ["-c", path, "-o", obj]
    if src.endswith(".cu"):
        cmd += ["-Xptxas", "-v"] if verbose else []
    res = subprocess.run(cmd, capture_output=True, text=True)
    if res.returncode != 0:
        raise RuntimeError(f"nvcc failed for {src}:\n{res.stdout}\n{res.stderr}")
    if verbose and res.stderr:
        sys.stderr.write(res.stderr)
    return obj


def build(verbose: bool = False) -> str:
    os.makedirs(BUILD, exist_ok=True)
    srcs = _sources()
    with cf.ThreadPoolExecutor(max_workers=min(8, len(srcs))) as ex:
        objs = list(ex.map(lambda s: _compile(s, verbose), srcs))
    if not os.path.exists(LIB) or any(os.path.getmtime(o) > os.path.getmtime(LIB) for o in objs):
        cudalib = os.path.join(os.path.dirname(os.path.dirname(nvcc())), "lib64")
        cmd = [nvcc()] + ARCH + ["-shared", "-cudart", "shared", "-Xcompiler", "-fopenmp", "-o", LIB + ".tmp"] + objs + \
              ["-Xlinker", "-rpath=" + cudalib]
        res = subprocess.run(cmd, capture_output=True, text=True)
        if res.returncode != 0:
            raise RuntimeError(f"link failed:\n{res.stdout}\n{res.stderr}")
        os.replace(LIB + ".tmp", LIB)
    return LIB


BASE_SRC = os.path.join(HERE, "baselines", "cufft_baseline.cu")
BASE_LIB = os.path.join(HERE, "libpcx_baselines.so")


def build_baselines() -> str:
    """libpcx_baselines.so: the cuFFT / cuBLAS baselines that the benchmark
    times beside libpcx (never loaded by libpcx itself)."""
    os.makedirs(BUILD, exist_ok=True)
    if os.path.exists(BASE_LIB) and os.path.getmtime(BASE_LIB) >= os.path.getmtime(BASE_SRC):
        return BASE_LIB
    cudalib = os.path.join(os.path.dirname(os.path.dirname(nvcc())), "lib64")
    cmd = [nvcc()] + ARCH + ["-O3", "-std=c++17", "-Xcompiler", "-fPIC", "-shared", "-cudart", "shared",
                             "-o", BASE_LIB + ".tmp", BASE_SRC, "-lcufft", "-lcublas", "-Xlinker", "-rpath=" + cudalib]
    res = subprocess.run(cmd, capture_output=True, text=True)
    if res.returncode != 0:
        raise RuntimeError(f"baseline build failed:\n{res.stdout}\n{res.stderr}")
    os.replace(BASE_LIB + ".tmp", BASE_LIB)
    return BASE_LIB


if __name__ == "__main__":
    print(build(verbose="-v" in sys.argv))
