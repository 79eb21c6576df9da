"""Writes tests/golden/solve_*.txt: the oracle's lowest eigenvalues for the
solve-parity tests of the GPU eigensolver (tests/test_gpu_solver.py), from
the oracle's textbook LOBPCG (oracle/eig.py) on the oracle's FFT-symbol
operator (oracle/fourier.py) to Res <= 1e-11.  Calls only oracle/ and the
input descriptions in workloads/.

    python tests/golden/make_solve_golden.py
"""
import os
import sys
import time

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, os.path.dirname(os.path.dirname(HERE)))

import workloads as wl  # noqa: E402
from oracle import eig, fourier, penalty, permittivity  # noqa: E402

# name, structure, N, k indices on its path, nev, block
CASES = [
    ("fcc_air_spheres_16", wl.fcc_air_spheres, 16, [0, 10, 29], 12, 16),
    ("diamond_rods_32", wl.diamond_rods, 32, [5], 12, 16),
]


def solve(structure, n, k, nev, block, seed):
    g = penalty.gamma_practical(k)
    blocks = permittivity.cell_blocks(structure, n)
    kap = fourier.kappa(n, structure.lattice, k)
    am = lambda e: permittivity.apply_m(blocks, e)
    deflate = not np.any(k)
    theta, _, res, its = eig.lobpcg(lambda x: fourier.apply_symbols(x, kap, am, g),
                                    lambda r: fourier.precondition(r, kap, g),
                                    wl.random_block(block, n, seed=seed), nev, tol=1e-11, maxit=2000,
                                    deflate=deflate)
    return theta, res, its


def main(only=None):
    for name, maker, n, kidx, nev, block in CASES:
        if only and name not in only:
            continue
        s = maker()
        path = wl.config_k(s.name)
        lines = [f"# oracle LOBPCG eigenvalues (omega_h^2), {name}: structure {s.name}, N = {n}, "
                 f"{nev} bands, block {block}, Res <= 1e-11",
                 "# k index on the structure's path, kx, ky, kz, then the eigenvalues ascending"]
        for i in kidx:
            t0 = time.time()
            theta, res, its = solve(s, n, path[i], nev, block, seed=100 + i)
            assert np.all(res <= 1e-11), res
            print(f"{name} k{i}: {its} iterations, {time.time() - t0:.1f} s, max res {res.max():.2e}")
            lines.append(" ".join([str(i)] + [repr(float(v)) for v in path[i]] + [repr(float(v)) for v in theta]))
        with open(os.path.join(HERE, f"solve_{name}.txt"), "w") as fh:
            fh.write("\n".join(lines) + "\n")


if __name__ == "__main__":
    main(sys.argv[1:])
