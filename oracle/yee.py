"""Real-space Yee operators (oracle; test infrastructure only).

Fields are numpy arrays whose last three axes are (z, y, x), x fastest,
matching the Kronecker order of Sec. 2.1 eq. yee_block (D_{s,1} = I (x) I (x) D_s
acts on the fastest index).  A vector field carries its three Cartesian
components on the axis just before: shape (..., 3, N, N, N).

Sec. 2.1 eq. yee_block:    D_i = D_{1,i} + i k_i D_{0,i}
Sec. 2.1 eq. yee_ABmatrix: A = [[0, -D3, D2], [D3, 0, -D1], [-D2, D1, 0]],
                           B = [D1, D2, D3]
Sec. 2.2 eq. ct_blocks (general lattice, reading "summed", the default):
    hat D_i = sum_j b_ji (D_{1,j} + i kt_j D_{0,j}),  b = A^{-1},  kt = A^T k
  i.e. the discrete form of grad_{A,k} = A^{-T}(grad_x' + i A^T k).  The
  printed formula sums over j without j appearing; the alternative reading
  "literal" keeps the printed Bloch term: sum_j b_ji D_{1,j} + i k_i D_{0,i}.
Sec. 2.3 eq. kc_formulation: Op = A M A^H + gamma B^H B.

Operators are kept as lists of terms (grid_axis, offset, complex weight) with
(T phi)_i = sum weight * phi_{i + offset e_axis}; the adjoint negates the
offsets and conjugates the weights.  Grid axis 0 is x (numpy axis -1),
1 is y (axis -2), 2 is z (axis -3).
"""
from __future__ import annotations

import numpy as np

from .stencils import stencil_offsets


def axis_terms(n: int, m: int, grid_axis: int, kt: float):
    """Terms of D_{1,axis} + i kt D_{0,axis} on an N^3 grid (h = 1/N)."""
    h = 1.0 / n
    terms = [(grid_axis, off, complex(w)) for off, w in stencil_offsets(m, 1, h)]
    terms += [(grid_axis, off, 1j * kt * w) for off, w in stencil_offsets(m, 0, h)]
    return terms


def dhat_terms(n: int, m: int, lattice, k, reading: str = "summed"):
    """[hat D_1, hat D_2, hat D_3] as term lists (Sec. 2.1 eq. yee_block and
    Sec. 2.2 eq. ct_blocks)."""
    a = np.asarray(lattice, dtype=np.float64)
    k = np.asarray(k, dtype=np.float64)
    b = np.linalg.inv(a)
    kt = a.T @ k
    h = 1.0 / n
    out = []
    for i in range(3):
        terms = []
        for j in range(3):
            if b[j, i] == 0.0:
                continue
            if reading == "summed":
                terms += [(ax, off, b[j, i] * w) for ax, off, w in axis_terms(n, m, j, kt[j])]
            elif reading == "literal":
                terms += [(j, off, complex(b[j, i] * w)) for off, w in stencil_offsets(m, 1, h)]
            else:
                raise ValueError(reading)
        if reading == "literal":
            terms += [(i, off, 1j * k[i] * w) for off, w in stencil_offsets(m, 0, h)]
        out.append(terms)
    return out


def adjoint(terms):
    return [(ax, -off, np.conj(w)) for ax, off, w in terms]


def apply_terms(terms, phi: np.ndarray) -> np.ndarray:
    """sum_t w_t * phi shifted so that out_i = phi_{i + offset} (periodic)."""
    out = np.zeros(phi.shape, dtype=np.complex128)
    for ax, off, w in terms:
        out += w * np.roll(phi, -off, axis=-1 - ax)
    return out


class YeeOperators:
    """A, A^H, B, B^H and the compensated operator for one (N, m, lattice, k)."""

    def __init__(self, n: int, lattice, k, m: int = 1, reading: str = "summed"):
        self.n = n
        self.d = dhat_terms(n, m, lattice, k, reading)
        self.dh = [adjoint(t) for t in self.d]

    def curl(self, e):
        """A E  (edges -> faces), Sec. 2.1 eq. yee_ABmatrix."""
        d = self.d
        f = np.empty(e.shape, dtype=np.complex128)
        f[..., 0, :, :, :] = -apply_terms(d[2], e[..., 1, :, :, :]) + apply_terms(d[1], e[..., 2, :, :, :])
        f[..., 1, :, :, :] = apply_terms(d[2], e[..., 0, :, :, :]) - apply_terms(d[0], e[..., 2, :, :, :])
        f[..., 2, :, :, :] = -apply_terms(d[1], e[..., 0, :, :, :]) + apply_terms(d[0], e[..., 1, :, :, :])
        return f

    def curl_adj(self, f):
        """A^H H  (faces -> edges): block (i, j) of A^H is (A_ji)^H."""
        dh = self.dh
        e = np.empty(f.shape, dtype=np.complex128)
        e[..., 0, :, :, :] = apply_terms(dh[2], f[..., 1, :, :, :]) - apply_terms(dh[1], f[..., 2, :, :, :])
        e[..., 1, :, :, :] = -apply_terms(dh[2], f[..., 0, :, :, :]) + apply_terms(dh[0], f[..., 2, :, :, :])
        e[..., 2, :, :, :] = apply_terms(dh[1], f[..., 0, :, :, :]) - apply_terms(dh[0], f[..., 1, :, :, :])
        return e

    def div(self, f):
        """B H (faces -> volumes)."""
        return sum(apply_terms(self.d[i], f[..., i, :, :, :]) for i in range(3))

    def div_adj(self, psi):
        """B^H psi (volumes -> faces)."""
        return np.stack([apply_terms(self.dh[i], psi) for i in range(3)], axis=-4)

    def compensated(self, hfield, apply_m, gamma: float):
        """(A M A^H + gamma B^H B) H, Sec. 2.3 eq. kc_formulation."""
        return self.curl(apply_m(self.curl_adj(hfield))) + gamma * self.div_adj(self.div(hfield))
