"""Staggered sampling and the discrete inverse permittivity (oracle; test
infrastructure only).

Sec. 2.1 eqs. yee_edgefacedofs / yee_volumedofs place, for 1-based grid
indices 1 <= i, j, k <= N and h = 1/N,
    E1 at ((i-1/2)h, j h, k h),  E2 at (i h, (j-1/2)h, k h),
    E3 at (i h, j h, (k-1/2)h),  volume centres at ((i-1/2)h, (j-1/2)h, (k-1/2)h),
in the fractional coordinates x' of the unit cube; array slot i-1 holds index
i.  A fractional point sits at the physical point A x' (Sec. 2.2 eq.
ct_replacement).

Sec. 1 eq. intro_permittivity: epsilon_1 is the INVERSE permittivity of the
material.  Sec. 3.1 eq. permittivity_diagonal_case: the diagonal blocks are
sampled pointwise at the edges, M_ii = (eps_ii - 1) I_i + I.  Sec. 3.2.1
eq. trivial_trivial (M_Trivial): the off-diagonal blocks eps_ij I_V are
sampled at the volume centres.  Lemma 3.5: M_Trivial is a direct sum of one
Hermitian 3x3 block per cell (same array slot for all three components).

With several materials (the paper has one plus vacuum) each diagonal entry
comes from the material at its edge point and the off-diagonals from the
material at the volume centre; with one material this is exactly M_Trivial.
"""
from __future__ import annotations

import numpy as np

SHAPE_SPHERE, SHAPE_SEGMENT, SHAPE_BOX, SHAPE_GYROID = 0, 1, 2, 3

POINT_SETS = ("E1", "E2", "E3", "V")


def fractional_points(n: int, which: str) -> np.ndarray:
    """(N, N, N, 3) fractional coordinates (x', y', z') of a point set,
    indexed [z][y][x] like the fields."""
    h = 1.0 / n
    idx = np.arange(1, n + 1, dtype=np.float64)       # 1-based i, j, k
    half = {"E1": (0.5, 0, 0), "E2": (0, 0.5, 0), "E3": (0, 0, 0.5), "V": (0.5, 0.5, 0.5)}[which]
    xs = (idx - half[0]) * h
    ys = (idx - half[1]) * h
    zs = (idx - half[2]) * h
    z, y, x = np.meshgrid(zs, ys, xs, indexing="ij")
    return np.stack([x, y, z], axis=-1)


def _dot3(a, b):
    """a . b over the last axis, summed left to right: (a0 b0 + a1 b1) + a2 b2."""
    return (a[..., 0] * b[..., 0] + a[..., 1] * b[..., 1]) + a[..., 2] * b[..., 2]


def _inside(shape_kind, params, p):
    """Membership of Cartesian points p (..., 3) in a unit-cube-periodic shape.

    sphere: |p - c| < r (surface outside); rod (flat-capped cylinder from a
    to b): the foot point on the axis lies within the closed segment and the
    distance to the axis is below r (caps closed, lateral surface open); box:
    lo <= p < hi per axis; gyroid: g(p) > t (mode 0) or |g(p)| > t (mode 1)
    with g = sin X cos Y + sin Y cos Z + sin Z cos X, X = 2 pi x.  Distances
    are evaluated left to right (see _dot3) so that a point on a boundary is
    classified the same way on every machine.  Pinned branch by branch in
    tests/test_oracle_permittivity.py (brute force over images, hand points,
    volume fractions, gyroid values)."""
    images = np.array([(a, b, c) for a in (-1, 0, 1) for b in (-1, 0, 1) for c in (-1, 0, 1)], dtype=np.float64)
    # After d -= round(d) every |d_i| <= 1/2, so an image other than (0,0,0)
    # has a coordinate of size >= 1/2 and lies at distance >= 1/2 from the
    # shape's centre: a shape whose reach is below 1/2 needs only image 0.
    centre_only = images[13:14]
    if shape_kind == SHAPE_SPHERE:
        c = np.array(params[:3])
        r = params[3]
        d = p - c
        d = d - np.round(d)
        hit = np.zeros(p.shape[:-1], dtype=bool)
        for im in (centre_only if r < 0.5 else images):
            q = d + im
            hit |= _dot3(q, q) < r * r
        return hit
    if shape_kind == SHAPE_SEGMENT:
        a = np.array(params[:3])
        b = np.array(params[3:6])
        r = params[6]
        mid = 0.5 * (a + b)
        axis = b - a
        length = np.sqrt((axis[0] * axis[0] + axis[1] * axis[1]) + axis[2] * axis[2])
        u = axis / length
        d = p - mid
        d = d - np.round(d)
        hit = np.zeros(p.shape[:-1], dtype=bool)
        # a hit needs |q|^2 = t^2 + |perp|^2 < (length/2)^2 + r^2
        for im in (centre_only if 0.5 * length + r < 0.5 else images):
            q = d + im
            t = _dot3(q, u)
            perp = q - t[..., None] * u
            hit |= (np.abs(t) <= 0.5 * length) & (_dot3(perp, perp) < r * r)
        return hit
    if shape_kind == SHAPE_BOX:
        lo = np.array(params[:3])
        hi = np.array(params[3:6])
        w = p - np.floor(p)
        hit = np.zeros(p.shape[:-1], dtype=bool)
        for im in images:
            q = w + im
            hit |= np.all((q >= lo) & (q < hi), axis=-1)
        return hit
    if shape_kind == SHAPE_GYROID:
        t, mode = params[0], int(params[1])
        x, y, z = (2 * np.pi * p[..., i] for i in range(3))
        g = np.sin(x) * np.cos(y) + np.sin(y) * np.cos(z) + np.sin(z) * np.cos(x)
        return (np.abs(g) > t) if mode == 1 else (g > t)
    raise ValueError(shape_kind)


def material_ids(structure, n: int, which: str) -> np.ndarray:
    """Material index at every point of a staggered point set; the first
    shape containing the point wins, else the background."""
    frac = fractional_points(n, which)
    a = np.asarray(structure.lattice, dtype=np.float64)
    phys = np.stack([_dot3(a[r], frac) for r in range(3)], axis=-1)   # A x'
    ids = np.full(frac.shape[:-1], structure.background, dtype=np.int64)
    done = np.zeros(frac.shape[:-1], dtype=bool)
    for s in structure.shapes:
        hit = _inside(s.kind, s.params, phys) & ~done
        ids[hit] = s.material
        done |= hit
    return ids


def inverse_permittivity(structure) -> np.ndarray:
    """epsilon_1 = eps^{-1} for every material (FP64)."""
    return np.linalg.inv(np.asarray(structure.eps, dtype=np.complex128))


def cell_blocks_from_ids(inv_eps, ids_e1, ids_e2, ids_e3, ids_v) -> np.ndarray:
    """(N, N, N, 3, 3) Hermitian per-cell blocks of M (Sec. 3.2.1)."""
    blocks = np.zeros(ids_v.shape + (3, 3), dtype=np.complex128)
    blocks[..., 0, 0] = inv_eps[ids_e1, 0, 0].real
    blocks[..., 1, 1] = inv_eps[ids_e2, 1, 1].real
    blocks[..., 2, 2] = inv_eps[ids_e3, 2, 2].real
    for i, j in ((0, 1), (0, 2), (1, 2)):
        blocks[..., i, j] = inv_eps[ids_v, i, j]
        blocks[..., j, i] = np.conj(inv_eps[ids_v, i, j])
    return blocks


def cell_blocks(structure, n: int) -> np.ndarray:
    inv = inverse_permittivity(structure)
    ids = [material_ids(structure, n, w) for w in POINT_SETS]
    return cell_blocks_from_ids(inv, *ids)


def apply_m(blocks: np.ndarray, e: np.ndarray) -> np.ndarray:
    """M E with one 3x3 block per cell; e has shape (..., 3, N, N, N)."""
    return np.einsum("zyxij,...jzyx->...izyx", blocks, e)


def assemble_m(blocks: np.ndarray) -> np.ndarray:
    """Dense 3N^3 x 3N^3 matrix of M (component-major ordering), for small N."""
    n3 = blocks.shape[0] * blocks.shape[1] * blocks.shape[2]
    b = blocks.reshape(n3, 3, 3)
    m = np.zeros((3 * n3, 3 * n3), dtype=np.complex128)
    r = np.arange(n3)
    for i in range(3):
        for j in range(3):
            m[i * n3 + r, j * n3 + r] = b[:, i, j]
    return m


def cell_min_eigenvalue(blocks: np.ndarray) -> np.ndarray:
    """Smallest eigenvalue of every cell block (HPD check, Lemma 3.5)."""
    return np.linalg.eigvalsh(blocks)[..., 0]
