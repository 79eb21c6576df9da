"""Seeded synthetic inputs shared by the oracle, the tests and the benchmark.

This module only *describes* inputs: lattices, shape lists, material
permittivity tensors, Bloch wave vectors and random complex blocks.  It holds
none of the method's arithmetic -- no staggered sample positions, no
permittivity inversion, no difference symbols, no penalty rule.  Both the CPU
oracle and the CUDA library turn these descriptions into discrete operators on
their own.

Conventions
-----------
* A structure is periodic with the Cartesian unit cube.  Shapes are given in
  Cartesian coordinates; every shape is tested against its periodic images.
* ``lattice`` holds the primitive vectors a1, a2, a3 as *columns* (Sec. 4,
  eq. exp_latticeconst).  The discrete grid lives on the fractional
  coordinates x' in [0,1)^3 and a point x' sits at the physical point A x'
  (Sec. 2.2, eq. ct_replacement).
* ``eps`` holds the relative PERMITTIVITY of each material (3x3 Hermitian
  positive definite).  The paper's epsilon_1 is its inverse (Sec. 1,
  eq. intro_permittivity); inverting is the consumer's job.
* A point takes the material of the first shape (in list order) that contains
  it, else ``background``.
* Random vectors are complex Gaussian blocks of shape (nvec, 3, N, N, N),
  component-major, then z, y, x with x fastest.
"""
from __future__ import annotations

import dataclasses
import math

import numpy as np

# Shape kinds (the integer codes are part of the C ABI, see include/pcx.h).
SHAPE_SPHERE = 0    # params: cx, cy, cz, r
SHAPE_SEGMENT = 1   # params: x0, y0, z0, x1, y1, z1, r   (finite cylinder, flat caps)
SHAPE_BOX = 2       # params: lox, loy, loz, hix, hiy, hiz (axis aligned)
SHAPE_GYROID = 3    # params: t, mode (0: g > t, 1: |g| > t)


@dataclasses.dataclass
class Shape:
    kind: int
    material: int
    params: tuple

    def packed(self) -> np.ndarray:
        p = np.zeros(9, dtype=np.float64)
        p[: len(self.params)] = self.params
        return p


@dataclasses.dataclass
class Structure:
    name: str
    lattice: np.ndarray            # (3,3) float64, columns a1 a2 a3
    eps: np.ndarray                # (n_mat, 3, 3) complex128 permittivity
    background: int
    shapes: list

    @property
    def n_mat(self) -> int:
        return int(self.eps.shape[0])


# ---------------------------------------------------------------------------
# lattices (Sec. 4, eq. exp_latticeconst) and Brillouin-zone points
# (Sec. 4, eq. exp_bzsym); values as printed in the paper.
# ---------------------------------------------------------------------------
SC = np.eye(3)
FCC = np.array([[0.0, 0.5, 0.5], [0.5, 0.0, 0.5], [0.5, 0.5, 0.0]]).T
BCC = np.array([[-0.5, 0.5, 0.5], [0.5, -0.5, 0.5], [0.5, 0.5, -0.5]]).T

PI = math.pi
FCC_POINTS = {
    "X": (0.0, 2 * PI, 0.0),
    "U": (PI / 2, 2 * PI, PI),
    "L": (PI, PI, PI),
    "G": (0.0, 0.0, 0.0),
    "W": (PI, 2 * PI, 0.0),
    "K": (1.5 * PI, 1.5 * PI, 0.0),
}
SC_POINTS = {"K": (0.0, 0.0, 0.0), "L": (PI, 0.0, 0.0), "M": (PI, PI, 0.0), "N": (PI, PI, PI)}


def k_path(points, labels, n_total):
    """n_total points spaced uniformly in arc length along the polyline
    through points[labels[0]], points[labels[1]], ... (both ends included)."""
    verts = np.array([points[l] for l in labels], dtype=np.float64)
    seg = np.linalg.norm(np.diff(verts, axis=0), axis=1)
    cum = np.concatenate([[0.0], np.cumsum(seg)])
    out = []
    for s in np.linspace(0.0, cum[-1], n_total):
        i = min(int(np.searchsorted(cum, s, side="right")) - 1, len(seg) - 1)
        t = 0.0 if seg[i] == 0 else (s - cum[i]) / seg[i]
        out.append(verts[i] + t * (verts[i + 1] - verts[i]))
    return np.array(out)


# ---------------------------------------------------------------------------
# material tensors
# ---------------------------------------------------------------------------
def seeded_rotation(rng) -> np.ndarray:
    """Real rotation: Q of QR(Gaussian 3x3), column signs fixed so that
    diag(R_qr) > 0, then det forced to +1."""
    q, r = np.linalg.qr(rng.standard_normal((3, 3)))
    q = q * np.sign(np.diag(r))
    if np.linalg.det(q) < 0:
        q[:, 0] = -q[:, 0]
    return q


def seeded_unitary(rng) -> np.ndarray:
    """Complex unitary: Q of QR(complex Gaussian 3x3) with unit-phase diag(R)."""
    z = rng.standard_normal((3, 3)) + 1j * rng.standard_normal((3, 3))
    q, r = np.linalg.qr(z)
    d = np.diag(r)
    return q * (d / np.abs(d))


def hermitian_pd(rng, lo, hi, complex_rotation=True) -> np.ndarray:
    """U diag(lam) U^H with lam ~ U[lo, hi]; every off-diagonal entry then has
    magnitude <= (hi - lo) / 2."""
    lam = rng.uniform(lo, hi, size=3)
    u = seeded_unitary(rng) if complex_rotation else seeded_rotation(rng)
    e = (u * lam) @ u.conj().T
    return 0.5 * (e + e.conj().T)


def gyrotropic(base_diag, rot, g) -> np.ndarray:
    """R diag(base) R^T plus the gyrotropic xy term: eps_12 += i g,
    eps_21 = conj(eps_12)."""
    e = (rot * np.asarray(base_diag, dtype=np.float64)) @ rot.T
    e = e.astype(np.complex128)
    e[0, 1] += 1j * g
    e[1, 0] -= 1j * g
    return e


def paper_anisotropic(eps_lattice, beta=0.875) -> np.ndarray:
    """Permittivity whose inverse is the paper's anisotropic epsilon_1
    (Sec. 4.1, eq. exp_permittivity)."""
    b = abs(beta)
    e1 = np.array(
        [[math.sqrt(1 + b * b), -1j * b, 0], [1j * b, math.sqrt(1 + b * b), 0], [0, 0, 1]],
        dtype=np.complex128,
    ) / eps_lattice
    return np.linalg.inv(e1)


VACUUM = np.eye(3, dtype=np.complex128)


# ---------------------------------------------------------------------------
# structures of the benchmark configurations
# ---------------------------------------------------------------------------
def sc_gyro_sphere(seed=20251117, radius=0.25) -> Structure:
    """Simple cubic, one sphere r=0.25 at the cell centre, eps =
    R diag(13,11,12) R^T + 0.5i gyrotropic xy term, vacuum background."""
    rng = np.random.default_rng(seed)
    rot = seeded_rotation(rng)
    eps = np.stack([VACUUM, gyrotropic((13.0, 11.0, 12.0), rot, 0.5)])
    shapes = [Shape(SHAPE_SPHERE, 1, (0.5, 0.5, 0.5, radius))]
    return Structure("sc-gyro-sphere", SC.copy(), eps, 0, shapes)


def fcc_air_spheres(seed=20251117, radius=0.3) -> Structure:
    """FCC lattice of air spheres (r=0.3) in a uniformly anisotropic
    background with eigenvalues in [8, 14]."""
    rng = np.random.default_rng(seed)
    bg = hermitian_pd(rng, 8.0, 14.0)
    eps = np.stack([bg, VACUUM])
    sites = [(0, 0, 0), (0, 0.5, 0.5), (0.5, 0, 0.5), (0.5, 0.5, 0)]
    shapes = [Shape(SHAPE_SPHERE, 1, (*s, radius)) for s in sites]
    return Structure("fcc-air-spheres", FCC.copy(), eps, 0, shapes)


DIAMOND_BONDS = [(0.25, 0.25, 0.25), (0.25, -0.25, -0.25), (-0.25, 0.25, -0.25), (-0.25, -0.25, 0.25)]


def diamond_rods(seed=20251117, radius=0.1) -> Structure:
    """Diamond network of dielectric rods (radius 0.1) on the FCC lattice:
    atoms on the FCC sites and the sites shifted by (1/4,1/4,1/4), one rod
    per nearest-neighbour bond (16 per cubic cell).  One seeded tensor per
    bond orientation, eigenvalues in [9, 13] (so every off-diagonal entry has
    magnitude <= 2), air background."""
    rng = np.random.default_rng(seed)
    mats = [VACUUM] + [hermitian_pd(rng, 9.0, 13.0) for _ in range(4)]
    sites = [(0, 0, 0), (0, 0.5, 0.5), (0.5, 0, 0.5), (0.5, 0.5, 0)]
    shapes = []
    for s in sites:
        b = np.add(s, (0.25, 0.25, 0.25))
        for o, d in enumerate(DIAMOND_BONDS):
            a = b - np.array(d)
            shapes.append(Shape(SHAPE_SEGMENT, 1 + o, (*b, *a, radius)))
    return Structure("diamond-rods", FCC.copy(), np.stack(mats), 0, shapes)


def woodpile(seed=20251117, width=0.25) -> Structure:
    """Simple cubic woodpile: four layers of height 1/4 along z with
    rectangular rods width x 1/4: along x at y=0, along y at x=0, along x at
    y=1/2, along y at x=1/2.  One seeded tensor per rod, eigenvalues in
    [4, 13], air background."""
    rng = np.random.default_rng(seed)
    mats = [VACUUM] + [hermitian_pd(rng, 4.0, 13.0) for _ in range(4)]
    w = width / 2
    shapes = [
        Shape(SHAPE_BOX, 1, (0.0, -w, 0.00, 1.0, w, 0.25)),
        Shape(SHAPE_BOX, 2, (-w, 0.0, 0.25, w, 1.0, 0.50)),
        Shape(SHAPE_BOX, 3, (0.0, 0.5 - w, 0.50, 1.0, 0.5 + w, 0.75)),
        Shape(SHAPE_BOX, 4, (0.5 - w, 0.0, 0.75, 0.5 + w, 1.0, 1.00)),
    ]
    return Structure("woodpile", SC.copy(), np.stack(mats), 0, shapes)


def random_inclusions(seed) -> Structure:
    """Learned-preconditioner training set member: 1-4 spheres or rods with
    radii in [0.1, 0.35] and tensors with eigenvalues in [2, 16] on the
    simple cubic lattice, air background."""
    rng = np.random.default_rng(seed)
    n = int(rng.integers(1, 5))
    mats = [VACUUM]
    shapes = []
    for i in range(n):
        mats.append(hermitian_pd(rng, 2.0, 16.0))
        r = float(rng.uniform(0.1, 0.35))
        c = rng.uniform(0.0, 1.0, size=3)
        if rng.uniform() < 0.5:
            shapes.append(Shape(SHAPE_SPHERE, i + 1, (*c, r)))
        else:
            d = rng.standard_normal(3)
            d = d / np.linalg.norm(d) * float(rng.uniform(0.3, 0.8))
            shapes.append(Shape(SHAPE_SEGMENT, i + 1, (*(c - d / 2), *(c + d / 2), r)))
    return Structure(f"random-{seed}", SC.copy(), np.stack(mats), 0, shapes)


def bcc_gyroid(double=False, anisotropic=True, eps_lattice=16.0, beta=0.875) -> Structure:
    """BCC-SG (material where g(x) > 1.1) or BCC-DG (|g(x)| > 1.1) on the BCC
    lattice (Sec. 4, eq. display:exp_latticeconst), with the paper's
    permittivity: epsilon_1 = I / eps_lattice (isotropic) or the gyrotropic
    tensor of eq. display:exp_permittivity (beta = 0.875), eps_lattice = 16
    for the BCC lattice; vacuum outside."""
    eps = paper_anisotropic(eps_lattice, beta) if anisotropic else eps_lattice * VACUUM
    shapes = [Shape(SHAPE_GYROID, 1, (1.1, 1 if double else 0))]
    name = ("bcc-dg" if double else "bcc-sg") + ("-aniso" if anisotropic else "-iso")
    return Structure(name, BCC.copy(), np.stack([VACUUM, eps]), 0, shapes)


BCC_POINTS = {"H'": (2 * PI, 0.0, 0.0), "G": (0.0, 0.0, 0.0), "P": (PI, PI, PI), "N": (PI, 0.0, PI),
              "H": (0.0, 2 * PI, 0.0)}


def ill_conditioned_sphere(seed=20251117, radius=0.345) -> Structure:
    """Sec. 4.4: a material whose inverse permittivity is
    U diag(1e-1, 1e-3, 1e-5) U^H (U a seeded unitary), so its permittivity
    is U diag(1e1, 1e3, 1e5) U^H, in a sphere of radius 0.345 at the centre
    of the simple cubic cell, vacuum outside (the sphere stands in for the
    SC-CURV geometry, whose cylinder axes the paper does not give)."""
    rng = np.random.default_rng(seed)
    u = seeded_unitary(rng)
    eps = u @ np.diag([1e1, 1e3, 1e5]).astype(np.complex128) @ u.conj().T
    eps = 0.5 * (eps + eps.conj().T)
    shapes = [Shape(SHAPE_SPHERE, 1, (0.5, 0.5, 0.5, radius))]
    return Structure("ill-conditioned-sphere", SC.copy(), np.stack([VACUUM, eps]), 0, shapes)


def homogeneous(eps, lattice=None) -> Structure:
    """One material filling the whole cell."""
    lat = SC.copy() if lattice is None else np.asarray(lattice, dtype=np.float64)
    return Structure("homogeneous", lat, np.stack([np.asarray(eps, dtype=np.complex128)]), 0, [])


# ---------------------------------------------------------------------------
# random blocks
# ---------------------------------------------------------------------------
def random_block(nvec, n, seed, dtype=np.complex128) -> np.ndarray:
    """Complex Gaussian block of shape (nvec, 3, n, n, n)."""
    rng = np.random.default_rng(seed)
    shape = (nvec, 3, n, n, n)
    x = rng.standard_normal(shape) + 1j * rng.standard_normal(shape)
    return x.astype(dtype)


def config_k(name):
    """Bloch wave vectors of the benchmark configurations (Cartesian)."""
    if name == "sc-gyro-sphere":
        return np.array([[2 * PI * 0.1, 2 * PI * 0.2, 2 * PI * 0.3]])
    if name == "fcc-air-spheres":
        return k_path(FCC_POINTS, ["G", "X", "W", "L"], 30)
    if name == "diamond-rods":
        return k_path(FCC_POINTS, ["X", "U", "L", "G", "X", "W", "K"], 40)
    if name == "woodpile":
        return np.array([[2 * PI * 0.1, 2 * PI * 0.2, 2 * PI * 0.3]])
    if name == "ill-conditioned-sphere":
        return np.array([[PI / 7, 3 * PI / 5, 4 * PI / 13]])
    if name.startswith("random"):
        return np.array([[PI, PI, PI]])
    raise KeyError(name)
