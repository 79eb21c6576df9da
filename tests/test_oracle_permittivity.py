"""Pins of the oracle's staggered sampling and discrete inverse permittivity."""
import math

import numpy as np
import pytest

import workloads as wl
from oracle import permittivity


def test_staggered_positions():
    """Sec. 2.1 eqs. yee_edgefacedofs / yee_volumedofs: slot (i-1, j-1, k-1)
    (x, y, z) of E1 sits at ((i-1/2)h, jh, kh), of E2 at (ih, (j-1/2)h, kh),
    of E3 at (ih, jh, (k-1/2)h), of the volume at ((i-1/2)h, (j-1/2)h, (k-1/2)h)."""
    n = 5
    h = 1.0 / n
    i, j, k = 2, 4, 1                 # 1-based
    slot = (k - 1, j - 1, i - 1)     # [z][y][x]
    want = {"E1": ((i - .5) * h, j * h, k * h), "E2": (i * h, (j - .5) * h, k * h),
            "E3": (i * h, j * h, (k - .5) * h), "V": ((i - .5) * h, (j - .5) * h, (k - .5) * h)}
    for w, p in want.items():
        np.testing.assert_allclose(permittivity.fractional_points(n, w)[slot], p, atol=1e-15)


def test_sphere_volume_fraction_and_symmetry():
    """The volume-centre indicator of a centred sphere has the sphere's
    volume fraction (up to O(h)) and the mirror symmetry x -> 1 - x."""
    n = 32
    s = wl.sc_gyro_sphere(radius=0.3)
    ids = permittivity.material_ids(s, n, "V")
    frac = np.mean(ids == 1)
    assert abs(frac - 4 / 3 * math.pi * 0.3 ** 3) < 0.02
    assert np.array_equal(ids, ids[:, :, ::-1]) and np.array_equal(ids, ids[::-1, :, :])


def test_periodic_images_and_first_shape_wins():
    """A sphere centred on a cell corner is seen through its periodic
    images; overlapping shapes resolve to the first in the list."""
    n = 16
    s = wl.Structure("t", wl.SC.copy(), np.stack([wl.VACUUM, 2 * wl.VACUUM, 3 * wl.VACUUM]), 0,
                     [wl.Shape(wl.SHAPE_SPHERE, 1, (0.0, 0.0, 0.0, 0.2)),
                      wl.Shape(wl.SHAPE_SPHERE, 2, (0.1, 0.1, 0.1, 0.3))])
    ids = permittivity.material_ids(s, n, "V")
    # volume centre nearest to the corner, seen from the far side of the cell
    assert ids[n - 1, n - 1, n - 1] == 1
    assert ids[0, 0, 0] == 1                   # inside both: first shape wins
    assert ids[3, 3, 3] == 2                   # only in the second sphere


def test_paper_anisotropic_tensor_satisfies_assumption():
    """Sec. 4.1 eq. exp_permittivity (beta = 0.875): epsilon_1 has
    eigenvalues (sqrt(1+beta^2) +- beta)/eps_lattice and 1/eps_lattice, all
    in (0, 1] (Assumption 3.1)."""
    b = 0.875
    inv = np.linalg.inv(wl.paper_anisotropic(13.0, b))
    ev = np.linalg.eigvalsh(inv)
    want = np.sort([(math.sqrt(1 + b * b) - b) / 13, 1 / 13, (math.sqrt(1 + b * b) + b) / 13])
    np.testing.assert_allclose(ev, want, rtol=1e-13)
    assert np.all((ev > 0) & (ev <= 1))


def test_trivial_matrix_hpd_bound_and_block_spectrum():
    """Lemma 3.5: the spectrum of M_Trivial is the union of its per-cell
    3x3 block spectra; Prop. 3.6: lambda_min(M_Trivial) >= lambda_min(hat
    epsilon_1) with hat eps_ii = min(eps_ii, 1)."""
    n = 6
    inv_target = np.linalg.inv(wl.paper_anisotropic(13.0))
    eps = np.linalg.inv(inv_target)
    s = wl.Structure("t", wl.SC.copy(), np.stack([wl.VACUUM, eps]), 0,
                     [wl.Shape(wl.SHAPE_SPHERE, 1, (0.5, 0.5, 0.5, 0.3))])
    blocks = permittivity.cell_blocks(s, n)
    dense = permittivity.assemble_m(blocks)
    np.testing.assert_allclose(dense, dense.conj().T, atol=0)
    spec = np.linalg.eigvalsh(dense)
    cells = np.sort(np.linalg.eigvalsh(blocks).ravel())
    np.testing.assert_allclose(spec, cells, atol=1e-14)
    e1 = inv_target.copy()
    for i in range(3):
        e1[i, i] = min(e1[i, i].real, 1.0)
    assert spec[0] >= np.linalg.eigvalsh(e1)[0] - 1e-15
    # the cells straddling the interface really mix edge and centre materials
    ids = [permittivity.material_ids(s, n, w) for w in permittivity.POINT_SETS]
    assert np.any(ids[0] != ids[3])


@pytest.mark.parametrize("maker", [wl.sc_gyro_sphere, wl.fcc_air_spheres, wl.diamond_rods, wl.woodpile])
def test_benchmark_structures_are_hpd(maker):
    n = 16
    blocks = permittivity.cell_blocks(maker(), n)
    assert permittivity.cell_min_eigenvalue(blocks).min() > 0


def test_non_hpd_cell_is_detected():
    """Two materials whose mixed cell block is indefinite: a strongly
    gyrotropic centre material next to edges of a weak one."""
    strong = np.linalg.inv(np.array([[1.0, 0.95j, 0], [-0.95j, 1.0, 0], [0, 0, 1.0]]))
    weak = np.diag([40.0, 40.0, 40.0]).astype(complex)
    s = wl.Structure("t", wl.SC.copy(), np.stack([weak, strong]), 0,
                     [wl.Shape(wl.SHAPE_BOX, 1, (0.2, 0.2, 0.2, 0.8, 0.8, 0.8))])
    blocks = permittivity.cell_blocks(s, 5)
    assert permittivity.cell_min_eigenvalue(blocks).min() < 0


def test_no_sampling_ties_on_the_sphere_config():
    """Configuration 1 (sphere r = 1/4 at the centre, N = 16): no sample
    point of any set lies on the sphere surface (distances squared differ
    from r^2 by far more than rounding)."""
    n = 16
    for w in permittivity.POINT_SETS:
        p = permittivity.fractional_points(n, w) - 0.5
        d2 = np.sum(p * p, axis=-1)
        assert np.abs(d2 - 0.0625).min() > 1e-6


# ---------------------------------------------------------------------------
# shape membership, branch by branch.  The reference here is a brute-force
# test over every periodic image n in {-2..2}^3 written from each shape's
# plain definition (a segment by its end points and a clamped parameter, a
# box by its corners), independent of the oracle's minimum-image shortcut.
# ---------------------------------------------------------------------------
_IMAGES2 = np.array([(a, b, c) for a in range(-2, 3) for b in range(-2, 3) for c in range(-2, 3)], dtype=float)


def _brute_segment(params, p):
    a = np.array(params[:3])
    b = np.array(params[3:6])
    r = params[6]
    ab = b - a
    hit = np.zeros(len(p), dtype=bool)
    for n in _IMAGES2:
        w = p - n - a
        s = (w @ ab) / (ab @ ab)               # parameter of the foot point
        foot = s[:, None] * ab
        hit |= (s >= 0) & (s <= 1) & (np.sum((w - foot) ** 2, axis=1) < r * r)
    return hit


def _brute_box(params, p):
    lo = np.array(params[:3])
    hi = np.array(params[3:6])
    hit = np.zeros(len(p), dtype=bool)
    for n in _IMAGES2:
        q = p - n
        hit |= np.all((q >= lo) & (q < hi), axis=1)
    return hit


def _brute_sphere(params, p):
    c = np.array(params[:3])
    r = params[3]
    hit = np.zeros(len(p), dtype=bool)
    for n in _IMAGES2:
        hit |= np.sum((p - n - c) ** 2, axis=1) < r * r
    return hit


_SEGMENTS = [
    (0.2, 0.3, 0.4, 0.7, 0.6, 0.55, 0.12),     # short tilted rod, minimum image suffices
    (0.9, 0.1, 0.5, 1.3, 0.45, 0.2, 0.1),      # crosses the cell faces
    (0.5 - 0.6 / 2 ** 0.5, 0.5 - 0.6 / 2 ** 0.5, 0.5,
     0.5 + 0.6 / 2 ** 0.5, 0.5 + 0.6 / 2 ** 0.5, 0.5, 0.2),   # reaches past 1/2: images needed
    (0.5 - 0.45 * 3 / 13 ** 0.5, 0.5 - 0.45 * 2 / 13 ** 0.5, 0.5,
     0.5 + 0.45 * 3 / 13 ** 0.5, 0.5 + 0.45 * 2 / 13 ** 0.5, 0.5, 0.3),   # half-length 0.45 < 1/2, but
    # the rim of a cap reaches x offset sqrt(0.45^2 + 0.3^2) = 0.54 > 1/2: images needed
    (0.25, 0.25, 0.25, 0.5, 0.5, 0.5, 0.1),    # one diamond bond
]


@pytest.mark.parametrize("seg", _SEGMENTS)
def test_segment_membership_matches_brute_force(seg):
    """Flat-capped rod: the oracle's minimum-image test agrees with the
    definition (foot point on [a, b], distance below r) over all images, on
    random points of the cell and on the sample points of a 24^3 grid."""
    rng = np.random.default_rng(7)
    p = np.concatenate([rng.uniform(-0.1, 1.1, size=(40000, 3)),
                        permittivity.fractional_points(24, "V").reshape(-1, 3)])
    got = permittivity._inside(wl.SHAPE_SEGMENT, seg, p)
    want = _brute_segment(seg, p)
    assert np.array_equal(got, want), np.count_nonzero(got != want)
    assert 0 < np.count_nonzero(want) < len(p)


def test_segment_hand_points():
    """Rod from (1/4, 1/2, 1/2) to (3/4, 1/2, 1/2), r = 1/8, exact in
    binary: the caps are closed (a point on a cap plane inside the radius is
    in), the lateral surface open, and nothing beyond a cap or the radius."""
    seg = (0.25, 0.5, 0.5, 0.75, 0.5, 0.5, 0.125)
    pts = {
        (0.5, 0.5, 0.5): True,            # centre
        (0.75, 0.5, 0.5): True,           # on the cap plane, on the axis
        (0.25, 0.5, 0.5625): True,        # on the other cap, off axis
        (0.7578125, 0.5, 0.5): False,     # just past the cap
        (0.5, 0.5, 0.625): False,         # on the lateral surface
        (0.5, 0.6171875, 0.5): True,      # just inside the lateral surface
        (0.5, 0.5, 0.6328125): False,     # just outside it
        (0.25 - 1e-3, 0.5, 0.5): False,   # before the first cap
        (1.5, 1.5, -0.5): True,           # periodic image of the centre
    }
    p = np.array(list(pts.keys()))
    got = permittivity._inside(wl.SHAPE_SEGMENT, seg, p)
    assert list(got) == list(pts.values())


def test_segment_image_only_point():
    """A diagonal rod of half-length 0.6 and radius 0.2 centred in the cell
    covers mid + (-0.49, 0.3, 0) only through its +x image: the foot point
    of mid + (0.51, 0.3, 0) lies at t = 0.573 < 0.6 and the distance squared
    to the axis is 0.022 < 0.04, while the minimum image is 0.56 from the
    axis."""
    seg = _SEGMENTS[2]
    p = np.array([[0.5 - 0.49, 0.8, 0.5]])
    assert permittivity._inside(wl.SHAPE_SEGMENT, seg, p)[0]


@pytest.mark.parametrize("n", [32, 64, 128])
def test_segment_volume_fraction(n):
    """The share of volume-centre samples inside one tilted rod of radius
    0.1 and length 0.45 approaches pi r^2 l (flat caps) at O(h)."""
    u = np.array([1.0, 2.0, 2.0]) / 3.0
    mid = np.array([0.5, 0.5, 0.5])
    a, b = mid - 0.225 * u, mid + 0.225 * u
    s = wl.Structure("rod", wl.SC.copy(), np.stack([wl.VACUUM, 2 * wl.VACUUM]), 0,
                     [wl.Shape(wl.SHAPE_SEGMENT, 1, (*a, *b, 0.1))])
    frac = np.mean(permittivity.material_ids(s, n, "V") == 1)
    vol = math.pi * 0.01 * 0.45
    assert abs(frac - vol) / vol < 2.0 / n


def test_box_membership():
    """Half-open box lo <= x < hi, seen through its periodic images."""
    box = (0.8, 0.25, 0.0, 1.2, 0.5, 1.0)    # crosses the x = 1 face
    pts = {
        (0.9, 0.3, 0.5): True,
        (0.1, 0.3, 0.5): True,       # image of the part beyond x = 1
        (0.2, 0.3, 0.5): False,      # x = 1.2 is the open end
        (0.8, 0.25, 0.0): True,      # the closed corner
        (0.9, 0.5, 0.5): False,      # y = hi is open
        (0.9, 0.3, 0.999): True,
        (0.5, 0.3, 0.5): False,
    }
    p = np.array(list(pts.keys()))
    assert list(permittivity._inside(wl.SHAPE_BOX, box, p)) == list(pts.values())
    rng = np.random.default_rng(3)
    q = rng.uniform(-0.5, 1.5, size=(20000, 3))
    for prm in [box, (0.0, -0.125, 0.25, 1.0, 0.125, 0.5), (0.3, 0.3, 0.3, 0.6, 0.7, 0.9)]:
        assert np.array_equal(permittivity._inside(wl.SHAPE_BOX, prm, q), _brute_box(prm, q))


def test_sphere_membership_matches_brute_force():
    rng = np.random.default_rng(5)
    q = rng.uniform(-0.2, 1.2, size=(30000, 3))
    for prm in [(0.5, 0.5, 0.5, 0.25), (0.05, 0.9, 0.5, 0.3), (0.5, 0.5, 0.5, 0.55)]:
        assert np.array_equal(permittivity._inside(wl.SHAPE_SPHERE, prm, q), _brute_sphere(prm, q))


def test_gyroid_point_values():
    """g(x) = sin X cos Y + sin Y cos Z + sin Z cos X with X = 2 pi x: g = 3/2
    at (1/8, 1/8, 1/8) (its maximum), -3/2 at the mirror point, 1 at
    (1/4, 0, 0) and (0, 1/4, 0) and (0, 0, 1/4), 0 at the origin and at
    (1/4, 1/4, 1/4), -1 at (3/4, 0, 0).  Mode 0 keeps g > t, mode 1 |g| > t."""
    p = np.array([[1 / 8, 1 / 8, 1 / 8], [-1 / 8, -1 / 8, -1 / 8], [0.25, 0, 0], [0, 0.25, 0], [0, 0, 0.25],
                  [0, 0, 0], [0.25, 0.25, 0.25], [0.75, 0, 0], [0.25, 0.25, 0], [0.25, 0.125, 0],
                  [0.25, 0, 0.125]])
    g = np.array([1.5, -1.5, 1.0, 1.0, 1.0, 0.0, 0.0, -1.0, 1.0, 2 ** 0.5, 1.0])
    # (1/4, 1/4, 0): sin(pi/2) cos(pi/2) + sin(pi/2) cos(0) + sin(0) cos(pi/2) = 1;
    # (1/4, 1/8, 0): cos(pi/4) + sin(pi/4) = sqrt 2, while the mirror gyroid
    # (y and z exchanged) has 1 there: the handedness is fixed
    for t in (-0.5, 0.5, 0.99, 1.01, 1.1, 1.49):
        assert list(permittivity._inside(wl.SHAPE_GYROID, (t, 0), p)) == list(g > t)
        assert list(permittivity._inside(wl.SHAPE_GYROID, (t, 1), p)) == list(np.abs(g) > t)


def test_gyroid_volume_fraction_is_odd_symmetric():
    """g is odd (g(-x) = -g(x)), so {g > t} and {g < -t} have the same
    volume: at N = 32 the samples of {g > 1.1} and of its point reflection
    through the origin, {g < -1.1}, are equinumerous and the mode-1 set is
    their disjoint union."""
    n = 32
    p = permittivity.fractional_points(n, "V").reshape(-1, 3)
    up = permittivity._inside(wl.SHAPE_GYROID, (1.1, 0), p)
    down = permittivity._inside(wl.SHAPE_GYROID, (1.1, 0), -p)
    both = permittivity._inside(wl.SHAPE_GYROID, (1.1, 1), p)
    assert np.count_nonzero(up) == np.count_nonzero(down) > 0
    assert np.count_nonzero(both) == 2 * np.count_nonzero(up)


def test_sphere_hand_points():
    """Sphere of radius 1/4 at the centre, exact in binary: the surface is
    outside, the inside strict, and periodic images count."""
    sph = (0.5, 0.5, 0.5, 0.25)
    pts = {(0.75, 0.5, 0.5): False, (0.7421875, 0.5, 0.5): True, (0.5, 0.25, 0.5): False,
           (0.5, 0.5, 0.5): True, (1.5, -0.5, 2.5): True, (0.75, 0.75, 0.5): False}
    p = np.array(list(pts.keys()))
    assert list(permittivity._inside(wl.SHAPE_SPHERE, sph, p)) == list(pts.values())
