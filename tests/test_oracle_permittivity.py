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
