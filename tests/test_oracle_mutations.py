"""Planted mistakes: each plausible error in the oracle must fail a pin.

Every case patches one oracle function with a realistic slip (a flipped
sign, a dropped term, a transposed operand, a shifted index) and asserts
that one of the pin tests then fails.  CPU only; the mistake is planted in
the oracle, never in the CUDA library.
"""
import numpy as np
import pytest

import test_oracle_operators as ops_pins
import test_oracle_permittivity as perm_pins
import test_oracle_spectrum as spec_pins
import test_oracle_stencils as st_pins
from oracle import fourier, permittivity, stencils, yee


def _fails(fn, *args):
    with pytest.raises(AssertionError):
        fn(*args)


def test_flipped_bloch_sign_in_symbols(monkeypatch):
    orig = fourier.kappa

    def bad(n, lattice, k, m=1, reading="summed"):
        return orig(n, lattice, -np.asarray(k, dtype=float), m, reading)

    monkeypatch.setattr(fourier, "kappa", bad)
    _fails(ops_pins.test_symbols_have_the_continuum_limit, "SC")
    _fails(ops_pins.test_symbol_form_equals_stencil_form, "SC", 1)


def test_dropped_average_in_bloch_term(monkeypatch):
    orig = yee.axis_terms

    def bad(n, m, grid_axis, kt):
        return [(ax, off, w) for ax, off, w in orig(n, m, grid_axis, kt) if w.imag == 0] + \
               [(grid_axis, 0, 1j * kt)]

    monkeypatch.setattr(yee, "axis_terms", bad)
    _fails(ops_pins.test_symbol_form_equals_stencil_form, "SC", 1)


def test_forward_instead_of_backward_difference(monkeypatch):
    orig = stencils.stencil_offsets

    def bad(m, kind, h):
        return [(-off - 1 if kind == 1 else off, w) for off, w in orig(m, kind, h)]

    monkeypatch.setattr(stencils, "stencil_offsets", bad)
    _fails(st_pins.test_yee_matrices_second_order)


def test_transposed_off_diagonal_blocks(monkeypatch):
    orig = permittivity.cell_blocks_from_ids

    def bad(inv_eps, *ids):
        return np.swapaxes(orig(inv_eps, *ids), -1, -2)

    monkeypatch.setattr(permittivity, "cell_blocks_from_ids", bad)
    _fails(ops_pins.test_homogeneous_m_is_the_constitutive_map)


def test_dropped_penalty_term(monkeypatch):
    def bad(self, hfield, apply_m, gamma):
        return self.curl(apply_m(self.curl_adj(hfield)))

    monkeypatch.setattr(yee.YeeOperators, "compensated", bad)
    _fails(ops_pins.test_symbol_form_equals_stencil_form, "SC", 1)
    _fails(spec_pins.test_lobpcg_matches_dense, (0.6, 1.3, -0.5))


def test_curl_symbol_with_conjugate(monkeypatch):
    orig = fourier.ka_matrix
    monkeypatch.setattr(fourier, "ka_matrix", lambda kap: orig(np.conj(kap)))
    _fails(ops_pins.test_symbol_form_equals_stencil_form, "FCC", 1)


def test_wrong_edge_position(monkeypatch):
    orig = permittivity.fractional_points

    def bad(n, which):
        p = orig(n, which)
        if which == "E1":
            p = p.copy()
            p[..., 0] += 0.5 / n
        return p

    monkeypatch.setattr(permittivity, "fractional_points", bad)
    _fails(perm_pins.test_staggered_positions)


def test_preconditioner_missing_penalty(monkeypatch):
    orig = fourier.precondition
    monkeypatch.setattr(fourier, "precondition", lambda r, kap, gamma, tiny=0.0: orig(r, kap, 1.0, tiny))
    _fails(spec_pins.test_preconditioned_rayleigh_quotient_bounds, (0.4, 2.2, -0.9))


def test_dft_with_wrong_sign(monkeypatch):
    orig = fourier.dft_matrix
    monkeypatch.setattr(fourier, "dft_matrix", lambda n: np.conj(orig(n)))
    _fails(st_pins.test_fft_route_equals_dft_matrix, 4)


def test_cross_dof_transfer_mistakes(monkeypatch):
    """M_CrossDoF: a transfer that pairs the wrong neighbours (D0 and D0^T
    swapped) fails the geometry pin, and a (j, i) block built with T_ij in
    place of its transpose fails the Hermiticity pin."""
    import test_oracle_crossdof as cd_pins
    from oracle import crossdof

    with monkeypatch.context() as mp:
        mp.setattr(crossdof, "_T_AXES", {k: (v[1], v[0]) for k, v in crossdof._T_AXES.items()})
        _fails(cd_pins.test_transfer_averages_the_four_nearest_dofs, 0, 1)

    with monkeypatch.context() as mp:
        mp.setattr(crossdof, "transfer_t", crossdof.transfer)   # the transpose forgotten
        _fails(cd_pins.test_hermitian_on_an_anisotropic_structure)


def _patched_inside(kind, branch):
    """permittivity._inside with one shape kind routed to a faulty branch."""
    orig = permittivity._inside

    def f(shape_kind, params, p):
        return branch(params, p) if shape_kind == kind else orig(shape_kind, params, p)

    return f


def _segment_variant(cap_strict=False, lateral_closed=False, reach_without_r=False, raw_axis=False):
    """The oracle's rod test with one slip switched on."""
    images = np.array([(a, b, c) for a in (-1, 0, 1) for b in (-1, 0, 1) for c in (-1, 0, 1)], dtype=float)

    def branch(params, p):
        a = np.array(params[:3])
        b = np.array(params[3:6])
        r = params[6]
        mid = 0.5 * (a + b)
        axis = b - a
        length = np.sqrt(axis @ axis)
        u = axis if raw_axis else axis / length
        d = p - mid
        d = d - np.round(d)
        reach = 0.5 * length if reach_without_r else 0.5 * length + r
        hit = np.zeros(p.shape[:-1], dtype=bool)
        for im in (images[13:14] if reach < 0.5 else images):
            q = d + im
            t = q @ u
            perp = q - t[..., None] * u
            in_len = np.abs(t) < 0.5 * length if cap_strict else np.abs(t) <= 0.5 * length
            pp = np.sum(perp * perp, axis=-1)
            hit |= in_len & ((pp <= r * r) if lateral_closed else (pp < r * r))
        return hit

    return branch


@pytest.mark.parametrize("slip", ["cap_strict", "lateral_closed", "reach_without_r", "raw_axis"])
def test_rod_membership_slips(monkeypatch, slip):
    """Open caps, a closed lateral surface, an image bound that forgets the
    radius and an unnormalised axis each fail a rod pin."""
    import test_oracle_permittivity as pp

    monkeypatch.setattr(permittivity, "_inside", _patched_inside(permittivity.SHAPE_SEGMENT,
                                                                _segment_variant(**{slip: True})))
    failures = 0
    for fn, args in [(pp.test_segment_hand_points, ()), (pp.test_segment_image_only_point, ())] + \
            [(pp.test_segment_membership_matches_brute_force, (s,)) for s in pp._SEGMENTS]:
        try:
            fn(*args)
        except AssertionError:
            failures += 1
    assert failures > 0, slip


def test_box_closed_upper_face(monkeypatch):
    import test_oracle_permittivity as pp

    def bad(params, p):
        lo, hi = np.array(params[:3]), np.array(params[3:6])
        w = p - np.floor(p)
        hit = np.zeros(p.shape[:-1], dtype=bool)
        for a in (-1, 0, 1):
            for b in (-1, 0, 1):
                for c in (-1, 0, 1):
                    q = w + np.array([a, b, c])
                    hit |= np.all((q >= lo) & (q <= hi), axis=-1)
        return hit

    monkeypatch.setattr(permittivity, "_inside", _patched_inside(permittivity.SHAPE_BOX, bad))
    _fails(pp.test_box_membership)


@pytest.mark.parametrize("slip", ["swap", "sign", "abs"])
def test_gyroid_slips(monkeypatch, slip):
    """sin and cos swapped, a flipped term, or the two modes exchanged each
    fail the gyroid point values."""
    import test_oracle_permittivity as pp

    def bad(params, p):
        t, mode = params[0], int(params[1])
        x, y, z = (2 * np.pi * p[..., i] for i in range(3))
        if slip == "swap":
            g = np.cos(x) * np.sin(y) + np.cos(y) * np.sin(z) + np.cos(z) * np.sin(x)
        elif slip == "sign":
            g = np.sin(x) * np.cos(y) - np.sin(y) * np.cos(z) + np.sin(z) * np.cos(x)
        else:
            g = np.sin(x) * np.cos(y) + np.sin(y) * np.cos(z) + np.sin(z) * np.cos(x)
            mode = 1 - mode
        return (np.abs(g) > t) if mode == 1 else (g > t)

    monkeypatch.setattr(permittivity, "_inside", _patched_inside(permittivity.SHAPE_GYROID, bad))
    _fails(pp.test_gyroid_point_values)


def test_sphere_closed_surface(monkeypatch):
    import test_oracle_permittivity as pp

    def bad(params, p):
        c, r = np.array(params[:3]), params[3]
        d = p - c
        d = d - np.round(d)
        return np.sum(d * d, axis=-1) <= r * r

    monkeypatch.setattr(permittivity, "_inside", _patched_inside(permittivity.SHAPE_SPHERE, bad))
    _fails(pp.test_sphere_hand_points)
