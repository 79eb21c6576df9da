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
