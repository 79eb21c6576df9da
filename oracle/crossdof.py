"""M_CrossDoF: the discrete inverse permittivity with symmetrised cross-DoF
transfer on its off-diagonal blocks (Sec. 3.2.2, eqs. crossdof_xytemplate,
crossdof_Tmat, crossdof_herm).  Test infrastructure only (see
oracle/__init__.py): plain FP64 numpy on fields of shape (..., 3, N, N, N)
indexed [component][z][y][x].

The diagonal blocks are those of M_Trivial: (eps_1)_cc of the material at the
E_c points.  Off the diagonal, E^j is carried to the E^i points by averaging
its four nearest DoFs, T_ij, and the block is symmetrised:

    block (i, j) = ( diag(e_ij at E_i) T_ij + T_ij diag(e_ij at E_j) ) / 2,
    block (j, i) = its conjugate transpose,

where e_ij is (eps_1)_ij of the material at each point.  With one material
in vacuum this is the paper's eps_ij (I_i T_ij + T_ij I_j) / 2 with the edge
indicators I_i; with several materials it is the reading above.

Reading of the transfer operators.  The Kronecker forms printed in eq.
crossdof_Tmat list the axes with x slowest, while the vectors here run x
fastest (the ordering of D_{s,1} = I_{N^2} (x) D_s in Sec. 2.1).  The
componentwise template of eq. crossdof_xytemplate decides: E^1 at
(i - 1/2, j, k) is the mean of E^2 at x in {i - 1, i} and y in
{j - 1/2, j + 1/2} (the printed template lists E^2_{i-1, j-1/2, k} twice;
the fourth point is E^2_{i-1, j+1/2, k}).  With 1-based DoF indices in
0-based array slots (E^1_{i-1/2, j, k} in slot [k-1][j-1][i-1],
E^2_{i, j-1/2, k} in slot [k-1][j-1][i-1], E^3_{i, j, k-1/2} likewise):

    T_12: D0 along x, D0^T along y      T_13: D0 along x, D0^T along z
    T_23: D0 along y, D0^T along z

with (D0 phi)_s = (phi_s + phi_{s-1}) / 2 and (D0^T phi)_s =
(phi_s + phi_{s+1}) / 2, periodic (eq. yee:D0D1).
"""
import numpy as np

from . import permittivity

# array axes of a field component [z][y][x]
_X, _Y, _Z = -1, -2, -3


def _d0(a, axis):
    """(phi_s + phi_{s-1}) / 2 along one axis, periodic."""
    return 0.5 * (a + np.roll(a, 1, axis=axis))


def _d0t(a, axis):
    """(phi_s + phi_{s+1}) / 2 along one axis, periodic (the transpose of D0)."""
    return 0.5 * (a + np.roll(a, -1, axis=axis))


# (D0 axis, D0^T axis) of T_ij
_T_AXES = {(0, 1): (_X, _Y), (0, 2): (_X, _Z), (1, 2): (_Y, _Z)}


def transfer(i: int, j: int, a: np.ndarray) -> np.ndarray:
    """T_ij a: values of component j carried to the points of component i."""
    d0_axis, d0t_axis = _T_AXES[(i, j)]
    return _d0t(_d0(a, d0_axis), d0t_axis)


def transfer_t(i: int, j: int, a: np.ndarray) -> np.ndarray:
    """T_ij^T a (from the points of component i to those of component j)."""
    d0_axis, d0t_axis = _T_AXES[(i, j)]
    return _d0(_d0t(a, d0_axis), d0t_axis)


class CrossDofM:
    """M_CrossDoF of a structure at grid n (eq. crossdof_herm)."""

    def __init__(self, structure, n: int):
        inv = permittivity.inverse_permittivity(structure)
        ids = [permittivity.material_ids(structure, n, w) for w in ("E1", "E2", "E3")]
        self.n = n
        # diagonal entries at the E_c points
        self.diag = [inv[ids[c], c, c].real for c in range(3)]
        # off-diagonal (eps_1)_ij at the E_i and at the E_j points
        self.off = {}
        for (i, j) in _T_AXES:
            self.off[(i, j)] = (inv[ids[i], i, j], inv[ids[j], i, j])

    def apply(self, e: np.ndarray) -> np.ndarray:
        """M_CrossDoF e for fields e of shape (..., 3, N, N, N)."""
        e = np.asarray(e, dtype=np.complex128)
        out = np.empty_like(e)
        for c in range(3):
            out[..., c, :, :, :] = self.diag[c] * e[..., c, :, :, :]
        for (i, j), (at_i, at_j) in self.off.items():
            ei, ej = e[..., i, :, :, :], e[..., j, :, :, :]
            # block (i, j) on E^j and its adjoint, block (j, i), on E^i
            out[..., i, :, :, :] += 0.5 * (at_i * transfer(i, j, ej) + transfer(i, j, at_j * ej))
            out[..., j, :, :, :] += 0.5 * (transfer_t(i, j, np.conj(at_i) * ei) + np.conj(at_j) * transfer_t(i, j, ei))
        return out

    def dense(self) -> np.ndarray:
        """The 3N^3 x 3N^3 matrix (component-major, cells z, y, x), small n."""
        n3 = self.n ** 3
        eye = np.eye(3 * n3, dtype=np.complex128).reshape(3 * n3, 3, self.n, self.n, self.n)
        cols = self.apply(eye).reshape(3 * n3, 3 * n3)
        return cols.T
