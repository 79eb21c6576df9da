"""Fourier-basis form of the compensated operator and the FFT-diagonal
preconditioner (oracle; test infrastructure only).

Lemma 2.1: a circulant C with first row (c_1..c_N) is F diag(lambda) F^H with
    lambda_i = sum_j c_j w^{(i-1)(j-1)},  F_ij = w^{(i-1)(j-1)} / sqrt(N),
    w = exp(+2 pi i / N).
Sec. 2.4: F3 = F (x) F (x) F and F3_3 = diag(F3, F3, F3).  Prop. 2.8:
    D_i = F3 K_i F3^H,  K_i = Lambda_1 + i k_i Lambda_0 on the axis of i,
    A = F3_3 K_A F3_3^H,  B^H B = F3_3 K_B F3_3^H,
    K_A = [[0, -K3, K2], [K3, 0, -K1], [-K2, K1, 0]],
    K_B = [K1^H; K2^H; K3^H] [K1 K2 K3].
Eq. matrixfree_kcform: with x = F3_3^H H the eigenproblem reads
    (K_A F3_3^H M F3_3 K_A^H + gamma K_B) x = w_h^2 x.
Eqs. matrixfree_diagP / matrixfree_finalform: preconditioner
    K_P^{-1},  K_P = K_A K_A^H + gamma K_B  (a 3x3 block per Fourier mode).
Under the coordinate change of Sec. 2.2 (reading "summed") the per-mode
symbol of hat D_i is  kappa_i(p) = sum_j b_ji (Lambda_1(p_j) + i kt_j Lambda_0(p_j)).

Fourier arrays use the same (…, 3, N, N, N) layout as real-space fields; the
last three axes are the mode indices (p3, p2, p1), p1 along x.
"""
from __future__ import annotations

import numpy as np

from .stencils import circulant_first_row


def dft_matrix(n: int) -> np.ndarray:
    """F of Lemma 2.1 (unitary, positive exponent)."""
    i = np.arange(n)
    return np.exp(2j * np.pi * np.outer(i, i) / n) / np.sqrt(n)


def circulant_symbol(first_row: np.ndarray) -> np.ndarray:
    """Eigenvalues lambda_p (p = 0..N-1) of a circulant, by the sum of
    Lemma 2.1 written out."""
    n = len(first_row)
    j = np.arange(n)
    w = np.exp(2j * np.pi / n)
    return np.array([np.sum(first_row * w ** ((p * j) % n)) for p in range(n)])


def lambda_tables(n: int, m: int = 1):
    """(Lambda_1, Lambda_0) diagonals of D1 and D0 (Prop. 2.8)."""
    return circulant_symbol(circulant_first_row(n, m, 1)), circulant_symbol(circulant_first_row(n, m, 0))


def kappa(n: int, lattice, k, m: int = 1, reading: str = "summed") -> np.ndarray:
    """(3, N, N, N) per-mode symbols kappa_i(p3, p2, p1) of hat D_i."""
    a = np.asarray(lattice, dtype=np.float64)
    k = np.asarray(k, dtype=np.float64)
    b = np.linalg.inv(a)
    kt = a.T @ k
    lam1, lam0 = lambda_tables(n, m)
    # 1D symbol along grid axis j broadcast to (p3, p2, p1)
    shapes = {0: (1, 1, n), 1: (1, n, 1), 2: (n, 1, 1)}
    out = np.zeros((3, n, n, n), dtype=np.complex128)
    for i in range(3):
        for j in range(3):
            if reading == "summed":
                sym = lam1 + 1j * kt[j] * lam0
            else:
                sym = lam1.astype(np.complex128)
            out[i] += b[j, i] * sym.reshape(shapes[j])
        if reading == "literal":
            out[i] += (1j * k[i] * lam0).reshape(shapes[i])
    return out


def ka_matrix(kap: np.ndarray) -> np.ndarray:
    """Per-mode 3x3 K_A = [[0,-K3,K2],[K3,0,-K1],[-K2,K1,0]]  -> (N,N,N,3,3)."""
    k1, k2, k3 = kap
    z = np.zeros_like(k1)
    return np.stack([np.stack([z, -k3, k2], -1), np.stack([k3, z, -k1], -1), np.stack([-k2, k1, z], -1)], -2)


def kb_matrix(kap: np.ndarray) -> np.ndarray:
    """Per-mode 3x3 K_B = [K1^H; K2^H; K3^H][K1 K2 K3]  -> (N,N,N,3,3)."""
    kk = np.moveaxis(kap, 0, -1)
    return np.conj(kk)[..., :, None] * kk[..., None, :]


def _per_mode(mat: np.ndarray, x: np.ndarray) -> np.ndarray:
    return np.einsum("zyxij,...jzyx->...izyx", mat, x)


def gamma_blocks(gamma):
    """gamma as a factor of (N, N, N, 3, 3) per-mode blocks: a scalar as is,
    a per-mode (N, N, N) array with two trailing axes added."""
    g = np.asarray(gamma, dtype=np.float64)
    return g[..., None, None] if g.ndim else float(g)


def f3(u: np.ndarray, explicit: bool = False) -> np.ndarray:
    """F3 applied to every component (last three axes)."""
    n = u.shape[-1]
    if explicit:
        f = dft_matrix(n)
        out = np.einsum("ap,...zyp->...zya", f, u)
        out = np.einsum("ap,...zpx->...zax", f, out)
        return np.einsum("ap,...pyx->...ayx", f, out)
    return np.fft.ifftn(u, axes=(-3, -2, -1)) * n ** 1.5


def f3h(v: np.ndarray, explicit: bool = False) -> np.ndarray:
    """F3^H applied to every component (last three axes)."""
    n = v.shape[-1]
    if explicit:
        fh = np.conj(dft_matrix(n)).T
        out = np.einsum("ap,...zyp->...zya", fh, v)
        out = np.einsum("ap,...zpx->...zax", fh, out)
        return np.einsum("ap,...pyx->...ayx", fh, out)
    return np.fft.fftn(v, axes=(-3, -2, -1)) / n ** 1.5


def apply_definition(x, yee, apply_m, gamma, explicit=False):
    """F3_3^H (A M A^H + gamma B^H B) F3_3 x: the compensated operator in the
    Fourier basis x = F3_3^H H (eq. matrixfree_kcform), built from the
    real-space stencils."""
    return f3h(yee.compensated(f3(x, explicit), apply_m, gamma), explicit)


def apply_symbols(x, kap, apply_m, gamma, explicit=False):
    """K_A F3_3^H M F3_3 K_A^H x + gamma K_B x  (Prop. 2.8 factorisation).
    gamma: a scalar, or per-mode (N, N, N) coefficients gamma_p."""
    ka = ka_matrix(kap)
    kah = np.conj(np.swapaxes(ka, -1, -2))
    u = _per_mode(kah, x)
    w = f3h(apply_m(f3(u, explicit)), explicit)
    return _per_mode(ka, w) + gamma * _per_mode(kb_matrix(kap), x)


def kp_matrix(kap, gamma) -> np.ndarray:
    """Per-mode K_P = K_A K_A^H + gamma K_B (eq. matrixfree_diagP); gamma a
    scalar or per-mode (N, N, N) coefficients."""
    ka = ka_matrix(kap)
    return ka @ np.conj(np.swapaxes(ka, -1, -2)) + gamma_blocks(gamma) * kb_matrix(kap)


def precondition(r, kap, gamma, tiny=0.0):
    """K_P^{-1} r per Fourier mode (eq. matrixfree_finalform), by inverting
    each 3x3 block.  A mode where every symbol vanishes (k = 0, p = 0) maps
    to zero: it is the null space H of Prop. 2.5 and is deflated."""
    kp = kp_matrix(kap, gamma)
    norm2 = np.sum(np.abs(kap) ** 2, axis=0)
    singular = norm2 <= tiny
    kp[singular] = np.eye(3)
    inv = np.linalg.inv(kp)
    inv[singular] = 0.0
    return _per_mode(inv, r)
