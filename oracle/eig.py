"""Eigenvalues of the compensated operator (oracle; test infrastructure only).

* ``dense_matrix``: the operator assembled column by column (small N only);
  its spectrum by LAPACK (numpy.linalg.eigvalsh).
* ``homogeneous_spectrum``: for a medium with one constant inverse
  permittivity P, F3_3^H M F3_3 = P on every mode, so the Fourier-basis
  operator is block diagonal with the 3x3 blocks
      H_p = K_A(p) P K_A(p)^H + gamma K_B(p)
  (Prop. 2.8, eq. matrixfree_kcform); its spectrum is the union of the block
  spectra.
* ``lobpcg``: textbook LOBPCG with soft locking (Sec. 4; Knyazev, SIAM J.
  Sci. Comput. 23 (2001) 517-541): Rayleigh-Ritz on span{X, W, P} with
  W = T R, R = A X - X Theta.  Converged columns stay in X and in the
  Rayleigh-Ritz step but get no new W or P columns.  Convergence test:
  Res_j = ||A x_j - theta_j x_j|| / ||x_j|| <= tol (Sec. 4,
  eq. exp_relativeresidual).
"""
from __future__ import annotations

import numpy as np
import scipy.linalg

from . import fourier


def dense_matrix(apply, dim: int, batch: int = 256) -> np.ndarray:
    """Dense matrix of a linear map on C^dim given as apply(block of columns)."""
    cols = []
    eye = np.eye(dim, dtype=np.complex128)
    for s in range(0, dim, batch):
        cols.append(apply(eye[s:s + batch]))
    return np.concatenate(cols, axis=0).T


def homogeneous_spectrum(kap: np.ndarray, inv_eps: np.ndarray, gamma) -> np.ndarray:
    """Sorted spectrum of the Fourier-basis operator for a homogeneous medium
    (gamma a scalar or per-mode (N, N, N) coefficients)."""
    ka = fourier.ka_matrix(kap)
    hp = ka @ inv_eps @ np.conj(np.swapaxes(ka, -1, -2)) + fourier.gamma_blocks(gamma) * fourier.kb_matrix(kap)
    return np.sort(np.linalg.eigvalsh(hp).ravel())


def _as_cols(x):
    return x.reshape(x.shape[0], -1).T


def _as_fields(c, shape):
    return c.T.reshape((c.shape[1],) + shape)


def lobpcg(apply, precond, x0, nev, tol=1e-10, maxit=1000, deflate=False, history=None):
    """LOBPCG with soft locking on blocks of fields of shape (n, 3, N, N, N).

    apply, precond: maps on such blocks.  deflate: zero the p = 0 mode of
    every search direction (k = 0, null space of Prop. 2.5).
    Returns (theta[:nev], X[:nev], residuals[:nev], iterations).
    """
    shape = x0.shape[1:]
    nblk = x0.shape[0]

    def defl(v):
        if deflate:
            v = v.copy()
            v[:, :, 0, 0, 0] = 0.0
        return v

    x = _as_cols(defl(x0))
    x, _ = np.linalg.qr(x)
    ax = _as_cols(apply(_as_fields(x, shape)))
    g = x.conj().T @ ax
    theta, c = scipy.linalg.eigh(0.5 * (g + g.conj().T))
    x, ax = x @ c, ax @ c
    p = ap = None
    res = None
    for it in range(1, maxit + 1):
        r = ax - x * theta
        res = np.linalg.norm(r, axis=0) / np.linalg.norm(x, axis=0)
        if history is not None:
            history.append(res[:nev].copy())
        if np.all(res[:nev] <= tol):
            return theta[:nev], _as_fields(x[:, :nev], shape), res[:nev], it - 1
        active = res > tol
        w = _as_cols(defl(precond(_as_fields(r[:, active], shape))))
        w = w - x @ (x.conj().T @ w)
        w, _ = np.linalg.qr(w)
        aw = _as_cols(apply(_as_fields(w, shape)))
        for use_p in (True, False):
            if use_p and p is not None:
                s = np.concatenate([x, w, p], axis=1)
                a_s = np.concatenate([ax, aw, ap], axis=1)
            else:
                s = np.concatenate([x, w], axis=1)
                a_s = np.concatenate([ax, aw], axis=1)
            ga = s.conj().T @ a_s
            gb = s.conj().T @ s
            if use_p and p is not None:
                # P nearly inside span[X W]: the Rayleigh-Ritz step would
                # amplify the rounding of ga by 1 / lambda_min of the scaled
                # gb; restart without P instead
                d = 1 / np.sqrt(np.diag(gb).real)
                lam = np.linalg.eigvalsh(0.5 * (gb + gb.conj().T) * d[:, None] * d[None, :])
                if lam[0] < 1e-12 * lam[-1]:
                    continue
            try:
                th, c = scipy.linalg.eigh(0.5 * (ga + ga.conj().T), 0.5 * (gb + gb.conj().T))
                break
            except np.linalg.LinAlgError:
                if not use_p or p is None:
                    raise
        theta = th[:nblk]
        c = c[:, :nblk]
        x_new = s @ c
        ax_new = a_s @ c
        # P: the part of the new Ritz vectors outside span(X), for active columns
        p_full = s[:, nblk:] @ c[nblk:, :]
        ap_full = a_s[:, nblk:] @ c[nblk:, :]
        nrm = np.linalg.norm(x_new, axis=0)
        x, ax = x_new / nrm, ax_new / nrm
        p, ap = p_full / nrm, ap_full / nrm
        r_next = ax - x * theta
        act = np.linalg.norm(r_next, axis=0) > tol
        p, ap = p[:, act], ap[:, act]
        if p.shape[1] == 0:
            p = ap = None
    return theta[:nev], _as_fields(x[:, :nev], shape), res[:nev], maxit
