"""Penalty coefficient gamma (oracle; test infrastructure only).

Prop. 2.5 eq. kc_settingofgamma (sufficient choice):
    gamma = max(1, lambda_m^A)                      if k = 0
    gamma = max(1, lambda_m^A) * max(1, |k|^-2)     if k != 0
Remark 2.6 eq. kc_settingofgamma1 (practical rule, valid when
lambda_m^A < 4 pi^2):
    gamma = 4 pi^2            if k = 0 or |k| > 1
    gamma = 4 pi^2 / |k|^2    if 0 < |k| < 1
The printed rule leaves |k| = 1 out; both branches give 4 pi^2 there, which
is the value taken.

Per-mode form (an extension of the rule, not the paper's scalar penalty):
Lemma kc_ABblock gives K_B(p) = conj(kappa_p) kappa_p^T, whose one nonzero
eigenvalue is |kappa_p|^2; the practical rule applied to each mode with that
eigenvalue in place of |k|^2 is
    gamma_p = 4 pi^2 max(1, |kappa_p|^-2),
so every penalty eigenvalue gamma_p |kappa_p|^2 = 4 pi^2 max(1, |kappa_p|^2)
is at least 4 pi^2 (the condition gamma lambda^B >= lambda_m^A of Prop. 2.5,
mode by mode) while the divergence-free eigenpairs do not change.

Projector form (also an extension): gamma_p = gamma / |kappa_p|^2, so that
gamma_p K_B(p) = gamma conj(kappa_p) kappa_p^T / |kappa_p|^2 is gamma times
the orthogonal projector onto conj(kappa_p) and every penalty eigenvalue is
gamma itself.
"""
from __future__ import annotations

import math

import numpy as np


def gamma_practical(k) -> float:
    kn = float(np.linalg.norm(np.asarray(k, dtype=np.float64)))
    four_pi2 = 4.0 * math.pi ** 2
    if kn == 0.0 or kn >= 1.0:
        return four_pi2
    return four_pi2 / kn ** 2


def gamma_sufficient(k, lambda_m: float) -> float:
    kn = float(np.linalg.norm(np.asarray(k, dtype=np.float64)))
    g = max(1.0, lambda_m)
    if kn == 0.0:
        return g
    return g * max(1.0, kn ** -2)


def gamma_per_mode(kap: np.ndarray, scale: float = 4.0 * math.pi ** 2) -> np.ndarray:
    """(N, N, N) per-mode coefficients gamma_p = scale max(1, |kappa_p|^-2)
    for the (3, N, N, N) symbols kap.  A mode with kappa_p = 0 has no penalty
    term (K_B(p) = 0); it gets `scale`."""
    k2 = np.sum(np.abs(kap) ** 2, axis=0)
    g = np.full(k2.shape, float(scale))
    small = (k2 > 0) & (k2 < 1)
    g[small] = scale / k2[small]
    return g


def gamma_projector(kap: np.ndarray, scale: float = 16.0 * math.pi ** 2) -> np.ndarray:
    """(N, N, N) coefficients gamma_p = scale / |kappa_p|^2 of the projector
    form; a mode with kappa_p = 0 (no penalty term) gets `scale`."""
    k2 = np.sum(np.abs(kap) ** 2, axis=0)
    g = np.full(k2.shape, float(scale))
    nz = k2 > 0
    g[nz] = scale / k2[nz]
    return g
