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
