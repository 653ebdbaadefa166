"""Truncation-error estimates of Section 7 (Tables 2 and 3).  Test infrastructure only.

All are absolute RMS errors  sqrt(1/N sum |Delta u|^2)  for N sources in a cube
of side L.  Q is sum |f|^2 (stokeslet, rotlet) or sum_n sum_lm f_l^2 q_m^2
(stresslet; the table's "q_l^2 n_m^2" with the source named f q here).
k_inf = pi / h = pi M / L (Section 7.1; k_inf = pi Mt / Ltilde with the same h).
R = sqrt(3) Ltilde.
"""
from __future__ import annotations

import math

import numpy as np


def q_sum(kernel: int, f, q=None) -> float:
    f = np.asarray(f, dtype=np.float64)
    if kernel == 1:
        q = np.asarray(q, dtype=np.float64)
        return float(np.sum(np.sum(f**2, axis=1) * np.sum(q**2, axis=1)))
    return float(np.sum(f**2))


def fourier_error(kernel: int, Q: float, xi: float, L: float, M: int, R: float) -> float:
    """Table 2 (est_fourier)."""
    kinf = math.pi * M / L
    ex = math.exp(-kinf**2 / (4.0 * xi**2))
    if kernel == 0:
        return math.sqrt(Q) * R * kinf**3 / (xi**2 * math.pi * L) * ex
    if kernel == 1:
        return math.sqrt(7.0 * Q / 6.0) * R * kinf**4 / (xi**2 * math.pi * L) * ex
    return math.sqrt(8.0 * xi**2 * Q / (3.0 * math.pi * L**3 * kinf)) * ex


def real_error(kernel: int, Q: float, xi: float, L: float, rc: float) -> float:
    """Table 3 (est_real)."""
    ex = math.exp(-xi**2 * rc**2)
    if kernel == 0:
        return math.sqrt(4.0 * Q * rc / L**3) * ex
    if kernel == 1:
        return math.sqrt(112.0 * Q * xi**4 * rc**3 / (9.0 * L**3)) * ex
    return math.sqrt(8.0 * Q / (3.0 * L**3 * rc)) * ex
