"""Closed forms of the oracle (FP64, numpy).  Test infrastructure only.

* Fourier transforms of the harmonic (H = 1/r) and biharmonic (B = r) Green's
  functions, plain (Section 3.2, eq. def_harm_biharm) and truncated at radius R
  (Section 4, eqs. HhatR and BhatR) with their k -> 0 limits.
* Screening functions in Fourier space (Section 3.1, Table 1).
* Self-interaction limit (Section 1.1, eq. Slimit).
"""
from __future__ import annotations

import math

import numpy as np

SQRT_PI = math.sqrt(math.pi)


def hhat(k):
    """Fourier transform of 1/r: 4 pi / k^2 (eq. def_harm_biharm)."""
    k = np.asarray(k, dtype=np.float64)
    return 4.0 * np.pi / k**2


def bhat(k):
    """Fourier transform of r: -8 pi / k^4 (eq. def_harm_biharm)."""
    k = np.asarray(k, dtype=np.float64)
    return -8.0 * np.pi / k**4


def hhat_trunc(k, R):
    """Truncated harmonic kernel 8 pi (sin(R k / 2) / k)^2, limit 2 pi R^2 at k = 0 (eq. HhatR)."""
    k = np.asarray(k, dtype=np.float64)
    out = np.empty_like(k)
    z = k == 0.0
    kk = k[~z]
    out[~z] = 8.0 * np.pi * (np.sin(R * kk / 2.0) / kk) ** 2
    out[z] = 2.0 * np.pi * R**2
    return out


def bhat_trunc(k, R, series_below: float = 1.0):
    """Truncated biharmonic kernel (eq. BhatR)

        4 pi [ (2 - R^2 k^2) cos(R k) + 2 R k sin(R k) - 2 ] / k^4,

    limit pi R^4 at k = 0.  For R k below ``series_below`` the numerator
    cancels to O((Rk)^4); there the Taylor series of the same quantity,
    (4 pi / k) int_0^R r^2 sin(k r) dr = 4 pi sum_n (-1)^n k^{2n} R^{2n+4} / ((2n+1)! (2n+4)),
    is used instead.
    """
    k = np.asarray(k, dtype=np.float64)
    out = np.empty_like(k)
    x = R * k
    small = x < series_below
    kk = k[~small]
    xx = x[~small]
    out[~small] = 4.0 * np.pi * ((2.0 - xx**2) * np.cos(xx) + 2.0 * xx * np.sin(xx) - 2.0) / kk**4
    ks = k[small]
    s = np.zeros_like(ks)
    for n in range(12):
        s += (-1.0) ** n * ks ** (2 * n) * R ** (2 * n + 4) / (math.factorial(2 * n + 1) * (2 * n + 4))
    out[small] = 4.0 * np.pi * s
    return out


def gamma_hat_ewald(k, xi):
    """Ewald screening in Fourier space: exp(-k^2 / 4 xi^2) (Table 1)."""
    k = np.asarray(k, dtype=np.float64)
    return np.exp(-k**2 / (4.0 * xi**2))


def gamma_hat_hasimoto(k, xi):
    """Hasimoto screening in Fourier space: exp(-k^2/4xi^2)(1 + k^2/4xi^2) (eq. hasimoto)."""
    k = np.asarray(k, dtype=np.float64)
    return np.exp(-k**2 / (4.0 * xi**2)) * (1.0 + k**2 / (4.0 * xi**2))


def self_coefficient(kernel: int, xi: float) -> float:
    """lim_{r->0} (K^R - K): -4 xi / sqrt(pi) times the identity for the stokeslet
    (eq. Slimit), zero for the stresslet and rotlet (Section 3.2)."""
    return -4.0 * xi / SQRT_PI if kernel == 0 else 0.0
