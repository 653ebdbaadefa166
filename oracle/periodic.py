"""O3: the triply periodic sums by plain Ewald summation (FP64, CPU).

TEST INFRASTRUCTURE ONLY (see the package header).

The sum over all periodic images of a cube of side L (Section 1.1: the
periodic problem that the earlier Spectral Ewald method treats), split with
the same screening as the free-space method (Section 3, Table 1: Hasimoto for
the stokeslet and stresslet, Ewald for the rotlet):

    u(x_m) = sum_n sum_{images p} K^R(x_m - x_n + p L)      (0 < |.| <= rc)
           + (1/L^3) sum_{k != 0} A(k) e^{-k^2/4xi^2} . sum_n s_n e^{i k.(x_m - x_n)}
           + u^self_m (stokeslet: -4 xi/sqrt(pi) f_m, eq. Slimit)

with k = 2 pi j / L over integer vectors j != 0.  The k = 0 term is left out:
the mean force is balanced by a uniform pressure gradient (Hasimoto's
convention), so the sum is defined for any net force.  The multipliers A(k)
are those of the free-space method (the module notes of ``oracle.se`` list
the readings: conjugated odd symbols, halved rotlet) with the plain
transforms of the biharmonic and harmonic kernels, Bhat = -8 pi/k^4 and
Hhat = 4 pi/k^2, in place of the truncated ones:

    stokeslet  A_jl  = -(k^2 delta_jl - k_j k_l)(1 + k^2/4xi^2) Bhat
    stresslet  A_jlm = -i[(k_m d_jl + k_j d_lm + k_l d_mj) k^2 - 2 k_j k_l k_m](1 + k^2/4xi^2) Bhat
    rotlet     A_jl  = -i eps_jlm k_m Hhat

The real-space part uses the oracle's screened kernels (the C loop of O2 for a
single displacement) over the 27 neighbouring images, so rc < L is required.
The Fourier sum keeps every j with e^{-k^2/4xi^2} above 1e-17.
"""
from __future__ import annotations

import math

import numpy as np

from . import greens
from ._lib import dptr, f64, lib
from .se import ROTLET, STOKESLET, STRESSLET, _eps, _kid


def sources(kid: int, f: np.ndarray, q: np.ndarray | None) -> np.ndarray:
    """Source components s_n: f_n (3) or, for the stresslet, f_l q_m (9, index 3l + m)."""
    if kid == STRESSLET:
        return (f[:, :, None] * q[:, None, :]).reshape(len(f), 9)
    return f


def multiply(kid: int, k: tuple, S: np.ndarray, xi: float) -> np.ndarray:
    """W_j(k) = A_j..(k) e^{-k^2/4xi^2} S_..(k) for k-vectors k = (kx, ky, kz) (each (nk,)),
    S the structure factors (ncomp, nk); returns (3, nk) complex."""
    k2 = k[0] ** 2 + k[1] ** 2 + k[2] ** 2
    kn = np.sqrt(k2)
    E = greens.gamma_hat_ewald(kn, xi)
    W = np.zeros((3, len(k2)), dtype=np.complex128)
    if kid == STOKESLET:
        hs = (1.0 + k2 / (4.0 * xi**2)) * greens.bhat(kn)
        for j in range(3):
            for l in range(3):
                A = -((k2 if j == l else 0.0) - k[j] * k[l]) * hs
                W[j] += E * A * S[l]
    elif kid == STRESSLET:
        hs = (1.0 + k2 / (4.0 * xi**2)) * greens.bhat(kn)
        for j in range(3):
            for l in range(3):
                for m in range(3):
                    poly = ((k[m] if j == l else 0.0) + (k[j] if l == m else 0.0) +
                            (k[l] if m == j else 0.0)) * k2 - 2.0 * k[j] * k[l] * k[m]
                    W[j] += E * (-1j) * poly * hs * S[3 * l + m]
    elif kid == ROTLET:
        hh = greens.hhat(kn)
        for j in range(3):
            for l in range(3):
                for m in range(3):
                    e = _eps(j, l, m)
                    if e:
                        W[j] += E * (-1j) * e * k[m] * hh * S[l]
    else:
        raise ValueError(kid)
    return W


def fourier_part(kernel, x, f, q, L: float, xi: float, chunk: int = 4096, targets=None) -> np.ndarray:
    """(1/L^3) sum_{k != 0} A(k) e^{-k^2/4xi^2} . sum_n s_n e^{i k.(x_m - x_n)} at the
    targets m (indices into x; default all)."""
    kid = _kid(kernel)
    x, f = f64(x), f64(f)
    xm = x if targets is None else x[np.asarray(targets, dtype=np.int64)]
    s = sources(kid, f, f64(q) if q is not None else None)
    kmax = 2.0 * xi * math.sqrt(math.log(1e17))
    jmax = int(math.ceil(kmax * L / (2.0 * math.pi)))
    r = np.arange(-jmax, jmax + 1)
    J = np.stack(np.meshgrid(r, r, r, indexing="ij"), -1).reshape(-1, 3)
    J = J[np.any(J != 0, axis=1)]
    kk = 2.0 * math.pi / L * J.astype(np.float64)
    kk = kk[np.einsum("ij,ij->i", kk, kk) <= kmax * kmax]
    u = np.zeros((len(xm), 3))
    for c0 in range(0, len(kk), chunk):
        kc = kk[c0:c0 + chunk]
        ph = np.exp(-1j * (x @ kc.T))                     # (N, nk): e^{-i k.x_n}
        S = s.T @ ph                                      # (ncomp, nk)
        W = multiply(kid, (kc[:, 0], kc[:, 1], kc[:, 2]), S, xi)
        pm = ph if targets is None else np.exp(-1j * (xm @ kc.T))
        u += np.real(np.conj(pm) @ W.T)                   # sum_k W(k) e^{i k.x_m}
    return u / L**3


def real_part(kernel, x, f, q, L: float, xi: float, rc: float, targets=None) -> np.ndarray:
    """Sum over all images within rc of the screened kernel K^R (Section 6), n = m
    excluded for the unshifted image, at the targets m (indices; default all)."""
    kid = _kid(kernel)
    if not rc < L:
        raise ValueError("rc must be below L")
    x, f = f64(x), f64(f)
    q = f64(q) if q is not None else None
    N = len(x)
    tid = np.arange(N) if targets is None else np.asarray(targets, dtype=np.int64)
    u = np.zeros((len(tid), 3))
    mi, ni = np.meshgrid(np.arange(len(tid)), np.arange(N), indexing="ij")
    mi, ni = mi.ravel(), ni.ravel()
    base = x[tid[mi]] - x[ni]
    for sx in (-1, 0, 1):
        for sy in (-1, 0, 1):
            for sz in (-1, 0, 1):
                r = base + L * np.array([sx, sy, sz], dtype=np.float64)
                r2 = np.einsum("ij,ij->i", r, r)
                keep = (r2 <= rc * rc) & (r2 > 0.0)
                if sx == 0 and sy == 0 and sz == 0:
                    keep &= tid[mi] != ni
                if not keep.any():
                    continue
                rk = np.ascontiguousarray(r[keep])
                G = np.zeros((len(rk), 27))
                lib().o_kernel_real(kid, len(rk), dptr(rk), xi, dptr(G))
                G = G.reshape(-1, 3, 3, 3)
                n = ni[keep]
                if kid == STRESSLET:
                    v = np.einsum("pjlm,pl,pm->pj", G, f[n], q[n])
                else:
                    v = np.einsum("pjl,pl->pj", G[:, :, :, 0], f[n])
                np.add.at(u, mi[keep], v)
    return u


def ewald(kernel, x, f, q=None, *, L: float = 1.0, xi: float, rc: float, parts: bool = False, targets=None):
    """The periodic sum at every point (or at the points with indices ``targets``):
    real-space + Fourier + self parts."""
    kid = _kid(kernel)
    uR = real_part(kid, x, f, q, L, xi, rc, targets=targets)
    uF = fourier_part(kid, x, f, q, L, xi, targets=targets)
    fm = f64(f) if targets is None else f64(f)[np.asarray(targets, dtype=np.int64)]
    uS = greens.self_coefficient(kid, xi) * fm if kid == STOKESLET else np.zeros_like(uF)
    if parts:
        return {"R": uR, "F": uF, "self": uS}
    return uR + uF + uS
