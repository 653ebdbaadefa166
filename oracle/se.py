"""O2: the plain FP64 CPU Spectral Ewald evaluation.  Test infrastructure only.

The steps follow the paper's order (Section 8 summary; Section 5.2 steps 1-5;
Section 4.3 precomputation), each written out without blocking or fusion:

  0. parameters  h = L/M, d = hP, m = C sqrt(pi P) (C = 0.976),
                 eta = (xi d / m)^2, delta_L (eq. deltaL_cond or delta_L = d),
                 Mt = M + delta_L/h, grid y_i = x0 - delta_L/2 + i h    (Sections 5.2-5.3)
  1. precompute  truncated Green's function on an oversampled Mg^3 grid,
                 inverse FFT, keep the 2 Mt values per dimension centred at
                 zero, forward FFT of size (2 Mt)^3                     (Section 4.3)
  2. spreading   eq. Hx over the P^3 block of each point                 (step 1)
  3. FFT         zero-padded to (2 Mt)^3                                (step 2)
  4. scaling     eq. gridfcnsc with A^{K,R}                              (step 3)
  5. IFFT        normalised, keep the Mt^3 octant                       (step 4)
  6. quadrature  eq. u_integr, trapezoidal weight h^3                    (step 5)
  7. real space  sum over 0 < |r| <= rc (every pair's distance checked)  (Section 6)
  8. self term   -4 xi/sqrt(pi) f_m, stokeslet only                      (eq. Slimit)

Readings of the paper taken here (each listed with its reason in the design notes):
  * Rotlet: the definition eps_jlm r_m / r^3 (eq. def_rotlet) is computed; the
    operator form (eq. rotlet_op), eq. RR_Op and eq. AR carry an extra factor 2
    and are halved.
  * Odd symbols (stresslet, rotlet): the Fourier multiplier is the transform of
    the kernel under the stated convention f^(k) = int f e^{-ik.x}, i.e. the
    operator with d/dx_m -> +i k_m; this is the complex conjugate of the printed
    eqs. AT and AR (which apply the operator to e^{-ik.x}).
  * Stresslet real space: delta-term coefficient (4 xi^3 r / sqrt(pi)) e^{-xi^2 r^2}.
  * Truncated Green's function: R = sqrt(3) * Ltilde; Mg = smallest even integer
    greater than (1 + sqrt(3)) Mt (Section 9).
"""
from __future__ import annotations

import math
from dataclasses import dataclass, field

import numpy as np
import scipy.fft as sfft

from . import greens
from ._lib import dptr, f64, iptr, lib

STOKESLET, STRESSLET, ROTLET = 0, 1, 2
KERNEL_IDS = {"stokeslet": STOKESLET, "stresslet": STRESSLET, "rotlet": ROTLET}
C_SHAPE = 0.976  # shape constant of m(P) = C sqrt(pi P) (Section 5.3)


def _kid(kernel) -> int:
    return KERNEL_IDS[kernel] if isinstance(kernel, str) else int(kernel)


@dataclass
class SEParams:
    """Parameters of one evaluation and the quantities derived from them."""
    L: float
    M: int
    P: int
    xi: float
    rc: float
    x0: tuple = (0.0, 0.0, 0.0)
    deltaL_policy: str = "d"
    h: float = field(init=False)
    d: float = field(init=False)
    m: float = field(init=False)
    eta: float = field(init=False)
    n_ext: int = field(init=False)
    deltaL: float = field(init=False)
    Mt: int = field(init=False)
    Mf: int = field(init=False)
    Ltilde: float = field(init=False)
    R: float = field(init=False)
    Mg: int = field(init=False)
    y0: np.ndarray = field(init=False)

    def __post_init__(self):
        self.h = self.L / self.M
        self.d = self.h * self.P
        self.m = C_SHAPE * math.sqrt(math.pi * self.P)
        self.eta = (self.xi * self.d / self.m) ** 2
        if self.deltaL_policy == "d":
            need = self.d
        elif self.deltaL_policy == "strict":
            # eq. deltaL_cond
            need = self.d if self.eta >= 1.0 else max(
                self.d, math.sqrt(2.0 * (1.0 - self.eta) * self.m**2 / self.xi**2))
        else:
            raise ValueError(self.deltaL_policy)
        self.n_ext = int(math.ceil(need / self.h - 1e-9))
        self.deltaL = self.n_ext * self.h
        self.Mt = self.M + self.n_ext
        self.Mf = 2 * self.Mt
        self.Ltilde = self.Mt * self.h
        self.R = math.sqrt(3.0) * self.Ltilde
        self.Mg = 2 * int(math.floor((1.0 + math.sqrt(3.0)) * self.Mt / 2.0)) + 2
        self.y0 = np.asarray(self.x0, dtype=np.float64) - self.deltaL / 2.0


def precompute_ghat(kind: str, p: SEParams) -> np.ndarray:
    """Section 4.3: the mollified truncated Green's function on the (2 Mt)^3 grid.

    kind 'B' (biharmonic, stokeslet and stresslet) or 'H' (harmonic, rotlet).
    Returns the complex FFT (real up to rounding), shape (Mf, Mf, Mf).
    """
    Mg, Mt, Mf, h = p.Mg, p.Mt, p.Mf, p.h
    kbar = sfft.fftfreq(Mg, 1.0 / Mg)  # integers in [-Mg/2, Mg/2 - 1]
    k1 = 2.0 * np.pi * kbar / (Mg * h)
    kk = np.sqrt(k1[:, None, None] ** 2 + k1[None, :, None] ** 2 + k1[None, None, :] ** 2)
    if kind == "B":
        gk = greens.bhat_trunc(kk, p.R)
    elif kind == "H":
        gk = greens.hhat_trunc(kk, p.R)
    else:
        raise ValueError(kind)
    del kk
    G = sfft.ifftn(gk, workers=-1)  # normalised by 1/Mg^3
    del gk
    # keep j in [-Mt, Mt-1] per dimension, stored wrap-ordered on the Mf grid
    j = np.arange(-Mt, Mt)
    src, dst = j % Mg, j % Mf
    Gt = np.zeros((Mf, Mf, Mf), dtype=np.complex128)
    Gt[np.ix_(dst, dst, dst)] = G[np.ix_(src, src, src)]
    del G
    return sfft.fftn(Gt, workers=-1)


def source_components(kernel: int, f: np.ndarray, q: np.ndarray | None) -> np.ndarray:
    """Per-point quantities that are spread: f (3 comps) or f_l q_m (9 comps, Section 9)."""
    if kernel == STRESSLET:
        return np.einsum("nl,nm->nlm", f, q).reshape(len(f), 9)
    return f.copy()


def spread(x: np.ndarray, src: np.ndarray, p: SEParams) -> np.ndarray:
    """Step 1 (eq. Hx): grid[c, iz, iy, ix] on the Mt^3 extended grid."""
    L = lib()
    x, src = f64(x), f64(src)
    nc = src.shape[1]
    grid = np.zeros((nc, p.Mt, p.Mt, p.Mt), dtype=np.float64)
    rc = L.o2_spread(len(x), dptr(x), nc, dptr(src), p.Mt, p.P, p.h, dptr(f64(p.y0)), p.xi,
                     p.eta, dptr(grid))
    if rc != 0:
        raise ValueError("a Gaussian support leaves the extended grid (point outside the box)")
    return grid


def gather(w: np.ndarray, xt: np.ndarray, p: SEParams) -> np.ndarray:
    """Step 5 (eq. u_integr): h^3 * sum_i w_i Gauss(x_t - y_i) for each target."""
    L = lib()
    xt = f64(xt)
    w = f64(w)
    nc = w.shape[0]
    out = np.zeros((len(xt), nc), dtype=np.float64)
    rc = L.o2_gather(len(xt), dptr(xt), nc, dptr(w), p.Mt, p.P, p.h, dptr(f64(p.y0)), p.xi,
                     p.eta, dptr(out))
    if rc != 0:
        raise ValueError("a target's Gaussian support leaves the extended grid")
    return out * p.h**3


def _kgrid(p: SEParams):
    kbar = sfft.fftfreq(p.Mf, 1.0 / p.Mf)  # [-Mt, Mt-1]; index Mt holds -Mt
    k1 = 2.0 * np.pi * kbar / (p.Mf * p.h)
    # grid arrays are indexed [z, y, x]
    kz = k1[:, None, None]
    ky = k1[None, :, None]
    kx = k1[None, None, :]
    return (kx, ky, kz)


def _eps(j, l, m):
    return int(np.sign((l - j) * (m - l) * (m - j)))


def scale(kernel: int, Ghat: np.ndarray, G: np.ndarray, p: SEParams, transpose: bool = False):
    """Step 3 (eq. gridfcnsc): W_j(k) = e^{-(1-eta) k^2 / 4 xi^2} sum A_j..(k) G_..(k).

    Multipliers (with B^R, H^R replaced by the precomputed Ghat):
      stokeslet  A_jl  = -(k^2 delta_jl - k_j k_l)(1 + k^2/4xi^2) B^R          (eq. AS)
      stresslet  A_jlm = -i[(k_m d_jl + k_j d_lm + k_l d_mj) k^2 - 2 k_j k_l k_m](1 + k^2/4xi^2) B^R
      rotlet     A_jl  = -i eps_jlm k_m H^R
    (odd symbols: conjugate of the printed eqs. AT, AR; rotlet halved, see module notes.)
    ``transpose`` applies A'_lj(k) = A_jl(-k), the multiplier of the transposed
    convolution (used by the gradient).
    """
    k = _kgrid(p)
    if transpose:
        k = tuple(-kc for kc in k)
    k2 = k[0] ** 2 + k[1] ** 2 + k[2] ** 2
    E = np.exp(-(1.0 - p.eta) * k2 / (4.0 * p.xi**2))
    W = np.zeros((3,) + G.shape[1:], dtype=np.complex128)
    if kernel == STOKESLET:
        hs = (1.0 + k2 / (4.0 * p.xi**2)) * Ghat
        for j in range(3):
            for l in range(3):
                A = -((k2 if j == l else 0.0) - k[j] * k[l]) * hs
                if transpose:
                    W[l] += E * A * G[j]
                else:
                    W[j] += E * A * G[l]
    elif kernel == STRESSLET:
        if transpose:
            raise NotImplementedError("stresslet transpose")
        hs = (1.0 + k2 / (4.0 * p.xi**2)) * Ghat
        for j in range(3):
            for l in range(3):
                for m in range(3):
                    poly = ((k[m] if j == l else 0.0) + (k[j] if l == m else 0.0) +
                            (k[l] if m == j else 0.0)) * k2 - 2.0 * k[j] * k[l] * k[m]
                    A = -1j * poly * hs
                    W[j] += E * A * G[3 * l + m]
    elif kernel == ROTLET:
        for j in range(3):
            for l in range(3):
                for m in range(3):
                    e = _eps(j, l, m)
                    if e == 0:
                        continue
                    A = -1j * e * k[m] * Ghat
                    if transpose:
                        W[l] += E * A * G[j]
                    else:
                        W[j] += E * A * G[l]
    else:
        raise ValueError(kernel)
    return W


def fourier_grid(kernel: int, src: np.ndarray, x: np.ndarray, p: SEParams, Ghat=None,
                 transpose: bool = False):
    """Steps 1-4: the scaled grid w (3, Mt, Mt, Mt) for the given sources."""
    if Ghat is None:
        Ghat = precompute_ghat("H" if kernel == ROTLET else "B", p)
    g = spread(x, src, p)
    G = sfft.fftn(g, s=(p.Mf, p.Mf, p.Mf), axes=(1, 2, 3), workers=-1)
    del g
    W = scale(kernel, Ghat, G, p, transpose=transpose)
    del G
    w = sfft.ifftn(W, axes=(1, 2, 3), workers=-1)
    del W
    return np.ascontiguousarray(w.real[:, : p.Mt, : p.Mt, : p.Mt])


def real_space(kernel: int, x, f, q, p: SEParams, targets=None, xt=None):
    """Section 6: screened real-space sum with every pair's distance checked."""
    L = lib()
    x, f = f64(x), f64(f)
    q = f64(q) if q is not None else None
    if xt is not None:
        xt = f64(xt)
        nt, tidx = len(xt), None
    else:
        tidx = np.arange(len(x), dtype=np.int64) if targets is None else np.ascontiguousarray(
            np.asarray(targets, dtype=np.int64))
        nt = len(tidx)
    u = np.zeros((nt, 3), dtype=np.float64)
    L.o2_real(kernel, len(x), dptr(x), dptr(f), dptr(q), nt, iptr(tidx), dptr(xt), p.xi, p.rc,
              dptr(u))
    return u


def se_eval(kernel, x, f, q=None, *, L=1.0, x0=(0.0, 0.0, 0.0), M, P, xi, rc,
            deltaL_policy="d", targets=None, xt=None, parts=False, Ghat=None):
    """u(x_m) = u^F + u^R + u^self (Section 8) at the targets.

    ``targets``: indices of sources used as targets (the n = m term excluded);
    default all.  ``xt``: arbitrary target points instead (nothing excluded,
    no self term).
    """
    kid = _kid(kernel)
    x = f64(x)
    f = f64(f)
    q = f64(q) if q is not None else None
    p = SEParams(L=L, M=M, P=P, xi=xi, rc=rc, x0=tuple(x0), deltaL_policy=deltaL_policy)
    src = source_components(kid, f, q)
    w = fourier_grid(kid, src, x, p, Ghat=Ghat)
    if xt is not None:
        xq = f64(xt)
    else:
        tidx = np.arange(len(x)) if targets is None else np.asarray(targets, dtype=np.int64)
        xq = x[tidx]
    uF = gather(w, xq, p)
    uR = real_space(kid, x, f, q, p, targets=targets, xt=xt)
    if xt is None and kid == STOKESLET:
        fm = f if targets is None else f[np.asarray(targets, dtype=np.int64)]
        uS = greens.self_coefficient(kid, xi) * fm
    else:
        uS = np.zeros_like(uF)
    if parts:
        return {"F": uF, "R": uR, "self": uS, "params": p}
    return uF + uR + uS


def se_grad(kernel, x, f, g, *, L=1.0, x0=(0.0, 0.0, 0.0), M, P, xi, rc, deltaL_policy="d",
            targets=None):
    """Gradients of the SE approximation of  L = sum_m g_m . u_m  (stokeslet, rotlet).

    grad_f: the SE operator applied to g with the transposed multiplier
            (A'_lj(k) = A_jl(-k); transposed real-space kernel G_jl(-r)).
    grad_x: h^3 sum_i [g_p . w_i + f_p . w'_i] grad Gauss(x_p - y_i)   (w from f,
            w' from g with the transposed multiplier), plus the real-space
            derivative  sum_{0<|r|<=rc} [g_p . dG^R(x_p - x_n) f_n - g_n . dG^R(x_n - x_p) f_p].
    The self term does not depend on x.
    """
    kid = _kid(kernel)
    if kid == STRESSLET:
        raise NotImplementedError
    Lb = lib()
    x, f, g = f64(x), f64(f), f64(g)
    p = SEParams(L=L, M=M, P=P, xi=xi, rc=rc, x0=tuple(x0), deltaL_policy=deltaL_policy)
    Ghat = precompute_ghat("H" if kid == ROTLET else "B", p)
    tidx = np.arange(len(x), dtype=np.int64) if targets is None else np.ascontiguousarray(
        np.asarray(targets, dtype=np.int64))
    # grad_f: transposed operator applied to g
    wT = fourier_grid(kid, g, x, p, Ghat=Ghat, transpose=True)
    gfF = gather(wT, x[tidx], p)
    # transposed real-space kernel: sum_m G^R_jl(x_m - x_n) g_mj
    gfR = np.zeros((len(tidx), 3))
    Lb.o2_real_T(kid, len(x), dptr(x), dptr(g), len(tidx), iptr(tidx), xi, rc, dptr(gfR))
    gfS = greens.self_coefficient(kid, xi) * g[tidx]
    grad_f = gfF + gfR + gfS
    # grad_x
    w = fourier_grid(kid, f, x, p, Ghat=Ghat)
    xt = np.ascontiguousarray(x[tidx])
    coefA = np.ascontiguousarray(g[tidx])
    coefB = np.ascontiguousarray(f[tidx])
    out = np.zeros((len(tidx), 3))
    rc_ = Lb.o2_gather_grad(len(tidx), dptr(xt), 3, dptr(coefA), dptr(f64(w)), dptr(coefB),
                            dptr(f64(wT)), p.Mt, p.P, p.h, dptr(f64(p.y0)), p.xi, p.eta, dptr(out))
    if rc_ != 0:
        raise ValueError("target outside the grid")
    gxF = out * p.h**3
    gxR = np.zeros((len(tidx), 3))
    Lb.o2_real_grad_x(kid, len(x), dptr(x), dptr(f), dptr(g), len(tidx), iptr(tidx), xi, rc,
                      dptr(gxR))
    return grad_f, gxF + gxR
