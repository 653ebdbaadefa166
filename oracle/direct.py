"""O1: FP64 direct sums (Section 1, eq. usumfree; Section 2, eq. usum).  Test
infrastructure only.  The loops live in csrc/oracle.c (o1_*)."""
from __future__ import annotations

import numpy as np

from ._lib import dptr, f64, iptr, lib
from .se import _kid


def direct(kernel, x, f, q=None, targets=None, xt=None):
    """u_m = sum_{n != m} K(x_m - x_n) . f_n at the targets (indices or points)."""
    kid = _kid(kernel)
    x, f = f64(x), f64(f)
    q = f64(q) if q is not None else None
    if kid == 1 and q is None:
        raise ValueError("stresslet needs q")
    if xt is not None:
        xt = f64(xt)
        nt, tidx = len(xt), None
    else:
        tidx = np.arange(len(x), dtype=np.int64) if targets is None else np.ascontiguousarray(
            np.asarray(targets, dtype=np.int64))
        nt = len(tidx)
    u = np.zeros((nt, 3))
    lib().o1_direct(kid, len(x), dptr(x), dptr(f), dptr(q), nt, iptr(tidx), dptr(xt), dptr(u))
    return u


def grad_x(kernel, x, f, g, q=None, targets=None):
    """d/dx_p of L = sum_m g_m . u_m (exact direct sum)."""
    kid = _kid(kernel)
    x, f, g = f64(x), f64(f), f64(g)
    q = f64(q) if q is not None else None
    tidx = np.arange(len(x), dtype=np.int64) if targets is None else np.ascontiguousarray(
        np.asarray(targets, dtype=np.int64))
    out = np.zeros((len(tidx), 3))
    lib().o1_grad_x(kid, len(x), dptr(x), dptr(f), dptr(q), dptr(g), len(tidx), iptr(tidx),
                    dptr(out))
    return out


def grad_f(kernel, x, g, targets=None):
    """d/df_n of L = sum_m g_m . u_m (stokeslet, rotlet): sum_m K(x_m - x_n)^T g_m."""
    kid = _kid(kernel)
    x, g = f64(x), f64(g)
    tidx = np.arange(len(x), dtype=np.int64) if targets is None else np.ascontiguousarray(
        np.asarray(targets, dtype=np.int64))
    out = np.zeros((len(tidx), 3))
    lib().o1_grad_f(kid, len(x), dptr(x), dptr(g), len(tidx), iptr(tidx), dptr(out))
    return out


def grad_fq(x, f, q, g, targets=None):
    """Stresslet: d/df_n and d/dq_n of L = sum_m g_m . u_m (exact direct sums)."""
    x, f, q, g = f64(x), f64(f), f64(q), f64(g)
    tidx = np.arange(len(x), dtype=np.int64) if targets is None else np.ascontiguousarray(
        np.asarray(targets, dtype=np.int64))
    gf = np.zeros((len(tidx), 3))
    gq = np.zeros((len(tidx), 3))
    lib().o1_grad_fq(len(x), dptr(x), dptr(f), dptr(q), dptr(g), len(tidx), iptr(tidx), dptr(gf), dptr(gq))
    return gf, gq


def kernel_full(kernel, r):
    """K(r) as (n, 3, 3, 3) (S and Omega use [..., 0])."""
    r = f64(np.atleast_2d(r))
    out = np.zeros((len(r), 27))
    lib().o_kernel_full(_kid(kernel), len(r), dptr(r), dptr(out))
    return out.reshape(-1, 3, 3, 3)


def kernel_real(kernel, r, xi):
    """K^R(r, xi) as (n, 3, 3, 3)."""
    r = f64(np.atleast_2d(r))
    out = np.zeros((len(r), 27))
    lib().o_kernel_real(_kid(kernel), len(r), dptr(r), float(xi), dptr(out))
    return out.reshape(-1, 3, 3, 3)


def kernel_real_grad(kernel, r, xi):
    """d/dr_a K^R_jl(r, xi) as (n, 3, 3, 3) indexed [a, j, l] (S and Omega)."""
    r = f64(np.atleast_2d(r))
    out = np.zeros((len(r), 27))
    if lib().o_kernel_real_grad(_kid(kernel), len(r), dptr(r), float(xi), dptr(out)) != 0:
        raise NotImplementedError
    return out.reshape(-1, 3, 3, 3)
