"""Generate erfc_poly.cuh: a polynomial Q(t) ~ erfcx(x) = exp(x^2) erfc(x) in the
variable t = 2 / (2 + x) for x in [0, X_MAX], so that the FP32 real-space kernel
evaluates erfc(x) = exp(-x^2) Q(t) and shares exp(-x^2) with the Gaussian term of
the screened kernels (Section 3.2).  The coefficients are a weighted
least-squares fit on Chebyshev nodes (relative error), computed here with
numpy/scipy; run this script to regenerate the header.
"""
import os

import numpy as np
from scipy.special import erfcx

X_MAX = 8.0
DEG = 10


def fit():
    tmin = 2.0 / (2.0 + X_MAX)
    k = np.arange(4000)
    tn = 0.5 * (1 + tmin) + 0.5 * (1 - tmin) * np.cos(np.pi * (k + 0.5) / len(k))
    x = 2.0 / tn - 2.0
    y = erfcx(x)
    V = np.vander(tn, DEG + 1, increasing=True)
    c, *_ = np.linalg.lstsq(V / y[:, None], np.ones_like(y), rcond=None)
    xs = np.linspace(0, X_MAX, 200001)
    ts = 2.0 / (2.0 + xs)
    approx = np.polyval(c[::-1], ts)
    err = np.max(np.abs(approx / erfcx(xs) - 1.0))
    # error after rounding the coefficients and evaluating in float32 (Horner)
    c32 = c.astype(np.float32)
    t32 = ts.astype(np.float32)
    acc = np.zeros_like(t32)
    for cc in c32[::-1]:
        acc = (acc * t32 + cc).astype(np.float32)
    err32 = np.max(np.abs(acc.astype(np.float64) / erfcx(xs) - 1.0))
    return c, err, err32


def main():
    c, err, err32 = fit()
    here = os.path.dirname(os.path.abspath(__file__))
    lines = [
        "// Generated by gen_erfc_poly.py: erfcx(x) ~ sum_k ERFC_Q[k] t^k, t = 2/(2+x), x in [0, %g]." % X_MAX,
        "// Max relative error of the fit %.2e (FP64), %.2e (FP32 Horner)." % (err, err32),
        "#pragma once",
        "#define SE_ERFC_XMAX %.1ff" % X_MAX,
        "#define SE_ERFC_DEG %d" % DEG,
        "__device__ __constant__ const float ERFC_Q[%d] = {" % (DEG + 1),
    ]
    lines += ["    %.9ef," % v for v in c]
    lines += ["};", ""]
    open(os.path.join(here, "erfc_poly.cuh"), "w").write("\n".join(lines))
    print("max rel err fp64 %.3e, fp32 %.3e" % (err, err32))


if __name__ == "__main__":
    main()
