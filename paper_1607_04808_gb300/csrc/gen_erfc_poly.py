"""Generate erfc_poly.cuh: polynomials Q(t) ~ erfcx(x) = exp(x^2) erfc(x) in the
variable t = 1 / (2 + x), so that the FP32 real-space kernel evaluates
erfc(x) = exp(-x^2) Q(t) and shares exp(-x^2) with the Gaussian terms of the
screened kernels (Section 3.2).  Two FP32 fits: degree 8 on x in [0, 5] (enough
for the cutoffs the parameter selection gives at FP32 tolerances) and degree
10 on [0, 8] (beyond 8, erfc(x) < 1e-28); one FP64 fit, degree 18 on [0, 8].  Weighted least squares on Chebyshev nodes
(relative error), with numpy; run this script to regenerate the header.
"""
import os

import numpy as np
from numpy.polynomial import chebyshev as cheb
from scipy.special import erfcx

FITS = [("Q5", 5.0, 8), ("Q8", 8.0, 10)]
# FP64: degree 18 on x in [0, 8], fitted in the Chebyshev basis of the
# shifted variable s = (2 t - (t_max + t_min)) / (t_max - t_min) in [-1, 1] and
# evaluated as a power series in s (coefficients below 0.5: well conditioned)
FIT64 = (8.0, 18)


def fit(xmax, deg):
    tmin, tmax = 1.0 / (2.0 + xmax), 0.5
    k = np.arange(4000)
    tn = 0.5 * (tmax + tmin) + 0.5 * (tmax - tmin) * np.cos(np.pi * (k + 0.5) / len(k))
    x = 1.0 / tn - 2.0
    y = erfcx(x)
    V = np.vander(tn, deg + 1, increasing=True)
    c, *_ = np.linalg.lstsq(V / y[:, None], np.ones_like(y), rcond=None)
    xs = np.linspace(0, xmax, 200001)
    ts = 1.0 / (2.0 + xs)
    err = np.max(np.abs(np.polyval(c[::-1], ts) / erfcx(xs) - 1.0))
    # error after rounding the coefficients and evaluating in float32 (Horner)
    c32 = c.astype(np.float32)
    t32 = ts.astype(np.float32)
    acc = np.zeros_like(t32)
    for cc in c32[::-1]:
        acc = (acc * t32 + cc).astype(np.float32)
    err32 = np.max(np.abs(acc.astype(np.float64) / erfcx(xs) - 1.0))
    return c, err, err32


def fit64(xmax, deg):
    tmin, tmax = 1.0 / (2.0 + xmax), 0.5
    k = np.arange(6000)
    tn = 0.5 * (tmax + tmin) + 0.5 * (tmax - tmin) * np.cos(np.pi * (k + 0.5) / len(k))
    y = erfcx(1.0 / tn - 2.0)
    sn = (2.0 * tn - (tmax + tmin)) / (tmax - tmin)
    c = cheb.cheb2poly(cheb.chebfit(sn, y, deg, w=1.0 / y))
    xs = np.linspace(0, xmax, 400001)
    ss = (2.0 / (2.0 + xs) - (tmax + tmin)) / (tmax - tmin)
    acc = np.zeros_like(ss)
    for cc in c[::-1]:
        acc = acc * ss + cc
    err = np.max(np.abs(acc / erfcx(xs) - 1.0))
    return c, 2.0 / (tmax - tmin), -(tmax + tmin) / (tmax - tmin), err


def main():
    here = os.path.dirname(os.path.abspath(__file__))
    lines = ["// Generated by gen_erfc_poly.py: erfcx(x) ~ sum_k Q[k] t^k, t = 1/(2+x).", "#pragma once"]
    for name, xmax, deg in FITS:
        c, err, err32 = fit(xmax, deg)
        lines += [
            "// x in [0, %g], degree %d: max relative error %.2e (FP64 fit), %.2e (FP32 Horner)."
            % (xmax, deg, err, err32),
            "#define SE_ERFC_DEG%s %d" % (name[1:], deg),
            "__device__ __constant__ const float ERFC_%s[%d] = {" % (name, deg + 1),
        ]
        lines += ["    %.9ef," % v for v in c]
        lines += ["};"]
        print("%s: max rel err fp64 %.3e, fp32 %.3e" % (name, err, err32))
    xmax, deg = FIT64
    c, sa, sb, err = fit64(xmax, deg)
    lines += [
        "// FP64: x in [0, %g], degree %d in s = SA t + SB (t = 1/(2+x)): max relative error %.2e." % (xmax, deg, err),
        "#define SE_ERFC_DEG64 %d" % deg,
        "#define SE_ERFC_XMAX64 %.1f" % xmax,
        "#define SE_ERFC_SA64 %.17e" % sa,
        "#define SE_ERFC_SB64 %.17e" % sb,
        "__device__ __constant__ const double ERFC_QD[%d] = {" % (deg + 1),
    ]
    lines += ["    %.17e," % v for v in c]
    lines += ["};"]
    print("QD: max rel err fp64 %.3e" % err)
    lines.append("")
    open(os.path.join(here, "erfc_poly.cuh"), "w").write("\n".join(lines))


if __name__ == "__main__":
    main()
