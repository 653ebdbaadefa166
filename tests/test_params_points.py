"""se_choose_params_points (host only, no GPU): parameter selection that counts
the neighbours of the actual points.  Uniform points must give the selection
for uniform points; clustered points (more pairs within every radius) must
move to a larger xi, a smaller cutoff and a finer grid with an FFT length
from the fast set; fixed parameters or an FFT cap leave the point-free
selection unchanged."""
from __future__ import annotations

import numpy as np
import pytest

import workloads as W


def pkg():
    from paper_1607_04808_gb300 import _build
    _build.build()
    import paper_1607_04808_gb300 as p
    return p


def in_box32(x, top=1.0):
    return np.minimum(x.astype(np.float32), np.nextafter(np.float32(top), np.float32(0)))


def same(a, b):
    """Equal selections (the point-aware one also gives the real-space cell width)."""
    return all(a[k] == b[k] for k in a)


def fast_fft(n, prec="fp32"):
    """The fast FFT lengths of the selection: 2^a 3^b (at most one 5), a multiple of
    4; FP32 leaves out the powers of two from 32 on (their single-precision
    real-to-complex transforms were measured an order of magnitude less accurate)."""
    if prec == "fp32" and n >= 32 and n & (n - 1) == 0:
        return False
    m, fives = n, 0
    while m % 2 == 0:
        m //= 2
    while m % 3 == 0:
        m //= 3
    while m % 5 == 0:
        m //= 5
        fives += 1
    return m == 1 and fives <= 1 and n % 4 == 0


@pytest.mark.parametrize("kernel,n", [("stokeslet", 200_000), ("stresslet", 100_000), ("rotlet", 50_000)])
def test_uniform_points_keep_the_uniform_choice(kernel, n):
    p = pkg()
    x = in_box32(W.uniform_points(n, 5))
    a = p.choose_params(kernel, n, tol=2e-6)
    b = p.choose_params_points(kernel, x, tol=2e-6)
    mfa, mfb = 2 * (a["M"] + a["P"]), 2 * (b["M"] + b["P"])
    # FP32 real-space cells from the density around the pairs: the mean density here
    w = 1.1 * (8.0 / n) ** (1.0 / 3.0)
    assert abs(b["cell_width"] / w - 1.0) < 0.1
    if fast_fft(mfa):
        assert same(a, b)
    else:
        # the point-aware selection moves to one of the two fast FFT lengths
        # around the uniform choice's
        lo, hi = mfa, mfa
        while not fast_fft(lo):
            lo -= 2
        while not fast_fft(hi):
            hi += 2
        assert mfb in (lo, hi) and b["P"] == a["P"]


def test_clustered_points_move_work_to_the_grid():
    p = pkg()
    n = 200_000
    x = in_box32(W.blob_points(n, 2))
    a = p.choose_params("stresslet", n, tol=2e-6)
    b = p.choose_params_points("stresslet", x, tol=2e-6)
    assert b["xi"] > 1.15 * a["xi"] and b["rc"] < a["rc"] / 1.15 and b["M"] > a["M"]
    assert b["P"] == a["P"] and fast_fft(2 * (b["M"] + b["P"]))
    # cells sized for the density around the pairs, well above the mean density
    assert b["cell_width"] < 0.7 * 1.1 * (8.0 / n) ** (1.0 / 3.0)
    # the same tolerance bookkeeping: xi rc (the real-space error's argument)
    # stays about the same
    assert abs(b["xi"] * b["rc"] - a["xi"] * a["rc"]) < 0.1 * a["xi"] * a["rc"]


def test_dense_sub_box_counts_as_clustered():
    """All points uniform in [0, 1/2)^3 of the unit box: eight times the density
    the box implies, so the selection must move as for clustered points."""
    p = pkg()
    n = 100_000
    x = in_box32(0.5 * W.uniform_points(n, 6))
    a = p.choose_params("stokeslet", n, tol=2e-6)
    b = p.choose_params_points("stokeslet", x, tol=2e-6)
    assert b["xi"] > 1.15 * a["xi"] and b["rc"] < a["rc"]


def test_fixed_parameters_and_caps_are_respected():
    p = pkg()
    n = 100_000
    x = in_box32(W.blob_points(n, 3))
    for kw in ({"max_fft": 256}, {"M": 64}, {"xi": 30.0}):
        assert same(p.choose_params("stokeslet", n, tol=2e-6, **kw), p.choose_params_points("stokeslet", x, tol=2e-6, **kw))


def test_fp64_points_and_boxes():
    p = pkg()
    n = 50_000
    box = (0.0, 0.0, 0.0, 1.0, 0.8, 1.2)
    x = W.uniform_points(n, 7, L=np.array(box[3:]), x0=np.zeros(3))
    b = p.choose_params_points("rotlet", x.astype(np.float64), box=box, tol=1e-10, prec="fp64")
    assert b["M"] > 0 and b["rc"] > 0 and b["xi"] > 0


def test_invalid_arguments():
    p = pkg()
    with pytest.raises(ValueError):
        p.choose_params_points("stokeslet", np.zeros((10, 2), np.float32))
    with pytest.raises(p.SEError) as ei:
        p.choose_params_points("stokeslet", np.zeros((0, 3), np.float32))
    assert ei.value.code == 1
    with pytest.raises(p.SEError) as ei:
        p.choose_params_points("stokeslet", np.zeros((5, 3), np.float32), box=(0, 0, 0, 1.0, 0.0, 1.0))
    assert ei.value.code == 1
