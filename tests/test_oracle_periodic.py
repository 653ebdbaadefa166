"""Pins of the periodic oracle O3 (plain Ewald summation) to facts that do not
come from the oracle itself:

* Hasimoto's result for a simple cubic array of point forces: the velocity a
  point force F induces at its own position through its periodic images is
  -2.837297 F / (6 pi mu L) (Hasimoto 1959).  With the kernel normalised as
  S = I/r + r r^T/r^3 (u = S f stands for 8 pi mu times the velocity) this is
  u = -(4/3) 2.8372975 f / L, isotropic, independent of the position and of xi.
* The Ewald split is exact: the sum does not depend on xi (the real-space and
  Fourier parts change by orders of magnitude more than their sum).
* Translation of all points (wrapped into the box) changes nothing.
* Cubic symmetry: the odd kernels (stresslet, rotlet) give zero for one point.
* Large boxes: for a fixed cloud, the difference from the free-space direct
  sum O1 falls like 1/L for the stokeslet (the images' far field of a net
  force) and like 1/L^3 for the stresslet and rotlet.
A planted mistake in the Fourier multipliers fails at least one of these.
"""
from __future__ import annotations

import numpy as np
import pytest

import workloads as W
from oracle import direct
from oracle import periodic as O3

HASIMOTO = 2.8372975  # simple cubic array, leading coefficient (Hasimoto 1959)
KN = ["stokeslet", "stresslet", "rotlet"]


def rel(a, b):
    return float(np.linalg.norm(a - b) / np.linalg.norm(b))


@pytest.mark.parametrize("L,xi,pos", [(1.0, 14.0, (0.3, 0.7, 0.1)), (1.0, 21.0, (0.0, 0.5, 0.99)),
                                      (2.5, 6.0, (2.0, 0.1, 1.3))])
def test_hasimoto_constant(L, xi, pos):
    f = np.array([[1.0, -2.0, 0.5]])
    u = O3.ewald("stokeslet", np.array([pos]), f, L=L, xi=xi, rc=6.3 / xi)
    np.testing.assert_allclose(u * L / f, -4.0 / 3.0 * HASIMOTO, rtol=3e-7)


@pytest.mark.parametrize("kernel", KN)
def test_xi_independence(kernel):
    x, f = W.stokeslet_uniform(40, 3)
    q = W.unit_vectors(40, 3) if kernel == "stresslet" else None
    p1 = O3.ewald(kernel, x, f, q, L=1.0, xi=14.0, rc=6.3 / 14.0, parts=True)
    u1 = p1["R"] + p1["F"] + p1["self"]
    u2 = O3.ewald(kernel, x, f, q, L=1.0, xi=19.0, rc=6.3 / 19.0)
    assert rel(u2, u1) <= 1e-12
    # the parts themselves move with xi
    p2 = O3.ewald(kernel, x, f, q, L=1.0, xi=19.0, rc=6.3 / 19.0, parts=True)
    assert rel(p2["F"], p1["F"]) > 1e-2


def test_translation_invariance():
    L = 1.3
    x, f = W.stokeslet_uniform(30, 5)
    x = x * L
    q = W.unit_vectors(30, 5)
    shift = np.array([0.41, -0.77, 1.9])
    xs = np.mod(x + shift, L)
    for kernel in KN:
        qq = q if kernel == "stresslet" else None
        u = O3.ewald(kernel, x, f, qq, L=L, xi=12.0, rc=6.3 / 12.0)
        us = O3.ewald(kernel, xs, f, qq, L=L, xi=12.0, rc=6.3 / 12.0)
        assert rel(us, u) <= 1e-12


@pytest.mark.parametrize("kernel", ["stresslet", "rotlet"])
def test_odd_kernels_vanish_for_one_point(kernel):
    x = np.array([[0.2, 0.6, 0.9]])
    f = np.array([[0.3, -1.0, 2.0]])
    q = np.array([[0.0, 0.6, 0.8]]) if kernel == "stresslet" else None
    pr = O3.ewald(kernel, x, f, q, L=1.0, xi=15.0, rc=6.3 / 15.0, parts=True)
    u = pr["R"] + pr["F"]
    assert np.abs(u).max() <= 1e-13 * max(1.0, np.abs(pr["F"]).max())


@pytest.mark.parametrize("kernel,order", [("stokeslet", 1), ("stresslet", 3), ("rotlet", 3)])
def test_large_box_limit(kernel, order):
    xs, fs = W.stokeslet_uniform(30, 4)
    xs = xs * 0.1
    q = W.unit_vectors(30, 4) if kernel == "stresslet" else None
    ref = direct.direct(kernel, xs, fs, q)
    errs = []
    for L in (1.0, 2.0):
        xi = 14.0 / L
        errs.append(rel(O3.ewald(kernel, xs, fs, q, L=L, xi=xi, rc=6.3 / xi), ref))
    assert errs[0] < (0.2 if order == 1 else 1e-3)
    ratio = errs[0] / errs[1]
    assert abs(ratio / 2**order - 1.0) < 0.05


def test_mutations_are_caught(monkeypatch):
    """Mistakes planted in the Fourier multipliers fail the pins above."""
    orig = O3.multiply
    x, f = W.stokeslet_uniform(20, 6)
    q = W.unit_vectors(20, 6)

    def xi_gap(kernel):
        qq = q if kernel == "stresslet" else None
        a = O3.ewald(kernel, x, f, qq, L=1.0, xi=14.0, rc=6.3 / 14.0)
        b = O3.ewald(kernel, x, f, qq, L=1.0, xi=19.0, rc=6.3 / 19.0)
        return rel(b, a)

    def hasimoto_gap():
        f1 = np.array([[1.0, 0.0, 0.0]])
        u = O3.ewald("stokeslet", np.array([[0.5, 0.5, 0.5]]), f1, L=1.0, xi=14.0, rc=6.3 / 14.0)
        return abs(u[0, 0] / (-4.0 / 3.0 * HASIMOTO) - 1.0)

    # (a) the sign of the odd symbols flipped
    monkeypatch.setattr(O3, "multiply", lambda kid, k, S, xi: (-orig(kid, k, S, xi) if kid != 0
                                                               else orig(kid, k, S, xi)))
    assert xi_gap("rotlet") > 1e-3 and xi_gap("stresslet") > 1e-3
    # (b) the Hasimoto factor (1 + k^2/4xi^2) dropped from the stokeslet
    def no_hasimoto(kid, k, S, xi):
        k2 = k[0] ** 2 + k[1] ** 2 + k[2] ** 2
        return orig(kid, k, S, xi) / (1.0 + k2 / (4.0 * xi**2))
    monkeypatch.setattr(O3, "multiply", no_hasimoto)
    assert xi_gap("stokeslet") > 1e-3
    # (c) a wrong overall factor on the Fourier part (a volume or normalisation slip)
    monkeypatch.setattr(O3, "multiply", lambda kid, k, S, xi: 1.5 * orig(kid, k, S, xi))
    assert hasimoto_gap() > 1e-3
    monkeypatch.setattr(O3, "multiply", orig)
    assert xi_gap("rotlet") < 1e-12 and hasimoto_gap() < 3e-7
