"""Rectangular boxes (se_plan_create_box) against the direct sum O1.

The free-space sums do not depend on the box: the box only fixes the grids.
The direct sum is therefore the exact answer for any box, and the FP64 path
must meet 1e-10 and the FP32 path 2e-6 (relative L2 and relative max error),
as for the cube.  One grid spacing h serves all dimensions; M counts the
intervals along the longest side and the truncation radius R is the diagonal
of the extended box (Section 4.1 with Ltilde per dimension).
"""
from __future__ import annotations

import numpy as np
import pytest
import torch

import workloads as W
from oracle import direct

pytestmark = pytest.mark.gpu

KN = ["stokeslet", "stresslet", "rotlet"]
GOOD = {2, 3, 5, 7}


@pytest.fixture(scope="module", autouse=True)
def _gpu():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1607_04808_gb300 import _build
    _build.build()
    torch.cuda.set_device(0)


def P():
    import paper_1607_04808_gb300 as pkg
    return pkg


def rel_l2(a, b):
    return float(np.linalg.norm(a - b) / np.linalg.norm(b))


def rel_max(a, b):
    return float(np.abs(a - b).max() / np.abs(b).max())


def points_in(box, n, seed, prec):
    """n uniform points in box = (x0, y0, z0, Lx, Ly, Lz), kept inside the
    half-open box after rounding to the path's precision."""
    x0, L = np.asarray(box[:3]), np.asarray(box[3:])
    x = W.uniform_points(n, seed, L=L, x0=x0)
    if prec == "fp32":
        top = np.nextafter((x0 + L).astype(np.float32), np.float32(-np.inf))
        x = np.minimum(x.astype(np.float32), top).astype(np.float64)
    return x


def as_prec(a, prec):
    if a is None:
        return None
    return a.astype(np.float32).astype(np.float64) if prec == "fp32" else a


def factors_ok(n):
    for p in sorted(GOOD):
        while n % p == 0:
            n //= p
    return n == 1


BOXES = [
    (-0.5, 0.2, 1.0, 2.0, 1.0, 0.5),   # x longest
    (0.0, 0.0, 0.0, 0.3, 1.2, 0.6),    # y longest
    (1.0, -1.0, 0.0, 0.7, 0.7, 1.4),   # z longest
]


@pytest.mark.parametrize("kernel", KN)
@pytest.mark.parametrize("box", BOXES, ids=["x", "y", "z"])
def test_fp64_box_vs_direct(kernel, box):
    pkg = P()
    n = 1500
    x = points_in(box, n, 41, "fp64")
    f = W.normal_vectors(n, 41)
    q = W.unit_vectors(n, 41) if kernel == "stresslet" else None
    plan = pkg.Plan(kernel, n, box, prec="fp64", tol=1e-10)
    t = lambda a: None if a is None else torch.tensor(a, device="cuda")  # noqa: E731
    u = plan.eval(t(x), t(f), t(q)).cpu().numpy()
    plan.check()
    g = plan.grid
    prm = plan.params
    plan.close()
    ref = direct.direct(kernel, x, f, q)
    assert rel_l2(u, ref) <= 1e-10
    assert rel_max(u, ref) <= 1e-10
    # grid sizes: M along the longest side, FFT-friendly lengths, 2 Mtilde
    longest = int(np.argmax(box[3:]))
    assert g["M"][longest] == prm["M"]
    for d in range(3):
        assert g["M"][d] * prm["h"] >= box[3 + d] * (1 - 1e-12)
        assert g["Mf"][d] == 2 * g["Mtilde"][d]
        assert factors_ok(g["Mf"][d]) and factors_ok(g["Mg"][d])
        assert g["Mg"][d] >= 2 * g["Mtilde"][d]
        if d != longest:
            assert g["M"][d] <= g["M"][longest]


@pytest.mark.parametrize("kernel", KN)
def test_fp32_box_vs_direct(kernel):
    pkg = P()
    box = (0.0, 0.0, 0.0, 1.0, 0.4, 0.7)
    n = 3000
    x = points_in(box, n, 42, "fp32")
    f = as_prec(W.normal_vectors(n, 42), "fp32")
    q = as_prec(W.unit_vectors(n, 42), "fp32") if kernel == "stresslet" else None
    plan = pkg.Plan(kernel, n, box, prec="fp32", tol=2e-6)
    t = lambda a: None if a is None else torch.tensor(a, dtype=torch.float32, device="cuda")  # noqa: E731
    u = plan.eval(t(x), t(f), t(q)).double().cpu().numpy()
    plan.check()
    plan.close()
    ref = direct.direct(kernel, x, f, q)
    assert rel_l2(u, ref) <= 2e-6
    assert rel_max(u, ref) <= 2e-6


@pytest.mark.parametrize("prec", ["fp64", "fp32"])
def test_thin_slab(prec):
    """A slab ten times thinner than wide: a single cell across its thickness."""
    pkg = P()
    box = (0.0, 0.0, 0.0, 1.0, 1.0, 0.1)
    n = 2000
    x = points_in(box, n, 43, prec)
    f = as_prec(W.normal_vectors(n, 43), prec)
    tol = 1e-10 if prec == "fp64" else 2e-6
    dt = torch.float64 if prec == "fp64" else torch.float32
    plan = pkg.Plan("stokeslet", n, box, prec=prec, tol=tol)
    u = plan.eval(torch.tensor(x, dtype=dt, device="cuda"),
                  torch.tensor(f, dtype=dt, device="cuda")).double().cpu().numpy()
    plan.check()
    plan.close()
    assert rel_l2(u, direct.direct("stokeslet", x, f)) <= tol


def test_cube_through_box_entry_matches_cube_entry():
    """(x0, y0, z0, L, L, L) through se_plan_create_box is the cube plan."""
    pkg = P()
    n = 1200
    x, f = W.stokeslet_uniform(n, 44)
    t = lambda a: torch.tensor(a, device="cuda")  # noqa: E731
    p4 = pkg.Plan("stokeslet", n, (0.0, 0.0, 0.0, 1.0), prec="fp64", tol=1e-10)
    p6 = pkg.Plan("stokeslet", n, (0.0, 0.0, 0.0, 1.0, 1.0, 1.0), prec="fp64", tol=1e-10)
    assert p4.params == p6.params and p4.grid == p6.grid
    u4 = p4.eval(t(x), t(f)).cpu().numpy()
    u6 = p6.eval(t(x), t(f)).cpu().numpy()
    p4.close()
    p6.close()
    assert rel_l2(u6, u4) <= 1e-14


@pytest.mark.parametrize("prec", ["fp64", "fp32"])
def test_box_targets_and_backward(prec):
    """Separate targets and the rotlet backward in a rectangular box."""
    pkg = P()
    box = (0.25, 0.0, -0.5, 0.6, 1.0, 0.8)
    n, nt = 1500, 400
    x = points_in(box, n, 45, prec)
    f = as_prec(W.normal_vectors(n, 45), prec)
    g = as_prec(W.normal_vectors(n, 46), prec)
    y = points_in(box, nt, 47, prec)
    tol = 1e-10 if prec == "fp64" else 2e-6
    dt = torch.float64 if prec == "fp64" else torch.float32
    t = lambda a: torch.tensor(a, dtype=dt, device="cuda")  # noqa: E731
    plan = pkg.Plan("rotlet", n, box, prec=prec, tol=tol)
    ut = plan.eval_targets(t(x), t(f), t(y)).double().cpu().numpy()
    plan.check()
    assert rel_l2(ut, direct.direct("rotlet", x, f, xt=y)) <= tol
    gf, gx = plan.backward(t(x), t(f), t(g))
    plan.check()
    tol_f, tol_x = (1e-9, 1e-8) if prec == "fp64" else (2e-6, 2e-5)
    assert rel_l2(gf.double().cpu().numpy(), direct.grad_f("rotlet", x, g)) <= tol_f
    assert rel_l2(gx.double().cpu().numpy(), direct.grad_x("rotlet", x, f, g)) <= tol_x
    plan.close()


def test_point_outside_the_short_side_is_reported():
    """A point inside the longest side's range but outside a shorter side."""
    pkg = P()
    box = (0.0, 0.0, 0.0, 1.0, 0.5, 0.5)
    n = 300
    x = points_in(box, n, 48, "fp64")
    x[7, 2] = 0.75  # beyond z0 + Lz
    f = W.normal_vectors(n, 48)
    plan = pkg.Plan("stokeslet", n, box, prec="fp64", tol=1e-8)
    plan.eval(torch.tensor(x, device="cuda"), torch.tensor(f, device="cuda"))
    with pytest.raises(pkg.SEError) as ei:
        plan.check()
    assert ei.value.code == 2  # SE_ERR_OUT_OF_BOX
    plan.close()
