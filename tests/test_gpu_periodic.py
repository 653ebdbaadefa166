"""Triply periodic plans (se_plan_create_periodic) against the periodic oracle O3.

O3 is a plain Ewald sum with its own Ewald parameter (the periodic sum does
not depend on it); it is pinned to Hasimoto's constant, xi-independence and
the large-box limit in test_oracle_periodic.py.  Bars as for free space: the
FP64 path 1e-10 and the FP32 path 2e-6 (relative L2 and relative max error);
FP32 runs are compared on the FP32-rounded inputs.
"""
from __future__ import annotations

import numpy as np
import pytest
import torch

import workloads as W
from oracle import periodic as O3

pytestmark = pytest.mark.gpu

KN = ["stokeslet", "stresslet", "rotlet"]
HASIMOTO = 2.8372975
XI_ORACLE = 14.0  # per unit box side


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


def oracle(kernel, x, f, q=None, L=1.0, targets=None):
    xi = XI_ORACLE / L
    return O3.ewald(kernel, x, f, q, L=L, xi=xi, rc=6.3 / xi, targets=targets)


def as_prec(a, prec):
    if a is None:
        return None
    return a.astype(np.float32).astype(np.float64) if prec == "fp32" else a


def inputs(n, seed, prec, box=(0.0, 0.0, 0.0, 1.0), stresslet=False):
    x = W.uniform_points(n, seed, L=box[3], x0=box[:3])
    if prec == "fp32":
        top = np.nextafter((np.asarray(box[:3]) + box[3]).astype(np.float32), np.float32(-np.inf))
        x = np.minimum(x.astype(np.float32), top).astype(np.float64)
    f = as_prec(W.normal_vectors(n, seed), prec)
    q = as_prec(W.unit_vectors(n, seed), prec) if stresslet else None
    return x, f, q


def run(kernel, x, f, q, prec, box=(0.0, 0.0, 0.0, 1.0), real_only=False, **kw):
    pkg = P()
    dt = torch.float32 if prec == "fp32" else torch.float64
    plan = pkg.Plan(kernel, len(x), box, prec=prec, periodic=True, **kw)
    t = lambda a: None if a is None else torch.tensor(a, dtype=dt, device="cuda")  # noqa: E731
    fn = plan.eval_real_space if real_only else plan.eval
    u = fn(t(x), t(f), t(q)).double().cpu().numpy()
    plan.check()
    info = (plan.params, plan.grid)
    plan.close()
    return u, info


@pytest.mark.parametrize("kernel", KN)
def test_fp64_vs_ewald(kernel):
    x, f, q = inputs(600, 51, "fp64", stresslet=kernel == "stresslet")
    u, (prm, grid) = run(kernel, x, f, q, "fp64", tol=1e-10)
    ref = oracle(kernel, x, f, q)
    assert rel_l2(u, ref) <= 1e-10
    assert rel_max(u, ref) <= 1e-10
    M = prm["M"]
    assert M % 2 == 0 and grid["Mf"] == (M, M, M) and prm["rc"] < 0.5


@pytest.mark.parametrize("kernel", KN)
def test_fp32_vs_ewald(kernel):
    x, f, q = inputs(2000, 52, "fp32", stresslet=kernel == "stresslet")
    u, _ = run(kernel, x, f, q, "fp32", tol=2e-6)
    ref = oracle(kernel, x, f, q)
    assert rel_l2(u, ref) <= 2e-6
    assert rel_max(u, ref) <= 2e-6


def test_offset_box_and_side():
    box = (-1.0, 0.5, 2.0, 1.7)
    x, f, _ = inputs(500, 53, "fp64", box=box)
    u, _ = run("rotlet", x, f, None, "fp64", box=box, tol=1e-10)
    # the oracle works in [0, L)^3: shift the points (the sum only sees differences)
    ref = oracle("rotlet", x - np.asarray(box[:3]), f, L=box[3])
    assert rel_l2(u, ref) <= 1e-10


@pytest.mark.parametrize("kernel", ["stokeslet", "rotlet"])
def test_fp32_offset_box_symmetric_path(kernel):
    """FP32 stokeslet and rotlet run the symmetric periodic kernel (wrapped rows,
    candidates moved to the image nearest their cluster); an offset box of side 1.7."""
    box = (-1.0, 0.5, 2.0, 1.7)
    x, f, _ = inputs(3000, 58, "fp32", box=box)
    u, _ = run(kernel, x, f, None, "fp32", box=box, tol=2e-6)
    ref = oracle(kernel, x - np.asarray(box[:3]), f, L=box[3])
    assert rel_l2(u, ref) <= 2e-6
    assert rel_max(u, ref) <= 2e-6


@pytest.mark.parametrize("prec,tol", [("fp64", 5e-8), ("fp32", 5e-6)])
def test_hasimoto_single_point(prec, tol):
    """One point force: its images give -(4/3) 2.8372975 f / L (Hasimoto 1959; the
    FP64 bar is the precision of the 8-digit constant)."""
    L = 2.0
    x = np.array([[0.3, 1.1, 1.9]])
    f = np.array([[1.0, -0.5, 2.0]])
    u, _ = run("stokeslet", x, f, None, prec, box=(0.0, 0.0, 0.0, L), xi=7.0,
               tol=1e-12 if prec == "fp64" else 2e-6)
    np.testing.assert_allclose(u * L / f, -4.0 / 3.0 * HASIMOTO, rtol=tol)


def test_xi_independence():
    x, f, q = inputs(400, 54, "fp64", stresslet=True)
    u1, p1 = run("stresslet", x, f, q, "fp64", xi=10.0, tol=1e-11)
    u2, p2 = run("stresslet", x, f, q, "fp64", xi=16.0, tol=1e-11)
    assert p1[0]["M"] != p2[0]["M"]
    assert rel_l2(u2, u1) <= 2e-10


@pytest.mark.parametrize("prec", ["fp64", "fp32"])
def test_real_space_part_vs_oracle(prec):
    x, f, _ = inputs(1500, 55, prec)
    u, (prm, _) = run("stokeslet", x, f, None, prec, real_only=True, tol=1e-10 if prec == "fp64" else 2e-6)
    ref = O3.real_part("stokeslet", x, f, None, 1.0, prm["xi"], prm["rc"])
    assert rel_l2(u, ref) <= (1e-12 if prec == "fp64" else 1e-6)


def test_medium_fp32_sampled():
    """N = 2e4 uniform points, FP32 stokeslet, 64 sampled points vs O3."""
    x, f, _ = inputs(20000, 56, "fp32")
    u, _ = run("stokeslet", x, f, None, "fp32", tol=2e-6)
    idx = np.random.default_rng(5).choice(len(x), 64, replace=False)
    ref = oracle("stokeslet", x, f, targets=idx)
    assert rel_l2(u[idx], ref) <= 2e-6


def test_unsupported_calls_are_refused():
    pkg = P()
    x, f, _ = inputs(100, 57, "fp64")
    plan = pkg.Plan("stokeslet", 100, (0.0, 0.0, 0.0, 1.0), prec="fp64", periodic=True, tol=1e-8)
    t = lambda a: torch.tensor(a, device="cuda")  # noqa: E731
    with pytest.raises(pkg.SEError) as ei:
        plan.eval_targets(t(x), t(f), t(x[:5]))
    assert ei.value.code == 8
    with pytest.raises(pkg.SEError) as ei:
        plan.backward(t(x), t(f), t(f))
    assert ei.value.code == 8
    plan.close()
    with pytest.raises(pkg.SEError) as ei:
        pkg.Plan("stokeslet", 100, (0.0, 0.0, 0.0, 1.0), prec="fp64", periodic=True, rc=0.6, xi=10.0,
                 M=40, P=16)
    assert ei.value.code == 1
