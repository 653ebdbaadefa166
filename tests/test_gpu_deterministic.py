"""Deterministic mode (se_plan_set_deterministic): the same inputs give
bit-identical results call after call, and those results are still the
method's, held to the FP32 bar against the FP64 direct sum (the oracle)."""
from __future__ import annotations

import numpy as np
import pytest
import torch

import workloads as W
from oracle import direct

pytestmark = pytest.mark.gpu

BOX = (0.0, 0.0, 0.0, 1.0)


@pytest.fixture(scope="module", autouse=True)
def _gpu():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1607_04808_gb300 import _build
    _build.build()
    torch.cuda.set_device(0)


def rel_l2(a, b):
    return float(np.linalg.norm(a - b) / np.linalg.norm(b))


def rel_max(a, b):
    return float(np.abs(a - b).max() / np.abs(b).max())


def as32(a):
    return None if a is None else np.minimum(np.asarray(a, dtype=np.float32),
                                             np.float32(1.0) - np.float32(2.0 ** -24))


def data(kernel, n, seed, blobs=False):
    if blobs:
        x, f, q = W.stresslet_blobs(n, seed)
    else:
        x, f = W.stokeslet_uniform(n, seed)
        q = W.unit_vectors(n, seed) if kernel == "stresslet" else None
    return as32(x), np.asarray(f, dtype=np.float32), (None if q is None else np.asarray(q, dtype=np.float32))


def dev(a):
    return None if a is None else torch.tensor(a, device="cuda")


# (kernel, N, clustered): dense tiles (about 270 points per tile: sub-tiles as
# clusters of CTAs), sparse tiles (the 8^3-tile kernel), and clustered points
# (bins of very different sizes; the stresslet's support P = 14)
CASES = [("stokeslet", 200_000, False), ("rotlet", 30_000, False), ("stresslet", 40_000, True)]


@pytest.mark.parametrize("kernel,n,blobs", CASES)
def test_repeated_evaluations_are_bit_identical(kernel, n, blobs):
    import paper_1607_04808_gb300 as pkg
    x, f, q = data(kernel, n, 91, blobs)
    xt, ft, qt = dev(x), dev(f), dev(q)
    plan = pkg.Plan(kernel, n, BOX, prec="fp32", tol=2e-6)
    u_def = plan.eval(xt, ft, qt).double().cpu().numpy()
    plan.set_deterministic(True)
    runs = []
    for k in range(3):
        if k == 1:
            # other work in between, on other inputs of the same size
            x2, f2, q2 = data(kernel, n, 92, blobs)
            plan.eval(dev(x2), dev(f2), dev(q2))
        runs.append(plan.eval(xt, ft, qt).clone())
    plan.check()
    for u in runs[1:]:
        assert torch.equal(u, runs[0])
    u = runs[0].double().cpu().numpy()
    # the same sums in another order: the default mode agrees to FP32 rounding
    assert rel_l2(u, u_def) <= 1e-6
    idx = np.random.default_rng(93).choice(n, 200, replace=False)
    ref = direct.direct(kernel, x, f, q, targets=idx)
    assert rel_l2(u[idx], ref) <= 2e-6
    if not blobs:
        assert rel_max(u[idx], ref) <= 2e-6
    plan.set_deterministic(False)
    u_off = plan.eval(xt, ft, qt).double().cpu().numpy()
    assert rel_l2(u_off, u) <= 1e-6
    plan.close()


def test_targets_bit_identical_and_scratch_grows():
    """se_eval_targets with more targets than sources: the mode's scratch grows
    with the target buffers, and repeated calls agree bit for bit."""
    import paper_1607_04808_gb300 as pkg
    n, nt = 20_000, 50_000
    x, f, _ = data("stokeslet", n, 94)
    y = as32(W.uniform_points(nt, 95))
    plan = pkg.Plan("stokeslet", n, BOX, prec="fp32", tol=2e-6)
    plan.set_deterministic(True)
    a = plan.eval_targets(dev(x), dev(f), dev(y)).clone()
    b = plan.eval_targets(dev(x), dev(f), dev(y)).clone()
    plan.check()
    assert torch.equal(a, b)
    idx = np.random.default_rng(96).choice(nt, 200, replace=False)
    ref = direct.direct("stokeslet", x, f, xt=y[idx])
    got = a.double().cpu().numpy()[idx]
    assert rel_l2(got, ref) <= 2e-6
    assert rel_max(got, ref) <= 2e-6
    plan.close()


def test_refused_where_not_built():
    import paper_1607_04808_gb300 as pkg
    plan = pkg.Plan("stokeslet", 5000, BOX, prec="fp64", tol=1e-10)
    with pytest.raises(pkg.SEError):
        plan.set_deterministic(True)
    plan.set_deterministic(False)  # turning it off is always accepted
    plan.close()
    per = pkg.Plan("stokeslet", 5000, BOX, prec="fp32", tol=2e-6, periodic=True)
    with pytest.raises(pkg.SEError):
        per.set_deterministic(True)
    per.close()


def test_other_support_widths():
    """A looser tolerance (a smaller support P, spread by the 8^3-tile kernel
    with its tile buffer): bit-identical repeats, and the default mode's
    result to FP32 rounding."""
    import paper_1607_04808_gb300 as pkg
    n = 20_000
    x, f, _ = data("stokeslet", n, 97)
    plan = pkg.Plan("stokeslet", n, BOX, prec="fp32", tol=1e-3)
    assert plan.params["P"] == 8
    u0 = plan.eval(dev(x), dev(f)).double().cpu().numpy()
    plan.set_deterministic(True)
    a = plan.eval(dev(x), dev(f)).clone()
    b = plan.eval(dev(x), dev(f)).clone()
    plan.check()
    assert torch.equal(a, b)
    assert rel_l2(a.double().cpu().numpy(), u0) <= 1e-6
    plan.close()
