"""Overlapped evaluation (se_plan_set_overlap): the Fourier part on the plan's
internal stream while the real-space sum runs on the caller's stream.  The
result must equal the sequential evaluation's up to the order of the FP32
atomics, meet the FP32 bar against the direct sum O1, and survive capture
into a CUDA graph."""
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


def P():
    import paper_1607_04808_gb300 as pkg
    return pkg


def rel_l2(a, b):
    return float(np.linalg.norm(a - b) / np.linalg.norm(b))


def fp32_inputs(n, seed, stresslet=False):
    x, f = W.stokeslet_uniform(n, seed)
    x = np.minimum(x.astype(np.float32), np.nextafter(np.float32(1), np.float32(0)))
    f = f.astype(np.float32)
    q = W.unit_vectors(n, seed).astype(np.float32) if stresslet else None
    return x, f, q


@pytest.mark.parametrize("kernel", ["stokeslet", "stresslet", "rotlet"])
def test_overlap_matches_sequential_and_direct(kernel):
    n = 40000
    x, f, q = fp32_inputs(n, 61, kernel == "stresslet")
    pkg = P()
    t = lambda a: None if a is None else torch.tensor(a, device="cuda")  # noqa: E731
    plan = pkg.Plan(kernel, n, BOX, prec="fp32", tol=2e-6)
    u_ov = plan.eval(t(x), t(f), t(q))
    plan.check()
    plan.set_overlap(False)
    u_seq = plan.eval(t(x), t(f), t(q))
    plan.check()
    plan.close()
    a, b = u_ov.double().cpu().numpy(), u_seq.double().cpu().numpy()
    assert rel_l2(a, b) <= 1e-6
    idx = np.random.default_rng(3).choice(n, 200, replace=False)
    d = lambda v: None if v is None else v.astype(np.float64)  # noqa: E731
    ref = direct.direct(kernel, d(x), d(f), d(q), targets=idx)
    assert rel_l2(a[idx], ref) <= 2e-6


def test_overlap_under_graph_capture():
    n = 30000
    x, f, _ = fp32_inputs(n, 62)
    x2, f2, _ = fp32_inputs(n, 63)
    pkg = P()
    plan = pkg.Plan("stokeslet", n, BOX, prec="fp32", tol=2e-6)
    xs = torch.tensor(x, device="cuda")
    fs = torch.tensor(f, device="cuda")
    us = torch.empty_like(xs)
    side = torch.cuda.Stream()
    side.wait_stream(torch.cuda.current_stream())
    with torch.cuda.stream(side):
        plan.eval(xs, fs, out=us)  # warm-up outside the capture
    torch.cuda.current_stream().wait_stream(side)
    torch.cuda.synchronize()
    g = torch.cuda.CUDAGraph()
    with torch.cuda.graph(g):
        plan.eval(xs, fs, out=us)
    xs.copy_(torch.tensor(x2, device="cuda"))
    fs.copy_(torch.tensor(f2, device="cuda"))
    g.replay()
    torch.cuda.synchronize()
    plan.check()
    got = us.double().cpu().numpy()
    ref = plan.eval(torch.tensor(x2, device="cuda"), torch.tensor(f2, device="cuda")).double().cpu().numpy()
    plan.close()
    assert rel_l2(got, ref) <= 1e-6


def test_overlap_refused_where_unavailable():
    pkg = P()
    plan = pkg.Plan("stokeslet", 100, BOX, prec="fp64", tol=1e-8)
    with pytest.raises(pkg.SEError) as ei:
        plan.set_overlap(True)
    assert ei.value.code == 8
    plan.set_overlap(False)
    plan.close()
