"""Plan options that change how the work is done, not what is computed: the
real-space cell width (se_params_t.cell_width) and stage timing of the
backward pass.  Results must agree with the default plan to FP32 rounding."""
from __future__ import annotations

import numpy as np
import pytest
import torch

import workloads as W

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


@pytest.mark.parametrize("kernel", ["stokeslet", "stresslet", "rotlet"])
@pytest.mark.parametrize("width", [0.02, 0.05])
def test_cell_width_changes_nothing_but_rounding(kernel, width):
    import paper_1607_04808_gb300 as pkg
    n = 30000
    x, f = W.stokeslet_uniform(n, 81)
    x = np.minimum(x.astype(np.float32), np.nextafter(np.float32(1), np.float32(0)))
    f = f.astype(np.float32)
    q = W.unit_vectors(n, 81).astype(np.float32) if kernel == "stresslet" else None
    t = lambda a: None if a is None else torch.tensor(a, device="cuda")  # noqa: E731
    ref_plan = pkg.Plan(kernel, n, BOX, prec="fp32", tol=2e-6)
    prm = ref_plan.params
    u0 = ref_plan.eval(t(x), t(f), t(q)).double().cpu().numpy()
    ref_plan.check()
    ref_plan.close()
    plan = pkg.Plan(kernel, n, BOX, prec="fp32", tol=2e-6, xi=prm["xi"], M=prm["M"], P=prm["P"], rc=prm["rc"],
                    cell_width=width)
    assert abs(plan.params["cell_width"] - width) < 1e-12
    u1 = plan.eval(t(x), t(f), t(q)).double().cpu().numpy()
    plan.check()
    plan.close()
    assert rel_l2(u1, u0) <= 1e-6


def test_backward_stage_times():
    import paper_1607_04808_gb300 as pkg
    n = 20000
    x, tq, g = W.rotlet_uniform(n, 82)
    x = np.minimum(x.astype(np.float32), np.nextafter(np.float32(1), np.float32(0)))
    t = lambda a: torch.tensor(a, dtype=torch.float32, device="cuda")  # noqa: E731
    plan = pkg.Plan("rotlet", n, BOX, prec="fp32", tol=2e-6)
    gf0, gx0 = plan.backward(t(x), t(tq), t(g))
    plan.set_timing(True)
    gf1, gx1 = plan.backward(t(x), t(tq), t(g))
    torch.cuda.synchronize()
    st = plan.stage_times(backward=True)
    plan.check()
    plan.close()
    assert list(st) == ["adj_bin", "adj_fourier", "adj_gather", "adj_real", "bin", "fourier", "grad_gather",
                        "grad_real"]
    assert all(v > 0 for v in st.values())
    # timing changes nothing but the order of the FP32 atomics
    assert rel_l2(gf1.double().cpu().numpy(), gf0.double().cpu().numpy()) <= 1e-6
    assert rel_l2(gx1.double().cpu().numpy(), gx0.double().cpu().numpy()) <= 1e-5


@pytest.mark.parametrize("kernel,prec", [("stokeslet", "fp32"), ("stresslet", "fp32"), ("rotlet", "fp32"),
                                         ("stokeslet", "fp64"), ("stresslet", "fp64")])
def test_keep_grid_reuses_forward_grid(kernel, prec):
    """With keep-grid on, the backward after se_eval on the same arrays skips
    the forward grid (fewer launches) and gives the gradients of a plan that
    recomputes it; after an evaluation on other arrays it recomputes."""
    import paper_1607_04808_gb300 as pkg
    n = 20000
    dt = torch.float32 if prec == "fp32" else torch.float64
    x, f = W.stokeslet_uniform(n, 83)
    x = np.minimum(x.astype(np.float32), np.nextafter(np.float32(1), np.float32(0)))
    g = W._rng(83, 5).standard_normal((n, 3))
    q = W.unit_vectors(n, 83) if kernel == "stresslet" else None
    t = lambda a: None if a is None else torch.tensor(a, dtype=dt, device="cuda")  # noqa: E731
    tx, tf, tq, tg = t(x), t(f), t(q), t(g)
    tf2 = t(-0.5 * f)
    want_q = kernel == "stresslet"
    ref = pkg.Plan(kernel, n, BOX, prec=prec, tol=2e-6 if prec == "fp32" else 1e-10)
    prm = ref.params
    plan = pkg.Plan(kernel, n, BOX, prec=prec, xi=prm["xi"], M=prm["M"], P=prm["P"], rc=prm["rc"])
    plan.set_keep_grid(True)
    ref.eval(tx, tf, tq)
    out0 = ref.backward(tx, tf, tg, q=tq, want_q=want_q)
    n_recompute = ref.launch_count()
    plan.eval(tx, tf, tq)
    out1 = plan.backward(tx, tf, tg, q=tq, want_q=want_q)
    n_kept = plan.launch_count()
    # a second backward on the same arrays still finds the grid
    out2 = plan.backward(tx, tf, tg, q=tq, want_q=want_q)
    assert plan.launch_count() == n_kept
    # after an evaluation with other strengths the grid belongs to those
    plan.eval(tx, tf2, tq)
    out3 = plan.backward(tx, tf, tg, q=tq, want_q=want_q)
    n_after = plan.launch_count()
    plan.check()
    ref.check()
    plan.close()
    ref.close()
    assert n_kept < n_recompute and n_after == n_recompute, (n_kept, n_recompute, n_after)
    tol = 1e-5 if prec == "fp32" else 1e-11  # FP32: the order of the spreading atomics
    for o in (out1, out2, out3):
        for a, b in zip(o, out0):
            if b is None:
                continue
            assert rel_l2(a.double().cpu().numpy(), b.double().cpu().numpy()) <= tol
