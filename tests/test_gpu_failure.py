"""Failure detection without a GPU fault: the gather's tile copy is a tensor
copy completed on an mbarrier, and its wait is bounded (one second).  With the
test flag SE_TEST_SKIP_TILE_COPY the copy is never issued, so every tile's
wait runs out: the kernel records the timeout in the plan's status and
returns, se_plan_check reports SE_ERR_TIMEOUT, and the same plan evaluates
correctly once the flag is cleared (the context stays usable)."""
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


def test_tile_copy_timeout_is_reported_and_the_plan_recovers():
    import paper_1607_04808_gb300 as pkg
    n = 3000
    x, f = W.stokeslet_uniform(n, 71)
    x = np.minimum(x.astype(np.float32), np.nextafter(np.float32(1), np.float32(0)))
    f = f.astype(np.float32)
    # M + P even (FFT length a multiple of 4): the gather stages its tiles by tensor copy
    plan = pkg.Plan("stokeslet", n, BOX, prec="fp32", tol=2e-6, M=36, P=12)
    assert plan.grid["Mf"][0] % 4 == 0
    xs, fs = torch.tensor(x, device="cuda"), torch.tensor(f, device="cuda")
    plan.set_test_flags(pkg.se.TEST_SKIP_TILE_COPY)
    plan.eval(xs, fs)
    with pytest.raises(pkg.SEError) as ei:
        plan.check()
    assert ei.value.code == 7  # SE_ERR_TIMEOUT
    plan.set_test_flags(0)
    u = plan.eval(xs, fs).double().cpu().numpy()
    plan.check()
    plan.close()
    idx = np.random.default_rng(4).choice(n, 128, replace=False)
    ref = direct.direct("stokeslet", x.astype(np.float64), f.astype(np.float64), targets=idx)
    assert float(np.linalg.norm(u[idx] - ref) / np.linalg.norm(ref)) <= 2e-6


def test_unknown_test_flag_is_refused():
    import paper_1607_04808_gb300 as pkg
    plan = pkg.Plan("stokeslet", 100, BOX, prec="fp32", tol=2e-6)
    with pytest.raises(pkg.SEError) as ei:
        plan.set_test_flags(2)
    assert ei.value.code == 1
    plan.close()
