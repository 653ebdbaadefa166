"""The allocation-free real-space entry point (se_real_space_noalloc).

For callers that may not allocate device memory, the library offers the
screened real-space sum with all temporaries in a fixed array inside the
library.  Its result must equal that of the regular entry point
(se_eval_real_space, which uses a plan's workspaces) within the tolerances
used elsewhere: two calls in a row, with different inputs, check that the
shared array is reset between calls.  This file is collected last.
"""
from __future__ import annotations

import ctypes

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


def _noalloc(kernel, prec, x, f, q, xi, rc):
    from paper_1607_04808_gb300 import se as sem
    L = sem.lib()
    fn = L.se_real_space_noalloc
    fn.restype = ctypes.c_int
    fn.argtypes = [ctypes.c_int, ctypes.c_int, ctypes.c_int64, ctypes.POINTER(ctypes.c_double),
                   ctypes.c_double, ctypes.c_double] + [ctypes.c_void_p] * 5
    u = torch.empty_like(x)
    boxa = (ctypes.c_double * 4)(*BOX)
    code = fn(sem.KERNELS[kernel], sem.PRECS[prec], x.shape[0], boxa, xi, rc,
              ctypes.c_void_p(x.data_ptr()), ctypes.c_void_p(f.data_ptr()),
              None if q is None else ctypes.c_void_p(q.data_ptr()), ctypes.c_void_p(u.data_ptr()),
              ctypes.c_void_p(torch.cuda.current_stream().cuda_stream))
    assert code == 0, L.se_last_error().decode()
    torch.cuda.synchronize()
    return u


@pytest.mark.parametrize("kernel", ["stokeslet", "stresslet", "rotlet"])
@pytest.mark.parametrize("prec", ["fp32", "fp64"])
def test_noalloc_matches_plan_entry_point(kernel, prec):
    import paper_1607_04808_gb300 as pkg
    dt = torch.float32 if prec == "fp32" else torch.float64
    tol = 1e-6 if prec == "fp32" else 1e-12
    N = 20000
    plan = pkg.Plan(kernel, N, BOX, prec=prec, tol=2e-6 if prec == "fp32" else 1e-10)
    prm = plan.params
    for seed in (21, 22):  # two calls in a row on different inputs
        x, f = W.stokeslet_uniform(N, seed)
        q = W.unit_vectors(N, seed) if kernel == "stresslet" else None
        tx = torch.tensor(x, dtype=dt, device="cuda")
        tf = torch.tensor(f, dtype=dt, device="cuda")
        tq = None if q is None else torch.tensor(q, dtype=dt, device="cuda")
        ref = plan.eval_real_space(tx, tf, tq).double().cpu().numpy()
        plan.check()
        got = _noalloc(kernel, prec, tx, tf, tq, prm["xi"], prm["rc"]).double().cpu().numpy()
        err = np.linalg.norm(got - ref) / np.linalg.norm(ref)
        assert err <= tol, (seed, err)
    plan.close()


@pytest.mark.parametrize("prec", ["fp32", "fp64"])
def test_noalloc_narrow_cutoff_wide_cells(prec):
    """A cutoff near L/24 with few points: the fixed cell list then caps the
    cells along x, which become wider than rc (a geometry no plan uses).  The
    sum must still equal the regular entry point's, on two calls in a row."""
    import paper_1607_04808_gb300 as pkg
    dt = torch.float32 if prec == "fp32" else torch.float64
    tol = 1e-6 if prec == "fp32" else 1e-12
    N, xi, rc = 3000, 60.0, 1.0 / 24.5
    plan = pkg.Plan("stokeslet", N, BOX, prec=prec, xi=xi, rc=rc, M=40, P=8)
    for seed in (23, 24):
        x, f = W.stokeslet_uniform(N, seed)
        tx = torch.tensor(x, dtype=dt, device="cuda")
        tf = torch.tensor(f, dtype=dt, device="cuda")
        ref = plan.eval_real_space(tx, tf).double().cpu().numpy()
        plan.check()
        got = _noalloc("stokeslet", prec, tx, tf, None, xi, rc).double().cpu().numpy()
        err = np.linalg.norm(got - ref) / np.linalg.norm(ref)
        assert err <= tol, (seed, err)
    plan.close()


def test_noalloc_rejects_oversized_requests():
    from paper_1607_04808_gb300 import se as sem
    x = torch.zeros((40000, 3), dtype=torch.float32, device="cuda")
    L = sem.lib()
    fn = L.se_real_space_noalloc
    fn.restype = ctypes.c_int
    fn.argtypes = [ctypes.c_int, ctypes.c_int, ctypes.c_int64, ctypes.POINTER(ctypes.c_double),
                   ctypes.c_double, ctypes.c_double] + [ctypes.c_void_p] * 5
    boxa = (ctypes.c_double * 4)(*BOX)
    p = ctypes.c_void_p(x.data_ptr())
    assert fn(0, 0, 40000, boxa, 30.0, 0.1, p, p, None, p, None) == 1  # N above the maximum
    assert fn(0, 0, 1000, boxa, 30.0, 0.01, p, p, None, p, None) == 1  # cell list above the maximum
