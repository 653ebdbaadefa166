"""A seeded matrix of mixed configurations through the C ABI: kernel, precision,
N (tiny to a few thousand), box shape (cube, rectangular, periodic cube) and
corner, each compared with the exact sum (O1, or O3 for periodic plans) at the
precision's bar.  The cases are drawn once from a fixed seed, so the matrix is
the same on every run."""
from __future__ import annotations

import numpy as np
import pytest
import torch

import workloads as W
from oracle import direct
from oracle import periodic as O3

pytestmark = pytest.mark.gpu

KN = ["stokeslet", "stresslet", "rotlet"]


def _cases(n_cases=18, seed=20261204):
    rng = np.random.default_rng(seed)
    out = []
    for i in range(n_cases):
        kernel = KN[i % 3]
        prec = "fp64" if (i // 3) % 2 == 0 else "fp32"
        shape = ["cube", "box", "periodic"][(i // 6) % 3]
        lo = 1 if prec == "fp64" else 200
        hi = 1500 if shape == "periodic" else 5000
        n = int(np.exp(rng.uniform(np.log(lo), np.log(hi))))
        x0 = tuple(float(v) for v in rng.uniform(-2.0, 2.0, 3))
        if shape == "box":
            sides = tuple(float(v) for v in rng.uniform(0.4, 1.6, 3))
        else:
            sides = (float(rng.uniform(0.5, 2.0)),) * 3
        out.append((i, kernel, prec, shape, n, x0, sides))
    return out


CASES = _cases()


@pytest.fixture(scope="module", autouse=True)
def _gpu():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1607_04808_gb300 import _build
    _build.build()
    torch.cuda.set_device(0)


@pytest.mark.parametrize("case", CASES, ids=[f"{c[0]}-{c[1]}-{c[2]}-{c[3]}-N{c[4]}" for c in CASES])
def test_random_configuration(case):
    import paper_1607_04808_gb300 as pkg
    i, kernel, prec, shape, n, x0, sides = case
    L = np.asarray(sides)
    x = W.uniform_points(n, 300 + i, L=L, x0=np.asarray(x0))
    f = W.normal_vectors(n, 300 + i)
    q = W.unit_vectors(n, 300 + i) if kernel == "stresslet" else None
    if prec == "fp32":
        top = np.nextafter((np.asarray(x0) + L).astype(np.float32), np.float32(-np.inf))
        x = np.minimum(x.astype(np.float32), top).astype(np.float64)
        f = f.astype(np.float32).astype(np.float64)
        q = None if q is None else q.astype(np.float32).astype(np.float64)
    bar = 1e-10 if prec == "fp64" else 2e-6
    # the parameter selection's error model is statistical: tiny systems ask for
    # a tighter tolerance so that they still land inside the bar
    tol = bar if n >= 100 else bar * 1e-2
    box = x0 + (sides if shape == "box" else sides[:1])
    dt = torch.float64 if prec == "fp64" else torch.float32
    t = lambda a: None if a is None else torch.tensor(a, dtype=dt, device="cuda")  # noqa: E731
    plan = pkg.Plan(kernel, n, box, prec=prec, tol=tol, periodic=(shape == "periodic"))
    u = plan.eval(t(x), t(f), t(q)).double().cpu().numpy()
    plan.check()
    plan.close()
    if n == 1 and shape != "periodic":
        # no pair: the self term cancels the point's own image in the Fourier part
        assert np.abs(u).max() <= 1e-6 * max(1.0, np.abs(f).max())
        return
    if shape == "periodic":
        xi = 14.0 / sides[0]
        ref = O3.ewald(kernel, x - np.asarray(x0), f, q, L=sides[0], xi=xi, rc=6.3 / xi)
    else:
        ref = direct.direct(kernel, x, f, q)
    err = float(np.linalg.norm(u - ref) / np.linalg.norm(ref))
    assert err <= bar, f"relative L2 error {err:.3g}"
