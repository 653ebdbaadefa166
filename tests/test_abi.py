"""The C-ABI library loads and exports every function include/*.h declares, and
its host-only entry points behave (no GPU needed)."""
from __future__ import annotations

import ctypes
import glob
import os
import re

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module")
def libse():
    from paper_1607_04808_gb300 import _build
    path = _build.build()
    return ctypes.CDLL(path)


def declared_functions():
    names = set()
    for h in glob.glob(os.path.join(ROOT, "include", "*.h")):
        src = open(h).read()
        src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
        for m in re.finditer(r"^\s*(?:const\s+)?[A-Za-z_][A-Za-z0-9_ ]*\*?\s*\**\s*\b(se_[a-z0-9_]+)\s*\(",
                             src, flags=re.M):
            names.add(m.group(1))
    return sorted(names)


def test_header_declares_the_boundary():
    names = declared_functions()
    for n in ("se_plan_create", "se_eval", "se_eval_backward", "se_plan_destroy",
              "se_plan_get_params", "se_last_error"):
        assert n in names


def test_every_declared_symbol_is_exported(libse):
    missing = [n for n in declared_functions() if not hasattr(libse, n)]
    assert not missing, missing


def test_version_and_error_strings(libse):
    libse.se_version.restype = ctypes.c_char_p
    assert b"sm_103a" in libse.se_version()
    libse.se_last_error.restype = ctypes.c_char_p
    assert isinstance(libse.se_last_error(), bytes)


def test_choose_params_host_only():
    import paper_1607_04808_gb300 as P
    p = P.choose_params("stokeslet", 1_000_000, 1.0, 2e-6, "fp32", max_fft=256)
    assert p["P"] == 12 and 2 * (p["M"] + p["P"]) <= 256
    assert 30 < p["xi"] < 45 and 0.07 < p["rc"] < 0.11
    p64 = P.choose_params("stokeslet", 1_000_000, 1.0, 1e-10, "fp64")
    assert p64["P"] >= 20
    # overrides are kept
    p2 = P.choose_params("rotlet", 1000, 1.0, 1e-8, "fp64", xi=7.0, M=30)
    assert p2["xi"] == 7.0 and p2["M"] == 30
    # larger domain at the same density: rc and xi unchanged, M scales with L (Section 8.1)
    a = P.choose_params("stokeslet", 20000, 2.0, 1e-8, "fp64", xi=7.0)
    b = P.choose_params("stokeslet", 160000, 4.0, 1e-8, "fp64", xi=7.0)
    assert abs(a["rc"] - b["rc"]) < 0.05 * a["rc"]
    assert 1.8 < b["M"] / a["M"] < 2.2


def test_choose_params_rejects_bad_input():
    import paper_1607_04808_gb300 as P
    with pytest.raises(P.SEError):
        P.choose_params("stokeslet", 0, 1.0, 1e-6)
    with pytest.raises(P.SEError):
        P.choose_params("stokeslet", 10, -1.0, 1e-6)


def test_plan_create_fails_loudly_without_gpu():
    import torch
    if torch.cuda.is_available():
        pytest.skip("a GPU is present")
    import paper_1607_04808_gb300 as P
    with pytest.raises(P.SEError):
        P.Plan("stokeslet", 100)
