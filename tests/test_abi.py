"""The C ABI without a GPU: libhrebsd.so builds and loads, exports every function that
include/hrebsd.h declares, and its host-only calls behave as documented (no kernel runs here).

The Gaussian of the field regularisation is pinned here: its FP32 taps must sum to exactly one
(a sum a few 1e-8 short would shrink the whole field by that much at every smoothing pass, a
systematic error that accumulates over the iterations of a level), be symmetric, and stay close to
the normalised weights exp(-k^2 / 2 sigma^2) / sum: each outer tap within half a unit in the last
place of the centre tap, the centre tap (which takes up their rounding) within r such units."""
import ctypes as C
import math
import os
import re

import numpy as np
import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module")
def P():
    import paper_1907_05993_gb300 as P
    P.load()
    return P


def declared_functions():
    src = open(os.path.join(ROOT, "include", "hrebsd.h")).read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    names = re.findall(r"^(?:int|long long|const char \*)\s*\*?\s*(hrebsd_\w+)\s*\(", src, flags=re.M)
    assert len(names) >= 30, names
    return sorted(set(names))


def test_every_declared_function_is_exported(P):
    lib = C.CDLL(P._build.LIB)
    missing = [n for n in declared_functions() if not hasattr(lib, n)]
    assert not missing, missing


def test_binding_covers_the_abi(P):
    lib = P.load()
    for n in declared_functions():
        f = getattr(lib, n)
        assert f.argtypes is not None, f"{n} has no ctypes signature in the binding"


def test_status_strings(P):
    lib = P.load()
    for code in (0, -1, -2, -3, -4, -5, -6, -7):
        s = lib.hrebsd_status_string(code).decode()
        assert s and s != "unknown status", code
    assert lib.hrebsd_status_string(-99).decode() == "unknown status"


@pytest.mark.parametrize("sigma", [0.4, 0.7, 1.0, 1.3, 1.6, 2.0])
def test_gauss_taps_sum_exactly_one(P, sigma):
    t = P.hrebsd_gauss_taps(sigma)
    r = math.ceil(3 * sigma)
    assert t.dtype == np.float32 and t.size == 2 * r + 1
    assert np.array_equal(t, t[::-1])
    assert math.fsum(float(x) for x in t) == 1.0          # exact sum of the FP32 values
    k = np.arange(-r, r + 1)
    s32 = float(np.float32(sigma))   # the ABI takes sigma in FP32
    w = np.exp(-k * k / (2 * s32 * s32))
    w /= w.sum()
    ulp0 = float(np.spacing(np.float32(w[r])))
    dev = np.abs(t - w) / ulp0
    # outer taps: rounded to a quantum of at most one unit of the centre tap; the centre tap takes
    # up the sum of their rounding errors
    assert np.all(np.delete(dev, r) <= 0.5 + 1e-9) and dev[r] <= r + 1e-9, dev


def test_gauss_taps_identity_and_limits(P):
    assert np.array_equal(P.hrebsd_gauss_taps(0.0), np.ones(1, np.float32))
    with pytest.raises(P.HrebsdError):
        P.hrebsd_gauss_taps(2.5)   # radius 8 > 6


def test_create_fails_loudly_without_a_gpu(P):
    import torch
    if torch.cuda.is_available():
        pytest.skip("a GPU is present")
    with pytest.raises(P.HrebsdError):
        P.hrebsd_create(0)
