"""The host search behind the tau and slice-level selections (csrc/search.h):
from every starting guess it returns the first index of a monotone predicate,
as a bisection from scratch does, in a logarithmic number of evaluations."""
import ctypes
import math
import os
import subprocess

import numpy as np
import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
HDR = os.path.join(ROOT, "paper_2005_10680_gb300", "csrc")

SHIM = r"""
#include "search.h"
extern "C" int first_true(int n, int hint, const unsigned char* truth, int fail_at,
                          int* answer, double* at, int* evals) {
    return hinted_first_true(
        n, hint,
        [&](int k, bool* p, double* v) -> int {
            if (k == fail_at) return 7;
            *p = truth[k] != 0;
            *v = 10.0 * k;
            return 0;
        },
        answer, at, evals);
}
"""


@pytest.fixture(scope="module")
def lib(tmp_path_factory):
    d = tmp_path_factory.mktemp("search")
    src = d / "shim.cpp"
    src.write_text(SHIM)
    so = d / "shim.so"
    subprocess.check_call(["g++", "-std=c++17", "-O1", "-shared", "-fPIC", "-I", HDR, "-o", str(so),
                           str(src)])
    L = ctypes.CDLL(str(so))
    L.first_true.argtypes = [ctypes.c_int, ctypes.c_int, ctypes.POINTER(ctypes.c_ubyte), ctypes.c_int,
                             ctypes.POINTER(ctypes.c_int), ctypes.POINTER(ctypes.c_double),
                             ctypes.POINTER(ctypes.c_int)]
    return L


def _run(lib, truth, hint, fail_at=-1):
    t = np.ascontiguousarray(truth, dtype=np.uint8)
    ans, at, ev = ctypes.c_int(-1), ctypes.c_double(-1.0), ctypes.c_int(0)
    st = lib.first_true(len(t), hint, t.ctypes.data_as(ctypes.POINTER(ctypes.c_ubyte)), fail_at,
                        ctypes.byref(ans), ctypes.byref(at), ctypes.byref(ev))
    return st, ans.value, at.value, ev.value


@pytest.mark.parametrize("n", [1, 2, 3, 7, 8, 9, 31, 64, 350])
def test_first_true_from_every_hint(lib, n):
    cap = 2 * math.ceil(math.log2(n + 1)) + 2
    for t in sorted({0, 1, n // 3, n // 2, n - 1, n}):
        truth = np.arange(n) >= t
        for hint in sorted({0, 1, t - 1, t, t + 1, n // 2, n - 1}):
            if not 0 <= hint < n:
                continue
            st, ans, at, ev = _run(lib, truth, hint)
            assert st == 0 and ans == t
            assert at == (10.0 * t if t < n else -1.0)
            assert ev <= cap
            if hint == t and 0 < t < n:
                assert ev == 2     # the guess and its neighbour settle it


def test_out_of_range_hints_and_errors(lib):
    truth = np.arange(20) >= 13
    assert _run(lib, truth, -5)[1] == 13
    assert _run(lib, truth, 99)[1] == 13
    st, ans, _, _ = _run(lib, truth, 5, fail_at=5)   # the guess is always evaluated
    assert st == 7 and ans == -1      # an evaluation error is returned, no answer
