"""The solver's stopping rules on the host (no GPU): the mixed solve's inner
tolerance per refinement step and the Krylov loop's stopping rule with its
stagnation exit, through the library's test hooks (include/nlh_selftest.h),
against the rules as include/nlh.h states them."""
import ctypes as C

import numpy as np
import pytest

from paper_2407_06834_gb300 import nlh


@pytest.fixture(scope="module")
def lib():
    return nlh.load()


def test_fixed_inner_tolerance(lib):
    f = lib.nlh_selftest_inner_tolerance
    tol = 1e-6
    # a step that cannot end the solve runs to the caller's tolerance
    assert f(1e-3, tol, 1.0) == 1e-3
    assert f(1e-3, tol, 3e-3) == 1e-3          # tol / (2 rel) = 1.7e-4 < 1e-3 / 4
    # one that can runs to exactly tol / (2 rel) (capped at 0.1)
    assert f(1e-3, tol, 2e-3) == pytest.approx(2.5e-4, rel=1e-15)
    assert f(1e-3, tol, 1e-3) == pytest.approx(5e-4, rel=1e-15)
    assert f(1e-3, tol, 2e-6) == 0.1
    # the reach test's 1e-4 floor binds for small inner tolerances
    assert f(1e-5, tol, 1e-2) == 1e-5          # tol / (2 rel) = 5e-5 < 1e-4
    assert f(1e-5, tol, 4e-3) == pytest.approx(1.25e-4, rel=1e-15)


def test_automatic_inner_tolerance(lib):
    f = lib.nlh_selftest_inner_tolerance
    tol = 1e-6
    assert f(0.0, tol, 1.0) == pytest.approx(1e-6, rel=1e-15)   # the first step aims at tol
    assert f(-1.0, tol, 1.0) == pytest.approx(1e-6, rel=1e-15)  # any inner <= 0 is automatic
    assert f(0.0, tol, 1.8e-6) == 0.1                           # a short second step
    assert f(0.0, tol, 1e-4) == pytest.approx(1e-2, rel=1e-15)
    assert f(0.0, 1e-9, 1.0) == 1e-7                            # floor below the FP32 operator
    assert f(0.0, tol, 50.0) == 1e-7                            # a start worse than zero


def _stop(lib, rels, tol, maxit=200, stag=0):
    a = np.ascontiguousarray(rels, dtype=np.float64)
    return lib.nlh_selftest_convergence(a.ctypes.data_as(C.c_void_p), len(a), tol, maxit, stag)


def test_convergence_and_maxit(lib):
    geo = [0.5 ** k for k in range(40)]
    k = _stop(lib, geo, 1e-6)
    assert geo[k] <= 1e-6 < geo[k - 1]
    assert _stop(lib, geo, 1e-6, stag=3) == k    # healthy descent: the exit never fires
    assert _stop(lib, [1.0] * 10, 1e-6, maxit=4) == 4
    assert _stop(lib, [1.0] * 10, 1e-6) == -1
    assert _stop(lib, [1.0, float("nan"), 0.5], 1e-6) == 1


def test_stagnation_exit(lib):
    tol = 1e-6
    # falls to 2e-6 and stays there (the FP32 operator's floor)
    rels = [1.0, 1e-2, 1e-4, 1e-5, 3e-6, 2e-6, 2.1e-6, 1.9e-6, 2.05e-6, 1.95e-6, 2e-6]
    # best 2e-6 at k = 5 (a 33 % fall from 3e-6), then three iterations within 8 tol
    # without a 30 % fall: stop at k = 8
    assert _stop(lib, rels, tol, stag=3) == 8
    assert _stop(lib, rels, tol, stag=0) == -1   # without the exit it would run to maxit
    # a plateau above 8 tol (a pause of CG's descent) ends the solve only after 9
    # iterations without a fall: best 5e-5 at k = 2, stop at k = 11
    assert _stop(lib, [1.0, 1e-3] + [5e-5] * 20, tol, stag=3) == 11
    # a pause of 8 iterations above 8 tol, then descent: the exit does not fire
    pause = [1.0, 1e-2, 1e-4] + [9e-5] * 8 + [1e-5 * 0.5 ** k for k in range(12)]
    k = _stop(lib, pause, tol, stag=3)
    assert pause[k] <= tol
    # slow but steady progress (30 % every other iteration) is not stagnation
    slow = [1e-5 * 0.69 ** (k // 2) for k in range(40)]
    k = _stop(lib, slow, tol, stag=3)
    assert slow[k] <= tol
    # an empty or invalid history
    assert _stop(lib, [], tol, stag=3) == -1
    assert lib.nlh_selftest_convergence(None, 3, tol, 200, 3) == -2
