"""The direct method's stopping rule (csrc/stoprule.h) on the host: on an error that decays
geometrically, the rate-corrected estimate recovers the true remaining error and the predicted
stopping step; the evaluation schedule respects its clamps."""
import ctypes
import math
import os
import shutil
import subprocess
import tempfile

import pytest

HERE = os.path.dirname(os.path.abspath(__file__))


@pytest.fixture(scope="module")
def lib():
    cxx = shutil.which("g++") or shutil.which("c++")
    if cxx is None:
        pytest.skip("no host C++ compiler")
    d = tempfile.mkdtemp()
    so = os.path.join(d, "stoprule_check.so")
    subprocess.run([cxx, "-O2", "-std=c++17", "-shared", "-fPIC", os.path.join(HERE, "native", "stoprule_check.cpp"),
                    "-o", so], check=True)
    L = ctypes.CDLL(so)
    D, I = ctypes.c_double, ctypes.c_int
    L.feed_geometric.argtypes = [D, D, ctypes.POINTER(I), I, D, ctypes.POINTER(D), ctypes.POINTER(D),
                                 ctypes.POINTER(I), ctypes.POINTER(D)]
    L.next_eval.restype = I
    L.next_eval.argtypes = [I, I, D]
    L.due.restype = I
    L.due.argtypes = [I, I, I, I]
    yield L
    shutil.rmtree(d, ignore_errors=True)


def _feed(L, c, rho, ks, tol):
    arr = (ctypes.c_int * len(ks))(*ks)
    est, lr, pr = ctypes.c_double(), ctypes.c_double(), ctypes.c_double()
    cv = ctypes.c_int()
    L.feed_geometric(c, rho, arr, len(ks), tol, ctypes.byref(est), ctypes.byref(lr), ctypes.byref(cv),
                     ctypes.byref(pr))
    return est.value, lr.value, cv.value, pr.value


@pytest.mark.parametrize("spacing", ["equal", "growing"])
def test_estimate_recovers_geometric_error(lib, spacing):
    c, rho = 1.0, 0.98
    ks = [25, 50, 75, 100] if spacing == "equal" else [25, 50, 100, 150]
    est, log_rho, _, _ = _feed(lib, c, rho, ks, 1e-12)
    assert log_rho < 0
    true_err = c * rho ** ks[-1]
    if spacing == "equal":  # the rate is exact for equal spacings, so is the estimate
        assert math.isclose(log_rho, math.log(rho), rel_tol=1e-9)
        assert math.isclose(est, true_err, rel_tol=1e-9)
    else:  # mean-spacing rate: the right order of magnitude
        assert true_err / 3 < est < true_err * 3


def test_stops_and_predicts(lib):
    c, rho, tol = 1.0, 0.98, 1e-8
    # far from tol: no stop, and the prediction points at where C rho^k = tol / 2
    est, log_rho, cv, pred = _feed(lib, c, rho, [25, 50, 75, 100], tol)
    assert cv == 0
    k_target = math.log(0.5 * tol / c) / math.log(rho)
    assert math.isclose(100 + pred, k_target, rel_tol=1e-6)
    # past the point: stop
    k = int(k_target) + 50
    _, _, cv, pred = _feed(lib, c, rho, [k - 75, k - 50, k - 25, k], tol)
    assert cv == 1 and pred == 0.0


def test_no_rate_without_decrease(lib):
    # equal changes (no decay seen): no rate, the estimate is the change itself
    arr = (ctypes.c_int * 3)(25, 50, 75)
    est, lr, pr = ctypes.c_double(), ctypes.c_double(), ctypes.c_double()
    cv = ctypes.c_int()
    lib.feed_geometric(1.0, 1.0, arr, 3, 1e-8, ctypes.byref(est), ctypes.byref(lr), ctypes.byref(cv), ctypes.byref(pr))
    assert lr.value == 0.0 and pr.value == -1.0 and cv.value == 0


def test_schedule_clamps(lib):
    chunk = 25
    assert lib.next_eval(100, chunk, -1.0) == 125           # no rate: 1.25 k
    assert lib.next_eval(1000, chunk, 5.0) == 1025          # at least one chunk ahead
    assert lib.next_eval(1000, chunk, 2000.0) == 1500       # at most 1.5 k
    assert lib.next_eval(1000, chunk, 300.0) == 1300        # the prediction in between
    assert lib.due(500, 475, 0, 0) == 0 and lib.due(500, 500, 0, 0) == 1
    assert lib.due(500, 300, 1, 0) == 1 and lib.due(500, 300, 0, 1) == 1  # last snapshot, stopped on device
