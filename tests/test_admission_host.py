"""The request server's admission policy (csrc/admission.h) on the host: least estimated work
first among the requests that fit the memory budget, the oldest first once it has waited too
long (and then nothing past it), nothing when nothing fits."""
import ctypes
import os
import shutil
import subprocess
import tempfile

import pytest

HERE = os.path.dirname(os.path.abspath(__file__))


@pytest.fixture(scope="module")
def pick():
    cxx = shutil.which("g++") or shutil.which("c++")
    if cxx is None:
        pytest.skip("no host C++ compiler")
    d = tempfile.mkdtemp()
    so = os.path.join(d, "admission_check.so")
    subprocess.run([cxx, "-O2", "-std=c++17", "-shared", "-fPIC", os.path.join(HERE, "native", "admission_check.cpp"),
                    "-o", so], check=True)
    L = ctypes.CDLL(so)
    D = ctypes.c_double
    L.pick.restype = ctypes.c_long
    L.pick.argtypes = [ctypes.POINTER(D), ctypes.POINTER(D), ctypes.c_long, D, D, D, D]

    def f(reqs, in_use, budget, waited=0.0, max_wait=2.0):
        n = len(reqs)
        fp = (D * max(n, 1))(*[r[0] for r in reqs])
        wk = (D * max(n, 1))(*[r[1] for r in reqs])
        return L.pick(fp, wk, n, in_use, budget, waited, max_wait)

    yield f
    shutil.rmtree(d, ignore_errors=True)


def test_least_work_first(pick):
    # (footprint, work) in arrival order
    reqs = [(100, 50.0), (100, 10.0), (100, 30.0)]
    assert pick(reqs, in_use=0, budget=1000) == 1


def test_only_what_fits(pick):
    reqs = [(100, 50.0), (900, 1.0), (100, 30.0)]
    assert pick(reqs, in_use=200, budget=1000) == 2  # the smallest work does not fit
    assert pick(reqs, in_use=950, budget=1000) == -1  # nothing fits


def test_oldest_first_after_max_wait(pick):
    reqs = [(500, 90.0), (100, 1.0)]
    assert pick(reqs, in_use=0, budget=1000, waited=3.0) == 0
    # the starving oldest does not fit yet: nothing is admitted past it
    assert pick(reqs, in_use=600, budget=1000, waited=3.0) == -1
    assert pick(reqs, in_use=600, budget=1000, waited=1.0) == 1


def test_empty_queue(pick):
    assert pick([], in_use=0, budget=1000) == -1
