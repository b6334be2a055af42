"""Plain C FP64 two-sided Lanczos (Algorithm 4) for any lattice size — TEST INFRASTRUCTURE ONLY.

The CPU counterpart of the whole direct method at sizes where no dense x* exists (8^4 to 16^4):
``krylov.c`` holds the matrix-free H_W(mu) (the definition with full 4x4 spin and 3x3 colour
products) and the two-sided Lanczos recurrence of Section 2.2; this module adds the deflation split
x_P, r, r~ of Algorithm 4 (``lanczos.deflation_vectors``), the small sign(H_k) e_1 by
eigendecomposition (``lanczos.sign_tridiag_e1``) and the combine x = x_P + beta V_k y. The shared
library is compiled with gcc (OpenMP over sites, no FMA contraction) on first use, or by
``build_lib()``; it is not part of the CUDA library and shares no code with it.

Pins (tests/test_oracle_krylov.py): the C operator equals ``deflation.sparse_hw`` (itself pinned
by three constructions, gamma5-hermiticity, gauge covariance and the free spectrum) and the free
field closed form; the recurrence coefficients equal ``lanczos.two_sided_lanczos`` at equal k; the
solve converges to the dense x* at 4^4.
"""
from __future__ import annotations

import ctypes
import os
import platform
import subprocess
import time

import numpy as np

from .lanczos import deflation_vectors, sign_tridiag_e1

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "krylov.c")
_LIB = os.path.join(_HERE, "_build", "libovlref-%s.so" % platform.machine())
_lib = None


def build_lib(force: bool = False) -> str:
    """Compile krylov.c into a shared library (gcc, -O2 -fopenmp, no FMA contraction so that the
    arithmetic is the same on every host)."""
    if force or not os.path.exists(_LIB) or os.path.getmtime(_LIB) < os.path.getmtime(_SRC):
        os.makedirs(os.path.dirname(_LIB), exist_ok=True)
        tmp = _LIB + ".%d.tmp" % os.getpid()
        cmd = ["gcc", "-O2", "-std=c11", "-fopenmp", "-fPIC", "-shared", "-ffp-contract=off",
               "-fcx-limited-range", _SRC, "-o", tmp, "-lm"]
        r = subprocess.run(cmd, capture_output=True, text=True)
        if r.returncode != 0:
            raise RuntimeError("oracle build failed: %s\n%s" % (" ".join(cmd), r.stderr))
        os.replace(tmp, _LIB)
    return _LIB


def _load():
    global _lib
    if _lib is None:
        lib = ctypes.CDLL(build_lib())
        P, I, D, L = ctypes.c_void_p, ctypes.c_int32, ctypes.c_double, ctypes.c_long
        lib.ovlref_threads.restype = ctypes.c_int
        lib.ovlref_threads.argtypes = [ctypes.c_int]
        lib.ovlref_apply_hw.restype = None
        lib.ovlref_apply_hw.argtypes = [P, I, D, D, P, P, P]
        lib.ovlref_lanczos_start.restype = ctypes.c_int
        lib.ovlref_lanczos_start.argtypes = [L, P, P, P, P, P]
        lib.ovlref_lanczos_steps.restype = ctypes.c_int
        lib.ovlref_lanczos_steps.argtypes = [P, I, D, D, P, L, ctypes.c_int, P, P, P, P, P, P, P, P, ctypes.c_int]
        lib.ovlref_combine.restype = None
        lib.ovlref_combine.argtypes = [L, ctypes.c_int, P, P, D, P]
        _lib = lib
    return _lib


def _c(a):
    return a.ctypes.data


def threads(n: int = 0) -> int:
    """Set (n > 0) and return the number of OpenMP threads the C oracle uses."""
    return int(_load().ovlref_threads(int(n)))


def apply_hw(links, dims, m_w, mu, psi, t_bc=-1):
    """H_W(mu) psi (canonical layouts) by the C operator."""
    lib = _load()
    u = np.ascontiguousarray(links, dtype=np.complex128)
    p = np.ascontiguousarray(psi, dtype=np.complex128)
    out = np.empty_like(p)
    d = np.array(dims, dtype=np.int32)
    lib.ovlref_apply_hw(_c(d), int(t_bc), float(m_w), float(mu), _c(u), _c(p), _c(out))
    return out


class DirectSolve:
    """Algorithm 4 for one right-hand side, advanced in pieces: ``start()``, then ``steps(m)``
    until k steps are done, then ``finish()`` -> x. Memory: the basis V_k (k n complex128)."""

    def __init__(self, links, dims, m_w, mu, b, k, t_bc=-1, R=None, L=None, lam=None):
        self.lib = _load()
        self.u = np.ascontiguousarray(links, dtype=np.complex128).reshape(-1)
        self.dims = np.array(dims, dtype=np.int32)
        self.shape = b.shape
        self.n = b.size
        self.m_w, self.mu, self.t_bc, self.kcap = float(m_w), float(mu), int(t_bc), int(k)
        self.b = np.ascontiguousarray(b, dtype=np.complex128).reshape(-1)
        self.R, self.L, self.lam = R, L, lam
        self.k = 0
        self.breakdown = False
        self.empty = False

    def start(self):
        n, k = self.n, self.kcap
        self.xp, r, rt = deflation_vectors(self.b, self.R, self.L, self.lam)
        r = np.ascontiguousarray(r)
        rt = np.ascontiguousarray(rt)
        self.V = np.empty((k, n), dtype=np.complex128)
        self.W = np.empty((2, n), dtype=np.complex128)
        self.av = np.empty(n, dtype=np.complex128)
        self.aw = np.empty(n, dtype=np.complex128)
        self.alpha = np.zeros(k, dtype=np.complex128)
        self.beta = np.zeros(k, dtype=np.complex128)
        self.delta = np.zeros(k, dtype=np.complex128)
        b0 = ctypes.c_double(0.0)
        st = self.lib.ovlref_lanczos_start(n, _c(r), _c(rt), _c(self.V), _c(self.W), ctypes.byref(b0))
        self.beta0 = b0.value
        self.empty = st != 0
        return self

    def steps(self, m: int) -> int:
        """Advance by up to m steps; returns the steps done so far."""
        if self.empty or self.breakdown or self.k >= self.kcap or m <= 0:
            return self.k
        kio = ctypes.c_int(self.k)
        st = self.lib.ovlref_lanczos_steps(_c(self.dims), self.t_bc, self.m_w, self.mu, _c(self.u), self.n,
                                           self.kcap, _c(self.V), _c(self.W), _c(self.av), _c(self.aw),
                                           _c(self.alpha), _c(self.beta), _c(self.delta), ctypes.byref(kio),
                                           int(m))
        self.k = kio.value
        self.breakdown = st != 0
        return self.k

    def finish(self):
        """x = x_P + beta V_k sign(H_k) e_1 (eigendecomposition of H_k)."""
        x = self.xp.astype(np.complex128).copy()
        k = self.k
        if self.empty or k == 0:
            self.y = np.zeros(0, dtype=np.complex128)
            return x.reshape(self.shape)
        self.y = np.ascontiguousarray(sign_tridiag_e1(self.alpha[:k], self.beta[:k - 1], self.delta[:k - 1]))
        self.lib.ovlref_combine(self.n, k, _c(self.V), _c(self.y), self.beta0, _c(x))
        return x.reshape(self.shape)


def direct_lanczos(links, dims, m_w, mu, b, k, t_bc=-1, R=None, L=None, lam=None):
    """Algorithm 4 with exactly k steps (fewer on breakdown). Returns (x, solve, seconds)."""
    t0 = time.perf_counter()
    s = DirectSolve(links, dims, m_w, mu, b, k, t_bc, R, L, lam).start()
    s.steps(k)
    x = s.finish()
    return x, s, time.perf_counter() - t0
