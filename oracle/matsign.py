"""Matrix sign function of a dense matrix (test infrastructure, oracle only).

Definition (Section 1, Eq. 1 and the line after it): for diagonalizable A = R Lambda R^-1,
f(A) = R f(Lambda) R^-1, and sign(z) = sign(Re z). The paper names two ways to evaluate
f on a small matrix (Section 2, after Eq. bloch_approx): an eigendecomposition, and
Roberts' Newton iteration X <- (X + X^-1)/2; the Newton form here uses determinantal
scaling (Higham, Functions of Matrices, Ch. 5), which the paper's reference covers.
"""
from __future__ import annotations

import numpy as np


class IllPosed(ValueError):
    """An eigenvalue lies (numerically) on the imaginary axis, where sign is undefined."""


def sign_eig(a: np.ndarray, b: np.ndarray | None = None, ill_tol: float = 1e-8):
    """sign(A) (or sign(A) b) as R diag(sign Re lambda) R^-1."""
    w, r = np.linalg.eig(a)
    scale = np.max(np.abs(w))
    if np.min(np.abs(w.real)) < ill_tol * scale:
        raise IllPosed("eigenvalue with |Re lambda| < %g max|lambda|" % ill_tol)
    s = np.sign(w.real)
    if b is None:
        return (r * s) @ np.linalg.inv(r)
    y = np.linalg.solve(r, b)
    return r @ (s[:, None] * y if y.ndim == 2 else s * y)


def sign_newton(a: np.ndarray, tol: float = 1e-14, maxit: int = 100):
    """sign(A) by Roberts' Newton iteration with determinantal scaling.

    X_0 = A;  X_{k+1} = (zeta_k X_k + (zeta_k X_k)^-1) / 2,  zeta_k = |det X_k|^(-1/n)
    while the relative change exceeds 1e-2, unscaled afterwards; stops when the relative
    change in the Frobenius norm drops below tol or stops decreasing.
    Returns (S, iterations).
    """
    x = np.array(a, dtype=np.complex128)
    n = x.shape[0]
    prev_change = np.inf
    scaling = True
    for it in range(1, maxit + 1):
        xinv = np.linalg.inv(x)
        if scaling:
            _, logdet = np.linalg.slogdet(x)
            zeta = np.exp(-logdet / n)
        else:
            zeta = 1.0
        xn = 0.5 * (zeta * x + xinv / zeta)
        change = np.linalg.norm(xn - x) / np.linalg.norm(xn)
        x = xn
        if change < 1e-2:
            scaling = False
        if change < tol or (not scaling and change >= prev_change and change < 1e-10):
            return x, it
        prev_change = change
    return x, maxit


def sign_hermitian(a: np.ndarray, b: np.ndarray | None = None):
    """sign(A) for Hermitian A via eigh: A (A^2)^(-1/2)."""
    w, q = np.linalg.eigh(a)
    s = np.sign(w)
    if b is None:
        return (q * s) @ np.conj(q).T
    return q @ (s * (np.conj(q).T @ b))
