"""Restarted FOM-LR(m, k) with a rational function (Algorithm 1, Section 4.1) — TEST INFRASTRUCTURE ONLY.

For f(t) = sum_i omega_i / (t - sigma_i) (Eq. rational_function) the action f(A) b is
sum_i omega_i x^(i) with (A - sigma_i) x^(i) = b (Eqs. schaefer_approx, multishift_eq). One Arnoldi
basis V_k, H_k of K_k(A, r) serves every shift: the FOM iterates are x_k^(i) = V_k (H_k - sigma_i)^-1
beta e_1 (Eq. rat_arnoldi), and their residuals are all multiples of v_{k+1} (Eq. collinearity):
r_k^(i) = rho_k^(i) v_{k+1}. So after k steps the remaining error is again a rational function of A,
with the same poles, applied to v_{k+1} - a restart with new weights rho^(i) and no instability.

Algorithm 1 in the paper's order, with LR deflation (P = R L^H, x_P = R f(Lambda) L^H b):
    x = x_P;  r = (I - P) b;  rho_i = 1
    while not all systems converged:
        beta = ||r||;  v_1 = r / beta;  k Arnoldi steps -> V_k, H_k, h_{k+1,k}, v_{k+1}
        y_i = beta rho_i (H_k - sigma_i I)^-1 e_1;  x += V_k sum_i omega_i y_i
        r = v_{k+1};  rho_i = -h_{k+1,k} e_k^T y_i;  r = (I - P) r        (projection step)
System i has converged when its residual |rho_i| ||r|| is at most tol times the first ||r||.

The sign function (Section 5): sign(H) b ~ H g(H) ... with g(t) = sum_i omega_i/(t^2 - sigma_i), i.e.
the algorithm above on A = H^2 for (I - P) b, then x = x_P + H X with x_P = R sign(Lambda) L^H b
(eigenvectors of H are eigenvectors of H^2, so the same P deflates both).

Arnoldi here is the textbook modified Gram-Schmidt process (the paper only says "k steps of
Arnoldi"); h_{j+1,j} = ||w|| > 0, so V_{k+1} and H_k are unique.

Pins (tests/test_oracle_fom.py): Arnoldi relation and orthonormality; FOM iterate = definition and
the residuals collinear with v_{k+1}; restarted iterates converge to the dense shifted solves and to
the dense g(A) b, with and without deflation; sign within Theorem 1's bound of x*.
"""
from __future__ import annotations

import numpy as np


def arnoldi(apply_a, v1, k):
    """k steps of Arnoldi (modified Gram-Schmidt) from the unit vector v1.
    Returns V (n x (k+1), columns v_1..v_{k+1}) and Hbar ((k+1) x k); fewer columns on a lucky
    breakdown (invariant subspace: h_{j+1,j} = 0)."""
    n = v1.size
    V = np.zeros((n, k + 1), dtype=np.complex128)
    H = np.zeros((k + 1, k), dtype=np.complex128)
    V[:, 0] = v1
    for j in range(k):
        w = apply_a(V[:, j])
        for i in range(j + 1):
            H[i, j] = np.vdot(V[:, i], w)
            w = w - H[i, j] * V[:, i]
        h = np.linalg.norm(w)
        H[j + 1, j] = h
        if h == 0.0:
            return V[:, :j + 1], H[:j + 2, :j + 1]
        V[:, j + 1] = w / h
    return V, H


def _project(r, R, L):
    """(I - P) r with P = R L^H."""
    if R is None or R.shape[1] == 0:
        return r
    return r - R @ (np.conj(L).T @ r)


def fom_lr(apply_a, b, omega, sigma, k, tol, max_cycles=1000, R=None, L=None, f_lam=None):
    """Algorithm 1: x ~ f(A) b, f(t) = sum_i omega_i/(t - sigma_i). With deflation, R, L are the
    n x m right/left eigenvectors (L^H R = I) and f_lam the m values f(lambda_j) for x_P.
    Returns (x, info) with info: cycles, matvecs, rho (last collinearity factors), xs (the s
    shifted solutions x^(i), accumulated like x), converged."""
    b = b.ravel().astype(np.complex128)
    omega = np.asarray(omega, dtype=np.float64)
    sigma = np.asarray(sigma, dtype=np.float64)
    s = len(sigma)
    if R is not None and R.shape[1] > 0:
        x = R @ (np.asarray(f_lam) * (np.conj(L).T @ b))
    else:
        x = np.zeros_like(b)
    xs = np.zeros((s, b.size), dtype=np.complex128)
    r = _project(b, R, L)
    r0 = np.linalg.norm(r)
    rho = np.ones(s, dtype=np.complex128)
    matvecs = 0
    cycles = 0
    converged = r0 == 0.0
    while not converged and cycles < max_cycles:
        beta = np.linalg.norm(r)
        V, H = arnoldi(apply_a, r / beta, k)
        kk = H.shape[1]
        matvecs += kk
        e1 = np.zeros(kk, dtype=np.complex128)
        e1[0] = 1.0
        ys = np.array([beta * rho[i] * np.linalg.solve(H[:kk, :kk] - sigma[i] * np.eye(kk), e1) for i in range(s)])
        x = x + V[:, :kk] @ (omega @ ys)
        xs = xs + ys @ V[:, :kk].T
        cycles += 1
        if V.shape[1] == kk:  # lucky breakdown: the Krylov space is invariant, the iterates are exact
            rho[:] = 0.0
            converged = True
            break
        rho = -H[kk, kk - 1] * ys[:, kk - 1]
        r = _project(V[:, kk], R, L)
        converged = bool(np.all(np.abs(rho) * np.linalg.norm(r) <= tol * r0))
    return x, {"cycles": cycles, "matvecs": matvecs, "rho": rho, "xs": xs, "converged": converged}


def sign_fom_lr(apply_h, b, omega, sigma, k, tol, max_cycles=1000, R=None, L=None, lam=None):
    """sign(H) b ~ x_P + H sum_i omega_i (H^2 - sigma_i)^-1 (I - P) b by Algorithm 1 on A = H^2
    (Section 5's g with sigma_i < 0). Returns (x, info) with info as fom_lr's."""
    shape = b.shape
    bf = b.ravel().astype(np.complex128)
    h = lambda v: apply_h(v.reshape(shape)).ravel()
    xp = np.zeros_like(bf)
    if R is not None and R.shape[1] > 0:
        xp = R @ (np.sign(np.real(lam)) * (np.conj(L).T @ bf))
    X, info = fom_lr(lambda v: h(h(v)), bf, omega, sigma, k, tol, max_cycles, R=R, L=L,
                     f_lam=np.zeros(R.shape[1]) if R is not None and R.shape[1] > 0 else None)
    info["matvecs"] *= 2
    return (xp + h(X)).reshape(shape), info
