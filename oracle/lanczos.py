"""Two-sided Lanczos approximations to f(A) b (test infrastructure, oracle only).

Direct two-sided Lanczos-LR(m, k), Algorithm 4, in the paper's order:
  x_P = R f(Lambda) L^H b;  r = b - R L^H b;  r~ = b - L R^H b   (modified shadow vector)
  v_1 = r / beta with beta = ||r||_2 (reading of "put v_1 = r"), w_1 = r~ scaled so that
  v_1^H w_1 = 1;  k steps of the two-sided Lanczos process (Eqs. 2sided1, 2sided2):
     A V_k = V_k H_k + h_{k+1,k} v_{k+1} e_k^T,  A^H W_k = W_k H_k^H + conj(h_{k,k+1}) w_{k+1} e_k^T,
  with W_k^H V_k = I and H_k = W_k^H A V_k tridiagonal;  x_k = x_P + beta V_k f(H_k) e_1
  (Eq. bloch_approx_unsym).
The split of each off-diagonal pair is not fixed by the paper; reading used:
  h_{j+1,j} = delta_j = sqrt(|w^H v|),  h_{j,j+1} = beta_j = (w^H v) / delta_j,
which reduces to Hermitian Lanczos (w_j = v_j) when A is Hermitian and r~ = r.

Multishift (Section 2.2 and Algorithm 3): for a rational f(t) = sum_i omega_i/(t - sigma_i)
the shifted iterates are x_k^(i) = beta V_k (H_k - sigma_i I)^-1 e_1 (the BiCG iterates of
(A - sigma_i) x = r). With the sign approximation g(t) = t sum_i omega_i/(t^2 - sigma_i) of
Section 5 the process runs on A^2 and x = x_P + A sum_i omega_i x^(i).
"""
from __future__ import annotations

import numpy as np

from .matsign import sign_eig


def _vdot(a, b):
    return np.vdot(a.ravel(), b.ravel())


def deflation_vectors(b, R=None, L=None, lam=None):
    """(x_P, r, r~) of Algorithm 4 (identity split when no deflation set is given)."""
    if R is None or R.shape[1] == 0:
        return np.zeros_like(b), b.copy(), b.copy()
    cl = np.conj(L).T @ b
    xp = R @ (np.sign(np.real(lam)) * cl)
    r = b - R @ cl
    rt = b - L @ (np.conj(R).T @ b)
    return xp, r, rt


def two_sided_lanczos(apply_a, apply_adag, r, rt, k):
    """k steps of two-sided Lanczos from (r, r~).

    Returns dict with beta0 = ||r||, V (n x k), alpha (k), beta (k-1, super-diagonal),
    delta (k-1, sub-diagonal), vnorm (k), breakdown step (or None).
    """
    n = r.size
    beta0 = np.linalg.norm(r)
    v = r.ravel() / beta0
    w = rt.ravel() / np.conj(_vdot(rt, v))  # v^H w = 1
    V = np.zeros((n, k), dtype=np.complex128)
    alpha = np.zeros(k, dtype=np.complex128)
    beta = np.zeros(max(k - 1, 0), dtype=np.complex128)
    delta = np.zeros(max(k - 1, 0), dtype=np.complex128)
    v_prev = np.zeros(n, dtype=np.complex128)
    w_prev = np.zeros(n, dtype=np.complex128)
    breakdown = None
    kk = k
    for j in range(k):
        V[:, j] = v
        av = apply_a(v)
        aw = apply_adag(w)
        alpha[j] = np.vdot(w, av)
        if j == k - 1:
            break
        bprev = beta[j - 1] if j > 0 else 0.0
        dprev = delta[j - 1] if j > 0 else 0.0
        vh = av - alpha[j] * v - bprev * v_prev
        wh = aw - np.conj(alpha[j]) * w - np.conj(dprev) * w_prev
        ip = np.vdot(wh, vh)
        if abs(ip) < 1e-14 * np.linalg.norm(vh) * np.linalg.norm(wh):
            breakdown = j + 1
            kk = j + 1
            break
        delta[j] = np.sqrt(abs(ip))
        beta[j] = ip / delta[j]
        v_prev, w_prev = v, w
        v = vh / delta[j]
        w = wh / np.conj(beta[j])
    return {
        "beta0": beta0,
        "V": V[:, :kk],
        "alpha": alpha[:kk],
        "beta": beta[: kk - 1],
        "delta": delta[: kk - 1],
        "breakdown": breakdown,
    }


def tridiag(alpha, beta, delta):
    """H_k with diagonal alpha, super-diagonal beta, sub-diagonal delta."""
    t = np.diag(np.asarray(alpha, dtype=np.complex128))
    if len(beta):
        t = t + np.diag(beta, 1) + np.diag(delta, -1)
    return t


def sign_tridiag_e1(alpha, beta, delta):
    """sign(H_k) e_1 by eigendecomposition (Eq. 1 on the projected matrix)."""
    t = tridiag(alpha, beta, delta)
    e1 = np.zeros(t.shape[0], dtype=np.complex128)
    e1[0] = 1.0
    return sign_eig(t, e1, ill_tol=0.0)


def direct_lanczos_lr(apply_a, apply_adag, b, k, R=None, L=None, lam=None):
    """Algorithm 4: returns (x_k, state) with b, x in the caller's shape."""
    shape = b.shape
    bf = b.ravel()
    xp, r, rt = deflation_vectors(bf, R, L, lam)
    st = two_sided_lanczos(lambda v: apply_a(v.reshape(shape)).ravel(),
                           lambda w: apply_adag(w.reshape(shape)).ravel(), r, rt, k)
    y = sign_tridiag_e1(st["alpha"], st["beta"], st["delta"])
    x = xp + st["beta0"] * (st["V"] @ y)
    st["y"] = y
    return x.reshape(shape), st


def multishift_iterates(apply_m, apply_mdag, r, rt, k, sigma):
    """x_k^(i) = beta V_k (H_k - sigma_i I)^-1 e_1 of two-sided Lanczos on M (Section 2.2)."""
    st = two_sided_lanczos(apply_m, apply_mdag, r.ravel(), rt.ravel(), k)
    t = tridiag(st["alpha"], st["beta"], st["delta"])
    kk = t.shape[0]
    e1 = np.zeros(kk, dtype=np.complex128)
    e1[0] = 1.0
    xs = []
    for sg in sigma:
        y = np.linalg.solve(t - sg * np.eye(kk), e1)
        xs.append(st["beta0"] * (st["V"] @ y))
    return np.array(xs), st


def bicg(apply_m, apply_mdag, rhs, shadow, sigma, k):
    """k steps of textbook BiCG (Fletcher 1976) for (M - sigma) x = rhs, shadow system with M^H."""
    x = np.zeros_like(rhs)
    r = rhs.copy()
    rt = shadow.copy()
    p = r.copy()
    pt = rt.copy()
    rho = np.vdot(rt, r)
    for _ in range(k):
        q = apply_m(p) - sigma * p
        qt = apply_mdag(pt) - np.conj(sigma) * pt
        a = rho / np.vdot(pt, q)
        x = x + a * p
        r = r - a * q
        rt = rt - np.conj(a) * qt
        rho_new = np.vdot(rt, r)
        bb = rho_new / rho
        rho = rho_new
        p = r + bb * p
        pt = rt + np.conj(bb) * pt
    return x


def rational_sign_dense(a_dense, b, omega, sigma):
    """g(A) b = A sum_i omega_i (A^2 - sigma_i)^-1 b (Section 5 form), dense solves."""
    a2 = a_dense @ a_dense
    n = a2.shape[0]
    acc = np.zeros_like(b, dtype=np.complex128)
    for w, sg in zip(omega, sigma):
        acc = acc + w * np.linalg.solve(a2 - sg * np.eye(n), b)
    return a_dense @ acc
