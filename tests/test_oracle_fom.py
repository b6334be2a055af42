"""Pins of the restarted FOM-LR oracle (Algorithm 1, oracle/fom.py), against what the mathematics
fixes: the Arnoldi relation and orthonormality, the FOM iterate's definition and the collinearity
of the shifted residuals (Eq. collinearity), convergence of the restarted iterates to dense
shifted solves and to the dense rational function, and the sign within Theorem 1's bound."""
import numpy as np
import pytest

import synth
from oracle import deflation, fom, lanczos, rational


@pytest.fixture(scope="module")
def small():
    dims = (2, 2, 4, 4)  # n = 768
    u = synth.gauge_links(dims, 12)
    h = deflation.sparse_hw(u, dims, -2.0, 0.3).toarray()  # dense: a = h @ h is formed explicitly
    b = synth.gaussian_source(dims, 13).ravel()
    return dims, u, h, b


def test_arnoldi_relation(small):
    _, _, h, b = small
    a = h @ h
    V, H = fom.arnoldi(lambda v: a @ v, b / np.linalg.norm(b), 25)
    assert np.abs(np.conj(V).T @ V - np.eye(V.shape[1])).max() < 1e-12
    assert np.abs(a @ V[:, :25] - V @ H).max() < 1e-12 * np.abs(a).max()
    assert np.all(np.diag(H, -1) > 0) and np.abs(np.tril(H, -2)).max() == 0.0


def test_fom_iterate_and_collinear_residuals(small):
    """One cycle: x^(i) = V_k (H_k - sigma_i)^-1 beta e_1 and b - (A - sigma_i) x^(i) = rho_i v_{k+1}
    with rho_i = -h_{k+1,k} e_k^T y_i."""
    _, _, h, b = small
    a = h @ h
    sig = np.array([-0.01, -0.3, -2.0])
    om = np.array([1.0, 0.5, 0.25])
    k = 20
    x, info = fom.fom_lr(lambda v: a @ v, b, om, sig, k, tol=0.0, max_cycles=1)
    V, H = fom.arnoldi(lambda v: a @ v, b / np.linalg.norm(b), k)
    e1 = np.zeros(k)
    e1[0] = 1.0
    for i in range(3):
        y = np.linalg.norm(b) * np.linalg.solve(H[:k, :k] - sig[i] * np.eye(k), e1)
        xi = V[:, :k] @ y
        assert np.linalg.norm(info["xs"][i] - xi) < 1e-12 * np.linalg.norm(xi)
        res = b - (a @ xi - sig[i] * xi)
        assert np.linalg.norm(res - info["rho"][i] * V[:, k]) < 1e-11 * np.linalg.norm(b)
    assert np.linalg.norm(x - om @ info["xs"]) < 1e-12 * np.linalg.norm(x)


@pytest.mark.parametrize("k", [8, 30])
def test_restarted_converges_to_dense_solves(small, k):
    _, _, h, b = small
    a = h @ h
    sig = np.array([-0.005, -0.1, -1.5, -9.0])
    om = np.array([0.3, 1.0, 2.0, 0.7])
    x, info = fom.fom_lr(lambda v: a @ v, b, om, sig, k, tol=1e-12, max_cycles=5000)
    assert info["converged"] and info["cycles"] > 1
    n = a.shape[0]
    for i in range(4):
        xd = np.linalg.solve(a - sig[i] * np.eye(n), b)
        assert np.linalg.norm(info["xs"][i] - xd) < 1e-9 * np.linalg.norm(xd)
    xg = sum(om[i] * np.linalg.solve(a - sig[i] * np.eye(n), b) for i in range(4))
    assert np.linalg.norm(x - xg) < 1e-9 * np.linalg.norm(xg)


def test_sign_fom_lr_vs_dense_rational_and_xstar(problem_4444):
    """4^4, mu = 0.3, Neuberger poles for the spectrum: restarted FOM on H^2 with k = 30 gives the
    dense g(H) b, which is within Theorem 1's bound (times the eigenvector condition) of x*."""
    p = problem_4444
    h = p["h"]
    hs = deflation.sparse_hw(p["links"], p["dims"], -2.0, 0.3)
    ev = p["eig"]
    lo, hi = 0.99 * np.abs(ev).min(), 1.01 * np.abs(ev).max()
    eps = 1e-8
    s, c, w, sg = rational.neuberger_for_spectrum(lo, hi, eps)
    x, info = fom.sign_fom_lr(lambda v: (hs @ v.ravel()).reshape(v.shape), p["b"], w, sg, 30, tol=1e-11)
    assert info["converged"]
    xg = lanczos.rational_sign_dense(h, p["b"].ravel(), w, sg)
    assert np.linalg.norm(x.ravel() - xg) < 1e-9 * np.linalg.norm(xg)
    assert np.linalg.norm(x - p["xstar"]) < 1e-6 * np.linalg.norm(p["xstar"])


def test_sign_fom_lr_with_deflation(problem_4444):
    """16 deflated eigenpairs: x_P exact on the deflated part, the rational part on (I - P) b with the
    projection step after every cycle; same dense result, fewer cycles (a larger gap)."""
    p = problem_4444
    hs = deflation.sparse_hw(p["links"], p["dims"], -2.0, 0.3)
    ev = p["eig"]
    hi = 1.01 * np.abs(ev).max()
    eps = 1e-8
    s, c, w, sg = rational.neuberger_for_spectrum(0.99 * p["gap16"], hi, eps)
    x, info = fom.sign_fom_lr(lambda v: (hs @ v.ravel()).reshape(v.shape), p["b"], w, sg, 30, tol=1e-11,
                              R=p["R16"], L=p["L16"], lam=p["lam16"])
    assert info["converged"]
    _, _, w0, sg0 = rational.neuberger_for_spectrum(0.99 * np.abs(ev).min(), hi, eps)
    _, info0 = fom.sign_fom_lr(lambda v: (hs @ v.ravel()).reshape(v.shape), p["b"], w0, sg0, 30, tol=1e-11)
    assert info["cycles"] < info0["cycles"]
    assert np.linalg.norm(x - p["xstar"]) < 1e-6 * np.linalg.norm(p["xstar"])
