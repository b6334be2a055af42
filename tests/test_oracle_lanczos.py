"""Pins for the oracle's Krylov methods and LR deflation (no GPU).

Two-sided Lanczos (Eqs. 2sided1/2): biorthogonality W^H V = I, H_k = W^H A V, the mu = 0
Hermitian limit (w_j = v_j, real symmetric T), exactness at k = n, convergence to the
eigendecomposition sign at 4^4 with deflation. Multishift (Section 2.2): V_k (H_k - sigma)^-1 e_1
equals textbook BiCG iterates and tends to the dense solve. LR deflation (Section 3): L^H R = I,
P^2 = P, Eq. exact_proj on eigenvector inputs, and the split of Eq. action.
"""
import numpy as np
import pytest

import synth
from oracle import deflation, lanczos, matsign, rational, wilson


def _ops(dims, seed, mu, t_bc=-1):
    u = synth.gauge_links(dims, seed)
    a = deflation.sparse_hw(u, dims, -2.0, mu, t_bc)
    ah = deflation.sparse_hw(u, dims, -2.0, -mu, t_bc)
    return u, a, ah


def _lanczos_with_w(a, ah, r, rt, k):
    """Re-run the oracle's recurrence keeping W, to check W^H V = I and H_k = W^H A V."""
    st = lanczos.two_sided_lanczos(lambda v: a @ v, lambda w: ah @ w, r, rt, k)
    v = st["V"]
    # rebuild w_j from A^H W = W H^H + ... : w_{j+1} = (A^H w_j - conj(a_j) w_j - conj(d_{j-1}) w_{j-1}) / conj(b_j)
    n, kk = v.shape
    w = np.zeros((n, kk), dtype=np.complex128)
    w[:, 0] = rt / np.conj(np.vdot(rt, v[:, 0]))
    for j in range(kk - 1):
        x = ah @ w[:, j] - np.conj(st["alpha"][j]) * w[:, j]
        if j > 0:
            x -= np.conj(st["delta"][j - 1]) * w[:, j - 1]
        w[:, j + 1] = x / np.conj(st["beta"][j])
    return st, v, w


def test_biorthogonality_and_projection():
    dims = (2, 2, 4, 4)
    _, a, ah = _ops(dims, 31, 0.3)
    b = synth.gaussian_source(dims, 32).ravel()
    st, v, w = _lanczos_with_w(a, ah, b, b, 30)
    k = v.shape[1]
    assert np.abs(np.conj(w).T @ v - np.eye(k)).max() < 1e-9
    t = lanczos.tridiag(st["alpha"], st["beta"], st["delta"])
    assert np.abs(np.conj(w).T @ (a @ v) - t).max() < 1e-9
    # delta_j = sqrt|w^H v| is real positive and |beta_j| = delta_j
    assert np.all(st["delta"].real > 0) and np.abs(st["delta"].imag).max() == 0
    assert np.abs(np.abs(st["beta"]) - st["delta"]).max() < 1e-12


def test_mu0_hermitian_limit():
    dims = (2, 2, 4, 4)
    _, a, ah = _ops(dims, 33, 0.0)
    b = synth.gaussian_source(dims, 34).ravel()
    st, v, w = _lanczos_with_w(a, ah, b, b, 25)
    assert np.abs(v - w).max() < 1e-10
    assert np.abs(st["alpha"].imag).max() < 1e-12
    assert np.abs(st["beta"] - st["delta"]).max() < 1e-12
    assert np.abs(np.conj(v).T @ v - np.eye(v.shape[1])).max() < 1e-9


@pytest.mark.parametrize("dims,eps", [((2, 2, 2, 2), 0.2), ((2, 2, 2, 4), 0.1)])
def test_exact_at_k_equal_n(dims, eps):
    """At k = n the Krylov space is the whole space and Algorithm 4 returns sign(A) b.

    Smooth links (small eps) keep |Re lambda| away from 0, so finite-precision loss of
    biorthogonality does not hide the exactness."""
    u = synth.gauge_links(dims, 35, eps)
    a = deflation.sparse_hw(u, dims, -2.0, 0.3)
    ah = deflation.sparse_hw(u, dims, -2.0, -0.3)
    b = synth.gaussian_source(dims, 36)
    xs = matsign.sign_eig(a.toarray(), b.ravel())
    n = b.size
    x, st = lanczos.direct_lanczos_lr(lambda v: (a @ v.ravel()).reshape(v.shape),
                                      lambda w: (ah @ w.ravel()).reshape(w.shape), b, n)
    assert st["breakdown"] is None
    assert np.linalg.norm(x.ravel() - xs) / np.linalg.norm(xs) < 1e-11
    # and half the space is visibly not enough
    xh, _ = lanczos.direct_lanczos_lr(lambda v: (a @ v.ravel()).reshape(v.shape),
                                      lambda w: (ah @ w.ravel()).reshape(w.shape), b, n // 4)
    assert np.linalg.norm(xh.ravel() - xs) / np.linalg.norm(xs) > 1e-9


def test_multishift_equals_bicg_and_dense():
    dims = (2, 2, 2, 4)
    u = synth.gauge_links(dims, 37, 0.2)
    a = deflation.sparse_hw(u, dims, -2.0, 0.3)
    ah = deflation.sparse_hw(u, dims, -2.0, -0.3)
    m = a @ a
    mh = ah @ ah
    r = synth.gaussian_source(dims, 38).ravel()
    sig = np.array([-0.01, -0.3, -2.0])
    k = 12
    xs, st = lanczos.multishift_iterates(lambda v: m @ v, lambda w: mh @ w, r, r, k, sig)
    for i, s in enumerate(sig):
        xb = lanczos.bicg(lambda v: m @ v, lambda w: mh @ w, r, r, s, k)
        assert np.linalg.norm(xs[i] - xb) / np.linalg.norm(xb) < 1e-8
    xs, st = lanczos.multishift_iterates(lambda v: m @ v, lambda w: mh @ w, r, r, 250, sig)
    md = m.toarray()
    for i, s in enumerate(sig):
        xd = np.linalg.solve(md - s * np.eye(len(r)), r)
        assert np.linalg.norm(xs[i] - xd) / np.linalg.norm(xd) < 1e-8


def test_rational_sign_within_theorem1_bound():
    dims = (2, 2, 2, 4)
    u, a, ah = _ops(dims, 39, 0.3)
    ad = a.toarray()
    b = synth.gaussian_source(dims, 40).ravel()
    ev = np.linalg.eigvals(ad)
    alpha, beta = np.abs(ev).min(), np.abs(ev).max()
    eps = 1e-8
    s, c, w, sg = rational.neuberger_for_spectrum(0.99 * alpha, 1.01 * beta, eps)
    xg = lanczos.rational_sign_dense(ad, b, w, sg)
    xs = matsign.sign_eig(ad, b)
    # spectrum inside the two circles => error bounded by eps times the eigenvector condition number
    _, r = np.linalg.eig(ad)
    kappa_r = np.linalg.cond(r)
    assert np.linalg.norm(xg - xs) / np.linalg.norm(b) < eps * kappa_r


def test_lr_deflation_identities():
    dims = (2, 2, 2, 4)
    u, a, ah = _ops(dims, 41, 0.3)
    ad = a.toarray()
    lam, R, L, gap = deflation.critical_dense(ad, 6)
    assert np.abs(np.conj(L).T @ R - np.eye(6)).max() < 1e-10
    p = R @ np.conj(L).T
    assert np.abs(p @ p - p).max() < 1e-10
    assert np.abs(ad @ R - R * lam).max() < 1e-10
    assert np.abs(np.conj(L).T @ ad - lam[:, None] * np.conj(L).T).max() < 1e-10
    assert gap >= np.abs(lam).max()
    # eigenvector input: x_P is exact, r = 0
    xp, r, rt = lanczos.deflation_vectors(R[:, 2], R, L, lam)
    assert np.abs(xp - np.sign(lam[2].real) * R[:, 2]).max() < 1e-10
    assert np.abs(r).max() < 1e-10
    # Eq. action: sign(A) b = x_P + sign(A) (I - P) b
    b = synth.gaussian_source(dims, 42).ravel()
    xp, r, rt = lanczos.deflation_vectors(b, R, L, lam)
    s = matsign.sign_eig(ad)
    assert np.abs(xp + s @ r - s @ b).max() < 1e-9
    # shadow: (I - P)^H b, free of left-eigenvector components' partners: R^H r~ = 0
    assert np.abs(np.conj(R).T @ rt).max() < 1e-10
    assert np.abs(np.conj(L).T @ r).max() < 1e-10


def test_sparse_critical_matches_dense():
    dims = (2, 2, 4, 4)
    u = synth.gauge_links(dims, 43)
    ad = deflation.sparse_hw(u, dims, -2.0, 0.3).toarray()
    lam_d, R_d, L_d, gap_d = deflation.critical_dense(ad, 8)
    lam_s, R_s, L_s, gap_s = deflation.critical_sparse(u, dims, -2.0, 0.3, 8)
    assert np.abs(np.sort_complex(lam_d) - np.sort_complex(lam_s)).max() < 1e-9
    assert abs(gap_d - gap_s) < 1e-9
    assert np.abs(np.conj(L_s).T @ R_s - np.eye(8)).max() < 1e-8
    b = synth.gaussian_source(dims, 44).ravel()
    xp_d, r_d, _ = lanczos.deflation_vectors(b, R_d, L_d, lam_d)
    xp_s, r_s, _ = lanczos.deflation_vectors(b, R_s, L_s, lam_s)
    assert np.linalg.norm(xp_d - xp_s) < 1e-8 * np.linalg.norm(b)


@pytest.mark.slow
def test_direct_lanczos_lr_converges_4444(problem_4444):
    p = problem_4444
    dims = p["dims"]
    a = deflation.sparse_hw(p["links"], dims, -2.0, 0.3)
    ah = deflation.sparse_hw(p["links"], dims, -2.0, -0.3)
    xs = p["xstar"]
    x, st = lanczos.direct_lanczos_lr(lambda v: (a @ v.ravel()).reshape(v.shape),
                                      lambda w: (ah @ w.ravel()).reshape(w.shape), p["b"], 600,
                                      p["R16"], p["L16"], p["lam16"])
    err = np.linalg.norm(x - xs) / np.linalg.norm(xs)
    assert err < 1e-8
