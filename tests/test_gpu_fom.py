"""GPU parity of restarted FOM-LR on A^2 (Algorithm 1 with Section 5's rational sign).

- one cycle (k steps) against the oracle's Algorithm 1 (oracle/fom.py) at equal k, FP64: 1e-10,
  at 4^4 and at 16^4 (the C operator of the oracle there);
- converged solves against the dense g(A) b (the solver's own error) and x* (within the rational
  bound), with and without 16 deflated eigenpairs; FP32 vectors to a stated bound;
- mu = 0.6 (eigenvalues far from the real axis): converges to the dense g(A) b;
- a batch of two right-hand sides equals the single solves, bitwise.
"""
import numpy as np
import pytest

import synth
from oracle import deflation, fom, krylov, lanczos, rational

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")


@pytest.fixture(scope="module")
def ovl():
    import paper_0910_1048_gb300 as m
    return m


@pytest.fixture(scope="module")
def ctx(ovl):
    c = ovl.ovl_ctx_create(0)
    yield c
    ovl.ovl_ctx_destroy(c)


def _rel(a, b):
    return np.linalg.norm(np.ravel(a) - np.ravel(b)) / np.linalg.norm(np.ravel(b))


def _solve(ovl, lat, b, **kw):
    p = ovl.ovl_sign_params_default(method=ovl.OVL_FOM_RESTARTED, **kw)
    bt = torch.from_numpy(np.ascontiguousarray(b)).cuda()
    xt = torch.empty_like(bt)
    st, info = ovl.ovl_apply_sign(lat, p, bt, xt)
    return st, info, xt.cpu().numpy()


@pytest.fixture(scope="module")
def p4f(ovl, ctx, problem_4444):
    p = problem_4444
    lat = ovl.ovl_create_lattice(ctx, p["dims"], -1)
    ovl.ovl_set_links(lat, p["links"], ovl.OVL_F64 | ovl.OVL_F32)
    ev = p["eig"]
    yield p, lat, 0.99 * float(np.abs(ev).min()), 1.01 * float(np.abs(ev).max())
    ovl.ovl_destroy_lattice(lat)


@pytest.mark.parametrize("k", [5, 20])
def test_one_cycle_equal_k_4444(ovl, p4f, k):
    p, lat, lo, hi = p4f
    st, info, x = _solve(ovl, lat, p["b"], mu=0.3, tol=0.0, k_max=k, restart_k=k, spec_lo=lo, spec_hi=hi, s=8)
    assert info[0]["iterations"] == k
    hs = deflation.sparse_hw(p["links"], p["dims"], -2.0, 0.3)
    w, sg = rational.neuberger_scaled(8, rational.scale_and_d(*rational.circle_from_gap(lo, hi))[0])
    xo, io = fom.sign_fom_lr(lambda v: (hs @ v.ravel()).reshape(v.shape), p["b"], w, sg, k, tol=0.0, max_cycles=1)
    assert _rel(x, xo) < 1e-10


def test_one_cycle_equal_k_1616(ovl, ctx):
    dims = (16, 16, 16, 16)
    u = synth.gauge_links(dims, 9)
    b = synth.gaussian_source(dims, 10)
    lat = ovl.ovl_create_lattice(ctx, dims, -1)
    ovl.ovl_set_links(lat, u, ovl.OVL_F64)
    k = 6
    st, info, x = _solve(ovl, lat, b, mu=0.3, tol=0.0, k_max=k, restart_k=k, spec_lo=0.05, spec_hi=2.7, s=6)
    ovl.ovl_destroy_lattice(lat)
    w, sg = rational.neuberger_scaled(6, rational.scale_and_d(*rational.circle_from_gap(0.05, 2.7))[0])
    xo, _ = fom.sign_fom_lr(lambda v: krylov.apply_hw(u, dims, -2.0, 0.3, v), b, w, sg, k, tol=0.0, max_cycles=1)
    assert _rel(x, xo) < 1e-10


def test_two_cycles_equal_k(ovl, p4f):
    """Two cycles: the restart (r = v_{k+1}, collinearity factors rho_i) as in Algorithm 1."""
    p, lat, lo, hi = p4f
    k = 12
    st, info, x = _solve(ovl, lat, p["b"], mu=0.3, tol=0.0, k_max=2 * k, restart_k=k, spec_lo=lo, spec_hi=hi, s=8)
    assert info[0]["evaluations"] == 2
    hs = deflation.sparse_hw(p["links"], p["dims"], -2.0, 0.3)
    w, sg = rational.neuberger_scaled(8, rational.scale_and_d(*rational.circle_from_gap(lo, hi))[0])
    xo, _ = fom.sign_fom_lr(lambda v: (hs @ v.ravel()).reshape(v.shape), p["b"], w, sg, k, tol=0.0, max_cycles=2)
    assert _rel(x, xo) < 1e-10


def test_converged_vs_dense_rational_and_xstar(ovl, p4f):
    p, lat, lo, hi = p4f
    eps = 1e-10
    st, info, x = _solve(ovl, lat, p["b"], mu=0.3, tol=eps, k_max=20000, restart_k=40, spec_lo=lo, spec_hi=hi)
    assert st == ovl.OVL_OK, info
    assert info[0]["residual"] <= eps
    s, c, w, sg = rational.neuberger_for_spectrum(lo, hi, eps)
    xg = lanczos.rational_sign_dense(p["h"], p["b"].ravel(), w, sg)
    assert _rel(x, xg) < 2e-9
    assert _rel(x, p["xstar"]) < 1e-8


def test_deflated_converged(ovl, p4f):
    p, lat, lo, hi = p4f
    ovl.ovl_set_deflation(lat, -2.0, 0.3, np.ascontiguousarray(p["R16"].T), np.ascontiguousarray(p["L16"].T),
                          p["lam16"])
    try:
        st, info, x = _solve(ovl, lat, p["b"], mu=0.3, tol=1e-10, k_max=20000, restart_k=30, use_deflation=1,
                             spec_lo=0.99 * p["gap16"], spec_hi=hi)
        st0, info0, _ = _solve(ovl, lat, p["b"], mu=0.3, tol=1e-10, k_max=20000, restart_k=30, spec_lo=lo,
                               spec_hi=hi)
    finally:
        ovl.ovl_set_deflation(lat, -2.0, 0.3, None, None, None)
    assert st == st0 == ovl.OVL_OK
    assert info[0]["iterations"] < info0[0]["iterations"]
    assert _rel(x, p["xstar"]) < 1e-8


def test_fp32_vectors(ovl, p4f):
    """FP32 basis and stencils, FP64 Hessenberg solves and accumulation: 1e-5 against x*."""
    p, lat, lo, hi = p4f
    st, info, x = _solve(ovl, lat, p["b"], mu=0.3, tol=1e-6, k_max=20000, restart_k=40, spec_lo=lo, spec_hi=hi,
                         precision=ovl.OVL_PREC_F32)
    assert st == ovl.OVL_OK, info
    assert _rel(x, p["xstar"]) < 1e-5


def test_mu_06_converges(ovl, ctx):
    """mu = 0.6 on 4^4 (eigenvalues of H_W up to 31 degrees off the real axis): restarted FOM on
    A = H_W^2 converges to the dense g(A) b of the same poles. (At mu = 1 a few eigenvalues lie more
    than 45 degrees off the axis, A is no longer positive real - the condition the paper states for
    the multishift methods on A^2 - and the restarted iteration diverges; the oracle does the same.)"""
    dims = (4, 4, 4, 4)
    u = synth.gauge_links(dims, 0)
    b = synth.gaussian_source(dims, 1000)
    h = deflation.sparse_hw(u, dims, -2.0, 0.6).toarray()
    ev = np.linalg.eigvals(h)
    lo, hi = 0.99 * float(np.abs(ev).min()), 1.01 * float(np.abs(ev).max())
    lat = ovl.ovl_create_lattice(ctx, dims, -1)
    ovl.ovl_set_links(lat, u, ovl.OVL_F64)
    st, info, x = _solve(ovl, lat, b, mu=0.6, tol=1e-9, k_max=20000, restart_k=40, spec_lo=lo, spec_hi=hi)
    ovl.ovl_destroy_lattice(lat)
    assert st == ovl.OVL_OK, info
    s, c, w, sg = rational.neuberger_for_spectrum(lo, hi, 1e-9)
    xg = lanczos.rational_sign_dense(h, b.ravel(), w, sg)
    assert _rel(x, xg) < 1e-7


def test_batch_equals_single(ovl, p4f):
    p, lat, lo, hi = p4f
    b2 = synth.gaussian_source(p["dims"], 71, nrhs=2)
    kw = dict(mu=0.3, tol=1e-9, k_max=20000, restart_k=30, spec_lo=lo, spec_hi=hi)
    st, info, x2 = _solve(ovl, lat, b2, **kw)
    for r in range(2):
        st1, info1, x1 = _solve(ovl, lat, b2[r], **kw)
        assert info1[0]["iterations"] == info[r]["iterations"]
        assert np.array_equal(x1, x2[r])
