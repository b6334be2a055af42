"""GPU parity of the rational (multishift BiCG-LR) variant, Algorithm 3 with Section 5.

x = x_P + A sum_i omega_i x^(i), (A^2 - sigma_i) x^(i) = r, A = H_W(mu).
- equal-k parity: with tol = 0 every shift runs exactly k steps; the oracle's shifted
  iterates beta V_k (H_k - sigma_i)^-1 e_1 of two-sided Lanczos on A^2 (Section 2.2) give the
  same x to 1e-9 (FP64);
- converged: against the dense g(A) b (solver error) and against x* (rational error within
  Theorem 1's eps times the eigenvector condition number), Neuberger from spectrum bounds
  (Eq. no_of_poles), with LR deflation, Zolotarev at mu = 0;
- FP32 vectors (1e-5) and FP16 12-real links (5e-3 against x*): stated bounds;
- a single custom pole (omega = 1, sigma = 0) gives A (A^2)^-1 b = A^-1 b.
"""
import numpy as np
import pytest

import synth
from oracle import deflation, lanczos, matsign, rational, wilson

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
    return np.linalg.norm(a - b) / np.linalg.norm(b)


def _solve(ovl, lat, b, **kw):
    p = ovl.ovl_sign_params_default(method=ovl.OVL_MULTISHIFT_BICG, **kw)
    bt = torch.from_numpy(np.ascontiguousarray(b)).cuda()
    xt = torch.empty_like(bt)
    st, info = ovl.ovl_apply_sign(lat, p, bt, xt)
    return st, info, xt.cpu().numpy()


@pytest.fixture(scope="module")
def p4m(ovl, ctx, problem_4444):
    p = problem_4444
    lat = ovl.ovl_create_lattice(ctx, p["dims"], -1)
    ovl.ovl_set_links(lat, p["links"], ovl.OVL_F64 | ovl.OVL_F32 | ovl.OVL_F16R12)
    ev = p["eig"]
    yield p, lat, float(np.abs(ev).min()), float(np.abs(ev).max())
    ovl.ovl_destroy_lattice(lat)


@pytest.mark.parametrize("k", [8, 30])
def test_equal_k_parity(ovl, p4m, k):
    p, lat, lo, hi = p4m
    st, info, x = _solve(ovl, lat, p["b"], mu=0.3, tol=0.0, k_max=k, spec_lo=0.9 * lo, spec_hi=1.1 * hi,
                         s=12, check_every=5)
    assert info[0]["iterations"] == k and info[0]["poles"] == 12
    w, sg = rational.neuberger_scaled(12, rational.scale_and_d(*rational.circle_from_gap(0.9 * lo, 1.1 * hi))[0])
    a = deflation.sparse_hw(p["links"], p["dims"], -2.0, 0.3)
    ah = deflation.sparse_hw(p["links"], p["dims"], -2.0, -0.3)
    m = a @ a
    mh = ah @ ah
    b = p["b"].ravel()
    xs, _ = lanczos.multishift_iterates(lambda v: m @ v, lambda v: mh @ v, b, b, k, sg)
    xo = a @ np.tensordot(w, xs, axes=1)
    assert _rel(x.ravel(), xo) < 1e-9


def test_neuberger_converged(ovl, p4m):
    p, lat, lo, hi = p4m
    eps = 1e-10
    st, info, x = _solve(ovl, lat, p["b"], mu=0.3, tol=eps, k_max=5000, spec_lo=0.99 * lo, spec_hi=1.01 * hi)
    assert st == ovl.OVL_OK, info
    s, c, w, sg = rational.neuberger_for_spectrum(0.99 * lo, 1.01 * hi, eps)
    assert info[0]["poles"] == s
    xg = lanczos.rational_sign_dense(p["h"], p["b"].ravel(), w, sg)
    assert _rel(x.ravel(), xg) < 2e-9          # solver error against g(A) b
    assert _rel(x.ravel(), p["xstar"].ravel()) < 1e-8   # total error against x*


def test_neuberger_with_deflation(ovl, p4m):
    p, lat, lo, hi = p4m
    ovl.ovl_set_deflation(lat, -2.0, 0.3, p["R16"].T.copy(), p["L16"].T.copy(), p["lam16"])
    st, info, x = _solve(ovl, lat, p["b"], mu=0.3, tol=1e-10, k_max=5000, spec_lo=0.99 * p["gap16"],
                         spec_hi=1.01 * hi, use_deflation=1)
    st0, info0, _ = _solve(ovl, lat, p["b"], mu=0.3, tol=1e-10, k_max=5000, spec_lo=0.99 * lo, spec_hi=1.01 * hi)
    ovl.ovl_set_deflation(lat, -2.0, 0.3, None, None, None)
    assert st == ovl.OVL_OK, info
    assert _rel(x, p["xstar"]) < 1e-8
    # pole reduction by deflation (Section 3) and fewer iterations
    assert info[0]["poles"] < info0[0]["poles"]
    assert info[0]["iterations"] < info0[0]["iterations"]


def test_zolotarev_mu0(ovl, ctx):
    dims = (4, 4, 4, 4)
    u = synth.gauge_links(dims, 7)
    h = wilson.dense_hw(u, dims, -2.0, 0.0)
    ev = np.linalg.eigvalsh(h)
    lo, hi = np.abs(ev).min(), np.abs(ev).max()
    b = synth.gaussian_source(dims, 8)
    xs = matsign.sign_hermitian(h, b.ravel()).reshape(b.shape)
    lat = ovl.ovl_create_lattice(ctx, dims, -1)
    ovl.ovl_set_links(lat, u, ovl.OVL_F64)
    st, info, x = _solve(ovl, lat, b, mu=0.0, tol=1e-11, k_max=5000, spec_lo=0.999 * lo, spec_hi=1.001 * hi,
                         rational_kind=ovl.OVL_RAT_ZOLOTAREV, s=20)
    assert st == ovl.OVL_OK, info
    assert _rel(x, xs) < 1e-9
    ovl.ovl_destroy_lattice(lat)


@pytest.mark.parametrize("prec,tol", [("f32", 1e-5), ("f16", 5e-3)])
def test_reduced_precision(ovl, p4m, prec, tol):
    p, lat, lo, hi = p4m
    pr = ovl.OVL_PREC_F32 if prec == "f32" else ovl.OVL_PREC_F32_F16LINKS
    st, info, x = _solve(ovl, lat, p["b"], mu=0.3, tol=1e-6, k_max=5000, spec_lo=0.99 * lo, spec_hi=1.01 * hi,
                         precision=pr)
    assert info[0]["iterations"] > 0
    assert _rel(x, p["xstar"]) < tol, (st, info)


def test_single_pole_is_inverse(ovl, p4m):
    p, lat, lo, hi = p4m
    om = np.array([1.0])
    sg = np.array([0.0])
    import ctypes
    st, info, x = _solve(ovl, lat, p["b"], mu=0.3, tol=1e-11, k_max=20000, rational_kind=ovl.OVL_RAT_CUSTOM, s=1,
                         omega=om.ctypes.data_as(ctypes.POINTER(ctypes.c_double)),
                         sigma=sg.ctypes.data_as(ctypes.POINTER(ctypes.c_double)))
    assert st == ovl.OVL_OK, info
    res = p["h"] @ x.ravel() - p["b"].ravel()
    assert np.linalg.norm(res) / np.linalg.norm(p["b"]) < 1e-8


def test_requires_spectrum_bounds(ovl, p4m):
    p, lat, lo, hi = p4m
    p_ = ovl.ovl_sign_params_default(method=ovl.OVL_MULTISHIFT_BICG, mu=0.3)
    bt = torch.from_numpy(p["b"]).cuda()
    with pytest.raises(ovl.OvlError) as e:
        ovl.ovl_apply_sign(lat, p_, bt, torch.empty_like(bt))
    assert "spec" in str(e.value)


def test_equal_k_parity_1616(ovl, ctx):
    """16^4 runs the one-thread-per-site multishift pair kernels; equal-k parity at k = 3."""
    dims = (16, 16, 16, 16)
    u = synth.gauge_links(dims, 9)
    b = synth.gaussian_source(dims, 10)
    lat = ovl.ovl_create_lattice(ctx, dims, -1)
    ovl.ovl_set_links(lat, u, ovl.OVL_F64)
    k = 3
    st, info, x = _solve(ovl, lat, b, mu=0.3, tol=0.0, k_max=k, spec_lo=0.05, spec_hi=2.7, s=6, check_every=1)
    w, sg = rational.neuberger_scaled(6, rational.scale_and_d(*rational.circle_from_gap(0.05, 2.7))[0])
    a = lambda v: wilson.apply_hw(u, v.reshape(b.shape), -2.0, 0.3).ravel()
    ah = lambda v: wilson.apply_hw(u, v.reshape(b.shape), -2.0, -0.3).ravel()
    xs, _ = lanczos.multishift_iterates(lambda v: a(a(v)), lambda v: ah(ah(v)), b.ravel(), b.ravel(), k, sg)
    xo = a(np.tensordot(w, xs, axes=1))
    assert _rel(x.ravel(), xo) < 1e-9
    ovl.ovl_destroy_lattice(lat)


@pytest.mark.parametrize("prec", ["f32", "f16"])
def test_reliable_updates_reach_fp64_accuracy(ovl, p4m, prec):
    """FP32 vectors (and FP16 12-real links) with FP64 reliable updates: below the FP32 floor
    every shifted system is refined with FP64 residuals, so the result matches the FP64
    rational result (dense g(A) b) to the requested tolerance."""
    p, lat, lo, hi = p4m
    eps = 1e-10
    pr = ovl.OVL_PREC_F32 if prec == "f32" else ovl.OVL_PREC_F32_F16LINKS
    st, info, x = _solve(ovl, lat, p["b"], mu=0.3, tol=eps, k_max=5000, spec_lo=0.99 * lo, spec_hi=1.01 * hi,
                         precision=pr)
    assert st == ovl.OVL_OK, info
    assert info[0]["residual"] <= eps
    s, c, w, sg = rational.neuberger_for_spectrum(0.99 * lo, 1.01 * hi, eps)
    xg = lanczos.rational_sign_dense(p["h"], p["b"].ravel(), w, sg)
    assert _rel(x.ravel(), xg) < 2e-9
    assert _rel(x.ravel(), p["xstar"].ravel()) < 1e-8
