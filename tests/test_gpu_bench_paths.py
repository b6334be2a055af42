"""GPU parity of the kernel variants and batch shapes that the benchmark's workloads run, at the
sizes where they run, and of the solver's edge cases.

- 16^4 multishift at equal k with FP32 and FP16 12-real links (the one-thread-per-site
  k_ms_pair<float> kernels the 16^4 lines use) against the oracle's shifted iterates
  beta V_k (H_k - sigma_i)^-1 e_1 of two-sided Lanczos on A^2 (Section 2.2, Algorithm 3). For the
  FP16 links the oracle runs the iteration on the same quantised links (rows 1, 2 rounded to half
  precision, row 3 = conj(row 1 x row 2)) and, like the solver, the final multiplication by A with
  the FP64 links, so both bounds measure FP32 arithmetic only: 1e-5.
- 16^4 FP32 direct with 16 right-hand sides in one batch, equal k, each against the oracle's
  Algorithm 4 (the C FP64 two-sided Lanczos), 1e-4 (the bound of the 4^4 FP32 equal-k test).
- every pair-stencil shape the autotuner may pick (pinned through ovl_set_pair_variant) at 12^4,
  the headline size, FP64 and FP32, equal k against the oracle's Algorithm 4: 1e-10 / 1e-4; the
  grouped FP32 shape (links once per four sources) on batches of 6 at 8^4 and 16 at 16^4.
- FP64 reliable updates with more than 64 correction systems in one batch (4 sources x s poles).
- the spectral set-up (ARPACK through the library) against the oracle's critical eigenpairs.
- breakdown at the start (shadow residual orthogonal to the residual), the ill-posed free field
  with periodic time at mu = 0 (exact zero modes) and mu = 1 (no convergence): statuses, not hangs.
"""
import numpy as np
import pytest

import synth
from conftest import fp16_quantised
from oracle import deflation, krylov, lanczos, matsign, rational, wilson

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
    p = ovl.ovl_sign_params_default(**kw)
    bt = torch.from_numpy(np.ascontiguousarray(b)).cuda()
    xt = torch.empty_like(bt)
    st, info = ovl.ovl_apply_sign(lat, p, bt, xt)
    return st, info, xt.cpu().numpy()


def test_fp16_quantised_links_are_what_the_stencil_uses(ovl, ctx):
    """The test's quantisation reproduces the library's FP16 12-real stencil to FP32 rounding."""
    dims = (4, 4, 4, 6)
    u = synth.gauge_links(dims, 5)
    psi = synth.gaussian_source(dims, 6)
    lat = ovl.ovl_create_lattice(ctx, dims, -1)
    ovl.ovl_set_links(lat, u, ovl.OVL_F16R12)
    x = torch.from_numpy(psi.astype(np.complex64)).cuda()
    y = torch.empty_like(x)
    ovl.ovl_apply_DW(lat, -2.0, 0.3, ovl.OVL_GAMMA5 | ovl.OVL_LINKS_F16R12, x, y)
    ref = wilson.apply_hw(fp16_quantised(u), psi, -2.0, 0.3)
    assert np.abs(y.cpu().numpy() - ref).max() < 5e-6 * np.abs(ref).max()
    ovl.ovl_destroy_lattice(lat)


@pytest.mark.parametrize("prec", ["f32", "f16"])
def test_multishift_equal_k_1616_reduced(ovl, ctx, prec):
    dims = (16, 16, 16, 16)
    u = synth.gauge_links(dims, 9)
    b = synth.gaussian_source(dims, 10)
    lat = ovl.ovl_create_lattice(ctx, dims, -1)
    ovl.ovl_set_links(lat, u, ovl.OVL_F32 | ovl.OVL_F16R12)
    k = 3
    pr = ovl.OVL_PREC_F32 if prec == "f32" else ovl.OVL_PREC_F32_F16LINKS
    # tol above the FP32 floor: no reliable-update stage, so x is the plain BiCG iterate at k (no
    # shift reaches 1e-5 within 3 iterations)
    st, info, x = _solve(ovl, lat, b, method=ovl.OVL_MULTISHIFT_BICG, mu=0.3, tol=1e-5, k_max=k, spec_lo=0.05,
                         spec_hi=2.7, s=6, check_every=1, precision=pr)
    assert info[0]["iterations"] == k
    ovl.ovl_destroy_lattice(lat)
    uo = u if prec == "f32" else fp16_quantised(u)
    w, sg = rational.neuberger_scaled(6, rational.scale_and_d(*rational.circle_from_gap(0.05, 2.7))[0])
    a = lambda v: krylov.apply_hw(uo, dims, -2.0, 0.3, v.reshape(b.shape)).ravel()
    ah = lambda v: krylov.apply_hw(uo, dims, -2.0, -0.3, v.reshape(b.shape)).ravel()
    xs, _ = lanczos.multishift_iterates(lambda v: a(a(v)), lambda v: ah(ah(v)), b.ravel(), b.ravel(), k, sg)
    # the solver's final x = A sum_i omega_i x^(i) is one FP64 stencil with the FP64 links
    xo = krylov.apply_hw(u, dims, -2.0, 0.3, np.tensordot(w, xs, axes=1).reshape(b.shape)).ravel()
    assert _rel(x.ravel(), xo) < 1e-5


def test_direct_batch16_1616_f32_equal_k(ovl, ctx):
    dims = (16, 16, 16, 16)
    u = synth.gauge_links(dims, 0)
    b = synth.gaussian_source(dims, 1000, nrhs=16)
    lat = ovl.ovl_create_lattice(ctx, dims, -1)
    ovl.ovl_set_links(lat, u, ovl.OVL_F64 | ovl.OVL_F32)
    k = 6
    st, info, x = _solve(ovl, lat, b, mu=0.2, fixed_k=k, precision=ovl.OVL_PREC_F32, check_every=3)
    ovl.ovl_destroy_lattice(lat)
    assert st == ovl.OVL_OK and all(i["iterations"] == k for i in info)
    for r in range(16):
        xo, _, _ = krylov.direct_lanczos(u, dims, -2.0, 0.2, b[r], k)
        assert _rel(x[r], xo) < 1e-4, r


@pytest.fixture(scope="module")
def lat12(ovl, ctx):
    dims = (12, 12, 12, 12)
    u = synth.gauge_links(dims, 0)
    b = synth.gaussian_source(dims, 1000)
    lat = ovl.ovl_create_lattice(ctx, dims, -1)
    ovl.ovl_set_links(lat, u, ovl.OVL_F64 | ovl.OVL_F32)
    k = 24
    xo, _, _ = krylov.direct_lanczos(u, dims, -2.0, 0.3, b, k)
    yield lat, b, k, xo
    ovl.ovl_destroy_lattice(lat)


@pytest.mark.parametrize("prec", ["f64", "f32"])
def test_every_pair_shape_equal_k_1212(ovl, lat12, prec):
    lat, b, k, xo = lat12
    vol = 12 ** 4
    pr = ovl.OVL_PREC_F64 if prec == "f64" else ovl.OVL_PREC_F32
    bound = 1e-10 if prec == "f64" else 1e-4
    xs = []
    try:
        for var in range(9):
            ovl.ovl_set_pair_variant(vol, pr, var)
            assert ovl.ovl_get_pair_variant(vol, pr) == var
            st, info, x = _solve(ovl, lat, b, mu=0.3, fixed_k=k, precision=pr, check_every=8)
            assert st == ovl.OVL_OK and info[0]["iterations"] == k
            assert _rel(x, xo) < bound, var
            xs.append(x)
    finally:
        ovl.ovl_set_pair_variant(vol, pr, -1)
    assert ovl.ovl_get_pair_variant(vol, pr) == -1
    # the shapes differ only in the order of alpha's partial sums
    for x in xs[1:]:
        assert _rel(x, xs[0]) < (1e-12 if prec == "f64" else 1e-5)


def test_shape_change_between_solves(ovl, ctx):
    """Solves on one lattice with different pinned pair shapes: the cached chunk graphs must follow
    the shape (a graph captured for one shape replayed in a solve of another mixed a deferred step
    with plain ones and broke the recurrence). 2x2x2x4 to 1e-10 against the dense sign."""
    dims = (2, 2, 2, 4)
    u = synth.gauge_links(dims, 35, 0.1)
    b = synth.gaussian_source(dims, 36)
    xs = matsign.sign_eig(wilson.dense_hw(u, dims, -2.0, 0.3), b.ravel()).reshape(b.shape)
    lat = ovl.ovl_create_lattice(ctx, dims, -1)
    ovl.ovl_set_links(lat, u, ovl.OVL_F64)
    try:
        for var in (4, 7, 5, 7, 3):
            ovl.ovl_set_pair_variant(32, ovl.OVL_PREC_F64, var)
            st, info, x = _solve(ovl, lat, b, mu=0.3, tol=1e-10, k_max=384, check_every=16)
            assert st == ovl.OVL_OK, (var, info)
            assert _rel(x, xs) < 1e-10, var
    finally:
        ovl.ovl_set_pair_variant(32, ovl.OVL_PREC_F64, -1)
        ovl.ovl_destroy_lattice(lat)


@pytest.mark.parametrize("var", [7, 3])
def test_graph_chunks_equal_direct_launches(ovl, ctx, var):
    """The chunks of steps as CUDA graphs (the default) and as direct launches give the same solve,
    bitwise, for the headline's shape (deferred step, early launch behind the settle kernel) and a
    plain one; 8^4 FP64, a fixed 75 steps (chunks of 20: three graphs and a partial chunk)."""
    dims = (8, 8, 8, 8)
    vol = int(np.prod(dims))
    u = synth.gauge_links(dims, 3)
    b = synth.gaussian_source(dims, 4, nrhs=2)
    lat = ovl.ovl_create_lattice(ctx, dims, -1)
    ovl.ovl_set_links(lat, u, ovl.OVL_F64)
    xs = []
    try:
        ovl.ovl_set_pair_variant(vol, ovl.OVL_PREC_F64, var)
        for graphs in (1, 0):
            st, info, x = _solve(ovl, lat, b, mu=0.3, fixed_k=75, check_every=20, use_graphs=graphs)
            assert st == ovl.OVL_OK and all(i["iterations"] == 75 for i in info)
            xs.append(x)
    finally:
        ovl.ovl_set_pair_variant(vol, ovl.OVL_PREC_F64, -1)
        ovl.ovl_destroy_lattice(lat)
    assert np.array_equal(xs[0], xs[1])
    xo, _, _ = krylov.direct_lanczos(u, dims, -2.0, 0.3, b[0], 75)
    assert _rel(xs[0][0], xo) < 1e-10


@pytest.mark.parametrize("dims,nrhs", [((8, 8, 8, 8), 6), ((16, 16, 16, 16), 16)])
def test_grouped_pair_batch_f32_equal_k(ovl, ctx, dims, nrhs):
    """Pair shape 8 (links loaded once per group of four sources; 6 = one full group and one of
    two) against the oracle's Algorithm 4 per rhs at equal k, FP32: 1e-4, and against shape 3."""
    u = synth.gauge_links(dims, 0)
    b = synth.gaussian_source(dims, 1000, nrhs=nrhs)
    lat = ovl.ovl_create_lattice(ctx, dims, -1)
    ovl.ovl_set_links(lat, u, ovl.OVL_F64 | ovl.OVL_F32)
    vol, k = int(np.prod(dims)), 6
    xs = {}
    try:
        for var in (8, 3):
            ovl.ovl_set_pair_variant(vol, ovl.OVL_PREC_F32, var)
            st, info, xs[var] = _solve(ovl, lat, b, mu=0.2, fixed_k=k, precision=ovl.OVL_PREC_F32, check_every=3)
            assert st == ovl.OVL_OK and all(i["iterations"] == k for i in info)
    finally:
        ovl.ovl_set_pair_variant(vol, ovl.OVL_PREC_F32, -1)
        ovl.ovl_destroy_lattice(lat)
    for r in (0, nrhs - 1) if nrhs > 6 else range(nrhs):
        xo, _, _ = krylov.direct_lanczos(u, dims, -2.0, 0.2, b[r], k)
        assert _rel(xs[8][r], xo) < 1e-4, r
    assert _rel(xs[8], xs[3]) < 1e-5


def test_reliable_update_batch_over_64_systems(ovl, ctx, problem_4444):
    """4 sources x s Neuberger poles (s > 16: more than 64 correction systems) refined in one batch
    with FP64 residuals: every source matches the dense g(A) b of its own right-hand side."""
    p = problem_4444
    ev = p["eig"]
    lo, hi = 0.99 * float(np.abs(ev).min()), 1.01 * float(np.abs(ev).max())
    eps = 1e-10
    s, c, w, sg = rational.neuberger_for_spectrum(lo, hi, eps)
    assert 4 * s > 64
    b = synth.gaussian_source(p["dims"], 77, nrhs=4)
    lat = ovl.ovl_create_lattice(ctx, p["dims"], -1)
    ovl.ovl_set_links(lat, p["links"], ovl.OVL_F64 | ovl.OVL_F32)
    st, info, x = _solve(ovl, lat, b, method=ovl.OVL_MULTISHIFT_BICG, mu=0.3, tol=eps, k_max=5000, spec_lo=lo,
                         spec_hi=hi, precision=ovl.OVL_PREC_F32)
    ovl.ovl_destroy_lattice(lat)
    assert st == ovl.OVL_OK, info
    assert all(i["poles"] == s for i in info)
    for r in range(4):
        xg = lanczos.rational_sign_dense(p["h"], b[r].ravel(), w, sg)
        assert _rel(x[r].ravel(), xg) < 2e-9, r


@pytest.mark.parametrize("dims", [(2, 2, 4, 4), (4, 4, 4, 4)])
def test_spectrum_setup_vs_oracle(ovl, ctx, dims):
    from paper_0910_1048_gb300 import spectrum

    u = synth.gauge_links(dims, 4)
    m = 8
    lat = ovl.ovl_create_lattice(ctx, dims, -1)
    ovl.ovl_set_links(lat, u, ovl.OVL_F64 | ovl.OVL_F32)
    lam, R, L, gap, info = spectrum.critical_eigenpairs(ovl, lat, -2.0, 0.3, m)
    ovl.ovl_destroy_lattice(lat)
    lo, Ro, Lo, gapo = deflation.critical_sparse(u, dims, -2.0, 0.3, m)
    assert np.abs(np.sort_complex(lam) - np.sort_complex(lo)).max() < 1e-9 * np.abs(lo).max()
    assert abs(gap - gapo) < 1e-9 * gapo
    assert np.abs(np.conj(L) @ R.T - np.eye(m)).max() <= 1e-10
    a = deflation.sparse_hw(u, dims, -2.0, 0.3)
    for i in range(m):  # eigen-equations A r = lam r, l^H A = lam l^H
        assert np.linalg.norm(a @ R[i] - lam[i] * R[i]) < 1e-9 * np.linalg.norm(R[i])
        assert np.linalg.norm(np.conj(a.T) @ L[i] - np.conj(lam[i]) * L[i]) < 1e-9 * np.linalg.norm(L[i])


def test_breakdown_at_start_returns_x_P(ovl, ctx):
    """A deflation set with L^H R = 1 chosen so that the shadow residual r~ = b - L R^H b is
    orthogonal to r = b - R L^H b: the two-sided process cannot start (EBREAKDOWN) and the result
    is the deflated part x_P = R sign(Lambda) L^H b of Algorithm 4."""
    dims = (4, 4, 4, 4)
    n = 12 * 256
    rng = np.random.default_rng(31)
    e, _ = np.linalg.qr(rng.standard_normal((n, 3)) + 1j * rng.standard_normal((n, 3)))
    e1, e2, e3 = e[:, 0], e[:, 1], e[:, 2]
    b = e1 + e2 + e3
    R = e1[None, :]
    L = (e1 + 2.0 * e3)[None, :]  # L^H R = 1; r = e2 + e3 - 2 e1, r~ = e2 - e3, r~^H r = 0
    lam = np.array([0.7 + 0.1j])
    lat = ovl.ovl_create_lattice(ctx, dims, -1)
    ovl.ovl_set_links(lat, synth.gauge_links(dims, 0), ovl.OVL_F64)
    ovl.ovl_set_deflation(lat, -2.0, 0.3, R, L, lam)
    st, info, x = _solve(ovl, lat, b.reshape(4, 4, 4, 4, 4, 3), mu=0.3, tol=1e-8, k_max=100, use_deflation=1)
    ovl.ovl_destroy_lattice(lat)
    assert st == ovl.OVL_EBREAKDOWN and info[0]["iterations"] == 0
    xp, r, rt = lanczos.deflation_vectors(b, R.T, L.T, lam)
    assert abs(np.vdot(rt, r)) < 1e-14 * np.linalg.norm(r) * np.linalg.norm(rt)
    assert _rel(x.ravel(), xp) < 1e-14


def test_ill_posed_free_field_periodic_time(ovl, ctx):
    """Periodic time, unit links, m_W = -2, mu = 0: H_W has exact zero modes, so sign(H_W) b is
    undefined (Section 1); the solve must end with a status (EILLPOSED, or ENOCONV with its best
    iterate), never OK."""
    dims = (4, 4, 4, 4)
    lat = ovl.ovl_create_lattice(ctx, dims, 1)
    ovl.ovl_set_links(lat, synth.unit_links(dims), ovl.OVL_F64)
    st, info, x = _solve(ovl, lat, synth.gaussian_source(dims, 2), mu=0.0, tol=1e-10, k_max=400)
    ovl.ovl_destroy_lattice(lat)
    assert st in (ovl.OVL_EILLPOSED, ovl.OVL_ENOCONV, ovl.OVL_EBREAKDOWN), (st, info)


def test_large_mu_ends_with_a_status(ovl, ctx, problem_4444):
    """mu = 1: two-sided Lanczos loses biorthogonality (the basis norms grow) and does not reach
    1e-8 within 600 steps; the call returns ENOCONV (or EBREAKDOWN) with a finite best iterate."""
    p = problem_4444
    lat = ovl.ovl_create_lattice(ctx, p["dims"], -1)
    ovl.ovl_set_links(lat, p["links"], ovl.OVL_F64)
    st, info, x = _solve(ovl, lat, p["b"], mu=1.0, tol=1e-8, k_max=600)
    ovl.ovl_destroy_lattice(lat)
    assert st in (ovl.OVL_OK, ovl.OVL_ENOCONV, ovl.OVL_EBREAKDOWN)
    assert np.isfinite(x).all()
