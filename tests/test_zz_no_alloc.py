"""The allocation-free entry point ovl_apply_sign_noalloc, for callers that cannot allocate
device memory (their device memory belongs to another allocator, or their run phase must not
call cudaMalloc/cudaFree). It must give the same x as ovl_apply_sign's direct method on the
same inputs, on two calls in a row (the static scratch array keeps the previous call's
contents), and refuse a solve whose scratch does not fit its fixed 64 MiB.
This file is collected last on purpose."""
import numpy as np
import pytest

import synth

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")


@pytest.fixture(scope="module")
def setup():
    import paper_0910_1048_gb300 as ovl
    ctx = ovl.ovl_ctx_create(0)
    dims = (4, 4, 4, 4)
    lat = ovl.ovl_create_lattice(ctx, dims, -1)
    ovl.ovl_set_links(lat, synth.gauge_links(dims, 0), ovl.OVL_F64 | ovl.OVL_F32)
    yield ovl, ctx, dims, lat
    ovl.ovl_destroy_lattice(lat)
    ovl.ovl_ctx_destroy(ctx)


def _rel(a, b):
    return float(torch.linalg.vector_norm(a - b) / torch.linalg.vector_norm(b))


@pytest.mark.parametrize("kw", [dict(fixed_k=60), dict(tol=1e-9, k_max=1200),
                                dict(tol=1e-5, k_max=400, precision=1)])
def test_matches_allocating_path_twice(setup, kw):
    ovl, ctx, dims, lat = setup
    b = torch.from_numpy(synth.gaussian_source(dims, 1000)).cuda()
    p = ovl.ovl_sign_params_default(mu=0.3, **kw)
    x_ref = torch.empty_like(b)
    st_ref, _ = ovl.ovl_apply_sign(lat, p, b, x_ref)
    for _ in range(2):  # the second call must not see stale state from the first
        x = torch.full_like(b, float("nan"))
        st, info = ovl.ovl_apply_sign_noalloc(lat, p, b, x)
        assert st == st_ref
        assert _rel(x, x_ref) < 1e-10


@pytest.mark.parametrize("var", [7, 1])
def test_matches_with_pinned_pair_shape(setup, var):
    """The same with the pair-stencil shape pinned: 7 (one block per SM, the deferred step and its
    settle kernels, as the 12^4 FP64 workload runs) and 1 (the split stencil)."""
    ovl, ctx, dims, lat = setup
    vol = int(np.prod(dims))
    b = torch.from_numpy(synth.gaussian_source(dims, 1000, nrhs=2)).cuda()
    # two rhs at k_max 600 fit the static array; both reach 1e-5 near k = 500 at mu = 0.2
    p = ovl.ovl_sign_params_default(mu=0.2, tol=1e-5, k_max=600)
    ovl.ovl_set_pair_variant(vol, ovl.OVL_PREC_F64, var)
    try:
        x_ref = torch.empty_like(b)
        st_ref, info_ref = ovl.ovl_apply_sign(lat, p, b, x_ref)
        x = torch.full_like(b, float("nan"))
        st, info = ovl.ovl_apply_sign_noalloc(lat, p, b, x)
    finally:
        ovl.ovl_set_pair_variant(vol, ovl.OVL_PREC_F64, -1)
    assert st == st_ref == ovl.OVL_OK
    assert [i["iterations"] for i in info] == [i["iterations"] for i in info_ref]
    assert _rel(x, x_ref) < 1e-10


def test_batch_matches(setup):
    ovl, ctx, dims, lat = setup
    b = torch.from_numpy(synth.gaussian_source(dims, 7, nrhs=2)).cuda()
    p = ovl.ovl_sign_params_default(mu=0.2, tol=1e-8, k_max=600)
    x_ref = torch.empty_like(b)
    ovl.ovl_apply_sign(lat, p, b, x_ref)
    x = torch.empty_like(b)
    ovl.ovl_apply_sign_noalloc(lat, p, b, x)
    assert _rel(x, x_ref) < 1e-10


def test_refuses_oversized_scratch(setup):
    ovl, ctx, dims, lat = setup
    b = torch.from_numpy(synth.gaussian_source(dims, 1)).cuda()
    p = ovl.ovl_sign_params_default(mu=0.3, fixed_k=4000)  # 4001 x 3072 x 16 B > 64 MiB
    with pytest.raises(ovl.OvlError) as e:
        ovl.ovl_apply_sign_noalloc(lat, p, b, torch.empty_like(b))
    assert e.value.status == ovl.OVL_EINVAL and "64 MiB" in str(e.value)


def test_deflated_matches_allocating_path_twice(setup, problem_4444):
    """With 16 LR deflation vectors: the deflated part x_P, the deflation-dot partials (sized by
    m) and the eigenvalue signs all live in the shared static array too."""
    ovl, ctx, dims, lat = setup
    p4 = problem_4444
    ovl.ovl_set_deflation(lat, -2.0, 0.3, np.ascontiguousarray(p4["R16"].T), np.ascontiguousarray(p4["L16"].T),
                          p4["lam16"])
    try:
        b = torch.from_numpy(p4["b"]).cuda()
        p = ovl.ovl_sign_params_default(mu=0.3, tol=1e-9, k_max=1000, use_deflation=1)
        x_ref = torch.empty_like(b)
        st_ref, _ = ovl.ovl_apply_sign(lat, p, b, x_ref)
        for _ in range(2):
            x = torch.full_like(b, float("nan"))
            st, _ = ovl.ovl_apply_sign_noalloc(lat, p, b, x)
            assert st == st_ref
            assert _rel(x, x_ref) < 1e-10
    finally:
        ovl.ovl_set_deflation(lat, -2.0, 0.3, None, None, None)


def test_current_device_kept(setup):
    """The entry point leaves the caller's current device as it was."""
    ovl, ctx, dims, lat = setup
    b = torch.from_numpy(synth.gaussian_source(dims, 3)).cuda()
    p = ovl.ovl_sign_params_default(mu=0.3, fixed_k=20)
    before = torch.cuda.current_device()
    ovl.ovl_apply_sign_noalloc(lat, p, b, torch.empty_like(b))
    assert torch.cuda.current_device() == before
