"""GPU parity of the Wilson stencil (ovl_apply_DW) against the oracle.

H_W = gamma5 D_W(mu) (Section 1) with the operator reading of the oracle. FP64 is compared
element by element to 1e-13 relative; FP32 links/arithmetic to 2e-6; FP16 12-real links to
3e-3 (half-precision link entries carry ~5e-4 relative rounding, reconstruction of the
third row doubles it). Ragged volumes (not a multiple of the 128-site block), extents of 2,
both time boundary conditions, the dagger/gamma5 flags, batches and both layouts are
covered; at the full bench sizes (16^4 and 32^4) randomly sampled sites are checked.
"""
import numpy as np
import pytest

import synth
from oracle import wilson

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


def _lattice(ovl, ctx, dims, seed, t_bc=-1, formats=None):
    u = synth.gauge_links(dims, seed)
    lat = ovl.ovl_create_lattice(ctx, dims, t_bc)
    ovl.ovl_set_links(lat, u, formats or (ovl.OVL_F64 | ovl.OVL_F32 | ovl.OVL_F16R12))
    return lat, u


def _ref(u, psi, mu, flags, ovl, t_bc):
    dag = bool(flags & ovl.OVL_DAGGER)
    g5 = bool(flags & ovl.OVL_GAMMA5)
    if dag:  # D^H = g5 D(-mu) g5
        y = wilson.apply_gamma5(wilson.apply_dw(u, wilson.apply_gamma5(psi), -2.0, -mu, t_bc))
    else:
        y = wilson.apply_dw(u, psi, -2.0, mu, t_bc)
    return wilson.apply_gamma5(y) if g5 else y


DIMS = [(4, 4, 4, 4), (6, 6, 6, 6), (2, 4, 6, 8), (2, 2, 2, 2), (8, 2, 4, 6)]


@pytest.mark.parametrize("dims", DIMS)
@pytest.mark.parametrize("t_bc", [-1, 1])
def test_dslash_f64_all_flags(ovl, ctx, dims, t_bc):
    lat, u = _lattice(ovl, ctx, dims, 11, t_bc, ovl.OVL_F64)
    psi = synth.gaussian_source(dims, 12, nrhs=2)
    inp = torch.from_numpy(psi).cuda()
    for flags in (0, ovl.OVL_GAMMA5, ovl.OVL_DAGGER, ovl.OVL_DAGGER | ovl.OVL_GAMMA5):
        for mu in (0.0, 0.3):
            out = torch.empty_like(inp)
            ovl.ovl_apply_DW(lat, -2.0, mu, flags, inp, out)
            got = out.cpu().numpy()
            ref = np.stack([_ref(u, psi[r], mu, flags, ovl, t_bc) for r in range(2)])
            assert np.abs(got - ref).max() <= 1e-13 * np.abs(ref).max(), (flags, mu)
    ovl.ovl_destroy_lattice(lat)


@pytest.mark.parametrize("dims", DIMS[:3])
@pytest.mark.parametrize("links,tol", [("f32", 2e-6), ("f16", 3e-3)])
def test_dslash_f32_links(ovl, ctx, dims, links, tol):
    lat, u = _lattice(ovl, ctx, dims, 13)
    psi = synth.gaussian_source(dims, 14)
    inp = torch.from_numpy(psi).to(torch.complex64).cuda()
    out = torch.empty_like(inp)
    flag = ovl.OVL_LINKS_F16R12 if links == "f16" else ovl.OVL_LINKS_F32
    ovl.ovl_apply_DW(lat, -2.0, 0.3, ovl.OVL_GAMMA5 | flag, inp, out)
    ref = wilson.apply_hw(u, psi, -2.0, 0.3)
    err = np.abs(out.cpu().numpy() - ref).max() / np.abs(ref).max()
    assert err < tol
    ovl.ovl_destroy_lattice(lat)


def test_set_links_again_rewrites_every_held_format(ovl, ctx):
    """A second ovl_set_links that names only FP64 still rewrites the FP32 and FP16 copies the
    lattice holds from the first call: the reduced-precision stencils then apply the new field."""
    dims = (4, 4, 4, 4)
    lat, _ = _lattice(ovl, ctx, dims, 21)
    u2 = synth.gauge_links(dims, 22)
    ovl.ovl_set_links(lat, u2, ovl.OVL_F64)
    psi = synth.gaussian_source(dims, 23)
    ref = wilson.apply_hw(u2, psi, -2.0, 0.3)
    inp = torch.from_numpy(psi).to(torch.complex64).cuda()
    for flag, tol in ((ovl.OVL_LINKS_F32, 2e-6), (ovl.OVL_LINKS_F16R12, 3e-3)):
        out = torch.empty_like(inp)
        ovl.ovl_apply_DW(lat, -2.0, 0.3, ovl.OVL_GAMMA5 | flag, inp, out)
        err = np.abs(out.cpu().numpy() - ref).max() / np.abs(ref).max()
        assert err < tol, (flag, err)
    ovl.ovl_destroy_lattice(lat)


@pytest.mark.parametrize("dtype", ["c128", "c64"])
def test_native_layout_roundtrip(ovl, ctx, dtype):
    dims = (6, 4, 2, 4)
    lat, u = _lattice(ovl, ctx, dims, 15)
    td = torch.complex128 if dtype == "c128" else torch.complex64
    psi = torch.from_numpy(synth.gaussian_source(dims, 16, nrhs=3)).to(td).cuda()
    nat = torch.empty_like(psi)
    ovl.ovl_to_native(lat, psi, nat)
    back = torch.empty_like(psi)
    ovl.ovl_from_native(lat, nat, back)
    torch.cuda.synchronize()
    assert torch.equal(back, psi)
    # native element (rhs, c, site) = canonical (rhs, site, c)
    n3 = nat.reshape(3, 12, -1).cpu()
    c3 = psi.reshape(3, -1, 12).cpu()
    assert torch.equal(n3, c3.transpose(1, 2))
    flags = ovl.OVL_GAMMA5 | (ovl.OVL_LINKS_F32 if dtype == "c64" else 0)
    o_can = torch.empty_like(psi)
    ovl.ovl_apply_DW(lat, -2.0, 0.3, flags, psi, o_can)
    o_nat = torch.empty_like(psi)
    ovl.ovl_apply_DW(lat, -2.0, 0.3, flags | ovl.OVL_NATIVE, nat, o_nat)
    o_back = torch.empty_like(psi)
    ovl.ovl_from_native(lat, o_nat, o_back)
    torch.cuda.synchronize()
    assert torch.equal(o_back, o_can)
    ovl.ovl_destroy_lattice(lat)


def test_gauge_covariance_on_gpu(ovl, ctx):
    dims = (8, 8, 8, 8)
    u = synth.gauge_links(dims, 17)
    g = synth.random_su3_field(dims, 18)
    psi = synth.gaussian_source(dims, 19)
    ug = wilson.gauge_transform(u, g)
    outs = []
    for links, src in ((u, psi), (ug, wilson.gauge_transform_spinor(psi, g))):
        lat = ovl.ovl_create_lattice(ctx, dims, -1)
        ovl.ovl_set_links(lat, links, ovl.OVL_F64)
        inp = torch.from_numpy(src).cuda()
        out = torch.empty_like(inp)
        ovl.ovl_apply_DW(lat, -2.0, 0.3, ovl.OVL_GAMMA5, inp, out)
        outs.append(out.cpu().numpy())
        ovl.ovl_destroy_lattice(lat)
    lhs = outs[1]
    rhs = wilson.gauge_transform_spinor(outs[0], g)
    assert np.abs(lhs - rhs).max() < 1e-12 * np.abs(rhs).max()


def test_rejects_bad_arguments(ovl, ctx):
    with pytest.raises(ovl.OvlError):
        ovl.ovl_create_lattice(ctx, (3, 4, 4, 4), -1)
    with pytest.raises(ovl.OvlError):
        ovl.ovl_create_lattice(ctx, (4, 4, 4, 4), 0)
    dims = (4, 4, 4, 4)
    lat = ovl.ovl_create_lattice(ctx, dims, -1)
    x = torch.zeros(12 * 256, dtype=torch.complex128, device="cuda")
    y = torch.zeros_like(x)
    with pytest.raises(ovl.OvlError) as e:
        ovl.ovl_apply_DW(lat, -2.0, 0.3, 0, x, y)  # no links yet
    assert "links" in str(e.value)
    ovl.ovl_set_links(lat, synth.gauge_links(dims, 1), ovl.OVL_F64)
    with pytest.raises(ovl.OvlError):
        ovl.ovl_apply_DW(lat, -2.0, 0.3, 0, x, x)  # aliasing
    with pytest.raises(ovl.OvlError):
        ovl.ovl_apply_DW(lat, -2.0, 0.3, ovl.OVL_LINKS_F32, x.to(torch.complex64), y.to(torch.complex64))
    ovl.ovl_destroy_lattice(lat)


@pytest.mark.parametrize("dims", [(16, 16, 16, 16), (32, 32, 32, 32)])
def test_full_size_sampled_sites(ovl, ctx, dims):
    """Bench sizes, launch configuration of the bench (FP32 and FP16 links, native layout)."""
    u = synth.gauge_links(dims, 21)
    lat = ovl.ovl_create_lattice(ctx, dims, -1)
    ovl.ovl_set_links(lat, u, ovl.OVL_F64 | ovl.OVL_F32 | ovl.OVL_F16R12)
    psi = synth.gaussian_source(dims, 22)
    inp = torch.from_numpy(psi).cuda()
    rng = np.random.default_rng(0)
    vol = synth.volume(dims)
    sites = np.concatenate([[0, vol - 1], rng.integers(0, vol, 254)])
    ref = wilson.apply_hw_at_sites(u, psi, -2.0, 0.3, sites)
    scale = np.abs(ref).max()
    for dt, flags, tol in ((torch.complex128, 0, 1e-13), (torch.complex64, ovl.OVL_LINKS_F32, 2e-6),
                           (torch.complex64, ovl.OVL_LINKS_F16R12, 3e-3)):
        x = inp.to(dt)
        nat = torch.empty_like(x)
        ovl.ovl_to_native(lat, x, nat)
        out = torch.empty_like(x)
        ovl.ovl_apply_DW(lat, -2.0, 0.3, ovl.OVL_GAMMA5 | ovl.OVL_NATIVE | flags, nat, out)
        can = torch.empty_like(x)
        ovl.ovl_from_native(lat, out, can)
        got = can.reshape(vol, 4, 3)[torch.from_numpy(sites).cuda()].cpu().numpy()
        assert np.abs(got - ref).max() <= tol * scale, (dt, flags)
    ovl.ovl_destroy_lattice(lat)
