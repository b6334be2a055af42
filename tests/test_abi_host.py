"""C-ABI checks that need no GPU: the library loads, exports every function declared in
include/ovl.h, and its host-side pieces agree with the oracle:
  - ovl_small_sign (sign(H_k) e_1, Section 2 / Algorithm 4's last line) vs eigendecomposition,
    for each route (rational g_s(cH) e_1, complex-symmetric eigenvectors, dense Newton);
  - ovl_rational_coeffs (Eq. pfe_s with Eq. no_of_poles; Zolotarev) vs the oracle's coefficients;
  - argument errors come back as EINVAL with a message, not a crash;
  - the pair-stencil shape table (ovl_set_pair_variant / ovl_get_pair_variant): set, read back,
    cleared, refused outside its range.
"""
import os
import re

import numpy as np
import pytest

import synth
from oracle import deflation, lanczos, rational

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module")
def ovl():
    import paper_0910_1048_gb300 as m
    return m


def _declared_functions():
    src = open(os.path.join(ROOT, "include", "ovl.h")).read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    return sorted(set(re.findall(r"\b(ovl_[a-zA-Z0-9_]+)\s*\(", src)))


def test_exports_every_declared_symbol(ovl):
    names = _declared_functions()
    assert len(names) >= 20
    for n in names:
        assert hasattr(ovl.lib, n), n
    assert ovl.ovl_version().startswith("ovl")


def _lanczos_t(mu, k, seed=51, dims=(2, 2, 4, 4)):
    u = synth.gauge_links(dims, seed)
    a = deflation.sparse_hw(u, dims, -2.0, mu)
    ah = deflation.sparse_hw(u, dims, -2.0, -mu)
    b = synth.gaussian_source(dims, seed + 1).ravel()
    st = lanczos.two_sided_lanczos(lambda v: a @ v, lambda w: ah @ w, b, b, k)
    return st["alpha"], st["beta"], st["delta"]


@pytest.mark.parametrize("mu,k", [(0.0, 30), (0.3, 10), (0.3, 60), (0.3, 150), (1.0, 80)])
@pytest.mark.parametrize("method", [0, 1, 2, 3])
def test_small_sign_matches_eig(ovl, mu, k, method):
    al, be, de = _lanczos_t(mu, k)
    ref = lanczos.sign_tridiag_e1(al, be, de)
    st, y = ovl.ovl_small_sign(al, be, de, method)
    if method == 1 and st != ovl.OVL_OK:
        pytest.skip("QL route declined (checked fallback exists): status %d" % st)
    assert st == ovl.OVL_OK
    # the eigenvector route is limited by cond(Z)^2 u; the rational and Newton routes are not
    tol = 1e-9 if method == 1 else 1e-11
    assert np.linalg.norm(y - ref) / np.linalg.norm(ref) < tol


@pytest.mark.parametrize("mu,k", [(0.3, 400), (0.8, 600)])
def test_rational_route_at_large_k(ovl, mu, k):
    """The rational route alone (method 3: its scale c and pole count s come from the Ritz values of
    H_k, no fallback) on H_k of the C oracle's Algorithm 4 at 4^4, against the eigendecomposition."""
    from oracle import krylov

    dims = (4, 4, 4, 4)
    s = krylov.DirectSolve(synth.gauge_links(dims, 0), dims, -2.0, mu, synth.gaussian_source(dims, 1000), k).start()
    s.steps(k)
    al, be, de = s.alpha[:k], s.beta[:k - 1], s.delta[:k - 1]
    ref = lanczos.sign_tridiag_e1(al, be, de)
    st, y = ovl.ovl_small_sign(al, be, de, 3)
    assert st == ovl.OVL_OK
    assert np.linalg.norm(y - ref) / np.linalg.norm(ref) < 1e-10


def test_small_sign_closed_forms(ovl):
    # 1x1 and a 2x2 with eigenvalues of opposite sign: sign(T) e1 from the 2x2 formula
    assert ovl.ovl_small_sign([2.0 + 1j], [], [])[1][0] == 1
    assert ovl.ovl_small_sign([-0.5 + 3j], [], [])[1][0] == -1
    a, d, b, c = 1.0, -2.0, 0.7, 0.4  # T = [[a, b], [c, d]]
    t = np.array([[a, b], [c, d]], dtype=complex)
    w, r = np.linalg.eig(t)
    ref = (r * np.sign(w.real)) @ np.linalg.inv(r)
    st, y = ovl.ovl_small_sign([a, d], [b], [c])
    assert st == 0 and np.abs(y - ref[:, 0]).max() < 1e-13


def test_small_sign_rejects_bad_args(ovl):
    with pytest.raises(ovl.OvlError) as e:
        ovl.ovl_small_sign([], [], [])
    assert e.value.status == ovl.OVL_EINVAL


@pytest.mark.parametrize("lo,hi,eps", [(0.05, 2.5, 1e-8), (0.1, 2.6, 1e-10), (0.2, 3.0, 1e-6)])
def test_neuberger_coeffs_match_oracle(ovl, lo, hi, eps):
    om, sg, err = ovl.ovl_rational_coeffs(ovl.OVL_RAT_NEUBERGER, 0, lo, hi, eps)
    s, c, w, sgo = rational.neuberger_for_spectrum(lo, hi, eps)
    assert len(om) == s
    assert np.abs(om - w).max() < 1e-12 * np.abs(w).max()
    assert np.abs(sg - sgo).max() < 1e-12 * np.abs(sgo).max()
    assert err <= eps


@pytest.mark.parametrize("n,lo,hi", [(1, 0.1, 1.0), (6, 1.0, 10.0), (20, 0.05, 2.6)])
def test_zolotarev_coeffs_match_oracle(ovl, n, lo, hi):
    om, sg, err = ovl.ovl_rational_coeffs(ovl.OVL_RAT_ZOLOTAREV, n, lo, hi)
    w, sgo, erro = rational.zolotarev(n, lo, hi)
    assert np.abs(om - w).max() < 1e-8 * np.abs(w).max()
    assert np.abs(sg - sgo).max() < 1e-10 * np.abs(sgo).max()
    assert abs(err - erro) < 1e-3 * erro + 1e-15


def test_rational_rejects_bad_interval(ovl):
    with pytest.raises(ovl.OvlError) as e:
        ovl.ovl_rational_coeffs(ovl.OVL_RAT_NEUBERGER, 0, 1.0, 0.5, 1e-8)
    assert e.value.status == ovl.OVL_EINVAL
    assert "lo" in str(e.value)


def test_submit_nrhs_inference(ovl):
    """A single canonical spinor is one right-hand side; a 7-D array is a batch."""
    one = np.zeros((4, 2, 2, 2, 4, 3), np.complex128)
    many = np.zeros((3, 4, 2, 2, 2, 4, 3), np.complex128)
    assert ovl._nrhs_of(one, None) == 1
    assert ovl._nrhs_of(many, None) == 3
    assert ovl._nrhs_of(one.ravel(), 1) == 1
    with pytest.raises(ValueError):
        ovl._nrhs_of(one.ravel(), None)


def test_sign_buffers_refused_before_the_library(ovl, monkeypatch):
    """b / x that would let a kernel write out of bounds or read a host pointer are refused in the
    binding: wrong dtype, sizes that are not whole spinors, x shorter than b, host/device mixes."""
    import torch

    n = 3072
    monkeypatch.setattr(ovl, "ovl_lattice_n", lambda lat: n)
    lat = ovl.ctypes.c_void_p(12345)
    good = np.zeros(n, np.complex128)
    cases = [
        (np.zeros(n, np.complex64), np.zeros(n, np.complex64)),       # not complex128
        (np.zeros(n + 1, np.complex128), np.zeros(n + 1, np.complex128)),  # not whole spinors
        (good, np.zeros(n - 12, np.complex128)),                        # x shorter than b
        (good, torch.zeros(n, dtype=torch.complex128)),                 # host / torch mix
        (torch.zeros(n, dtype=torch.complex128), torch.zeros(n, dtype=torch.complex128)),  # CPU tensors
        (np.zeros((2, n), np.complex128)[:, ::2], good),                # not contiguous
    ]
    p = ovl.ovl_sign_params_default()
    for b, x in cases:
        with pytest.raises((TypeError, ValueError)):
            ovl.ovl_apply_sign(lat, p, b, x)
        with pytest.raises((TypeError, ValueError)):
            ovl.ovl_apply_sign_noalloc(lat, p, b, x)


def test_stencil_and_set_up_buffers_refused_before_the_library(ovl, monkeypatch):
    """The stencil and layout calls take CUDA tensors only (a host pointer would reach a kernel);
    links and deflation vectors must be complex128 of the lattice's sizes (a short or mistyped
    buffer would be read out of bounds by the copies)."""
    import torch

    n = 3072
    monkeypatch.setattr(ovl, "ovl_lattice_n", lambda lat: n)
    lat = ovl.ctypes.c_void_p(12345)
    spinor_cases = [
        (np.zeros(n, np.complex128), np.zeros(n, np.complex128)),                     # host arrays
        (torch.zeros(n, dtype=torch.complex128), torch.zeros(n, dtype=torch.complex128)),  # CPU tensors
    ]
    for fn in (lambda a, b: ovl.ovl_apply_DW(lat, -2.0, 0.3, 0, a, b),
               lambda a, b: ovl.ovl_to_native(lat, a, b),
               lambda a, b: ovl.ovl_from_native(lat, a, b)):
        for a, b in spinor_cases:
            with pytest.raises(TypeError):
                fn(a, b)
    links = 3 * n  # 4 directions x 9 colour entries per site = 36 V = 3 n
    for U in (np.zeros(links - 9, np.complex128),                  # too short
              torch.zeros(links, dtype=torch.complex64),            # complex64 tensor
              torch.zeros(2 * links, dtype=torch.complex128)[::2],  # not contiguous
              [0.0] * links):                                        # not an array
        with pytest.raises((TypeError, ValueError)):
            ovl.ovl_set_links(lat, U, ovl.OVL_F64)
    m = 2
    R = np.zeros((m, n), np.complex128)
    for args in ((R, np.zeros((m, n - 1), np.complex128), np.zeros(m, np.complex128)),   # L too short
                 (R, R, np.zeros(m + 1, np.complex128)),                                 # lambda too long
                 (R, torch.zeros(m * n, dtype=torch.complex64), np.zeros(m, np.complex128))):
        with pytest.raises((TypeError, ValueError)):
            ovl.ovl_set_deflation(lat, -2.0, 0.3, *args)


def test_pair_variant_table(ovl):
    vol = 6 * 6 * 6 * 10  # a volume no other test solves
    assert ovl.ovl_get_pair_variant(vol, ovl.OVL_PREC_F32) == -1
    ovl.ovl_set_pair_variant(vol, ovl.OVL_PREC_F32, 5)
    assert ovl.ovl_get_pair_variant(vol, ovl.OVL_PREC_F32) == 5
    assert ovl.ovl_get_pair_variant(vol, ovl.OVL_PREC_F64) == -1
    ovl.ovl_set_pair_variant(vol, ovl.OVL_PREC_F32, -1)
    assert ovl.ovl_get_pair_variant(vol, ovl.OVL_PREC_F32) == -1
    for args in [(vol, ovl.OVL_PREC_F64, 9), (vol, ovl.OVL_PREC_F64, -2), (0, ovl.OVL_PREC_F64, 1),
                 (vol, 3, 1), (1 << 27, ovl.OVL_PREC_F64, 0)]:
        with pytest.raises(ovl.OvlError) as e:
            ovl.ovl_set_pair_variant(*args)
        assert e.value.status == ovl.OVL_EINVAL and "ovl_set_pair_variant" in str(e.value)
    assert ovl.ovl_get_pair_variant(vol, 7) == -1
