"""Spectral set-up for deflation and rational approximations, driven through the library.

The paper computes the critical eigenpairs once per matrix and leaves that cost out of its
timings (Section 6, footnote on deflation cost). This module produces them for a lattice
already loaded in the library: ARPACK (scipy) runs in shift-invert form on the host while
every operator application runs on the GPU through the C ABI:
  A^-1 v = A (A^2)^-1 v  is one multishift solve with the single pole omega = 1, sigma = 0;
  A v                    is ovl_apply_DW with the gamma5 flag.
Right eigenvectors come from A = H_W(mu), left ones from A^H = H_W(-mu) (conjugate
eigenvalues); the pairs are matched and scaled to L^H R = I (Section 3).
"""
from __future__ import annotations

import ctypes

import numpy as np


def _inverse_operator(ovl, lat, m_W, mu, tol, k_max, precision=None):
    """A^-1 as a host matvec. precision: OVL_PREC_F64 (default) or OVL_PREC_F32 (FP32 links and
    vectors with FP64 reliable updates to the same tol; the lattice needs FP32 links)."""
    n = ovl.ovl_lattice_n(lat)
    om = np.array([1.0])
    sg = np.array([0.0])
    prec = ovl.OVL_PREC_F64 if precision is None else precision
    p = ovl.ovl_sign_params_default(method=ovl.OVL_MULTISHIFT_BICG, m_W=m_W, mu=mu, tol=tol, k_max=k_max,
                                    rational_kind=ovl.OVL_RAT_CUSTOM, s=1, check_every=50, precision=prec)
    p.omega = om.ctypes.data_as(ctypes.POINTER(ctypes.c_double))
    p.sigma = sg.ctypes.data_as(ctypes.POINTER(ctypes.c_double))
    calls = [0]

    def matvec(v):
        b = np.ascontiguousarray(np.asarray(v, dtype=np.complex128).reshape(n))
        x = np.empty_like(b)
        st, info = ovl.ovl_apply_sign(lat, p, b, x)
        if st != ovl.OVL_OK:
            raise ovl.OvlError(st, "inverse solve did not converge: %r" % info[0])
        calls[0] += 1
        return x

    return matvec, calls, (om, sg)


def critical_eigenpairs(ovl, lat, m_W, mu, m, tol=1e-10, solve_tol=1e-12, k_max=20000, extra=2, ncv=None,
                        precision=None):
    """(lam[m], R[m][n], L[m][n], gap, info): the m eigenvalues of H_W(mu) smallest in modulus,
    canonical-layout right/left eigenvectors with L^H R = I, and gap = |lambda_{m+1}|.
    precision selects the inverse solves (see _inverse_operator); both reach solve_tol."""
    import scipy.sparse.linalg as spla

    n = ovl.ovl_lattice_n(lat)
    nev = m + extra
    ncv = ncv or max(2 * nev + 8, 40)
    mv_r, calls_r, keep_r = _inverse_operator(ovl, lat, m_W, mu, solve_tol, k_max, precision)
    mv_l, calls_l, keep_l = _inverse_operator(ovl, lat, m_W, -mu, solve_tol, k_max, precision)
    op_r = spla.LinearOperator((n, n), matvec=mv_r, dtype=np.complex128)
    op_l = spla.LinearOperator((n, n), matvec=mv_l, dtype=np.complex128)
    v0 = np.ones(n, dtype=np.complex128)
    th_r, vr = spla.eigs(op_r, k=nev, which="LM", tol=tol, ncv=ncv, v0=v0)
    th_l, vl = spla.eigs(op_l, k=nev, which="LM", tol=tol, ncv=ncv, v0=v0)
    lam_r = 1.0 / th_r  # eigenvalues of A from those of A^-1
    lam_l = 1.0 / th_l  # eigenvalues of A^H
    order = np.argsort(np.abs(lam_r))
    lam_r, vr = lam_r[order], vr[:, order]
    R = vr[:, :m].T.copy()
    lam = lam_r[:m].copy()
    L = np.empty_like(R)
    for i in range(m):
        j = int(np.argmin(np.abs(lam_l - np.conj(lam[i]))))
        L[i] = vl[:, j]
    g = np.einsum("in,in->i", np.conj(L), R)
    L = L / np.conj(g)[:, None]
    # the off-diagonal overlaps of eigenvectors of distinct eigenvalues vanish only to the
    # eigensolver's accuracy: replace L by the combination conj(G^-1) L (G = L^H R), which makes
    # L^H R = I to rounding while leaving each l_i a left eigenvector to that same accuracy
    G = np.conj(L) @ R.T
    L = np.conj(np.linalg.inv(G)) @ L
    gap = float(np.abs(lam_r[m]))
    info = {"inverse_solves": calls_r[0] + calls_l[0], "max_LR_offdiag": float(np.abs(np.conj(L) @ R.T - np.eye(m)).max())}
    del keep_r, keep_l
    return lam, R, L, gap, info


def smallest_modulus(ovl, lat, m_W, mu, tol=1e-4, precision=None):
    """|lambda|_min of H_W(mu): the largest-modulus eigenvalue of A^-1 by ARPACK, every A^-1
    application a GPU multishift solve with the single pole (omega, sigma) = (1, 0)."""
    import scipy.sparse.linalg as spla

    n = ovl.ovl_lattice_n(lat)
    mv, _, keep = _inverse_operator(ovl, lat, m_W, mu, 1e-8, 20000, precision)
    op = spla.LinearOperator((n, n), matvec=mv, dtype=np.complex128)
    th = spla.eigs(op, k=1, which="LM", tol=tol, return_eigenvectors=False, v0=np.ones(n, np.complex128))
    del keep
    return float(1.0 / np.abs(th).max())


def largest_modulus(ovl, lat, m_W, mu, tol=1e-6):
    """|lambda|_max of H_W(mu) by ARPACK with GPU matrix-vector products."""
    import scipy.sparse.linalg as spla
    import torch

    n = ovl.ovl_lattice_n(lat)
    dev_in = torch.empty(n, dtype=torch.complex128, device="cuda")
    dev_out = torch.empty_like(dev_in)

    def matvec(v):
        dev_in.copy_(torch.from_numpy(np.ascontiguousarray(np.asarray(v, dtype=np.complex128).reshape(n))))
        ovl.ovl_apply_DW(lat, m_W, mu, ovl.OVL_GAMMA5, dev_in, dev_out)
        return dev_out.cpu().numpy()

    op = spla.LinearOperator((n, n), matvec=matvec, dtype=np.complex128)
    th = spla.eigs(op, k=1, which="LM", tol=tol, return_eigenvectors=False, v0=np.ones(n, np.complex128))
    return float(np.abs(th).max())
