"""Critical eigenpairs for LR deflation (test infrastructure, oracle only).

Section 3 (LR deflation): R_m holds right and L_m left eigenvectors of m critical
eigenvalues, A R_m = R_m Lambda_m, L_m^H A = Lambda_m L_m^H, normalised so that
L_m^H R_m = I_m; P = R_m L_m^H is an oblique projector (P^2 = P) and
f(A) P b = R_m f(Lambda_m) L_m^H b (Eq. exact_proj).
"Critical" is read as smallest modulus, matching the numerical section's deflation gap
("modulus of the smallest non-deflated eigenvalue").
"""
from __future__ import annotations

import numpy as np
import scipy.sparse as sp
import scipy.sparse.linalg as spla

from .gamma import GAMMA, GAMMA5
from .wilson import kappa


def critical_dense(a: np.ndarray, m: int):
    """(lam[m], R[n,m], L[n,m], gap) from a full eigendecomposition; gap = |lambda_{m+1}|."""
    w, r = np.linalg.eig(a)
    rinv = np.linalg.inv(r)
    order = np.argsort(np.abs(w))
    idx = order[:m]
    gap = float(np.abs(w[order[m]])) if m < len(w) else 0.0
    return w[idx], r[:, idx], np.conj(rinv[idx, :]).T, gap


def sparse_hw(links, dims, m_w, mu, t_bc=-1):
    """H_W(mu) = gamma5 D_W(mu) as a scipy CSR matrix (same reading as ``wilson``)."""
    lx, ly, lz, lt = (int(d) for d in dims)
    vol = lx * ly * lz * lt
    k = kappa(m_w)
    t, z, y, x = np.meshgrid(np.arange(lt), np.arange(lz), np.arange(ly), np.arange(lx), indexing="ij")
    t, z, y, x = t.ravel(), z.ravel(), y.ravel(), x.ravel()
    site = ((t * lz + z) * ly + y) * lx + x
    ext = (lx, ly, lz, lt)
    coords = [x, y, z, t]
    u = links.reshape(4, vol, 3, 3)
    one = np.eye(4, dtype=np.complex128)
    rows, cols, vals = [], [], []
    ii, jj = np.meshgrid(np.arange(12), np.arange(12), indexing="ij")
    g5 = np.kron(GAMMA5, np.eye(3))

    def add(src_sites, dst_sites, blocks):
        rows.append((12 * src_sites[:, None, None] + ii[None]).ravel())
        cols.append((12 * dst_sites[:, None, None] + jj[None]).ravel())
        vals.append(np.einsum("ab,sbc->sac", g5, blocks).ravel())

    add(site, site, np.broadcast_to(np.eye(12, dtype=np.complex128), (vol, 12, 12)))
    for nu in range(4):
        cf = [c.copy() for c in coords]
        cf[nu] = (coords[nu] + 1) % ext[nu]
        cb = [c.copy() for c in coords]
        cb[nu] = (coords[nu] - 1) % ext[nu]
        sf = ((cf[3] * lz + cf[2]) * ly + cf[1]) * lx + cf[0]
        sb = ((cb[3] * lz + cb[2]) * ly + cb[1]) * lx + cb[0]
        ef = np.full(vol, np.exp(mu) if nu == 3 else 1.0, dtype=np.complex128)
        eb = np.full(vol, np.exp(-mu) if nu == 3 else 1.0, dtype=np.complex128)
        if nu == 3:
            ef[coords[3] == lt - 1] *= t_bc
            eb[coords[3] == 0] *= t_bc
        bf = -k * ef[:, None, None] * np.einsum("st,xab->xsatb", one - GAMMA[nu], u[nu]).reshape(vol, 12, 12)
        ubd = np.conj(np.swapaxes(u[nu][sb], -1, -2))
        bb = -k * eb[:, None, None] * np.einsum("st,xab->xsatb", one + GAMMA[nu], ubd).reshape(vol, 12, 12)
        add(site, sf, bf)
        add(site, sb, bb)
    n = 12 * vol
    mat = sp.coo_matrix((np.concatenate(vals), (np.concatenate(rows), np.concatenate(cols))), shape=(n, n))
    return mat.tocsr()


def critical_sparse(links, dims, m_w, mu, m, t_bc=-1, ncv=None, tol=1e-13, extra=4):
    """(lam[m], R, L, gap) by ARPACK shift-invert at 0 on H_W(mu) (right) and H_W(-mu) (left).

    Left eigenvectors of A = H_W(mu) are right eigenvectors of A^H = H_W(-mu) with
    conjugated eigenvalues; pairs are matched by eigenvalue and scaled to L^H R = I.
    """
    a = sparse_hw(links, dims, m_w, mu, t_bc).tocsc()
    ah = sparse_hw(links, dims, m_w, -mu, t_bc).tocsc()
    nev = m + extra
    wr, vr = spla.eigs(a, k=nev, sigma=0.0, which="LM", ncv=ncv, tol=tol)
    wl, vl = spla.eigs(ah, k=nev, sigma=0.0, which="LM", ncv=ncv, tol=tol)
    order = np.argsort(np.abs(wr))
    wr, vr = wr[order], vr[:, order]
    lam = wr[:m]
    R = vr[:, :m]
    L = np.empty_like(R)
    for i in range(m):
        j = int(np.argmin(np.abs(wl - np.conj(lam[i]))))
        L[:, i] = vl[:, j]
    # biorthonormalise: L^H R should be diagonal for distinct eigenvalues
    g = np.conj(L).T @ R
    L = L / np.conj(np.diag(g))[None, :]
    gap = float(np.abs(wr[m]))
    return lam, R, L, gap
