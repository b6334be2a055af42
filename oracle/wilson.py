"""Wilson-Dirac operator at chemical potential mu (test infrastructure, oracle only).

The paper's kernel is H_W = gamma5 D_W(mu) (Section 1; parameters m_W = -2, m_q = 0,
mu = 0.3 in Section 6) and defers D_W's notation to its reference [Bloch:2006cd].
Reading used (kappa normalisation, kappa = 1/(2 m_W + 8), = 1/4 at m_W = -2):

  (D_W psi)(x) = psi(x)
     - kappa sum_{nu=x,y,z} [ (1 - g_nu) U_nu(x) psi(x+nu) + (1 + g_nu) U_nu(x-nu)^H psi(x-nu) ]
     - kappa [ e^{+mu} (1 - g_t) U_t(x) psi(x+t) + e^{-mu} (1 + g_t) U_t(x-t)^H psi(x-t) ]

periodic in space, periodic (t_bc = +1) or antiperiodic (t_bc = -1, default) in time;
a hop that crosses the t boundary is multiplied by t_bc. Positive mu sits on forward
temporal hops. Spinor index (site, spin, colour), colour fastest; canonical site index
((t*Lz + z)*Ly + y)*Lx + x.
"""
from __future__ import annotations

import numpy as np

from .gamma import GAMMA, GAMMA5

# numpy axis of each direction in a [Lt][Lz][Ly][Lx] site array
_AXIS = {0: 3, 1: 2, 2: 1, 3: 0}


def kappa(m_w: float) -> float:
    return 1.0 / (2.0 * m_w + 8.0)


def _coords(dims):
    lx, ly, lz, lt = dims
    t, z, y, x = np.meshgrid(np.arange(lt), np.arange(lz), np.arange(ly), np.arange(lx), indexing="ij")
    return x.ravel(), y.ravel(), z.ravel(), t.ravel()


def site_index(dims, x, y, z, t):
    lx, ly, lz, lt = dims
    return ((t * lz + z) * ly + y) * lx + x


def dense_dw(links: np.ndarray, dims, m_w: float, mu: float, t_bc: int = -1) -> np.ndarray:
    """Dense n x n D_W(mu), n = 12 V, built site by site and hop by hop."""
    dims = tuple(int(d) for d in dims)
    lx, ly, lz, lt = dims
    vol = lx * ly * lz * lt
    n = 12 * vol
    k = kappa(m_w)
    d = np.eye(n, dtype=np.complex128)
    u = links.reshape(4, vol, 3, 3)
    one = np.eye(4, dtype=np.complex128)
    ext = (lx, ly, lz, lt)
    xs, ys, zs, ts = _coords(dims)
    for s in range(vol):
        c = [int(xs[s]), int(ys[s]), int(zs[s]), int(ts[s])]
        for nu in range(4):
            fwd = list(c)
            fwd[nu] = (c[nu] + 1) % ext[nu]
            bwd = list(c)
            bwd[nu] = (c[nu] - 1) % ext[nu]
            sf = site_index(dims, *fwd)
            sb = site_index(dims, *bwd)
            ef = np.exp(mu) if nu == 3 else 1.0
            eb = np.exp(-mu) if nu == 3 else 1.0
            if nu == 3 and c[3] == lt - 1:
                ef *= t_bc
            if nu == 3 and c[3] == 0:
                eb *= t_bc
            blk_f = -k * ef * np.kron(one - GAMMA[nu], u[nu, s])
            blk_b = -k * eb * np.kron(one + GAMMA[nu], np.conj(u[nu, sb]).T)
            d[12 * s:12 * s + 12, 12 * sf:12 * sf + 12] += blk_f
            d[12 * s:12 * s + 12, 12 * sb:12 * sb + 12] += blk_b
    return d


def dense_hw(links, dims, m_w, mu, t_bc=-1) -> np.ndarray:
    """Dense H_W(mu) = gamma5 D_W(mu)."""
    dims = tuple(int(d) for d in dims)
    vol = int(np.prod(dims))
    g5 = np.kron(np.eye(vol), np.kron(GAMMA5, np.eye(3)))
    return g5 @ dense_dw(links, dims, m_w, mu, t_bc)


def apply_dw(links: np.ndarray, psi: np.ndarray, m_w: float, mu: float, t_bc: int = -1) -> np.ndarray:
    """Matrix-free D_W(mu) psi on canonical arrays (psi[Lt][Lz][Ly][Lx][4][3])."""
    k = kappa(m_w)
    lt = psi.shape[0]
    out = psi.astype(np.complex128, copy=True)
    one = np.eye(4, dtype=np.complex128)
    for nu in range(4):
        ax = _AXIS[nu]
        u = links[nu]
        pf = np.roll(psi, -1, axis=ax)
        ub = np.roll(u, 1, axis=ax)
        pb = np.roll(psi, 1, axis=ax)
        if nu == 3:
            pf = pf.copy()
            pb = pb.copy()
            pf[lt - 1] *= t_bc
            pb[0] *= t_bc
        hf = np.einsum("...ab,...sb->...sa", u, pf)
        hb = np.einsum("...ba,...sb->...sa", np.conj(ub), pb)
        ef = np.exp(mu) if nu == 3 else 1.0
        eb = np.exp(-mu) if nu == 3 else 1.0
        out -= k * ef * np.einsum("st,...tb->...sb", one - GAMMA[nu], hf)
        out -= k * eb * np.einsum("st,...tb->...sb", one + GAMMA[nu], hb)
    return out


def apply_gamma5(psi: np.ndarray) -> np.ndarray:
    return np.einsum("st,...tb->...sb", GAMMA5, psi)


def apply_hw(links, psi, m_w, mu, t_bc=-1) -> np.ndarray:
    """Matrix-free H_W(mu) psi = gamma5 D_W(mu) psi."""
    return apply_gamma5(apply_dw(links, psi, m_w, mu, t_bc))


def apply_dw_at_sites(links, psi, m_w, mu, sites, t_bc=-1) -> np.ndarray:
    """(D_W(mu) psi)(x) for a list of canonical site indices only; returns [len(sites)][4][3].

    Computed one site at a time from its eight neighbours, for spot checks of
    lattices too large to sweep in Python.
    """
    lt, lz, ly, lx = psi.shape[:4]
    dims = (lx, ly, lz, lt)
    ext = (lx, ly, lz, lt)
    k = kappa(m_w)
    vol = lx * ly * lz * lt
    pf = psi.reshape(vol, 4, 3)
    u = links.reshape(4, vol, 3, 3)
    one = np.eye(4, dtype=np.complex128)
    res = np.empty((len(sites), 4, 3), dtype=np.complex128)
    for i, s in enumerate(sites):
        s = int(s)
        c = [s % lx, (s // lx) % ly, (s // (lx * ly)) % lz, s // (lx * ly * lz)]
        acc = pf[s].copy()
        for nu in range(4):
            fwd = list(c)
            fwd[nu] = (c[nu] + 1) % ext[nu]
            bwd = list(c)
            bwd[nu] = (c[nu] - 1) % ext[nu]
            sf = site_index(dims, *fwd)
            sb = site_index(dims, *bwd)
            ef = np.exp(mu) if nu == 3 else 1.0
            eb = np.exp(-mu) if nu == 3 else 1.0
            if nu == 3 and c[3] == lt - 1:
                ef *= t_bc
            if nu == 3 and c[3] == 0:
                eb *= t_bc
            acc -= k * ef * (one - GAMMA[nu]) @ (pf[sf] @ u[nu, s].T)
            acc -= k * eb * (one + GAMMA[nu]) @ (pf[sb] @ np.conj(u[nu, sb]))
        res[i] = acc
    return res


def apply_hw_at_sites(links, psi, m_w, mu, sites, t_bc=-1) -> np.ndarray:
    return np.einsum("st,...tb->...sb", GAMMA5, apply_dw_at_sites(links, psi, m_w, mu, sites, t_bc))


def gauge_transform(links: np.ndarray, g: np.ndarray) -> np.ndarray:
    """U_nu(x) -> G(x) U_nu(x) G(x+nu)^H (periodic shift; boundary signs live in D_W)."""
    out = np.empty_like(links)
    for nu in range(4):
        gf = np.roll(g, -1, axis=_AXIS[nu])
        out[nu] = np.einsum("...ab,...bc,...dc->...ad", g, links[nu], np.conj(gf))
    return out


def gauge_transform_spinor(psi: np.ndarray, g: np.ndarray) -> np.ndarray:
    return np.einsum("...ab,...sb->...sa", g, psi)
