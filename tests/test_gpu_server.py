"""Serving: requests of mixed lattices, mu, tolerances and batch sizes admitted by memory
footprint while others run (ovl_submit / ovl_poll). Each result must be the same as the
same request solved alone through ovl_apply_sign (the kernels' arithmetic per right-hand side
does not depend on what else runs, so equality is exact), and the solves must still match
the oracle's sign where one is available.
"""
import time

import numpy as np
import pytest

import synth
from oracle import matsign, wilson

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")


@pytest.fixture(scope="module")
def ovl():
    import paper_0910_1048_gb300 as m
    return m


@pytest.fixture(scope="module")
def env(ovl):
    ctx = ovl.ovl_ctx_create(0)
    fields = []
    for dims, seed in (((4, 4, 4, 4), 0), ((4, 4, 4, 4), 5), ((6, 6, 6, 6), 1), ((2, 2, 2, 4), 35)):
        u = synth.gauge_links(dims, seed, 0.1 if dims == (2, 2, 2, 4) else 0.5)
        lat = ovl.ovl_create_lattice(ctx, dims, -1)
        ovl.ovl_set_links(lat, u, ovl.OVL_F64 | ovl.OVL_F32)
        fields.append((dims, u, lat))
    yield ctx, fields
    for _, _, lat in fields:
        ovl.ovl_destroy_lattice(lat)
    ovl.ovl_ctx_destroy(ctx)


def _alone(ovl, lat, b, mu, tol, k_max, precision):
    p = ovl.ovl_sign_params_default(mu=mu, tol=tol, k_max=k_max, precision=precision)
    x = np.zeros_like(b)
    st, info = ovl.ovl_apply_sign(lat, p, np.ascontiguousarray(b), x)
    return st, x


def test_mixed_stream_matches_alone(ovl, env):
    ctx, fields = env
    rng = np.random.default_rng(42)
    # budget for about two 4^4 FP64 requests at k_max = 400 at a time
    budget = 2 * (401 * 12 * 256 * 16 + 4 * 12 * 256 * 16 + 3 * 12 * 256 * 16 + (1 << 20)) + (1 << 21)
    budget = max(budget, 3 * (401 * 12 * 1296 * 16))  # room for a 6^4 request
    srv = ovl.ovl_server_create(ctx, budget, max_slots=3)
    ids = [ovl.ovl_server_add_field(srv, f[2]) for f in fields]
    reqs = []
    for i in range(10):
        fi = int(rng.integers(0, len(fields)))
        dims = fields[fi][0]
        nrhs = int(rng.integers(1, 3))
        mu = float(rng.uniform(0.0, 0.5))
        tol = float(rng.choice([1e-6, 1e-8]))
        prec = ovl.OVL_PREC_F64 if i % 3 else ovl.OVL_PREC_F32
        b = synth.gaussian_source(dims, 1000 + i, nrhs=nrhs)
        t = ovl.ovl_submit(srv, ids[fi], b, mu, tol, k_max=400, precision=prec)
        reqs.append((t, fi, b, mu, tol, prec, nrhs))
        time.sleep(float(rng.exponential(0.01)))  # arrivals while earlier ones run
    results = {}
    deadline = time.time() + 300
    while len(results) < len(reqs) and time.time() < deadline:
        for t, fi, b, mu, tol, prec, nrhs in reqs:
            if t in results:
                continue
            x = np.zeros_like(b)
            st, info = ovl.ovl_poll(srv, t, nrhs, x)
            if st != ovl.OVL_PENDING:
                results[t] = (st, x, info)
        time.sleep(0.01)
    ovl.ovl_server_destroy(srv)
    assert len(results) == len(reqs)
    for t, fi, b, mu, tol, prec, nrhs in reqs:
        st, x, info = results[t]
        st1, x1 = _alone(ovl, fields[fi][2], b, mu, tol, 400, prec)
        assert st == st1
        assert np.array_equal(x, x1), "request %d differs alone vs in the mix" % t


def test_server_result_matches_oracle(ovl, env):
    ctx, fields = env
    dims, u, lat = fields[3]
    b = synth.gaussian_source(dims, 36)
    xs = matsign.sign_eig(wilson.dense_hw(u, dims, -2.0, 0.3), b.ravel()).reshape(b.shape)
    srv = ovl.ovl_server_create(ctx, 1 << 30, max_slots=2)
    fid = ovl.ovl_server_add_field(srv, lat)
    t = ovl.ovl_submit(srv, fid, b, 0.3, 1e-10, k_max=384)
    x = np.zeros_like(b)
    for _ in range(3000):
        st, info = ovl.ovl_poll(srv, t, 1, x)
        if st != ovl.OVL_PENDING:
            break
        time.sleep(0.01)
    assert st == ovl.OVL_OK, info
    assert np.linalg.norm(x - xs) / np.linalg.norm(xs) < 1e-9
    with pytest.raises(ovl.OvlError) as e:
        ovl.ovl_poll(srv, t, 1, x)  # results are handed out once
    assert e.value.status == ovl.OVL_ENOTFOUND
    ovl.ovl_server_destroy(srv)


def test_two_pass_request(ovl, env):
    """A direct request with two_pass = 1: admitted under a budget too small for its one-pass basis,
    and its result bitwise the same as the two-pass solve alone; a two-pass multishift is refused."""
    ctx, fields = env
    dims, u, lat = fields[2]  # 6^4
    b = synth.gaussian_source(dims, 41, nrhs=2)
    p = ovl.ovl_sign_params_default(mu=0.4, tol=1e-9, k_max=3000, two_pass=1)
    xa = np.zeros_like(b)
    st_a, _ = ovl.ovl_apply_sign(lat, p, np.ascontiguousarray(b), xa)
    # one-pass basis: 2 x 3001 x 12 x 1296 x 16 B = 1.9 GB; the budget admits only the two-pass state
    srv = ovl.ovl_server_create(ctx, 256 << 20, max_slots=2)
    fid = ovl.ovl_server_add_field(srv, lat)
    with pytest.raises(ovl.OvlError):
        ovl.ovl_submit(srv, fid, b, 0.4, 1e-9, k_max=3000)
    t = ovl.ovl_submit(srv, fid, b, 0.4, 1e-9, k_max=3000, two_pass=1)
    res = _drain(ovl, srv, [dict(t=t, b=b, nrhs=2)])
    st, x, info = res[t]
    assert st == st_a == ovl.OVL_OK, info
    assert np.array_equal(x, xa)
    with pytest.raises(ovl.OvlError) as e:
        ovl.ovl_submit(srv, fid, b, 0.4, 1e-9, method=ovl.OVL_MULTISHIFT_BICG, spec_lo=0.05, spec_hi=2.7,
                       two_pass=1)
    assert e.value.status == ovl.OVL_EINVAL
    ovl.ovl_server_destroy(srv)


def test_admission_rejects_oversized(ovl, env):
    ctx, fields = env
    srv = ovl.ovl_server_create(ctx, 1 << 20, max_slots=1)  # 1 MiB: nothing fits
    fid = ovl.ovl_server_add_field(srv, fields[0][2])
    with pytest.raises(ovl.OvlError) as e:
        ovl.ovl_submit(srv, fid, synth.gaussian_source(fields[0][0], 1), 0.3, 1e-8)
    assert e.value.status == ovl.OVL_EINVAL and "budget" in str(e.value)
    ovl.ovl_server_destroy(srv)


def _drain(ovl, srv, reqs, timeout=300):
    results = {}
    deadline = time.time() + timeout
    while len(results) < len(reqs) and time.time() < deadline:
        for r in reqs:
            t, b, nrhs = r["t"], r["b"], r["nrhs"]
            if t in results:
                continue
            x = np.zeros_like(b)
            st, info = ovl.ovl_poll(srv, t, nrhs, x)
            if st != ovl.OVL_PENDING:
                results[t] = (st, x, info)
        time.sleep(0.01)
    return results


def test_mixed_methods_stream_matches_alone(ovl, env, problem_4444):
    """Requests that choose the method and precision (FP64 direct, direct with the field's 16-pair
    deflation set, FP32 multishift with FP64 reliable updates, Zolotarev) run concurrently; each
    result equals the same request solved alone, bitwise."""
    ctx, fields = env
    p4 = problem_4444
    lat0 = fields[0][2]  # 4^4, seed-0 links: the links of problem_4444
    ovl.ovl_set_deflation(lat0, -2.0, 0.3, np.ascontiguousarray(p4["R16"].T), np.ascontiguousarray(p4["L16"].T),
                          p4["lam16"])
    lo, hi = 0.99 * float(np.abs(p4["eig"]).min()), 1.01 * float(np.abs(p4["eig"]).max())
    kinds = [dict(), dict(use_deflation=1), dict(method=ovl.OVL_MULTISHIFT_BICG, precision=ovl.OVL_PREC_F32,
                                                 spec_lo=lo, spec_hi=hi),
             dict(method=ovl.OVL_MULTISHIFT_BICG, rational_kind=ovl.OVL_RAT_ZOLOTAREV, s=24, spec_lo=lo,
                  spec_hi=hi, precision=ovl.OVL_PREC_F32)]
    srv = ovl.ovl_server_create(ctx, 8 << 30, max_slots=4)
    fid = ovl.ovl_server_add_field(srv, lat0)
    reqs = []
    try:
        for i in range(8):
            kw = dict(kinds[i % len(kinds)])
            kw.setdefault("precision", ovl.OVL_PREC_F64)
            nrhs = 1 + i % 2
            b = synth.gaussian_source(p4["dims"], 2000 + i, nrhs=nrhs)
            t = ovl.ovl_submit(srv, fid, b, 0.3, 1e-8, k_max=3000, nrhs=nrhs, **kw)
            reqs.append(dict(t=t, b=b, nrhs=nrhs, kw=kw))
            time.sleep(0.005)
        results = _drain(ovl, srv, reqs)
    finally:
        ovl.ovl_server_destroy(srv)
    assert len(results) == len(reqs)
    for r in reqs:
        st, x, info = results[r["t"]]
        kw = dict(r["kw"])
        p = ovl.ovl_sign_params_default(mu=0.3, tol=1e-8, k_max=3000, **kw)
        x1 = np.zeros_like(r["b"])
        st1, _ = ovl.ovl_apply_sign(lat0, p, np.ascontiguousarray(r["b"]), x1)
        assert st == st1 == ovl.OVL_OK, (kw, st, st1)
        assert np.array_equal(x, x1), kw
    ovl.ovl_set_deflation(lat0, -2.0, 0.3, None, None, None)


def test_field_updates_seen_and_destroy_refused(ovl, env):
    """A field's links are read at every solve: after ovl_set_links on a served field, a new
    request sees the new links (equal to a solve on a fresh lattice holding them); destroying a
    field that a server holds is refused until the server is gone."""
    ctx, fields = env
    dims, u1, lat1 = fields[1]
    srv = ovl.ovl_server_create(ctx, 4 << 30, max_slots=2)
    fid = ovl.ovl_server_add_field(srv, lat1)
    b = synth.gaussian_source(dims, 55)
    try:
        with pytest.raises(ovl.OvlError) as e:
            ovl.ovl_destroy_lattice(lat1)
        assert e.value.status == ovl.OVL_EBUSY
        ra = dict(t=ovl.ovl_submit(srv, fid, b, 0.2, 1e-8, k_max=2000), b=b, nrhs=1)
        xa = _drain(ovl, srv, [ra])[ra["t"]][1]
        u2 = synth.gauge_links(dims, 6)
        ovl.ovl_set_links(lat1, u2, ovl.OVL_F64 | ovl.OVL_F32)
        rb = dict(t=ovl.ovl_submit(srv, fid, b, 0.2, 1e-8, k_max=2000), b=b, nrhs=1)
        stb, xb, _ = _drain(ovl, srv, [rb])[rb["t"]]
    finally:
        ovl.ovl_server_destroy(srv)
        ovl.ovl_set_links(lat1, u1, ovl.OVL_F64 | ovl.OVL_F32)
    fresh = ovl.ovl_create_lattice(ctx, dims, -1)
    ovl.ovl_set_links(fresh, u2, ovl.OVL_F64 | ovl.OVL_F32)
    x2 = np.zeros_like(b)
    st2, _ = ovl.ovl_apply_sign(fresh, ovl.ovl_sign_params_default(mu=0.2, tol=1e-8, k_max=2000), b, x2)
    ovl.ovl_destroy_lattice(fresh)
    assert stb == st2 == ovl.OVL_OK
    assert np.array_equal(xb, x2)
    assert not np.allclose(xa, xb)
