"""Pins of the C FP64 Krylov oracle (oracle/krylov.c): the operator, the recurrence, the solve.

Each check compares against something other than the C code itself: the sparse H_W of
``oracle.deflation`` (pinned by its own constructions and invariants), the free-field closed
form of ``oracle.freefield`` (momentum space, any size), gamma5-hermiticity, the Python
recurrence of ``oracle.lanczos`` at equal k, and the dense x* = sign(H_W) b (eigendecomposition).
"""
import numpy as np
import pytest

import synth
from oracle import deflation, freefield, krylov, lanczos


@pytest.mark.parametrize("dims,t_bc,mu", [((4, 4, 4, 4), -1, 0.3), ((2, 4, 6, 4), 1, 0.7), ((4, 2, 2, 6), -1, 0.0)])
def test_operator_equals_sparse(dims, t_bc, mu):
    u = synth.gauge_links(dims, 3)
    psi = synth.gaussian_source(dims, 5)
    a = deflation.sparse_hw(u, dims, -2.0, mu, t_bc)
    got = krylov.apply_hw(u, dims, -2.0, mu, psi, t_bc)
    ref = (a @ psi.ravel()).reshape(psi.shape)
    assert np.abs(got - ref).max() <= 1e-14 * np.abs(ref).max()


def test_operator_free_field_closed_form():
    dims = (6, 4, 4, 8)
    u = synth.unit_links(dims)
    psi = synth.gaussian_source(dims, 7)
    got = krylov.apply_hw(u, dims, -2.0, 0.4, psi)
    dpsi = freefield.apply_dw_free(psi, dims, -2.0, 0.4)
    ref = dpsi.copy()
    ref[..., 2:, :] *= -1  # gamma5 = diag(1, 1, -1, -1)
    assert np.abs(got - ref).max() <= 1e-12 * np.abs(ref).max()


def test_operator_gamma5_hermiticity():
    """<w, H(mu) v> = <H(-mu) w, v>: H_W(mu)^H = H_W(-mu)."""
    dims = (4, 4, 2, 6)
    u = synth.gauge_links(dims, 11)
    v = synth.gaussian_source(dims, 12)
    w = synth.gaussian_source(dims, 13)
    lhs = np.vdot(w, krylov.apply_hw(u, dims, -2.0, 0.5, v))
    rhs = np.vdot(krylov.apply_hw(u, dims, -2.0, -0.5, w), v)
    assert abs(lhs - rhs) <= 1e-12 * abs(lhs)


def test_recurrence_equals_python_oracle():
    dims = (4, 4, 4, 4)
    u = synth.gauge_links(dims, 0)
    b = synth.gaussian_source(dims, 1000)
    a = deflation.sparse_hw(u, dims, -2.0, 0.3)
    ah = deflation.sparse_hw(u, dims, -2.0, -0.3)
    k = 30
    st = lanczos.two_sided_lanczos(lambda v: a @ v, lambda w: ah @ w, b.ravel(), b.ravel(), k)
    s = krylov.DirectSolve(u, dims, -2.0, 0.3, b, k).start()
    s.steps(k)
    assert s.k == k and not s.breakdown
    assert abs(s.beta0 - st["beta0"]) <= 1e-14 * st["beta0"]
    scale = np.abs(st["alpha"]).max()
    assert np.abs(s.alpha[:k] - st["alpha"]).max() <= 1e-11 * scale
    assert np.abs(s.beta[:k - 1] - st["beta"]).max() <= 1e-11 * scale
    assert np.abs(s.delta[:k - 1] - st["delta"]).max() <= 1e-11 * scale
    assert np.abs(s.V[:k].T - st["V"]).max() <= 1e-10


def test_steps_in_pieces_equal_one_run():
    dims = (4, 4, 2, 4)
    u = synth.gauge_links(dims, 2)
    b = synth.gaussian_source(dims, 3)
    x1, s1, _ = krylov.direct_lanczos(u, dims, -2.0, 0.2, b, 40)
    s2 = krylov.DirectSolve(u, dims, -2.0, 0.2, b, 40).start()
    for m in (7, 13, 1, 19):
        s2.steps(m)
    x2 = s2.finish()
    assert s2.k == 40
    assert np.array_equal(x1, x2)


def test_converges_to_dense_sign(problem_4444):
    p = problem_4444
    x, s, _ = krylov.direct_lanczos(p["links"], p["dims"], -2.0, 0.3, p["b"], 1100)
    rel = np.linalg.norm(x - p["xstar"]) / np.linalg.norm(p["xstar"])
    assert rel < 1e-10


def test_deflated_solve(problem_4444):
    """Algorithm 4 with the 16 critical eigenpairs (x_P exact on the deflated part): fewer steps
    than the undeflated solve to the same accuracy."""
    p = problem_4444
    x, s, _ = krylov.direct_lanczos(p["links"], p["dims"], -2.0, 0.3, p["b"], 800, R=p["R16"], L=p["L16"],
                                    lam=p["lam16"])
    rel = np.linalg.norm(x - p["xstar"]) / np.linalg.norm(p["xstar"])
    assert rel < 1e-10


def test_free_field_8888_closed_form():
    """At 8^4 (no dense x*), the unit-link solve against the momentum-space closed form."""
    dims = (8, 8, 8, 8)
    u = synth.unit_links(dims)
    b = synth.gaussian_source(dims, 21)
    xs = freefield.sign_hw_free(b, dims, -2.0, 0.3)
    x, s, _ = krylov.direct_lanczos(u, dims, -2.0, 0.3, b, 400)
    rel = np.linalg.norm(x - xs) / np.linalg.norm(xs)
    assert rel < 1e-9, rel
