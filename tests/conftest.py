"""Shared fixtures. GPU tests are marked ``gpu``; everything else runs on CPU."""
import os
import sys

import numpy as np
import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)


def pytest_configure(config):
    config.addinivalue_line("markers", "gpu: needs a CUDA GPU (GB300) and the built library")
    config.addinivalue_line("markers", "slow: takes more than a few seconds on CPU")


def read_paper_values():
    """The values the paper prints (tests/golden/paper_values.txt, each line citing its passage),
    as {key: float}."""
    vals = {}
    with open(os.path.join(ROOT, "tests", "golden", "paper_values.txt")) as f:
        for line in f:
            line = line.split("#", 1)[0].strip()
            if line:
                k, v = (x.strip() for x in line.split("=", 1))
                vals[k] = float(v)
    return vals


@pytest.fixture(scope="session")
def paper():
    return read_paper_values()


def fp16_quantised(u):
    """Links as the FP16 12-real format stores them: the first two rows' real and imaginary parts
    rounded to float32 and then to float16, the third row rebuilt as conj(row1 x row2) (SU(3)).
    Oracles that run on these links see the same operator as the library's FP16-link stencil, so
    a comparison measures the FP32 arithmetic alone."""
    q = u.copy()
    r01 = u[..., :2, :]
    rr = r01.real.astype(np.float32).astype(np.float16).astype(np.float64)
    ri = r01.imag.astype(np.float32).astype(np.float16).astype(np.float64)
    q[..., :2, :] = rr + 1j * ri
    q[..., 2, :] = np.conj(np.cross(q[..., 0, :], q[..., 1, :]))
    return q


@pytest.fixture(scope="session")
def problem_4444():
    """4^4, seed-0 links, m_W=-2, mu=0.3, antiperiodic t, Gaussian b (seed 1000):
    dense H_W, x* = sign(H_W) b by eigendecomposition, and 16 critical eigenpairs."""
    import synth
    from oracle import deflation, matsign

    dims = (4, 4, 4, 4)
    u = synth.gauge_links(dims, 0)
    b = synth.gaussian_source(dims, 1000)
    h = deflation.sparse_hw(u, dims, -2.0, 0.3).toarray()
    w, r = np.linalg.eig(h)
    rinv = np.linalg.inv(r)
    xs = r @ (np.sign(w.real) * (rinv @ b.ravel()))
    order = np.argsort(np.abs(w))
    idx = order[:16]
    return {
        "dims": dims, "links": u, "b": b, "h": h, "xstar": xs.reshape(b.shape),
        "lam16": w[idx], "R16": r[:, idx], "L16": np.conj(rinv[idx, :]).T,
        "gap16": float(abs(w[order[16]])), "eig": w,
    }
