"""CGLS on B^H B m = B^H d with d = B m_true (m_true: 1% sparse spikes, N(0,1) amplitudes):
the GPU run (forward + adjoint kernels) against the same iteration driven by the FP64
oracle, and monotone residuals at N = 1024."""
import numpy as np
import pytest

import oracle
from paper_1305_4650_gb300 import workloads as wl

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def bf():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1305_4650_gb300 import build, bf as bfmod
    build.build()
    return bfmod


def cgls_oracle(P, d, iters):
    m = np.zeros_like(d)
    r = d.copy()
    s = oracle.butterfly_adjoint(P, r)
    p = s.copy()
    gamma = np.vdot(s, s).real
    hist = [np.linalg.norm(r)]
    for _ in range(iters):
        q = oracle.butterfly(P, p)
        alpha = gamma / np.vdot(q, q).real
        m = m + alpha * p
        r = r - alpha * q
        s = oracle.butterfly_adjoint(P, r)
        gn = np.vdot(s, s).real
        p = s + (gn / gamma) * p
        gamma = gn
        hist.append(np.linalg.norm(r))
    return m, np.array(hist)


@pytest.mark.parametrize("precision,tol", [("fp64", 1e-9), ("mixed", 1e-3)])
def test_cgls_matches_oracle_n32(bf, precision, tol):
    import torch
    from paper_1305_4650_gb300.autograd import cgls
    spec = wl.genradon2d(L=5)
    P = oracle.Problem(**spec.oracle_kwargs())
    mt = wl.sparse_spikes(spec, 0.01, dtype=np.complex128)
    d = oracle.butterfly(P, mt)
    _, href = cgls_oracle(P, d, 20)
    plan = bf.Plan.from_spec(spec, precision=precision)
    dt = torch.complex128 if precision == "fp64" else torch.complex64
    _, hist = cgls(plan, torch.from_numpy(d).to(dt).cuda(), 20)
    plan.close()
    hist = np.array(hist)
    assert np.all(np.diff(hist) <= 1e-6 * hist[0])
    assert np.max(np.abs(hist - href) / href[0]) <= tol


def test_cgls_n1024_residual_decreases(bf):
    import torch
    from paper_1305_4650_gb300.autograd import cgls
    spec = wl.genradon2d()
    plan = bf.Plan.from_spec(spec, precision="mixed")
    mt = torch.from_numpy(wl.sparse_spikes(spec, 0.01)).cuda()
    d = plan.apply(mt)
    m, hist = cgls(plan, d, 20)
    plan.close()
    hist = np.array(hist)
    assert np.all(np.diff(hist) <= 1e-5 * hist[0]), hist
    assert hist[-1] < 0.2 * hist[0]
