"""Arbitrary source and target point sets on the GPU (bf_plan_create_points) against the
oracle's point-set butterfly: clustered and uniform random points, empty and crowded
leaf boxes, several right-hand sides, FP64 and mixed precision."""
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


def _pts(rng, lo, w, n, d, clustered):
    u = rng.random((n, d))
    if clustered:
        u = np.where(rng.random((n, 1)) < 0.7, 0.15 + 0.1 * u, u)
    return np.asarray(lo[:d]) + u * np.asarray(w[:d])


CASES = [
    (wl.genradon2d(L=5), 3000, 2000, 1, "mixed", True),
    (wl.genradon2d(L=5), 1500, 900, 3, "fp64", False),
    (wl.hypradon(6), 5000, 4000, 2, "mixed", True),
    (wl.dft64().with_(L=3, d=3, q=4, precision="mixed"), 700, 600, 1, "mixed", False),
    (wl.genradon2d(L=4).with_(phase="separable", scale=3.0), 800, 500, 1, "mixed_sfu", True),
]


@pytest.mark.parametrize("spec,nsrc,ntgt,nrhs,prec,clustered", CASES)
def test_points_match_the_oracle(bf, spec, nsrc, ntgt, nrhs, prec, clustered):
    import torch
    rng = np.random.default_rng(nsrc + ntgt)
    x_lo, x_w, y_lo, y_w = spec.domain()
    y = _pts(rng, y_lo, y_w, nsrc, spec.d, clustered)
    x = _pts(rng, x_lo, x_w, ntgt, spec.d, clustered)
    plan = bf.Plan.from_spec(spec, max_nrhs=nrhs, precision=prec, sources=y, targets=x)
    dt = np.complex128 if prec == "fp64" else np.complex64
    g = (rng.standard_normal((nrhs, nsrc)) + 1j * rng.standard_normal((nrhs, nsrc))).astype(dt)
    out = plan.apply(torch.from_numpy(g).cuda()).cpu().numpy()
    assert out.shape == (nrhs, ntgt)
    P = oracle.Problem(**spec.oracle_kwargs())
    ref = oracle.butterfly_points(P, y, g.astype(np.complex128), x)
    tol = {"fp64": 1e-11, "mixed": 1e-5, "mixed_sfu": 2e-5}[prec]
    for j in range(nrhs):
        assert np.linalg.norm(out[j] - ref[j]) <= tol * np.linalg.norm(ref[j]), j
    plan.close()


def test_grid_points_through_the_point_path(bf):
    # the plan's own grid points, shuffled: same operator as the grid plan (FP32 rounding apart)
    import torch
    spec = wl.genradon2d(L=6)
    P = oracle.Problem(**spec.oracle_kwargs())
    rng = np.random.default_rng(3)
    ps, pt = rng.permutation(spec.npts), rng.permutation(spec.npts)
    y, x = oracle.grid_points(P, True)[ps], oracle.grid_points(P, False)[pt]
    pp = bf.Plan.from_spec(spec, sources=y, targets=x)
    pg = bf.Plan.from_spec(spec)
    g = torch.from_numpy(wl.source_values(spec, 1, np.complex64, seed=4)).cuda()
    fg = pg.apply(g)[0]
    fp = pp.apply(g[:, torch.from_numpy(ps).cuda()].contiguous())[0]
    torch.cuda.synchronize()
    fgp = fg[torch.from_numpy(pt).cuda()]
    assert (torch.linalg.vector_norm(fp - fgp) / torch.linalg.vector_norm(fgp)).item() < 2e-6
    pp.close()
    pg.close()


def test_empty_point_sets_and_unsupported_calls(bf):
    import torch
    spec = wl.hypradon(5)
    x_lo, x_w, y_lo, y_w = spec.domain()
    rng = np.random.default_rng(11)
    x = _pts(rng, x_lo, x_w, 50, 2, False)
    p0 = bf.Plan.from_spec(spec, sources=np.zeros((0, 2)), targets=x)
    f = p0.apply(torch.zeros((1, 0), dtype=torch.complex64, device="cuda"))
    assert f.shape == (1, 50) and torch.count_nonzero(f).item() == 0
    y = _pts(rng, y_lo, y_w, 40, 2, False)
    p1 = bf.Plan.from_spec(spec, sources=y, targets=np.zeros((0, 2)))
    f = p1.apply(torch.ones((1, 40), dtype=torch.complex64, device="cuda"))
    assert f.shape == (1, 0)
    with pytest.raises(bf.BfError) as e:
        p0.apply_adjoint(torch.ones((1, 50), dtype=torch.complex64, device="cuda"))
    assert e.value.code == 2
    with pytest.raises(bf.BfError) as e:
        p1.autotune(1)
    assert e.value.code == 2
    p0.close()
    p1.close()
