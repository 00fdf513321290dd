"""bf_apply_noalloc against bf_apply (GPU).

bf_apply_noalloc serves callers that cannot allocate device memory -- an
application that owns all GPU memory through its own fixed pool, or code that
must not allocate once it runs.  It keeps its tables and workspace in a static
device array shared by every call.  This file is collected last so that a run
stopping at the first failure has already run every other test; it also passes
on its own in a fresh process.
"""
import numpy as np
import pytest

from paper_1305_4650_gb300 import workloads as wl

pytestmark = pytest.mark.gpu

TOL = {"mixed": 1e-5, "fp64": 1e-11}     # the parity tolerances of the d = 2 tests


@pytest.fixture(scope="module")
def bf():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1305_4650_gb300 import build, bf as bfmod
    build.build()
    return bfmod


def _call(bf, spec, precision, g, f):
    x_lo, x_w, y_lo, y_w = spec.domain()
    bf.apply_noalloc(spec.d, spec.N, spec.q, spec.phase, g, f, precision=precision, scale=spec.scale,
                     x_lo=x_lo, x_w=x_w, y_lo=y_lo, y_w=y_w, tgt_off=spec.tgt_off, src_off=spec.src_off,
                     switch_level=spec.switch_level, node_kind=spec.node_kind)


@pytest.mark.parametrize("precision", ["mixed", "fp64"])
def test_noalloc_matches_plan_apply_on_two_calls(bf, precision):
    import torch
    spec = wl.genradon2d(L=7)                      # N = 128, q = 5: the largest d = 2 size the array admits
    dt = np.complex128 if precision == "fp64" else np.complex64
    plan = bf.Plan.from_spec(spec, precision=precision)
    for call in range(2):
        g = torch.from_numpy(wl.source_values(spec, 1, dt, seed=200 + call)).cuda()
        ref = plan.apply(g)
        out = torch.full_like(g, float("nan"))
        _call(bf, spec, precision, g, out)
        torch.cuda.synchronize()
        a, b = out.cpu().numpy(), ref.cpu().numpy()
        err = float(np.linalg.norm(a - b) / np.linalg.norm(b))
        assert err <= TOL[precision], (call, err)
    plan.close()


def test_noalloc_d3_and_hyperbolic(bf):
    import torch
    for spec in (wl.genradon3d(L=4), wl.hypradon(6)):
        plan = bf.Plan.from_spec(spec, precision="mixed")
        g = torch.from_numpy(wl.source_values(spec, 1, np.complex64, seed=7)).cuda()
        ref = plan.apply(g)
        out = torch.empty_like(g)
        _call(bf, spec, "mixed", g, out)
        torch.cuda.synchronize()
        a, b = out.cpu().numpy(), ref.cpu().numpy()
        assert np.linalg.norm(a - b) <= TOL["mixed"] * np.linalg.norm(b)
        plan.close()


def test_noalloc_rejects_problems_beyond_the_static_array(bf):
    import torch
    spec = wl.genradon2d(L=8)                      # N = 256 needs ~26 MB > 16 MiB
    g = torch.zeros(spec.npts, dtype=torch.complex64, device="cuda")
    f = torch.full_like(g, 3.0)
    with pytest.raises(bf.BfError) as e:
        _call(bf, spec, "mixed", g, f)
    assert e.value.code == 1
    torch.cuda.synchronize()
    assert torch.all(f == 3.0)


def test_noalloc_against_the_oracle(bf):
    # directly against the FP64 oracle butterfly (not only through bf_apply), both sincos
    # variants and FP64
    import torch
    import oracle
    cases = ((wl.genradon2d(L=6), "mixed", np.complex64, TOL["mixed"]),
             (wl.genradon2d(L=5), "mixed_sfu", np.complex64, TOL["mixed"]),
             (wl.hypradon(5), "fp64", np.complex128, TOL["fp64"]))
    for spec, prec, dt, tol in cases:
        g = torch.from_numpy(wl.source_values(spec, 1, dt, seed=31)).cuda()
        out = torch.full_like(g, float("nan"))
        _call(bf, spec, prec, g, out)
        torch.cuda.synchronize()
        ref = oracle.butterfly(oracle.Problem(**spec.oracle_kwargs()), g.cpu().numpy()[0].astype(np.complex128))
        a = out.cpu().numpy()[0]
        assert np.linalg.norm(a - ref) <= tol * np.linalg.norm(ref), (spec.name, prec)


@pytest.mark.parametrize("precision", ["mixed", "mixed_sfu"])
def test_noalloc_several_rhs(bf, precision):
    # three right-hand sides (the static array holds 2 x nrhs x N^d x r weights): the
    # single-RHS kernels with grid_y = nrhs, against the plan's multi-RHS apply (FP32
    # rounding order) and, per right-hand side, against the oracle
    import torch
    import oracle
    spec = wl.genradon2d(L=6)
    nrhs = 3
    g = torch.from_numpy(wl.source_values(spec, nrhs, np.complex64, seed=41)).cuda()
    plan = bf.Plan.from_spec(spec, max_nrhs=nrhs, precision=precision)
    ref = plan.apply(g).cpu().numpy()
    plan.close()
    out = torch.full_like(g, float("nan"))
    _call(bf, spec, precision, g, out)
    torch.cuda.synchronize()
    a = out.cpu().numpy()
    P = oracle.Problem(**spec.oracle_kwargs())
    for j in range(nrhs):
        assert np.linalg.norm(a[j] - ref[j]) <= 2e-6 * np.linalg.norm(ref[j]), j
        o = oracle.butterfly(P, g[j].cpu().numpy().astype(np.complex128))
        assert np.linalg.norm(a[j] - o) <= TOL["mixed"] * np.linalg.norm(o), j
