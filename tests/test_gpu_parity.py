"""GPU parity: the sm_103a butterfly against the FP64 CPU oracle (same q, same
readings), element by element on seeded inputs.

Tolerances (relative l2 over all compared outputs):
  * FP64 GPU vs oracle butterfly: 1e-11 (same arithmetic, different summation order);
  * mixed vs oracle butterfly: 1e-5 for d = 2 and 1e-4 for d = 3.  The mixed path
    keeps complex64 weights (unit roundoff 2^-24 ~ 6e-8); each of the ~2L+2 steps
    adds a few roundings per term and the Chebyshev interpolation amplifies them
    by its Lebesgue constant (< 2.5 for q <= 8), giving a few 1e-7 per level;
    the phase is computed to ~2^-44 relative before the FP32 sincospif.
"""
import numpy as np
import pytest

import oracle
from paper_1305_4650_gb300 import workloads as wl

pytestmark = pytest.mark.gpu

TOL = {("fp64", 2): 1e-11, ("fp64", 3): 1e-11, ("mixed", 2): 1e-5, ("mixed", 3): 1e-4,
       ("mixed_sfu", 2): 1e-5, ("mixed_sfu", 3): 1e-4}


@pytest.fixture(scope="module")
def bf():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1305_4650_gb300 import build, bf as bfmod
    build.build()
    return bfmod


def rel(a, b):
    return float(np.linalg.norm(a - b) / np.linalg.norm(b))


def run_gpu(bfmod, spec, g, precision, fuse_levels=0):
    import torch
    plan = bfmod.Plan.from_spec(spec, max_nrhs=g.shape[0], precision=precision, fuse_levels=fuse_levels)
    gt = torch.from_numpy(np.ascontiguousarray(g)).cuda()
    f = plan.apply(gt)
    torch.cuda.synchronize()
    out = f.cpu().numpy()
    plan.close()
    return out


def spec_of(d, L, q, phase, **kw):
    base = dict(x_lo=(0.0,) * 3, x_w=(1.0,) * 3)
    if phase == "hypradon":
        base = dict(x_lo=(1.0, 0.0, 0.0), y_lo=(1.0, 0.0, 0.0), y_w=(1.0, 1.0, 1.0), scale=float(1 << L))
    base.update(kw)
    return wl.Spec(f"t_{d}_{L}_{q}_{phase}", d, L, q, phase, **base)


CASES = [
    # d, L, q, phase, extra
    (2, 1, 3, "dot", {}),                                   # N = 2: m = 0, init + switch + one row level
    (2, 2, 2, "genradon", {}),
    (2, 3, 5, "dot", {"tgt_off": 0.3, "src_off": 0.6}),
    (2, 4, 4, "separable", {"tgt_off": 0.25, "src_off": 0.7}),
    (2, 5, 5, "genradon", {}),
    (2, 5, 3, "hypradon", {}),
    (2, 6, 6, "genradon", {"m": 1}),
    (2, 7, 5, "genradon", {}),                              # odd L, several tiles and passes
    (2, 6, 8, "dot", {"node_kind": 1}),
    (3, 1, 2, "dot", {}),
    (3, 2, 3, "genradon", {"tgt_off": 0.5}),
    (3, 3, 4, "genradon", {}),
    (3, 4, 2, "separable", {"src_off": 0.2}),
    (3, 4, 4, "dot", {"m": 3}),
]


@pytest.mark.parametrize("precision", ["fp64", "mixed", "mixed_sfu"])
@pytest.mark.parametrize("case", CASES, ids=[f"d{c[0]}L{c[1]}q{c[2]}{c[3]}" for c in CASES])
def test_parity_small(bf, case, precision):
    d, L, q, phase, kw = case
    spec = spec_of(d, L, q, phase, **kw)
    dt = np.complex128 if precision == "fp64" else np.complex64
    g = wl.source_values(spec, 2, dt, seed=11 + L)
    assert precision in ("fp64", "mixed", "mixed_sfu")
    ref = oracle.butterfly(oracle.Problem(**spec.oracle_kwargs()), g.astype(np.complex128))
    out = run_gpu(bf, spec, g, precision)
    assert rel(out, ref) <= TOL[(precision, d)], rel(out, ref)


@pytest.mark.parametrize("precision", ["fp64", "mixed"])
def test_fusion_depth_does_not_change_results(bf, precision):
    spec = spec_of(2, 7, 4, "genradon", tgt_off=0.1)
    dt = np.complex128 if precision == "fp64" else np.complex64
    g = wl.source_values(spec, 1, dt, seed=5)
    outs = [run_gpu(bf, spec, g, precision, fuse_levels=k) for k in (1, 2, 3)]
    # every output is computed by the same per-pair arithmetic whatever the tile depth
    assert np.array_equal(outs[0], outs[1]) and np.array_equal(outs[0], outs[2])


def test_separable_phase_is_exact_on_gpu(bf):
    spec = spec_of(2, 6, 3, "separable", tgt_off=0.4, src_off=0.3)
    g = wl.source_values(spec, 1, np.complex128, seed=3)
    P = oracle.Problem(**spec.oracle_kwargs())
    direct = oracle.direct_sum(P, g[0])
    out = run_gpu(bf, spec, g, "fp64")[0]
    assert rel(out, direct) < 1e-12


def test_nrhs_zero_is_a_noop_and_bad_sizes_raise(bf):
    import torch
    spec = spec_of(2, 3, 3, "dot")
    plan = bf.Plan.from_spec(spec, max_nrhs=2, precision="mixed")
    g = torch.zeros(0, dtype=torch.complex64, device="cuda")
    f = torch.full((4,), 7.0, dtype=torch.complex64, device="cuda")
    plan.apply_ptr(g.data_ptr(), f.data_ptr(), 0)
    torch.cuda.synchronize()
    assert torch.all(f == 7.0)
    with pytest.raises(bf.BfError):
        plan.apply_ptr(g.data_ptr(), f.data_ptr(), 3)          # nrhs > max_nrhs
    with pytest.raises(bf.BfError):
        plan.apply_ptr(g.data_ptr() + 8, f.data_ptr(), 1)      # misaligned pointer
    with pytest.raises(TypeError):
        plan.apply(torch.zeros(64, dtype=torch.complex128, device="cuda"))
    plan.close()


def test_host_apply_matches_device_apply(bf):
    spec = spec_of(2, 5, 5, "genradon")
    g = wl.source_values(spec, 3, np.complex64, seed=9)
    dev = run_gpu(bf, spec, g, "mixed")
    plan = bf.Plan.from_spec(spec, max_nrhs=3, precision="mixed")
    host = plan.apply_host(g)
    plan.close()
    assert np.array_equal(host, dev)


# ------------------------------------------------------ full benchmark sizes

def _sampled_parity(bfmod, spec, precision, box, tol):
    """Full-size GPU apply, compared at all targets of level-m target boxes with the oracle
    butterfly restricted to each box (identical arithmetic for those outputs): the given box
    and one near the end of the Morton order (other CTAs, tiles and corners of the domain)."""
    dt = np.complex128 if precision == "fp64" else np.complex64
    g = wl.source_values(spec, 1, dt)
    out = run_gpu(bfmod, spec, g, precision)[0]
    P = oracle.Problem(**spec.oracle_kwargs())
    lvl = spec.switch_level
    errs = []
    for b in (box, (1 << (spec.d * lvl)) - 2):
        ref = oracle.butterfly(P, g[0].astype(np.complex128), restrict=(lvl, b))
        tg = oracle.restricted_targets(P, lvl, b)
        errs.append(rel(out[tg], ref[tg]))
    assert max(errs) <= tol, errs
    return max(errs)


def test_parity_genradon2d_full_size_mixed(bf):
    spec = wl.genradon2d()                                   # d=2, N=1024, q=5
    _sampled_parity(bf, spec, "mixed", box=(1 << (2 * spec.switch_level)) // 3, tol=TOL[("mixed", 2)])


def test_parity_genradon2d_full_size_mixed_sfu(bf):
    spec = wl.genradon2d()
    _sampled_parity(bf, spec, "mixed_sfu", box=(1 << (2 * spec.switch_level)) // 3, tol=TOL[("mixed_sfu", 2)])


def test_parity_genradon3d_full_size_mixed_sfu(bf):
    spec = wl.genradon3d()
    _sampled_parity(bf, spec, "mixed_sfu", box=300, tol=TOL[("mixed_sfu", 3)])


def test_parity_genradon2d_full_size_fp64(bf):
    spec = wl.genradon2d(precision="fp64")
    _sampled_parity(bf, spec, "fp64", box=17, tol=TOL[("fp64", 2)])


def test_parity_genradon3d_full_size_mixed(bf):
    spec = wl.genradon3d()                                   # d=3, N=64, q=4
    _sampled_parity(bf, spec, "mixed", box=300, tol=TOL[("mixed", 3)])


def test_parity_dft64_full(bf):
    spec = wl.dft64()                                        # d=2, N=64, q=5, FP64, all outputs
    g = wl.source_values(spec, 1, np.complex128)
    out = run_gpu(bf, spec, g, "fp64")[0]
    P = oracle.Problem(**spec.oracle_kwargs())
    assert rel(out, oracle.butterfly(P, g[0])) <= TOL[("fp64", 2)]
