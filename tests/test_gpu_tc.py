"""The switch on the tensor cores (BF_PREC_BF16X3, BF_PREC_TF32X3): tcgen05 GEMM self-checks, then the
butterfly with several right-hand sides against the FP64 oracle.

Tolerance: relative l2 <= 1e-4 against the same-q oracle butterfly, per right-hand side
(the batched-RHS split-product tolerance of the method's GPU forms).  The switch's BF16x3
products carry a relative error below 2^-16 each (the dropped lo.lo term and the BF16
rounding of the lo parts), ~1e-5 on a 25-term sum; every other step is the mixed path
(a few 1e-7).  Against the all-FP32 multi-RHS apply the difference is the switch's
error alone: 5e-5.
"""
import numpy as np
import pytest

import oracle
from paper_1305_4650_gb300 import workloads as wl

pytestmark = pytest.mark.gpu

TOL_ORACLE = 1e-4
TOL_FP32 = 5e-5


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


def test_umma_selfcheck_exact(bf):
    # small-integer operands: every BF16 product and FP32 sum is exact
    err, timed_out = bf.selfcheck_umma(split=False)
    assert not timed_out
    assert err == 0.0, err


def test_umma_selfcheck_split(bf):
    # values in [-1, 1) through the BF16x3 split: 64-term sums to ~2^-16 relative
    err, timed_out = bf.selfcheck_umma(split=True)
    assert not timed_out
    assert err < 1e-4, err


def _apply(bf, spec, nrhs, precision, seed, autotune=False):
    import torch
    plan = bf.Plan.from_spec(spec, max_nrhs=nrhs, precision=precision)
    if autotune:
        plan.autotune(nrhs, reps=1)
    g = torch.from_numpy(wl.source_values(spec, nrhs, np.complex64, seed=seed)).cuda()
    f = plan.apply(g)
    torch.cuda.synchronize()
    passes = plan.passes(nrhs)
    timed_out = plan.table_info()["timed_out"]
    plan.close()
    return g.cpu().numpy(), f.cpu().numpy(), passes, timed_out


@pytest.mark.parametrize("phase,L,q,nrhs", [("hypradon", 5, 5, 2), ("hypradon", 6, 5, 16), ("hypradon", 7, 5, 19),
                                            ("genradon", 5, 5, 5), ("dot", 4, 5, 3), ("separable", 5, 5, 4),
                                            ("genradon", 6, 4, 7), ("hypradon", 5, 3, 17), ("genradon", 4, 2, 3),
                                            ("hypradon", 2, 5, 20), ("genradon", 1, 5, 3)])
def test_bf16x3_against_oracle(bf, phase, L, q, nrhs):
    spec = (wl.hypradon(L) if phase == "hypradon" else wl.genradon2d(L=L).with_(phase=phase)).with_(q=q)
    g, out, passes, timed_out = _apply(bf, spec, nrhs, "bf16x3", seed=900 + L + q)
    assert not timed_out
    assert [p["kind"] for p in passes].count("switch_tc") == 1
    ref = oracle.butterfly(oracle.Problem(**spec.oracle_kwargs()), g.astype(np.complex128))
    for j in range(nrhs):
        assert rel(out[j], ref[j]) <= TOL_ORACLE, (j, rel(out[j], ref[j]))


@pytest.mark.parametrize("m", [0, 1, 3, 4])
def test_bf16x3_every_switch_level(bf, m):
    spec = wl.hypradon(5).with_(m=m)
    g, out, passes, _ = _apply(bf, spec, 6, "bf16x3", seed=950 + m)
    sw = [p for p in passes if p["kind"] == "switch_tc"]
    assert len(sw) == 1 and sw[0]["l0"] == m
    ref = oracle.butterfly(oracle.Problem(**spec.oracle_kwargs()), g.astype(np.complex128))
    for j in range(6):
        assert rel(out[j], ref[j]) <= TOL_ORACLE


def test_bf16x3_one_rhs_is_the_mixed_apply(bf):
    # one right-hand side runs the mixed single-RHS kernels: bit-identical
    spec = wl.hypradon(6)
    _, a, pa, _ = _apply(bf, spec, 1, "bf16x3", seed=5)
    _, b, pb, _ = _apply(bf, spec, 1, "mixed", seed=5)
    assert pa == pb
    assert np.array_equal(a, b)


@pytest.mark.parametrize("L,nrhs", [(7, 16), (8, 16), (9, 16), (9, 19)])
def test_bf16x3_benchmark_sizes(bf, L, nrhs):
    # the 48-problem batch's sizes (N = 128, 256, 512) with 16 and 19 right-hand sides,
    # autotuned: against the FP32 multi-RHS apply everywhere and against the oracle
    # restricted to one level-m target box (two boxes at N = 512)
    spec = wl.hypradon(L)
    g, out, passes, timed_out = _apply(bf, spec, nrhs, "bf16x3", seed=960 + L, autotune=True)
    assert not timed_out
    assert any(p["kind"] == "switch_tc" for p in passes)
    _, f32, _, _ = _apply(bf, spec, nrhs, "mixed", seed=960 + L)
    for j in range(nrhs):
        assert rel(out[j], f32[j]) <= TOL_FP32, (j, rel(out[j], f32[j]))
    P = oracle.Problem(**spec.oracle_kwargs())
    lvl = spec.switch_level
    boxes = [(1 << (2 * lvl)) // 3] + ([(1 << (2 * lvl)) - 5] if L == 9 else [])
    for box in boxes:
        tg = oracle.restricted_targets(P, lvl, box)
        for j in (0, nrhs - 1):
            ref = oracle.butterfly(P, g[j].astype(np.complex128), restrict=(lvl, box))
            assert rel(out[j][tg], ref[tg]) <= TOL_ORACLE, (box, j)


def test_bf16x3_refuses_tables_and_batches(bf):
    spec = wl.hypradon(5)
    with pytest.raises(bf.BfError):
        bf.Plan.from_spec(spec, max_nrhs=4, precision="bf16x3", phase_tables=True)
    plan = bf.Plan.from_spec(spec, max_nrhs=4, precision="bf16x3")
    with pytest.raises(bf.BfError):
        bf.Batch([plan], [4])
    plan.close()


# ---- the column merge levels on the tensor cores (bf_params.tc_levels = 1)

def _apply_levels(bf, spec, nrhs, seed, autotune=False):
    import torch
    plan = bf.Plan.from_spec(spec, max_nrhs=nrhs, precision="bf16x3", tc_levels=True)
    if autotune:
        plan.autotune(nrhs, reps=1)
    g = torch.from_numpy(wl.source_values(spec, nrhs, np.complex64, seed=seed)).cuda()
    f = plan.apply(g)
    torch.cuda.synchronize()
    passes = plan.passes(nrhs)
    timed_out = plan.table_info()["timed_out"]
    plan.close()
    return g.cpu().numpy(), f.cpu().numpy(), passes, timed_out


@pytest.mark.parametrize("phase,L,q,nrhs", [("hypradon", 5, 5, 2), ("hypradon", 6, 5, 16), ("hypradon", 7, 5, 19),
                                            ("genradon", 6, 5, 5), ("dot", 4, 5, 3), ("separable", 5, 5, 4),
                                            ("genradon", 6, 4, 7), ("hypradon", 5, 3, 17), ("genradon", 4, 2, 3),
                                            ("hypradon", 2, 5, 20), ("genradon", 1, 5, 3)])
def test_tc_levels_against_oracle(bf, phase, L, q, nrhs):
    spec = (wl.hypradon(L) if phase == "hypradon" else wl.genradon2d(L=L).with_(phase=phase)).with_(q=q)
    g, out, passes, timed_out = _apply_levels(bf, spec, nrhs, seed=700 + L + q)
    assert not timed_out
    kinds = [p["kind"] for p in passes]
    assert kinds.count("col_tc") == spec.switch_level and kinds.count("switch_tc") == 1 and "col" in kinds
    ref = oracle.butterfly(oracle.Problem(**spec.oracle_kwargs()), g.astype(np.complex128))
    for j in range(nrhs):
        assert rel(out[j], ref[j]) <= TOL_ORACLE, (j, rel(out[j], ref[j]))


@pytest.mark.parametrize("L,nrhs", [(8, 16), (9, 16), (9, 19)])
def test_tc_levels_benchmark_sizes(bf, L, nrhs):
    # against the FP32 multi-RHS apply everywhere and the restricted oracle on one box
    spec = wl.hypradon(L)
    g, out, passes, timed_out = _apply_levels(bf, spec, nrhs, seed=760 + L, autotune=True)
    assert not timed_out
    _, f32, _, _ = _apply(bf, spec, nrhs, "mixed", seed=760 + L)
    for j in range(nrhs):
        assert rel(out[j], f32[j]) <= 2 * TOL_FP32, (j, rel(out[j], f32[j]))
    P = oracle.Problem(**spec.oracle_kwargs())
    lvl = spec.switch_level
    box = (1 << (2 * lvl)) // 3
    tg = oracle.restricted_targets(P, lvl, box)
    ref = oracle.butterfly(P, g[0].astype(np.complex128), restrict=(lvl, box))
    assert rel(out[0][tg], ref[tg]) <= TOL_ORACLE


def test_tc_levels_only_with_bf16x3(bf):
    # the option changes nothing for the other precisions' schedules
    spec = wl.hypradon(5)
    p = bf.Plan.from_spec(spec, max_nrhs=4, precision="mixed", tc_levels=True)
    assert all(x["kind"] in ("col", "row") for x in p.passes(4))
    p.close()


# ---- TF32x3 (BF_PREC_TF32X3): the same switch with TF32 parts, kind::tf32

def test_umma_tf32_selfcheck_exact(bf):
    err, timed_out = bf.selfcheck_umma(split=False, fmt="tf32")
    assert not timed_out
    assert err == 0.0, err


def test_umma_tf32_selfcheck_split(bf):
    # values in [-1, 1) through the TF32x3 split: 32-term sums to ~2^-21 relative
    err, timed_out = bf.selfcheck_umma(split=True, fmt="tf32")
    assert not timed_out
    assert err < 1e-6, err


TOL_TF32_ORACLE = 1e-5      # the mixed tolerance: the TF32x3 products are at FP32 rounding


@pytest.mark.parametrize("phase,L,q,nrhs", [("hypradon", 5, 5, 2), ("hypradon", 6, 5, 16), ("hypradon", 7, 5, 19),
                                            ("genradon", 5, 5, 5), ("dot", 4, 5, 3), ("separable", 5, 5, 4),
                                            ("genradon", 6, 4, 7), ("hypradon", 5, 3, 17), ("genradon", 4, 2, 3),
                                            ("hypradon", 2, 5, 20), ("genradon", 1, 5, 3)])
def test_tf32x3_against_oracle(bf, phase, L, q, nrhs):
    spec = (wl.hypradon(L) if phase == "hypradon" else wl.genradon2d(L=L).with_(phase=phase)).with_(q=q)
    g, out, passes, timed_out = _apply(bf, spec, nrhs, "tf32x3", seed=1900 + L + q)
    assert not timed_out
    assert [p["kind"] for p in passes].count("switch_tc") == 1
    ref = oracle.butterfly(oracle.Problem(**spec.oracle_kwargs()), g.astype(np.complex128))
    for j in range(nrhs):
        assert rel(out[j], ref[j]) <= TOL_TF32_ORACLE, (j, rel(out[j], ref[j]))


def test_tf32x3_one_rhs_is_the_mixed_apply(bf):
    spec = wl.hypradon(6)
    _, a, pa, _ = _apply(bf, spec, 1, "tf32x3", seed=15)
    _, b, pb, _ = _apply(bf, spec, 1, "mixed", seed=15)
    assert pa == pb
    assert np.array_equal(a, b)


@pytest.mark.parametrize("L,nrhs", [(8, 16), (9, 16), (9, 19)])
def test_tf32x3_benchmark_sizes(bf, L, nrhs):
    # against the FP32 multi-RHS apply (the switch's products differ by ~2^-22) and the
    # restricted oracle on one level-m box; BF16x3 of the same input is ~10x further off
    spec = wl.hypradon(L)
    g, out, passes, timed_out = _apply(bf, spec, nrhs, "tf32x3", seed=1960 + L, autotune=True)
    assert not timed_out
    assert any(p["kind"] == "switch_tc" for p in passes)
    _, f32, _, _ = _apply(bf, spec, nrhs, "mixed", seed=1960 + L)
    _, b16, _, _ = _apply(bf, spec, nrhs, "bf16x3", seed=1960 + L)
    e32 = [rel(out[j], f32[j]) for j in range(nrhs)]
    e16 = [rel(b16[j], f32[j]) for j in range(nrhs)]
    assert max(e32) <= 2e-6, max(e32)
    assert max(e32) < 0.5 * min(e16), (max(e32), min(e16))
    P = oracle.Problem(**spec.oracle_kwargs())
    lvl = spec.switch_level
    box = (1 << (2 * lvl)) // 3
    tg = oracle.restricted_targets(P, lvl, box)
    ref = oracle.butterfly(P, g[0].astype(np.complex128), restrict=(lvl, box))
    assert rel(out[0][tg], ref[tg]) <= TOL_TF32_ORACLE


def test_tf32x3_refuses_tables_and_batches_and_ignores_tc_levels(bf):
    spec = wl.hypradon(5)
    with pytest.raises(bf.BfError):
        bf.Plan.from_spec(spec, max_nrhs=4, precision="tf32x3", phase_tables=True)
    plan = bf.Plan.from_spec(spec, max_nrhs=4, precision="tf32x3")
    with pytest.raises(bf.BfError):
        bf.Batch([plan], [4])
    plan.close()
    p = bf.Plan.from_spec(spec, max_nrhs=4, precision="tf32x3", tc_levels=True)
    assert [x["kind"] for x in p.passes(4)].count("col_tc") == 0
    p.close()


# ---- staging of the switch's weights: one tiled bulk copy (TMA) per unit, or cp.async

@pytest.mark.parametrize("prec", ["bf16x3", "tf32x3"])
@pytest.mark.parametrize("L,nrhs", [(6, 2), (7, 16), (8, 19)])
def test_tiled_and_cpasync_staging_agree(bf, prec, L, nrhs):
    # the same arithmetic on the same staged bytes: bit-identical; 19 right-hand sides make
    # a second block of 16 whose last 13 rows lie past max_nrhs (read as zero, unused)
    import torch
    spec = wl.hypradon(L)
    g = torch.from_numpy(wl.source_values(spec, nrhs, np.complex64, seed=2100 + L)).cuda()
    outs, tiled = [], []
    for cp in (False, True):
        plan = bf.Plan.from_spec(spec, max_nrhs=nrhs, precision=prec, tc_cpasync=cp)
        tiled.append(plan.tc_info()["tiled_copies"])
        outs.append(plan.apply(g))
        torch.cuda.synchronize()
        assert not plan.table_info()["timed_out"]
        plan.close()
    assert tiled == [True, False]
    assert torch.equal(outs[0], outs[1])


def test_staging_reported_per_precision(bf):
    spec = wl.hypradon(5)
    for prec, expect in (("bf16x3", True), ("tf32x3", True), ("mixed", False)):
        p = bf.Plan.from_spec(spec, max_nrhs=4, precision=prec)
        assert p.tc_info()["tiled_copies"] == expect, prec
        p.close()
    p = bf.Plan.from_spec(spec, max_nrhs=1, precision="bf16x3")    # one right-hand side: no switch pass
    assert p.tc_info()["tiled_copies"] is False
    p.close()


def test_tiled_staging_autotuned_benchmark_size(bf):
    # the autotuned schedule of the N = 512 problem with 16 right-hand sides, both stagings
    import torch
    spec = wl.hypradon(9)
    g = torch.from_numpy(wl.source_values(spec, 16, np.complex64, seed=2200)).cuda()
    outs = []
    for cp in (False, True):
        plan = bf.Plan.from_spec(spec, max_nrhs=16, precision="bf16x3", tc_cpasync=cp)
        plan.autotune(16, reps=1)
        outs.append(plan.apply(g))
        torch.cuda.synchronize()
        plan.close()
    assert torch.equal(outs[0], outs[1])
