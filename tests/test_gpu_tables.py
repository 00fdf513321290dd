"""Phase tables (bf_params.phase_tables): every phase factor evaluated once at plan
creation and read back by the apply.  The factors are the ones the evaluating kernels
compute, so the apply equals the evaluating multi-RHS apply bit for bit, and the oracle
to the mixed tolerance."""
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


def _table_bytes(plan, spec):
    # r (5 per pair and level, init, final) + r^2 at the switch, complex64, per point
    r, L = spec.r, spec.L
    return 8 * spec.npts * (r * 5 * L + r + (r + 1) + r * r)


@pytest.mark.parametrize("spec,nrhs,prec", [(wl.genradon2d(L=6), 3, "mixed"), (wl.hypradon(7), 16, "mixed"),
                                            (wl.hypradon(5), 19, "mixed_sfu"), (wl.genradon2d(L=3).with_(q=4), 2, "mixed"),
                                            (wl.dft64().with_(precision="mixed"), 5, "mixed")])
def test_tables_equal_evaluated_phases(bf, spec, nrhs, prec):
    import torch
    pt = bf.Plan.from_spec(spec, max_nrhs=nrhs, precision=prec, phase_tables=True)
    pc = bf.Plan.from_spec(spec, max_nrhs=nrhs, precision=prec)
    info = pt.table_info()
    assert info["bytes"] == _table_bytes(pt, spec) and info["build_ms"] > 0
    assert pc.table_info()["bytes"] == 0
    g = torch.from_numpy(wl.source_values(spec, nrhs, np.complex64, seed=61)).cuda()
    ft, fc = pt.apply(g), pc.apply(g)
    torch.cuda.synchronize()
    assert not pt.table_info()["timed_out"]
    assert torch.equal(ft, fc)
    ref = oracle.butterfly(oracle.Problem(**spec.oracle_kwargs()), g.cpu().numpy().astype(np.complex128))
    tol = 1e-5 if prec == "mixed" else 2e-5
    out = ft.cpu().numpy()
    assert np.linalg.norm(out - ref) <= tol * np.linalg.norm(ref)
    pt.close()
    pc.close()


def _tile_table_bytes(spec):
    # single-RHS table: one float (the reduced phase) per factor, (2^d + 1) r per pair and level
    # (2^d r modulations of the children's weights, r demodulations), and r^2 per pair at the
    # switch unless the phase is a sum over dimensions (factorised switch)
    r, L = spec.r, spec.L
    sw = 0 if spec.phase in ("dot", "separable") else r * r
    return 4 * spec.npts * (((1 << spec.d) + 1) * r * L + sw)


def _spec3(L, q, phase, **kw):
    base = dict(x_lo=(0.0,) * 3, x_w=(1.0,) * 3)
    base.update(kw)
    return wl.Spec(f"t3_{L}_{q}_{phase}", 3, L, q, phase, **base)


@pytest.mark.parametrize("spec,prec", [(wl.genradon2d(L=6), "mixed"), (wl.genradon2d(L=7), "mixed_sfu"),
                                       (wl.hypradon(7), "mixed"), (wl.hypradon(5), "mixed_sfu"),
                                       (wl.genradon2d(L=3).with_(q=4), "mixed"), (wl.genradon2d(L=5).with_(q=3), "mixed"),
                                       (wl.dft64().with_(precision="mixed"), "mixed"), (wl.genradon2d(L=1), "mixed"),
                                       (wl.genradon2d(L=2).with_(q=2), "mixed"), (wl.hypradon(3), "mixed_sfu"),
                                       (wl.genradon3d(L=3), "mixed"), (wl.genradon3d(L=4), "mixed_sfu"),
                                       (_spec3(4, 3, "genradon", tgt_off=0.3), "mixed"), (_spec3(3, 2, "genradon"), "mixed_sfu"),
                                       (_spec3(4, 4, "dot"), "mixed"), (_spec3(3, 3, "separable", src_off=0.2), "mixed"),
                                       (_spec3(1, 4, "genradon"), "mixed"), (_spec3(5, 2, "genradon", m=1), "mixed")])
def test_single_rhs_table_equals_evaluated_phases(bf, spec, prec):
    # plans of one right-hand side record the reduced phase that the single-RHS kernels feed to
    # their sincos, so reading it gives the evaluating apply bit for bit
    import torch
    pt = bf.Plan.from_spec(spec, precision=prec, phase_tables=True)
    pc = bf.Plan.from_spec(spec, precision=prec)
    info = pt.table_info()
    assert info["bytes"] == _tile_table_bytes(spec) and info["build_ms"] > 0
    assert pt.passes(1) == pc.passes(1)
    g = torch.from_numpy(wl.source_values(spec, 1, np.complex64, seed=63)).cuda()
    ft, fc = pt.apply(g), pc.apply(g)
    torch.cuda.synchronize()
    assert not pt.table_info()["timed_out"]
    assert torch.equal(ft, fc)
    for i in range(len(pt.passes(1))):   # one pass at a time reads the same table blocks
        pt.apply_pass(i, g.data_ptr(), ft.data_ptr(), 1)
    torch.cuda.synchronize()
    assert torch.equal(ft, fc)
    ref = oracle.butterfly(oracle.Problem(**spec.oracle_kwargs()), g.cpu().numpy().astype(np.complex128))
    tol = (1e-5 if prec == "mixed" else 2e-5) if spec.d == 2 else 1e-4
    assert np.linalg.norm(ft.cpu().numpy() - ref) <= tol * np.linalg.norm(ref)
    pt.close()
    pc.close()


def test_tables_one_rhs_and_autotune(bf):
    # autotune keeps the schedule the table was recorded for
    import torch
    spec = wl.genradon2d(L=7)
    pt = bf.Plan.from_spec(spec, precision="mixed", phase_tables=True)
    before = pt.passes(1)
    assert pt.autotune(1, reps=2) > 0
    assert pt.passes(1) == before
    g = torch.from_numpy(wl.source_values(spec, 1, np.complex64, seed=62)).cuda()
    out = pt.apply(g)
    single = bf.Plan.from_spec(spec, precision="mixed").apply(g)
    torch.cuda.synchronize()
    assert torch.equal(out, single)
    ref = oracle.butterfly(oracle.Problem(**spec.oracle_kwargs()), g.cpu().numpy().astype(np.complex128))
    assert np.linalg.norm(out.cpu().numpy() - ref) <= 1e-5 * np.linalg.norm(ref)
    pt.close()


def test_tables_refused_where_not_built(bf):
    with pytest.raises(bf.BfError) as e:
        bf.Plan.from_spec(wl.hypradon(5).with_(q=6), precision="mixed", phase_tables=True)
    assert e.value.code == 2
    with pytest.raises(bf.BfError) as e:
        bf.Plan.from_spec(wl.hypradon(5), precision="fp64", phase_tables=True)
    assert e.value.code == 2
    with pytest.raises(bf.BfError) as e:     # d = 3 has no multi-RHS kernels to record factors
        bf.Plan.from_spec(wl.genradon3d(L=3), max_nrhs=2, precision="mixed", phase_tables=True)
    assert e.value.code == 2
    with pytest.raises(bf.BfError) as e:
        bf.Plan.from_spec(wl.genradon3d(L=3), precision="fp64", phase_tables=True)
    assert e.value.code == 2


def test_single_rhs_table_full_size(bf):
    # the benchmark size (N = 1024, q = 5; a 7.9 GB table): the table apply equals the evaluating
    # apply bit for bit, and a level-m target box matches the restricted oracle butterfly
    import torch
    spec = wl.genradon2d()
    pt = bf.Plan.from_spec(spec, precision="mixed", phase_tables=True)
    assert pt.table_info()["bytes"] == _tile_table_bytes(spec)
    pc = bf.Plan.from_spec(spec, precision="mixed")
    g = torch.from_numpy(wl.source_values(spec, 1, np.complex64, seed=64)).cuda()
    ft, fc = pt.apply(g), pc.apply(g)
    torch.cuda.synchronize()
    assert not pt.table_info()["timed_out"]
    assert torch.equal(ft, fc)
    P = oracle.Problem(**spec.oracle_kwargs())
    box = (1 << (2 * spec.switch_level)) // 5
    tg = oracle.restricted_targets(P, spec.switch_level, box)
    ref = oracle.butterfly(P, g[0].cpu().numpy().astype(np.complex128), restrict=(spec.switch_level, box))[tg]
    out = ft[0].cpu().numpy()[tg]
    assert np.linalg.norm(out - ref) <= 1e-5 * np.linalg.norm(ref)
    pt.close()
    pc.close()


def test_single_rhs_table_full_size_d3(bf):
    # d = 3, N = 64, q = 4 (a 7.9 GB table): bit-identical to the evaluating apply, and a
    # level-3 target box against the restricted oracle butterfly
    import torch
    spec = wl.genradon3d()
    pt = bf.Plan.from_spec(spec, precision="mixed", phase_tables=True)
    assert pt.table_info()["bytes"] == _tile_table_bytes(spec)
    pc = bf.Plan.from_spec(spec, precision="mixed")
    g = torch.from_numpy(wl.source_values(spec, 1, np.complex64, seed=65)).cuda()
    ft, fc = pt.apply(g), pc.apply(g)
    torch.cuda.synchronize()
    assert not pt.table_info()["timed_out"]
    assert torch.equal(ft, fc)
    P = oracle.Problem(**spec.oracle_kwargs())
    box = 300
    tg = oracle.restricted_targets(P, spec.switch_level, box)
    ref = oracle.butterfly(P, g[0].cpu().numpy().astype(np.complex128), restrict=(spec.switch_level, box))[tg]
    out = ft[0].cpu().numpy()[tg]
    assert np.linalg.norm(out - ref) <= 1e-4 * np.linalg.norm(ref)
    pt.close()
    pc.close()
