"""Many independent problems of uneven size in one call (bf_apply_batched), also
captured in a CUDA graph; every result equals the single-problem apply and the oracle."""
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


def _problems():
    # uneven N and RHS counts, as in the 48-problem hyperbolic Radon batch but small
    out = []
    for i, (L, k) in enumerate([(5, 3), (6, 1), (4, 7), (7, 2), (5, 16), (6, 5)]):
        out.append((wl.hypradon(L), k, 500 + i))
    return out


def test_batched_equals_single_and_oracle(bf):
    import torch
    probs = _problems()
    plans = [bf.Plan.from_spec(s, max_nrhs=k, precision="mixed") for s, k, _ in probs]
    gs = [torch.from_numpy(wl.source_values(s, k, np.complex64, seed=sd)).cuda() for s, k, sd in probs]
    fs = [torch.empty_like(g) for g in gs]
    bf.apply_batched(plans, gs, fs, [k for _, k, _ in probs])
    torch.cuda.synchronize()
    for (s, k, _), p, g, f in zip(probs, plans, gs, fs):
        single = p.apply(g)
        torch.cuda.synchronize()
        assert torch.equal(single, f)
        ref = oracle.butterfly(oracle.Problem(**s.oracle_kwargs()), g.cpu().numpy().astype(np.complex128))
        out = f.cpu().numpy()
        assert np.linalg.norm(out - ref) <= 1e-5 * np.linalg.norm(ref)
    for p in plans:
        p.close()


def test_batched_in_a_cuda_graph(bf):
    import torch
    probs = _problems()
    plans = [bf.Plan.from_spec(s, max_nrhs=k, precision="mixed") for s, k, _ in probs]
    gs = [torch.from_numpy(wl.source_values(s, k, np.complex64, seed=sd)).cuda() for s, k, sd in probs]
    fs = [torch.empty_like(g) for g in gs]
    nr = [k for _, k, _ in probs]
    bf.apply_batched(plans, gs, fs, nr)                 # first call outside the capture
    torch.cuda.synchronize()
    ref = [f.clone() for f in fs]
    graph = torch.cuda.CUDAGraph()
    with torch.cuda.graph(graph):
        bf.apply_batched(plans, gs, fs, nr)
    for f in fs:
        f.zero_()
    graph.replay()
    graph.replay()
    torch.cuda.synchronize()
    for a, b in zip(fs, ref):
        assert torch.equal(a, b)
    for p in plans:
        p.close()


@pytest.mark.parametrize("L,q,nrhs,prec", [(5, 5, 7, "mixed"), (6, 3, 4, "mixed"), (7, 5, 2, "mixed"),
                                           (8, 5, 9, "mixed"), (9, 5, 16, "mixed"), (4, 4, 17, "mixed"),
                                           (6, 8, 5, "mixed"), (5, 2, 3, "mixed"), (1, 5, 3, "mixed"),
                                           (2, 5, 20, "mixed"), (3, 6, 2, "mixed"), (7, 5, 11, "mixed_sfu")])
def test_multi_rhs_equals_one_rhs_at_a_time(bf, L, q, nrhs, prec):
    # several right-hand sides share each phase evaluation (cached once per stage in
    # shared memory); the per-RHS arithmetic follows the single-RHS kernels up to the
    # order of a few products, so results agree to a few FP32 roundings
    import torch
    spec = wl.genradon2d(L=L).with_(q=q)
    plan = bf.Plan.from_spec(spec, max_nrhs=nrhs, precision=prec)
    g = torch.from_numpy(wl.source_values(spec, nrhs, np.complex64, seed=40 + L)).cuda()
    many = plan.apply(g)
    ones = torch.stack([plan.apply(g[j:j + 1].contiguous())[0] for j in range(nrhs)])
    torch.cuda.synchronize()
    for j in range(nrhs):
        err = (torch.linalg.vector_norm(many[j] - ones[j]) / torch.linalg.vector_norm(ones[j])).item()
        assert err < 2e-6, (j, err)
    plan.close()


def test_multi_rhs_against_oracle_beyond_one_cta_of_rhs(bf):
    # 19 right-hand sides: two CTAs along the RHS axis (16 + 3), odd L, hyperbolic Radon
    import torch
    spec = wl.hypradon(7)
    nrhs = 19
    plan = bf.Plan.from_spec(spec, max_nrhs=nrhs, precision="mixed")
    g = torch.from_numpy(wl.source_values(spec, nrhs, np.complex64, seed=77)).cuda()
    out = plan.apply(g).cpu().numpy()
    ref = oracle.butterfly(oracle.Problem(**spec.oracle_kwargs()), g.cpu().numpy().astype(np.complex128))
    for j in range(nrhs):
        assert np.linalg.norm(out[j] - ref[j]) <= 1e-5 * np.linalg.norm(ref[j]), j
    plan.close()


def test_multi_rhs_bench_size_against_restricted_oracle(bf):
    # the benchmark's multi-RHS configuration (hyperbolic Radon N = 512, 16 right-hand sides, autotuned
    # schedule): every right-hand side at all targets of one level-m box against the restricted oracle
    import torch
    spec = wl.hypradon(9)
    nrhs = 16
    plan = bf.Plan.from_spec(spec, max_nrhs=nrhs, precision="mixed")
    plan.autotune(nrhs, reps=1)
    g = torch.from_numpy(wl.source_values(spec, nrhs, np.complex64, seed=78)).cuda()
    out = plan.apply(g).cpu().numpy()
    P = oracle.Problem(**spec.oracle_kwargs())
    lvl = spec.switch_level
    box = (1 << (2 * lvl)) // 3
    tg = oracle.restricted_targets(P, lvl, box)
    gh = g.cpu().numpy().astype(np.complex128)
    for j in (0, 7, 15):
        ref = oracle.butterfly(P, gh[j], restrict=(lvl, box))[tg]
        assert np.linalg.norm(out[j][tg] - ref) <= 1e-5 * np.linalg.norm(ref), j
    plan.close()


# ------------------------------------------------------------ persistent batch

def _batch_problems():
    # uneven N, 1..19 RHS (19: two blocks of right-hand sides), odd and even L
    out = []
    for i, (L, k) in enumerate([(5, 3), (6, 1), (4, 7), (7, 2), (5, 16), (6, 5), (3, 19), (8, 4)]):
        out.append((wl.hypradon(L), k, 700 + i))
    return out


def _make(bf, probs, precision="mixed"):
    import torch
    plans = [bf.Plan.from_spec(s, max_nrhs=k, precision=precision) for s, k, _ in probs]
    gs = [torch.from_numpy(wl.source_values(s, k, np.complex64, seed=sd)).cuda() for s, k, sd in probs]
    fs = [torch.empty_like(g) for g in gs]
    return plans, gs, fs


@pytest.mark.parametrize("precision", ["mixed", "mixed_sfu"])
def test_persistent_batch_equals_per_problem_apply(bf, precision):
    # one launch runs every pass of every problem; each unit executes the per-pass
    # kernel's code on the same data, so results equal the per-problem applies bit for bit
    import torch
    probs = _batch_problems()
    plans, gs, fs = _make(bf, probs, precision)
    batch = bf.Batch(plans, [k for _, k, _ in probs])
    info = batch.info()
    assert info["units"] > info["grid"] > 0
    batch.apply(gs, fs)
    torch.cuda.synchronize()
    assert not batch.status()
    for (s, k, _), p, g, f in zip(probs, plans, gs, fs):
        single = p.apply(g)
        torch.cuda.synchronize()
        if k >= 2:
            assert torch.equal(single, f), (s.N, k)
        else:   # one RHS: the per-problem apply takes the single-RHS kernels (other rounding order)
            assert (torch.linalg.vector_norm(single - f) / torch.linalg.vector_norm(single)).item() < 2e-6
    # and against the oracle on two of them
    for j in (0, 6):
        s = probs[j][0]
        ref = oracle.butterfly(oracle.Problem(**s.oracle_kwargs()), gs[j].cpu().numpy().astype(np.complex128))
        out = fs[j].cpu().numpy()
        tol = 1e-5 if precision == "mixed" else 2e-5
        assert np.linalg.norm(out - ref) <= tol * np.linalg.norm(ref)
    batch.close()
    for p in plans:
        p.close()


def test_persistent_batch_in_a_cuda_graph(bf):
    import torch
    probs = _batch_problems()
    plans, gs, fs = _make(bf, probs)
    batch = bf.Batch(plans, [k for _, k, _ in probs])
    batch.apply(gs, fs)
    torch.cuda.synchronize()
    ref = [f.clone() for f in fs]
    graph = torch.cuda.CUDAGraph()
    with torch.cuda.graph(graph):
        batch.apply(gs, fs)
    for f in fs:
        f.zero_()
    graph.replay()
    graph.replay()
    torch.cuda.synchronize()
    assert not batch.status()
    for a, b in zip(fs, ref):
        assert torch.equal(a, b)
    batch.close()
    for p in plans:
        p.close()


def test_persistent_batch_wait_times_out_without_hanging(bf):
    # every dependency target set one above what can be reached and a 20 ms limit: the
    # first wait gives up, sets the flag, later units skip; the context stays usable
    import time
    import torch
    probs = _batch_problems()[:4]
    plans, gs, fs = _make(bf, probs)
    batch = bf.Batch(plans, [k for _, k, _ in probs])
    t0 = time.perf_counter()
    assert batch.selftest_timeout(gs, fs)
    assert time.perf_counter() - t0 < 10.0
    batch.apply(gs, fs)
    torch.cuda.synchronize()
    assert not batch.status()
    for (_, k, _), p, g, f in zip(probs, plans, gs, fs):
        single = p.apply(g)
        if k >= 2:
            assert torch.equal(single, f)
        else:
            assert (torch.linalg.vector_norm(single - f) / torch.linalg.vector_norm(single)).item() < 2e-6
    batch.close()
    for p in plans:
        p.close()


def test_persistent_batch_rejects_mixed_configurations(bf):
    s = wl.hypradon(5)
    a = bf.Plan.from_spec(s, max_nrhs=2, precision="mixed")
    b = bf.Plan.from_spec(s.with_(q=4), max_nrhs=2, precision="mixed")
    c = bf.Plan.from_spec(s, max_nrhs=2, precision="fp64")
    with pytest.raises(bf.BfError) as e:
        bf.Batch([a, b], [2, 2])
    assert e.value.code == 2
    with pytest.raises(bf.BfError) as e:
        bf.Batch([a, c], [2, 2])
    assert e.value.code == 2
    with pytest.raises(bf.BfError) as e:
        bf.Batch([a, a], [2, 2])
    assert e.value.code == 1
    with pytest.raises(bf.BfError) as e:
        bf.Batch([a], [3])
    assert e.value.code == 1
    for p in (a, b, c):
        p.close()
