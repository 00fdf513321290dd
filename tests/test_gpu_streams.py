"""One workspace per plan: an apply issued on another stream while the plan's previous
apply is still running is refused (BF_ERR_UNSUPPORTED, nothing queued); the same stream,
or another stream once the previous apply has completed, is accepted."""
import numpy as np
import pytest

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


def test_apply_from_another_stream_while_busy_is_refused(bf):
    import torch
    spec = wl.genradon2d(L=8)
    plan = bf.Plan.from_spec(spec, precision="mixed")
    g = torch.from_numpy(wl.source_values(spec, 1, np.complex64, seed=3)).cuda()
    f1, f2 = torch.empty_like(g), torch.empty_like(g)
    s1, s2 = torch.cuda.Stream(), torch.cuda.Stream()
    ref = plan.apply(g)
    torch.cuda.synchronize()
    with torch.cuda.stream(s1):
        torch.cuda._sleep(200_000_000)          # keeps s1, and the apply queued behind it, busy
        plan.apply(g, f1, stream=s1)
    f2.fill_(7.0)
    with pytest.raises(bf.BfError) as e:
        plan.apply(g, f2, stream=s2)            # s1's apply has not completed
    assert e.value.code == 2
    with pytest.raises(bf.BfError):
        plan.apply_adjoint(g, f2, stream=s2)
    plan.apply(g, f1, stream=s1)                # the same stream stays ordered: accepted
    s1.synchronize()
    plan.apply(g, f2, stream=s2)                # s1 is idle now: accepted
    s2.synchronize()
    assert torch.equal(f1, ref) and torch.equal(f2, ref)
    plan.close()


def test_graph_capture_is_not_checked(bf):
    # a capture on a side stream after applies on the current stream
    import torch
    spec = wl.genradon2d(L=6)
    plan = bf.Plan.from_spec(spec, precision="mixed")
    g = torch.from_numpy(wl.source_values(spec, 1, np.complex64, seed=4)).cuda()
    f = torch.empty_like(g)
    plan.apply(g, f)
    torch.cuda.synchronize()
    ref = f.clone()
    graph = torch.cuda.CUDAGraph()
    with torch.cuda.graph(graph):
        plan.apply(g, f)
    f.zero_()
    graph.replay()
    torch.cuda.synchronize()
    assert torch.equal(f, ref)
    plan.close()
