"""The schedule autotuner (bf_plan_autotune): the schedule it keeps covers every level
once, and the apply it times gives the oracle's result (the schedule changes only the
FP32 rounding order)."""
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


def _covers(passes, L, m):
    col = [p for p in passes if p["kind"] == "col"]
    row = [p for p in passes if p["kind"] == "row"]
    lv = 0
    for p in col:
        assert p["l0"] == lv
        lv += p["k"]
    assert lv == m and col[0]["init"] and col[-1]["switch"]
    for p in row:
        assert p["l0"] == lv
        lv += p["k"]
    assert lv == L and row[-1]["final"]


@pytest.mark.parametrize("spec,nrhs,prec", [(wl.genradon2d(L=7), 1, "mixed"), (wl.hypradon(7), 6, "mixed"),
                                            (wl.genradon3d(L=4), 1, "mixed"), (wl.hypradon(6), 3, "fp64"),
                                            (wl.genradon2d(L=6), 17, "mixed_sfu")])
def test_autotuned_schedule_is_valid_and_exact(bf, spec, nrhs, prec):
    import torch
    plan = bf.Plan.from_spec(spec, max_nrhs=nrhs, precision=prec)
    ms = plan.autotune(nrhs, reps=2)
    assert ms > 0
    _covers(plan.passes(nrhs), spec.L, spec.switch_level)
    dt = np.complex128 if prec == "fp64" else np.complex64
    g = torch.from_numpy(wl.source_values(spec, nrhs, dt, seed=91)).cuda()
    out = plan.apply(g).cpu().numpy()
    ref = oracle.butterfly(oracle.Problem(**spec.oracle_kwargs()), g.cpu().numpy().astype(np.complex128))
    tol = {"fp64": 1e-11, "mixed": 1e-5 if spec.d == 2 else 1e-4, "mixed_sfu": 2e-5}[prec]
    assert np.linalg.norm(out - ref) <= tol * np.linalg.norm(ref)
    plan.close()
