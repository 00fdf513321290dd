"""The mixed path's hand-written arithmetic against CUDA's FP64 on the GPU."""
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


def test_sincos_against_fp64_sincospi(bf):
    # minimax truncation < 4e-8 plus a few FP32 roundings of values <= 1
    assert bf.selfcheck_sincos(1 << 22) < 1.5e-7


@pytest.mark.parametrize("spec", [wl.genradon2d(), wl.genradon3d(), wl.hypradon(9), wl.dft64().with_(precision="mixed"),
                                  wl.genradon2d(L=6).with_(phase="separable")],
                         ids=["genradon2d", "genradon3d", "hypradon512", "dft64", "separable64"])
def test_double_float_phase_against_fp64(bf, spec):
    # |Phi| reaches ~2e3 cycles.  The double-float evaluation keeps ~44 bits before the
    # mod-1 reduction; the reduced phase is then one FP32 number of magnitude < 2, so
    # the error is a few of its roundings (< 3e-7 cycles) whatever |Phi| is.  Evaluating
    # Phi in plain FP32 would err by ~|Phi| * 6e-8, i.e. ~1e-4 cycles here.
    plan = bf.Plan.from_spec(spec, precision="mixed")
    err = plan.selfcheck_phase(1 << 20)
    plan.close()
    assert err < 3e-7, err
