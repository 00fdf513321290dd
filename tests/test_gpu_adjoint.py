"""GPU adjoint butterfly: parity with the oracle's exact adjoint, the dot-product
identity at full size, gradcheck through torch.autograd, and the dense adjoint."""
import numpy as np
import pytest

import oracle
from paper_1305_4650_gb300 import workloads as wl

pytestmark = pytest.mark.gpu

TOL = {("fp64", 2): 1e-11, ("fp64", 3): 1e-11, ("mixed", 2): 1e-5, ("mixed", 3): 1e-4}


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


def spec_of(d, L, q, phase, **kw):
    base = dict(x_lo=(0.0,) * 3, x_w=(1.0,) * 3)
    if phase == "hypradon":
        base = dict(x_lo=(1.0, 0.0, 0.0), y_lo=(1.0, 0.0, 0.0), y_w=(1.0, 1.0, 1.0), scale=float(1 << L))
    base.update(kw)
    return wl.Spec(f"t_{d}_{L}_{q}_{phase}", d, L, q, phase, **base)


CASES = [
    (2, 1, 3, "dot", {}),
    (2, 3, 5, "genradon", {"tgt_off": 0.3, "src_off": 0.6}),
    (2, 4, 4, "separable", {"tgt_off": 0.25, "src_off": 0.7}),
    (2, 5, 5, "genradon", {}),
    (2, 5, 3, "hypradon", {"m": 1}),
    (2, 7, 5, "genradon", {}),
    (3, 2, 3, "genradon", {"tgt_off": 0.5}),
    (3, 3, 4, "genradon", {}),
    (3, 4, 2, "dot", {"m": 3, "src_off": 0.2}),
]


@pytest.mark.parametrize("precision", ["fp64", "mixed"])
@pytest.mark.parametrize("case", CASES, ids=[f"d{c[0]}L{c[1]}q{c[2]}{c[3]}" for c in CASES])
def test_adjoint_parity_small(bf, case, precision):
    import torch
    d, L, q, phase, kw = case
    spec = spec_of(d, L, q, phase, **kw)
    dt = np.complex128 if precision == "fp64" else np.complex64
    h = wl.source_values(spec, 2, dt, seed=31 + L)
    ref = oracle.butterfly_adjoint(oracle.Problem(**spec.oracle_kwargs()), h.astype(np.complex128))
    plan = bf.Plan.from_spec(spec, max_nrhs=2, precision=precision)
    out = plan.apply_adjoint(torch.from_numpy(h).cuda())
    torch.cuda.synchronize()
    plan.close()
    assert rel(out.cpu().numpy(), ref) <= TOL[(precision, d)]


@pytest.mark.parametrize("spec,precision,tol", [(wl.genradon2d(), "mixed", 2e-6), (wl.genradon2d(), "fp64", 1e-12),
                                                (wl.genradon3d(), "mixed", 2e-6)],
                         ids=["genradon2d-mixed", "genradon2d-fp64", "genradon3d-mixed"])
def test_adjoint_dot_product_full_size(bf, spec, precision, tol):
    # <B g, h> = <g, B^H h> for the approximate operator, at the benchmark sizes
    import torch
    plan = bf.Plan.from_spec(spec, precision=precision)
    dt = np.complex128 if precision == "fp64" else np.complex64
    g = torch.from_numpy(wl.source_values(spec, 1, dt, seed=1)).cuda()
    h = torch.from_numpy(wl.source_values(spec, 1, dt, seed=2)).cuda()
    Bg = plan.apply(g)
    BHh = plan.apply_adjoint(h)
    lhs = torch.vdot(h.flatten().to(torch.complex128), Bg.flatten().to(torch.complex128))
    rhs = torch.vdot(BHh.flatten().to(torch.complex128), g.flatten().to(torch.complex128))
    scale = (torch.linalg.vector_norm(Bg.to(torch.complex128)) * torch.linalg.vector_norm(h.to(torch.complex128))).item()
    plan.close()
    assert abs((lhs - rhs).item()) <= tol * scale


def test_gradcheck_n32(bf):
    import torch
    from paper_1305_4650_gb300.autograd import butterfly
    spec = wl.genradon2d(L=5, precision="fp64")
    plan = bf.Plan.from_spec(spec, precision="fp64")
    g = torch.from_numpy(wl.source_values(spec, 1, np.complex128, seed=4)[0]).cuda().requires_grad_(True)
    # the full Jacobian (2 x 1024 real directions each way), not a random projection
    assert torch.autograd.gradcheck(lambda x: butterfly(x, plan), (g,), eps=1e-6, atol=1e-8, rtol=1e-6,
                                    fast_mode=False)
    plan.close()


def test_adjoint_against_dense_adjoint_n32(bf):
    # B^H h approximates K^H h to the butterfly's own accuracy; dense K from the oracle's direct sum
    import torch
    spec = wl.genradon2d(L=5, precision="fp64").with_(phase="hypradon", scale=32.0, x_lo=(1.0, 0.0, 0.0),
                                                      y_lo=(1.0, 0.0, 0.0), y_w=(1.0, 1.0, 1.0), q=8)
    P = oracle.Problem(**spec.oracle_kwargs())
    n = spec.npts
    K = oracle.direct_sum(P, np.eye(n, dtype=np.complex128)).T          # K[i, j] = K(x_i, y_j)
    h = wl.source_values(spec, 1, np.complex128, seed=8)[0]
    plan = bf.Plan.from_spec(spec, precision="fp64")
    out = plan.apply_adjoint(torch.from_numpy(h).cuda()).cpu().numpy()
    fwd = plan.apply(torch.from_numpy(h).cuda()).cpu().numpy()
    plan.close()
    err_fwd = rel(fwd, K @ h)
    err_adj = rel(out, K.conj().T @ h)
    # the oracle gives 1.1e-4 for both directions at q = 8 (Section 1.4 interpolation error)
    assert err_adj < 3e-4 and err_adj < 2 * err_fwd
