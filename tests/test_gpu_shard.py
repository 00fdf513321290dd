"""Sharded apply over 2, 4 and 8 ranks (bf_apply_shard + one all-reduce), each rank its own
process with its own plan; here all ranks share the one GPU of the test machine and the
all-reduce runs on the CPU (gloo).  The kernels of different ranks never wait on each other:
every rank computes its part, then the host exchange sums the parts.

The sum of the parts must equal the unsharded apply up to rounding order (the last merge
adds the children of different ranks in another order) and match the FP64 oracle within
the parity tolerances.
"""
import json
import os
import socket

import numpy as np
import pytest

pytestmark = pytest.mark.gpu

# (name, d, L, q, phase, precision, nrhs, worlds)
CASES = [("genradon2d_mixed", 2, 6, 5, "genradon", "mixed", 1, (2, 4)),
         ("hypradon_fp64", 2, 5, 5, "hypradon", "fp64", 1, (2, 4)),
         ("hypradon_mixed_3rhs", 2, 6, 5, "hypradon", "mixed", 3, (2, 4)),
         ("hypradon_bf16x3_5rhs", 2, 6, 5, "hypradon", "bf16x3", 5, (2,)),
         ("genradon2d_sfu_oddL", 2, 5, 4, "genradon", "mixed_sfu", 1, (2,)),
         ("genradon3d_mixed", 3, 4, 4, "genradon", "mixed", 1, (2, 8))]
TOL_SUM = {"mixed": 1e-6, "mixed_sfu": 1e-6, "bf16x3": 1e-6, "fp64": 1e-13}
TOL_ORACLE = {"mixed": 1e-5, "mixed_sfu": 1e-5, "bf16x3": 1e-4, "fp64": 1e-11}


def _spec(d, L, q, phase, precision):
    from paper_1305_4650_gb300 import workloads as wl
    if phase == "hypradon":
        return wl.hypradon(L, precision).with_(q=q)
    return (wl.genradon2d(L, precision) if d == 2 else wl.genradon3d(L, precision)).with_(q=q)


def _worker(rank, world, port, out_path):
    import torch
    import torch.distributed as dist
    from paper_1305_4650_gb300 import bf, sharding, workloads as wl
    dist.init_process_group("gloo", init_method=f"tcp://127.0.0.1:{port}", rank=rank, world_size=world)
    torch.cuda.set_device(0)
    res = {}
    for name, d, L, q, phase, prec, nrhs, worlds in CASES:
        if world not in worlds:
            continue
        spec = _spec(d, L, q, phase, prec)
        dt = np.complex128 if prec == "fp64" else np.complex64
        g_np = wl.source_values(spec, nrhs, dt, seed=70 + L)
        g = torch.from_numpy(g_np).cuda()
        plan = bf.Plan.from_spec(spec, max_nrhs=nrhs, precision=prec)
        f = sharding.sharded_apply(plan, g, host_reduce=True)
        full = plan.apply(g)
        torch.cuda.synchronize()
        plan.close()
        if rank == 0:
            a, b = f.cpu().numpy(), full.cpu().numpy()
            res[name] = {"sum_vs_full": float(np.linalg.norm(a - b) / np.linalg.norm(b)), "prec": prec}
            np.save(out_path + f".{name}.npy", a.reshape(nrhs, -1))
    if rank == 0:
        with open(out_path, "w") as fh:
            json.dump(res, fh)
    dist.barrier()
    dist.destroy_process_group()


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


@pytest.fixture(scope="module")
def built():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1305_4650_gb300 import build
    build.build()


@pytest.mark.parametrize("world", [2, 4, 8])
def test_sharded_apply_sums_to_the_apply_and_matches_the_oracle(built, world, tmp_path):
    import torch.multiprocessing as mp
    import oracle
    from paper_1305_4650_gb300 import workloads as wl
    out = str(tmp_path / f"shard{world}.json")
    mp.start_processes(_worker, args=(world, _free_port(), out), nprocs=world, start_method="spawn", join=True)
    res = json.load(open(out))
    cases = [c for c in CASES if world in c[7]]
    assert sorted(res) == sorted(c[0] for c in cases)
    for name, d, L, q, phase, prec, nrhs, _ in cases:
        assert res[name]["sum_vs_full"] <= TOL_SUM[prec], (name, res[name])
        spec = _spec(d, L, q, phase, prec)
        dt = np.complex128 if prec == "fp64" else np.complex64
        g = wl.source_values(spec, nrhs, dt, seed=70 + L).astype(np.complex128)
        a = np.load(out + f".{name}.npy")
        P = oracle.Problem(**spec.oracle_kwargs())
        for j in range(nrhs):
            ref = oracle.butterfly(P, g[j])
            assert np.linalg.norm(a[j] - ref) <= TOL_ORACLE[prec] * np.linalg.norm(ref), (name, j)


def test_shard_arguments_are_checked(built):
    import torch
    from paper_1305_4650_gb300 import bf
    spec = _spec(2, 4, 5, "genradon", "mixed")
    plan = bf.Plan.from_spec(spec)
    g = torch.zeros(spec.npts, dtype=torch.complex64, device="cuda")
    for sg, sr in ((3, 0), (1, 2), (-1, 0), (2, 4)):
        with pytest.raises(bf.BfError) as e:
            plan.apply_shard(g, sg, sr)
        assert e.value.code == 1
    ref = plan.apply(g)
    assert torch.equal(plan.apply_shard(g, 0, 0), ref)      # shard_g = 0: the whole apply
    plan.close()
