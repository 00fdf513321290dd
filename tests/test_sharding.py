"""Multi-GPU distribution of the pair space (design, host logic), on the CPU.

1. The ownership map is a balanced partition at every level, merge blocks are local
   for the first levels and need teams of at most 2^d ranks afterwards, the first ranks
   own contiguous source ranges and the last ones target boxes in bit-reversed order.
2. A stand-in linear butterfly (random 3 x 3 translation matrices per pair and child,
   not the Chebyshev operators) runs sharded over 2 gloo ranks, exchanging partial
   sums with send/recv exactly where the schedule says, and matches the serial run.
"""
import os
import socket

import numpy as np
import pytest

from paper_1305_4650_gb300 import sharding as sh


@pytest.mark.parametrize("d,L,g", [(2, 3, 1), (2, 3, 2), (2, 4, 3), (2, 4, 4), (3, 2, 3), (2, 5, 5), (3, 3, 4)])
def test_ownership_partition_and_teams(d, L, g):
    G, n = 1 << g, 1 << (d * L)
    for level in range(L + 1):
        nA, nB = 1 << (d * level), 1 << (d * (L - level))
        counts = np.zeros(G, int)
        for A in range(nA):
            for B in range(nB):
                counts[sh.owner(d, L, g, level, A, B)] += 1
        assert np.all(counts == n // G), (level, counts)
    stages = sh.schedule(d, L, g)
    assert sum(not s.exchange for s in stages) == sh.local_levels(d, L, g)
    for st in stages:
        l = st.level
        for Ap in range(1 << (d * l)):
            for Bp in range(1 << (d * (L - l - 1))):
                ins, outs = sh.block_ranks(d, L, g, l, Ap, Bp)
                team = set(ins) | set(outs)
                if not st.exchange:
                    assert len(team) == 1
                else:
                    assert set(ins) == set(outs) and len(team) == st.team_size <= (1 << d)
    # last level: ranks own targets by A's newest digits, i.e. the source order bit-reversed
    for A in range(n):
        assert sh.owner(d, L, g, L, A, 0) == sh.digit_rev(A, L, d) >> (d * L - g)
    # first level: ranks own contiguous ranges of source boxes
    for B in range(n):
        assert sh.owner(d, L, g, 0, 0, B) == B >> (d * L - g)


# ----------------------------------------------------------------- gloo run

R = 3


def _T(seed, level, A, B, a):
    rng = np.random.default_rng([seed, level, A, B, a])
    return rng.standard_normal((R, R))


def _serial(d, L, w0, seed):
    w = {(0, B): w0[B] for B in range(1 << (d * L))}
    for l in range(L):
        nw = {}
        for (A, B), v in w.items():
            Bp, c = B >> d, B & ((1 << d) - 1)
            for a in range(1 << d):
                key = ((A << d) + a, Bp)
                nw[key] = nw.get(key, 0) + _T(seed, l, A, B, a) @ v
        w = nw
    return w


def _worker(rank, world, port, d, L, seed, q):
    import torch
    import torch.distributed as dist
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        g = world.bit_length() - 1
        w0 = np.random.default_rng(seed).standard_normal((1 << (d * L), R))
        w = {(0, B): w0[B] for B in range(1 << (d * L)) if sh.owner(d, L, g, 0, 0, B) == rank}
        for st in sh.schedule(d, L, g):
            l = st.level
            part = {}
            for (A, B), v in w.items():
                Bp = B >> d
                for a in range(1 << d):
                    key = ((A << d) + a, Bp)
                    part[key] = part.get(key, 0) + _T(seed, l, A, B, a) @ v
            if st.exchange:
                # sum-scatter over the team: send every partial output to its owner
                out_keys = sorted(part)
                peer = 1 - rank
                mine = {k: v for k, v in part.items() if sh.owner(d, L, g, l + 1, *k) == rank}
                send = [k for k in out_keys if sh.owner(d, L, g, l + 1, *k) == peer]
                n_send = torch.tensor([len(send)])
                n_recv = torch.tensor([0])
                reqs = [dist.isend(n_send, peer), dist.irecv(n_recv, peer)]
                for r_ in reqs:
                    r_.wait()
                buf_s = torch.tensor(np.array([[*k, *part[k]] for k in send], dtype=np.float64).reshape(-1, 2 + R))
                buf_r = torch.zeros((int(n_recv.item()), 2 + R), dtype=torch.float64)
                reqs = [dist.isend(buf_s, peer), dist.irecv(buf_r, peer)]
                for r_ in reqs:
                    r_.wait()
                for row in buf_r.numpy():
                    key = (int(row[0]), int(row[1]))
                    assert key in mine or sh.owner(d, L, g, l + 1, *key) == rank
                    mine[key] = mine.get(key, 0) + row[2:]
                part = mine
            else:
                assert all(sh.owner(d, L, g, l + 1, *k) == rank for k in part)
            w = part
        ref = _serial(d, L, w0, seed)
        err = max(float(np.max(np.abs(v - ref[k]))) for k, v in w.items())
        assert len(w) == len(ref) // world
        q.put((rank, err))
    except Exception as e:  # report to the parent
        q.put((rank, repr(e)))
    finally:
        dist.destroy_process_group()


@pytest.mark.parametrize("d,L", [(2, 3), (3, 2)])
def test_sharded_run_two_gloo_ranks(d, L):
    import torch.multiprocessing as mp
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        port = s.getsockname()[1]
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    procs = [ctx.Process(target=_worker, args=(r, 2, port, d, L, 7, q)) for r in range(2)]
    for p in procs:
        p.start()
    res = [q.get(timeout=120) for _ in procs]
    for p in procs:
        p.join(timeout=60)
    for rank, err in res:
        assert isinstance(err, float) and err < 1e-9, (rank, err)
