"""Distribution of the butterfly's pair space over G = 2^g GPUs (design; host logic only).

This restates the data distribution of the paper's parallel algorithm (Section 2: the
bitwise bisections of Algorithm 2, the p <= N^d scheme of Algorithm 4) for the
Morton-ordered pair layout used here.  Every level holds N^d pairs (A, B): A a target
box with d*l Morton bits, B a source box with d*(L-l) bits.

A pair's key is its source digits (most significant first) followed by its target digits
newest first: key = B * 2^(d l) + rev(A), with rev reversing A's base-2^d digits.  A pair
belongs to the rank given by the top g bits of its key.

* At level 0 the key is B: ranks partition the source domain.  A merge turns the inputs'
  lowest source digit c into the outputs' newest target digit alpha at the same place
  in the key, so a merge block stays on one rank while that digit lies below the top g
  bits: these first levels are purely local.
* Afterwards the digit overlaps the rank bits: the block's 2^d inputs and 2^d outputs sit
  on one team of up to 2^d ranks (identical but for those bits).  Each rank applies the
  translation to the inputs it holds, and the team sums the contributions and scatters
  the outputs to their owners -- the paper's SumScatter (a reduce-scatter over the team).
* At the last level the key is rev(A): ranks own target boxes by A's newest digits, the
  source bisection order bit-reversed (Section 2.2).

The product path (``sharded_apply``, over ``bf_apply_shard``) keeps the local levels of
this distribution and replaces the team exchanges of the last levels by one all-reduce of
the targets: for G <= 2^d ranks only the last merge mixes ranks, so every rank runs the
last pass on all pairs with the other ranks' weights read as zero and the partial target
values are summed (N^d values per right-hand side instead of N^d r weights).
"""
from __future__ import annotations

from dataclasses import dataclass


def digit_rev(x: int, n: int, d: int) -> int:
    """Reverse the n base-2^d digits of x."""
    y = 0
    for _ in range(n):
        y = (y << d) | (x & ((1 << d) - 1))
        x >>= d
    return y


def key(d: int, level: int, A: int, B: int) -> int:
    return (B << (d * level)) | digit_rev(A, level, d)


def owner(d: int, L: int, g: int, level: int, A: int, B: int) -> int:
    """Rank that holds pair (A, B) at `level` among 2^g ranks."""
    return key(d, level, A, B) >> (d * L - g)


def local_levels(d: int, L: int, g: int) -> int:
    """Number of leading merge levels (l -> l+1) that need no exchange: d (L - l - 1) >= g."""
    return sum(1 for l in range(L) if d * (L - l - 1) >= g)


@dataclass(frozen=True)
class Stage:
    level: int            # merge level l -> l + 1
    exchange: bool        # False: every block is local to one rank
    team_size: int        # ranks that share a merge block (1 when local)


def schedule(d: int, L: int, g: int) -> list[Stage]:
    """Per merge level: local or a sum-scatter over teams of team_size ranks."""
    out = []
    for l in range(L):
        nb_out = d * (L - l - 1)                          # key bits above the block's digit
        width = min(d, max(0, g - nb_out))                # rank bits inside that digit
        out.append(Stage(l, width > 0, 1 << width))
    return out


def block_ranks(d: int, L: int, g: int, level: int, Ap: int, Bp: int):
    """Ranks holding the 2^d inputs (Ap, Bp*2^d + c) and the 2^d outputs (Ap*2^d + a, Bp)
    of the merge block (Ap, Bp) at `level`."""
    ins = [owner(d, L, g, level, Ap, (Bp << d) + c) for c in range(1 << d)]
    outs = [owner(d, L, g, level + 1, (Ap << d) + a, Bp) for a in range(1 << d)]
    return ins, outs


def shard_bits(world: int, d: int) -> int:
    """g with world = 2^g ranks; one exchange (the final all-reduce) needs g <= d."""
    g = world.bit_length() - 1
    if world < 1 or (1 << g) != world or g > d:
        raise ValueError(f"world size {world} must be a power of two <= 2^d = {1 << d}")
    return g


def sharded_apply(plan, g, group=None, stream=None, host_reduce: bool = False):
    """f = B g over the ranks of a torch.distributed group: each rank computes its part on its
    own GPU (bf_apply_shard with the rank's source boxes) and one all-reduce sums the parts.
    host_reduce: reduce CPU copies (for backends without device tensors, e.g. gloo)."""
    import torch.distributed as dist
    world = dist.get_world_size(group)
    rank = dist.get_rank(group)
    f = plan.apply_shard(g, shard_bits(world, plan.d), rank, stream=stream)
    if world == 1:
        return f
    if host_reduce:
        h = f.cpu()
        dist.all_reduce(h, op=dist.ReduceOp.SUM, group=group)
        f.copy_(h)
    else:
        dist.all_reduce(f, op=dist.ReduceOp.SUM, group=group)
    return f
