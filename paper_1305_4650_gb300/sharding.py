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

No run here uses more than one GPU; tests/test_sharding.py checks this algebra and runs
an exchange with world_size 2 on the CPU (gloo).
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
