"""Seeded synthetic workloads for the butterfly: problem geometry and inputs.

This module holds no arithmetic of the method: it only names the benchmark
problems (sizes, domains, phase kind, precision) and draws their inputs from a
seeded PCG64 generator.  Both the CUDA path's tests/benchmark and the CPU oracle
are fed from here; neither is imported by this module.

Problems (kernel exp(2 pi i Phi(x, y)); the paper's experiments are Section 3):

* ``dft64``      d=2, N=64, q=5, Phi = x.p, x = j/N on [0,1)^2, p integer in [-32,32)^2, FP64.
* ``genradon2d`` d=2, N=1024, q=5, Phi = x.p + sqrt(a0(x)^2 p0^2 + a1(x)^2 p1^2) with
                 a0 = (2 + sin 2pi x0 sin 2pi x1)/3, a1 = (2 + cos 2pi x0 cos 2pi x1)/3
                 (the generalized Radon analogue of Section 3.2 with the 2 pi scale), complex64.
* ``genradon3d`` d=3, N=64, q=4, a_k = (2 + sin 2pi x_k cos 2pi x_{k+1 mod 3})/3, complex64.
* ``hypradon``   d=2 hyperbolic Radon (Section 3.1): x=(w,h) on [1,2)x[0,1), y=(tau,p) on
                 [1,2)x[0,1), Phi = N w sqrt(tau^2 + p^2 h^2); 48 problems, N in {128,256,512},
                 1..16 right-hand sides each.
* ``adjoint``    the genradon2d operator with its adjoint; sparse spike model for CG.

Complex inputs have i.i.d. N(0,1) real and imaginary parts, drawn in FP64 and
rounded to the run's complex type; callers feeding the FP64 oracle pass the
rounded values back up-cast, so input rounding is not counted as error.
"""
from __future__ import annotations

from dataclasses import dataclass, field, replace

import numpy as np


@dataclass(frozen=True)
class Spec:
    """Geometry and discretisation of one butterfly problem."""
    name: str
    d: int
    L: int
    q: int
    phase: str                       # "dot" | "genradon" | "hypradon" | "separable"
    scale: float = 1.0
    precision: str = "mixed"         # "fp64" | "mixed"
    x_lo: tuple = (0.0, 0.0, 0.0)
    x_w: tuple = (1.0, 1.0, 1.0)
    y_lo: tuple | None = None        # None: [-N/2, N/2)^d (integer frequencies)
    y_w: tuple | None = None
    m: int | None = None             # switch level, floor(L/2) if None
    node_kind: int = 0
    tgt_off: float = 0.0
    src_off: float = 0.0
    seed: int = 1000

    @property
    def N(self) -> int:
        return 1 << self.L

    @property
    def npts(self) -> int:
        return self.N ** self.d

    @property
    def r(self) -> int:
        return self.q ** self.d

    @property
    def switch_level(self) -> int:
        return self.L // 2 if self.m is None else self.m

    def domain(self):
        N = self.N
        y_lo = self.y_lo if self.y_lo is not None else (-N / 2,) * 3
        y_w = self.y_w if self.y_w is not None else (float(N),) * 3
        return tuple(self.x_lo), tuple(self.x_w), tuple(y_lo), tuple(y_w)

    def with_(self, **kw) -> "Spec":
        return replace(self, **kw)

    def oracle_kwargs(self) -> dict:
        x_lo, x_w, y_lo, y_w = self.domain()
        return dict(d=self.d, L=self.L, q=self.q, phase=self.phase, scale=self.scale,
                    m=self.switch_level, node_kind=self.node_kind, x_lo=x_lo, x_w=x_w,
                    y_lo=y_lo, y_w=y_w, tgt_off=self.tgt_off, src_off=self.src_off)


def dft64() -> Spec:
    return Spec("dft64_d2_q5", 2, 6, 5, "dot", precision="fp64", seed=1001)


def genradon2d(L: int = 10, precision: str = "mixed") -> Spec:
    return Spec(f"genradon2d_N{1 << L}_q5", 2, L, 5, "genradon", precision=precision, seed=1002)


def genradon3d(L: int = 6, precision: str = "mixed") -> Spec:
    return Spec(f"genradon3d_N{1 << L}_q4", 3, L, 4, "genradon", precision=precision, seed=1003)


def hypradon(L: int, precision: str = "mixed") -> Spec:
    return Spec(f"hypradon_N{1 << L}_q5", 2, L, 5, "hypradon", scale=float(1 << L),
                precision=precision, x_lo=(1.0, 0.0, 0.0), y_lo=(1.0, 0.0, 0.0),
                y_w=(1.0, 1.0, 1.0), seed=1004)


def hypradon_batch(seed: int = 1004):
    """48 problems: 16 each of N = 128, 256, 512; RHS counts uniform in 1..16 (drawn first)."""
    rng = np.random.default_rng(seed)
    Ls = [7] * 16 + [8] * 16 + [9] * 16
    nrhs = rng.integers(1, 17, size=len(Ls))
    return [(hypradon(L), int(k)) for L, k in zip(Ls, nrhs)], rng


def source_values(spec: Spec, nrhs: int = 1, dtype=np.complex64, seed: int | None = None,
                  rng: np.random.Generator | None = None) -> np.ndarray:
    """(nrhs, N^d) complex values, real and imaginary parts i.i.d. N(0,1), rounded to dtype."""
    if rng is None:
        rng = np.random.default_rng(spec.seed if seed is None else seed)
    n = spec.npts
    a = rng.standard_normal((nrhs, n)) + 1j * rng.standard_normal((nrhs, n))
    return a.astype(dtype)


def sparse_spikes(spec: Spec, density: float = 0.01, seed: int | None = None,
                  dtype=np.complex64) -> np.ndarray:
    """m_true for the CG model problem: density*N^d positions without replacement,
    real N(0,1) amplitudes stored as complex."""
    rng = np.random.default_rng(spec.seed + 7 if seed is None else seed)
    n = spec.npts
    k = max(1, int(round(density * n)))
    idx = rng.choice(n, size=k, replace=False)
    m = np.zeros(n, np.complex128)
    m[idx] = rng.standard_normal(k)
    return m.astype(dtype)
