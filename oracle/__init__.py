"""FP64 CPU oracle for the Chebyshev-interpolation butterfly (test infrastructure).

Only ``tests/``, ``__graft_entry__.smoke()`` and ``bench.py``'s CPU-baseline and
reference legs may import this package.  The product path (the CUDA library
and its Python binding) never imports, links or calls it, and the oracle
imports nothing from the product.

Contents (all in ``bf_oracle.c``, plain C99 + OpenMP, FP64):

* ``direct_sum``  -- f(x) = sum_y exp(2 pi i Phi(x,y)) g(y), the operator of
  Section 1 of Poulson-Demanet-Maxwell-Ying, "A Parallel Butterfly Algorithm";
* ``butterfly``   -- Algorithm 1 with the analytic Chebyshev interpolation of
  Section 1.4 (column space, middle switch, row space);
* ``butterfly_adjoint`` -- the exact conjugate transpose of ``butterfly``;
* ``direct_sum_points`` / ``butterfly_points`` -- the same for arbitrary source and
  target point sets (init sums the sources of each leaf box, final evaluates the
  leaf box's interpolant at each target);
* ``cheb_nodes`` / ``lagrange1`` / ``phi`` -- the building blocks, exposed so the
  tests can pin them.

Parity is pinned by ``tests/test_oracle.py``: the DFT special case against
numpy.fft, an exact plane wave for a delta source, Parseval, exactness of the
butterfly for an additively separable phase, error falling with q, brute force
on tiny N, adjoint identities, and the paper's ~1% sup-norm accuracy claim for
r = 5^3 (Section 3.2).
"""
from __future__ import annotations

import ctypes
import os
import subprocess
from dataclasses import dataclass, field

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "bf_oracle.c")
_BUILD = os.path.join(_HERE, "_build")
_LIB = os.path.join(_BUILD, "libbf_oracle.so")

PHASES = {"dot": 0, "genradon": 1, "hypradon": 2, "separable": 3, "genradon_paper": 4}


def build(force: bool = False) -> str:
    """Compile the oracle with gcc (plain C99, -O2, OpenMP).  Returns the .so path."""
    os.makedirs(_BUILD, exist_ok=True)
    if not force and os.path.exists(_LIB) and os.path.getmtime(_LIB) >= os.path.getmtime(_SRC):
        return _LIB
    tmp = _LIB + f".tmp{os.getpid()}"
    cmd = ["gcc", "-std=gnu99", "-O2", "-fPIC", "-shared", "-fopenmp", "-fno-fast-math",
           "-ffp-contract=off", _SRC, "-o", tmp, "-lm"]
    subprocess.run(cmd, check=True)
    os.replace(tmp, _LIB)
    return _LIB


class _Problem(ctypes.Structure):
    _fields_ = [("d", ctypes.c_int32), ("L", ctypes.c_int32), ("q", ctypes.c_int32),
                ("m", ctypes.c_int32), ("phase", ctypes.c_int32), ("node_kind", ctypes.c_int32),
                ("scale", ctypes.c_double),
                ("x_lo", ctypes.c_double * 3), ("x_w", ctypes.c_double * 3),
                ("y_lo", ctypes.c_double * 3), ("y_w", ctypes.c_double * 3),
                ("tgt_off", ctypes.c_double), ("src_off", ctypes.c_double)]


_lib = None


def _bind(path: str):
    """Load an oracle shared library and declare its entry points."""
    lib = ctypes.CDLL(path)
    P = ctypes.POINTER(_Problem)
    cp = ctypes.c_void_p
    lib.orc_direct_sum.argtypes = [P, cp, ctypes.c_int64, cp, cp]
    lib.orc_butterfly.argtypes = [P, cp, cp, ctypes.c_int, ctypes.c_int64]
    lib.orc_butterfly_adjoint.argtypes = [P, cp, cp]
    lib.orc_direct_sum_points.argtypes = [P, ctypes.c_int64, cp, cp, ctypes.c_int64, cp, cp]
    lib.orc_butterfly_points.argtypes = [P, ctypes.c_int64, cp, cp, ctypes.c_int64, cp, cp]
    lib.orc_phi.argtypes = [P, cp, cp]
    lib.orc_phi.restype = ctypes.c_double
    lib.orc_cheb_nodes.argtypes = [ctypes.c_int, ctypes.c_int, cp]
    lib.orc_lagrange1.argtypes = [ctypes.c_int, cp, ctypes.c_int, ctypes.c_double]
    lib.orc_lagrange1.restype = ctypes.c_double
    lib.orc_flat_from_morton.argtypes = [P, ctypes.c_int64]
    lib.orc_flat_from_morton.restype = ctypes.c_int64
    lib.orc_num_threads.restype = ctypes.c_int
    lib.orc_set_num_threads.argtypes = [ctypes.c_int]
    return lib


def _load():
    global _lib
    if _lib is None:
        _lib = _bind(build())
    return _lib


def use_library(path: str | None):
    """Point the wrappers at another build of bf_oracle.c (None: the default build).
    Used by the mutation test, which compiles deliberately broken copies."""
    global _lib
    _lib = None if path is None else _bind(path)


@dataclass
class Problem:
    """One butterfly problem: N = 2**L points per dimension, q nodes, phase kind."""
    d: int
    L: int
    q: int
    phase: str
    scale: float = 1.0
    m: int | None = None            # switch level; floor(L/2) if None
    node_kind: int = 0              # 0 Chebyshev-Lobatto, 1 first kind
    x_lo: tuple = (0.0, 0.0, 0.0)
    x_w: tuple = (1.0, 1.0, 1.0)
    y_lo: tuple | None = None       # default [-N/2, N/2)^d
    y_w: tuple | None = None
    tgt_off: float = 0.0
    src_off: float = 0.0

    @property
    def N(self) -> int:
        return 1 << self.L

    @property
    def npts(self) -> int:
        return self.N ** self.d

    def _c(self) -> _Problem:
        N = self.N
        y_lo = self.y_lo if self.y_lo is not None else (-N / 2,) * 3
        y_w = self.y_w if self.y_w is not None else (float(N),) * 3
        pad = lambda t: (ctypes.c_double * 3)(*(list(t) + [0.0] * 3)[:3])
        return _Problem(self.d, self.L, self.q, self.L // 2 if self.m is None else self.m,
                        PHASES[self.phase], self.node_kind, self.scale,
                        pad(self.x_lo), pad(self.x_w), pad(y_lo), pad(y_w),
                        self.tgt_off, self.src_off)


def _c128(a: np.ndarray) -> np.ndarray:
    return np.ascontiguousarray(a, dtype=np.complex128)


def _check(rc: int, what: str):
    if rc != 0:
        raise ValueError(f"oracle {what} failed with code {rc}")


def direct_sum(P: Problem, g: np.ndarray, targets: np.ndarray | None = None) -> np.ndarray:
    """Direct O(N^{2d}) sum.  g: (N^d,) or (nrhs, N^d).  targets: flat target indices."""
    lib = _load()
    g = _c128(g)
    batch = g.reshape(-1, P.npts)
    tg = None if targets is None else np.ascontiguousarray(targets, dtype=np.int64)
    nt = P.npts if tg is None else tg.size
    out = np.zeros((batch.shape[0], nt), np.complex128)
    pc = P._c()
    for i in range(batch.shape[0]):
        gi = np.ascontiguousarray(batch[i])
        _check(lib.orc_direct_sum(ctypes.byref(pc), gi.ctypes.data, nt,
                                  None if tg is None else tg.ctypes.data, out[i].ctypes.data),
               "direct_sum")
    return out.reshape(g.shape[:-1] + (nt,)) if g.ndim > 1 else out[0]


def butterfly(P: Problem, g: np.ndarray, restrict: tuple[int, int] | None = None) -> np.ndarray:
    """CPU butterfly (Algorithm 1).  restrict=(level, box) limits the work to the
    target boxes on the path to that box; outputs inside it are unchanged."""
    lib = _load()
    g = _c128(g)
    batch = g.reshape(-1, P.npts)
    out = np.zeros_like(batch)
    rl, rb = (-1, 0) if restrict is None else restrict
    pc = P._c()
    for i in range(batch.shape[0]):
        gi = np.ascontiguousarray(batch[i])
        _check(lib.orc_butterfly(ctypes.byref(pc), gi.ctypes.data, out[i].ctypes.data, rl, rb),
               "butterfly")
    return out.reshape(g.shape)


def butterfly_adjoint(P: Problem, f: np.ndarray) -> np.ndarray:
    """Exact conjugate transpose of ``butterfly``."""
    lib = _load()
    f = _c128(f)
    batch = f.reshape(-1, P.npts)
    out = np.zeros_like(batch)
    pc = P._c()
    for i in range(batch.shape[0]):
        fi = np.ascontiguousarray(batch[i])
        _check(lib.orc_butterfly_adjoint(ctypes.byref(pc), fi.ctypes.data, out[i].ctypes.data),
               "butterfly_adjoint")
    return out.reshape(f.shape)


def _points(P: Problem, pts) -> np.ndarray:
    a = np.ascontiguousarray(pts, dtype=np.float64)
    if a.ndim != 2 or a.shape[1] != P.d:
        raise ValueError("points must be an (n, d) array")
    return a


def direct_sum_points(P: Problem, y, g: np.ndarray, x) -> np.ndarray:
    """f_i = sum_j exp(2 pi i Phi(x_i, y_j)) g_j for arbitrary points; g: (nsrc,) or (nrhs, nsrc)."""
    lib = _load()
    y, x = _points(P, y), _points(P, x)
    g = _c128(g)
    batch = g.reshape((1 if g.ndim == 1 else g.shape[0]), y.shape[0])
    out = np.zeros((batch.shape[0], x.shape[0]), np.complex128)
    pc = P._c()
    for i in range(batch.shape[0]):
        gi = np.ascontiguousarray(batch[i])
        _check(lib.orc_direct_sum_points(ctypes.byref(pc), y.shape[0], y.ctypes.data, gi.ctypes.data, x.shape[0],
                                         x.ctypes.data, out[i].ctypes.data), "direct_sum_points")
    return out.reshape(g.shape[:-1] + (x.shape[0],)) if g.ndim > 1 else out[0]


def butterfly_points(P: Problem, y, g: np.ndarray, x) -> np.ndarray:
    """CPU butterfly for arbitrary sources y (nsrc, d) and targets x (ntgt, d)."""
    lib = _load()
    y, x = _points(P, y), _points(P, x)
    g = _c128(g)
    batch = g.reshape((1 if g.ndim == 1 else g.shape[0]), y.shape[0])
    out = np.zeros((batch.shape[0], x.shape[0]), np.complex128)
    pc = P._c()
    for i in range(batch.shape[0]):
        gi = np.ascontiguousarray(batch[i])
        _check(lib.orc_butterfly_points(ctypes.byref(pc), y.shape[0], y.ctypes.data, gi.ctypes.data, x.shape[0],
                                        x.ctypes.data, out[i].ctypes.data), "butterfly_points")
    return out.reshape(g.shape[:-1] + (x.shape[0],)) if g.ndim > 1 else out[0]


def grid_points(P: Problem, is_src: bool) -> np.ndarray:
    """The uniform grid points of the plan, row-major flat order: (N^d, d)."""
    N = 1 << P.L
    y_lo = P.y_lo if P.y_lo is not None else (-N / 2,) * 3
    y_w = P.y_w if P.y_w is not None else (float(N),) * 3
    lo = y_lo if is_src else P.x_lo
    w = y_w if is_src else P.x_w
    off = P.src_off if is_src else P.tgt_off
    idx = np.indices((N,) * P.d).reshape(P.d, -1).T
    return np.stack([lo[k] + (idx[:, k] + off) * (w[k] / N) for k in range(P.d)], axis=1)


def restricted_targets(P: Problem, level: int, box: int) -> np.ndarray:
    """Flat indices of the targets inside target box ``box`` (Morton) at ``level``."""
    lib = _load()
    pc = P._c()
    n = 1 << (P.d * (P.L - level))
    return np.array([lib.orc_flat_from_morton(ctypes.byref(pc), (box << (P.d * (P.L - level))) + i)
                     for i in range(n)], dtype=np.int64)


def phi(P: Problem, x, y) -> float:
    lib = _load()
    xa = np.ascontiguousarray(np.resize(np.asarray(x, np.float64), 3))
    ya = np.ascontiguousarray(np.resize(np.asarray(y, np.float64), 3))
    return lib.orc_phi(ctypes.byref(P._c()), xa.ctypes.data, ya.ctypes.data)


def cheb_nodes(q: int, kind: int = 0) -> np.ndarray:
    lib = _load()
    z = np.zeros(q, np.float64)
    lib.orc_cheb_nodes(q, kind, z.ctypes.data)
    return z


def lagrange1(z: np.ndarray, t: int, xi: float) -> float:
    lib = _load()
    z = np.ascontiguousarray(z, np.float64)
    return lib.orc_lagrange1(len(z), z.ctypes.data, t, xi)


def num_threads() -> int:
    return _load().orc_num_threads()


def set_num_threads(n: int) -> None:
    _load().orc_set_num_threads(n)
