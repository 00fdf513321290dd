"""Python binding of the C ABI in include/bf.h (argument marshalling only).

Every step of the butterfly runs in the sm_103a kernels of ``libbf_gb300.so``;
this module only converts arguments.  PyTorch supplies device memory and the
current stream.  If the library has not been built, every entry point raises
instead of falling back to anything else.
"""
from __future__ import annotations

import ctypes
import os

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(HERE, "_build", "libbf_gb300.so")

PHASE = {"dot": 0, "genradon": 1, "hypradon": 2, "separable": 3}
PREC = {"fp64": 0, "mixed": 1, "mixed_sfu": 2, "bf16x3": 3, "tf32x3": 4}
STATUS = {0: "BF_OK", 1: "BF_ERR_INVALID_ARG", 2: "BF_ERR_UNSUPPORTED", 3: "BF_ERR_NOMEM",
          4: "BF_ERR_CUDA", 5: "BF_ERR_TIMEOUT", 6: "BF_ERR_INTERNAL"}

EXPORTS = ["bf_params_default", "bf_plan_create", "bf_apply", "bf_apply_adjoint", "bf_apply_host",
           "bf_apply_batched", "bf_destroy", "bf_status_string", "bf_last_cuda_error", "bf_plan_info",
           "bf_apply_pass", "bf_pass_info", "bf_pass_count", "bf_selfcheck_sincos", "bf_selfcheck_phase", "bf_measure_fma_rate",
           "bf_measure_phase_rate", "bf_batch_create", "bf_batch_apply", "bf_batch_status",
           "bf_batch_selftest_timeout", "bf_batch_info", "bf_batch_wait_stats", "bf_batch_destroy", "bf_plan_autotune",
           "bf_plan_table_info", "bf_plan_create_points", "bf_plan_points_info", "bf_plan_tc_info"]


class BfError(RuntimeError):
    def __init__(self, code: int, what: str):
        super().__init__(f"{what}: {STATUS.get(code, code)}")
        self.code = code


class BfParams(ctypes.Structure):
    _fields_ = [("x_lo", ctypes.c_double * 3), ("x_w", ctypes.c_double * 3),
                ("y_lo", ctypes.c_double * 3), ("y_w", ctypes.c_double * 3),
                ("phase_scale", ctypes.c_double), ("tgt_off", ctypes.c_double), ("src_off", ctypes.c_double),
                ("precision", ctypes.c_int32), ("switch_level", ctypes.c_int32), ("node_kind", ctypes.c_int32),
                ("max_nrhs", ctypes.c_int32), ("fuse_levels", ctypes.c_int32), ("phase_tables", ctypes.c_int32),
                ("tc_levels", ctypes.c_int32), ("tc_cpasync", ctypes.c_int32), ("reserved", ctypes.c_int32 * 4)]


_lib = None


def load():
    """Load the CUDA library (raises if it is missing: there is no fallback)."""
    global _lib
    if _lib is None:
        if not os.path.exists(LIB_PATH):
            raise RuntimeError(f"butterfly CUDA library not built: {LIB_PATH} missing "
                               "(run __graft_entry__.build() or python -m paper_1305_4650_gb300.build)")
        lib = ctypes.CDLL(LIB_PATH)
        vp, i64, i32 = ctypes.c_void_p, ctypes.c_int64, ctypes.c_int
        lib.bf_params_default.argtypes = [i32, i64, ctypes.POINTER(BfParams)]
        lib.bf_plan_create.argtypes = [i32, i64, i32, i32, ctypes.POINTER(BfParams), ctypes.POINTER(vp)]
        lib.bf_apply.argtypes = [vp, vp, vp, i32, vp]
        lib.bf_apply_adjoint.argtypes = [vp, vp, vp, i32, vp]
        lib.bf_apply_host.argtypes = [vp, vp, vp, i32, vp]
        lib.bf_apply_batched.argtypes = [ctypes.POINTER(vp), ctypes.POINTER(vp), ctypes.POINTER(vp),
                                         ctypes.POINTER(i32), i32, vp]
        lib.bf_destroy.argtypes = [vp]
        lib.bf_status_string.argtypes = [i32]
        lib.bf_status_string.restype = ctypes.c_char_p
        lib.bf_last_cuda_error.argtypes = [vp, ctypes.POINTER(i32)]
        lib.bf_plan_info.argtypes = [vp, ctypes.POINTER(i32), ctypes.POINTER(i64), ctypes.POINTER(i32),
                                     ctypes.POINTER(i32), ctypes.POINTER(i32), ctypes.POINTER(i32),
                                     ctypes.POINTER(i64)]
        lib.bf_apply_pass.argtypes = [vp, i32, vp, vp, i32, vp]
        lib.bf_pass_info.argtypes = [vp, i32, i32, ctypes.POINTER(i32), ctypes.POINTER(i32), ctypes.POINTER(i32),
                                     ctypes.POINTER(i32)]
        lib.bf_pass_count.argtypes = [vp, i32, ctypes.POINTER(i32)]
        lib.bf_selfcheck_sincos.argtypes = [i32, ctypes.POINTER(ctypes.c_double)]
        lib.bf_selfcheck_phase.argtypes = [vp, i32, ctypes.POINTER(ctypes.c_double)]
        lib.bf_measure_fma_rate.argtypes = [i32, ctypes.POINTER(ctypes.c_double)]
        lib.bf_measure_phase_rate.argtypes = [vp, i32, ctypes.POINTER(ctypes.c_double)]
        lib.bf_selfcheck_umma.argtypes = [i32, ctypes.POINTER(ctypes.c_double), ctypes.POINTER(i32)]
        lib.bf_selfcheck_umma_tf32.argtypes = [i32, ctypes.POINTER(ctypes.c_double), ctypes.POINTER(i32)]
        lib.bf_apply_shard.argtypes = [vp, vp, vp, i32, i32, i32, vp]
        lib.bf_batch_create.argtypes = [ctypes.POINTER(vp), ctypes.POINTER(i32), i32, ctypes.POINTER(vp)]
        lib.bf_batch_apply.argtypes = [vp, ctypes.POINTER(vp), ctypes.POINTER(vp), vp]
        lib.bf_batch_status.argtypes = [vp, ctypes.POINTER(i32)]
        lib.bf_batch_selftest_timeout.argtypes = [vp, ctypes.POINTER(vp), ctypes.POINTER(vp), vp, ctypes.POINTER(i32)]
        lib.bf_batch_info.argtypes = [vp, ctypes.POINTER(i32), ctypes.POINTER(i32), ctypes.POINTER(i32),
                                      ctypes.POINTER(i64)]
        lib.bf_batch_destroy.argtypes = [vp]
        lib.bf_plan_autotune.argtypes = [vp, i32, i32, vp, ctypes.POINTER(ctypes.c_double)]
        lib.bf_plan_create_points.argtypes = [i32, i64, i32, i32, ctypes.POINTER(BfParams), i64, vp, i64, vp,
                                              ctypes.POINTER(vp)]
        lib.bf_plan_points_info.argtypes = [vp, ctypes.POINTER(i32), ctypes.POINTER(i64), ctypes.POINTER(i64)]
        lib.bf_plan_tc_info.argtypes = [vp, ctypes.POINTER(i32)]
        lib.bf_plan_table_info.argtypes = [vp, ctypes.POINTER(i64), ctypes.POINTER(ctypes.c_double),
                                           ctypes.POINTER(i32)]
        lib.bf_batch_wait_stats.argtypes = [vp, ctypes.POINTER(ctypes.c_double), ctypes.POINTER(i64)]
        for name in EXPORTS:
            getattr(lib, name).restype = getattr(lib, name).restype or ctypes.c_int
        lib.bf_status_string.restype = ctypes.c_char_p
        _lib = lib
    return _lib


def _check(code: int, what: str, plan=None):
    if code != 0:
        if code == 4 and plan is not None and plan.value:
            e = ctypes.c_int()
            load().bf_last_cuda_error(plan, ctypes.byref(e))
            what = f"{what} (cudaError {e.value})"
        raise BfError(code, what)


def _stream_ptr(stream) -> int:
    import torch
    if stream is None:
        stream = torch.cuda.current_stream()
    return int(stream.cuda_stream) if hasattr(stream, "cuda_stream") else int(stream)


class Plan:
    """A butterfly plan: owns device workspace and geometry tables."""

    def __init__(self, d: int, N: int, q: int, phase: str, precision: str = "mixed", scale: float = 1.0,
                 x_lo=None, x_w=None, y_lo=None, y_w=None, tgt_off: float = 0.0, src_off: float = 0.0,
                 switch_level: int = -1, node_kind: int = 0, max_nrhs: int = 1, fuse_levels: int = 0,
                 phase_tables: bool = False, sources=None, targets=None, tc_levels: bool = False,
                 tc_cpasync: bool = False):
        lib = load()
        p = BfParams()
        _check(lib.bf_params_default(d, N, ctypes.byref(p)), "bf_params_default")
        for name, val in (("x_lo", x_lo), ("x_w", x_w), ("y_lo", y_lo), ("y_w", y_w)):
            if val is not None:
                arr = getattr(p, name)
                for k, v in enumerate(list(val)[:3]):
                    arr[k] = float(v)
        p.phase_scale = scale
        p.tgt_off, p.src_off = tgt_off, src_off
        p.precision = PREC[precision]
        p.switch_level = switch_level
        p.node_kind = node_kind
        p.max_nrhs = max_nrhs
        p.fuse_levels = fuse_levels
        p.phase_tables = 1 if phase_tables else 0
        p.tc_levels = 1 if tc_levels else 0
        p.tc_cpasync = 1 if tc_cpasync else 0
        h = ctypes.c_void_p()
        if sources is None and targets is None:
            _check(lib.bf_plan_create(d, N, q, PHASE[phase], ctypes.byref(p), ctypes.byref(h)), "bf_plan_create")
            self.nsrc = self.ntgt = N ** d
        else:
            ys = np.ascontiguousarray(np.asarray(sources, dtype=np.float64).reshape(-1, d))
            xs = np.ascontiguousarray(np.asarray(targets, dtype=np.float64).reshape(-1, d))
            _check(lib.bf_plan_create_points(d, N, q, PHASE[phase], ctypes.byref(p), ys.shape[0],
                                             ys.ctypes.data if ys.size else None, xs.shape[0],
                                             xs.ctypes.data if xs.size else None, ctypes.byref(h)),
                   "bf_plan_create_points")
            self.nsrc, self.ntgt = ys.shape[0], xs.shape[0]
        self._h = h
        self.d, self.N, self.q, self.precision, self.max_nrhs = d, N, q, precision, max_nrhs
        self.npts = N ** d
        self.cdtype = np.complex128 if precision == "fp64" else np.complex64

    @classmethod
    def from_spec(cls, spec, max_nrhs: int = 1, precision: str | None = None, fuse_levels: int = 0,
                  phase_tables: bool = False, sources=None, targets=None, tc_levels: bool = False,
                  tc_cpasync: bool = False) -> "Plan":
        """Plan for a workload spec; sources / targets ((n, d) arrays) make a point-set plan."""
        x_lo, x_w, y_lo, y_w = spec.domain()
        return cls(spec.d, spec.N, spec.q, spec.phase, precision or spec.precision, spec.scale,
                   x_lo, x_w, y_lo, y_w, spec.tgt_off, spec.src_off, spec.switch_level, spec.node_kind,
                   max_nrhs, fuse_levels, phase_tables, sources, targets, tc_levels, tc_cpasync)

    @property
    def handle(self) -> int:
        return self._h.value

    def torch_dtype(self):
        import torch
        return torch.complex128 if self.precision == "fp64" else torch.complex64

    def _nrhs(self, t, n=None) -> int:
        import torch
        n = self.npts if n is None else n
        if not isinstance(t, torch.Tensor) or not t.is_cuda:
            raise TypeError("expected a CUDA tensor")
        if t.dtype != self.torch_dtype():
            raise TypeError(f"expected dtype {self.torch_dtype()}, got {t.dtype}")
        if not t.is_contiguous() or (n and t.numel() % n) or (not n and t.numel()):
            raise ValueError("expected a contiguous tensor of nrhs x points elements")
        return t.numel() // n if n else (t.shape[0] if t.dim() > 1 else 1)

    def apply(self, g, f=None, stream=None):
        """f = B g for CUDA tensors of shape (nsrc,) or (nrhs, nsrc); f: (nrhs, ntgt)
        (nsrc = ntgt = N^d for grid plans)."""
        import torch
        n = self._nrhs(g, self.nsrc)
        if f is None:
            f = torch.empty((n, self.ntgt) if g.dim() > 1 else (self.ntgt,), dtype=g.dtype, device=g.device)
        elif self._nrhs(f, self.ntgt) != n:
            raise ValueError("g and f differ in size")
        _check(load().bf_apply(self._h, g.data_ptr(), f.data_ptr(), n, _stream_ptr(stream)), "bf_apply", self._h)
        return f

    def apply_shard(self, g, shard_g: int, shard_r: int, f=None, stream=None):
        """f_r: rank shard_r's part of B g when the sources are split over 2^shard_g ranks by the
        top Morton bits of their leaf boxes (bf_apply_shard); the sum over ranks is B g."""
        import torch
        n = self._nrhs(g, self.nsrc)
        if f is None:
            f = torch.empty((n, self.ntgt) if g.dim() > 1 else (self.ntgt,), dtype=g.dtype, device=g.device)
        elif self._nrhs(f, self.ntgt) != n:
            raise ValueError("g and f differ in size")
        _check(load().bf_apply_shard(self._h, g.data_ptr(), f.data_ptr(), n, shard_g, shard_r, _stream_ptr(stream)),
               "bf_apply_shard", self._h)
        return f

    def apply_adjoint(self, f, g=None, stream=None):
        """g = B^H f (grid plans)."""
        import torch
        n = self._nrhs(f, self.ntgt)
        if g is None:
            g = torch.empty((n, self.nsrc) if f.dim() > 1 else (self.nsrc,), dtype=f.dtype, device=f.device)
        elif self._nrhs(g, self.nsrc) != n:
            raise ValueError("f and g differ in size")
        _check(load().bf_apply_adjoint(self._h, f.data_ptr(), g.data_ptr(), n, _stream_ptr(stream)),
               "bf_apply_adjoint", self._h)
        return g

    def apply_host(self, g: np.ndarray, f: np.ndarray | None = None, stream=None) -> np.ndarray:
        """Host-buffer apply: H2D copy, butterfly, D2H copy, stream synchronised."""
        g = np.ascontiguousarray(g, dtype=self.cdtype)
        if (self.nsrc and g.size % self.nsrc) or (not self.nsrc and g.size):
            raise ValueError("g must hold nrhs x nsrc values")
        n = g.size // self.nsrc if self.nsrc else (g.shape[0] if g.ndim > 1 else 1)
        if f is None:
            f = np.empty((n, self.ntgt) if g.ndim > 1 else (self.ntgt,), dtype=self.cdtype)
        st = 0 if stream is None else _stream_ptr(stream)
        _check(load().bf_apply_host(self._h, g.ctypes.data, f.ctypes.data, n, st), "bf_apply_host", self._h)
        return f

    def apply_ptr(self, g_ptr: int, f_ptr: int, nrhs: int, stream_ptr: int = 0) -> None:
        _check(load().bf_apply(self._h, g_ptr, f_ptr, nrhs, stream_ptr), "bf_apply", self._h)

    def apply_host_ptr(self, g_ptr: int, f_ptr: int, nrhs: int, stream_ptr: int = 0) -> None:
        _check(load().bf_apply_host(self._h, g_ptr, f_ptr, nrhs, stream_ptr), "bf_apply_host", self._h)

    def apply_pass(self, i: int, g_ptr: int, f_ptr: int, nrhs: int, stream_ptr: int = 0) -> None:
        """Run pass i of the apply schedule only (instrumentation)."""
        _check(load().bf_apply_pass(self._h, i, g_ptr, f_ptr, nrhs, stream_ptr), "bf_apply_pass", self._h)

    def table_info(self) -> dict:
        """Bytes of the plan's phase table (0 without), the milliseconds its construction took, and
        whether a wait for a table copy ever gave up (synchronises the device)."""
        b, ms, t = ctypes.c_int64(), ctypes.c_double(), ctypes.c_int()
        _check(load().bf_plan_table_info(self._h, ctypes.byref(b), ctypes.byref(ms), ctypes.byref(t)),
               "bf_plan_table_info")
        return dict(bytes=b.value, build_ms=ms.value, timed_out=bool(t.value))

    def tc_info(self) -> dict:
        """Whether the tensor-core switch stages its weights by tiled bulk copies (TMA)."""
        t = ctypes.c_int()
        _check(load().bf_plan_tc_info(self._h, ctypes.byref(t)), "bf_plan_tc_info")
        return dict(tiled_copies=bool(t.value))

    def autotune(self, nrhs: int = 1, reps: int = 3, stream=None) -> float:
        """Time candidate tile schedules for nrhs right-hand sides, keep the fastest; ms per apply."""
        ms = ctypes.c_double()
        _check(load().bf_plan_autotune(self._h, nrhs, reps, _stream_ptr(stream), ctypes.byref(ms)),
               "bf_plan_autotune", self._h)
        return ms.value

    def launches(self, nrhs: int = 1) -> int:
        """Kernel launches (passes) of one apply of nrhs right-hand sides."""
        n = ctypes.c_int()
        _check(load().bf_pass_count(self._h, nrhs, ctypes.byref(n)), "bf_pass_count")
        return n.value

    def passes(self, nrhs: int = 1) -> list[dict]:
        """The pass schedule bf_apply runs for nrhs right-hand sides."""
        i32 = ctypes.c_int
        out = []
        for i in range(self.launches(nrhs)):
            kind, l0, k, fl = i32(), i32(), i32(), i32()
            _check(load().bf_pass_info(self._h, nrhs, i, ctypes.byref(kind), ctypes.byref(l0), ctypes.byref(k),
                                       ctypes.byref(fl)), "bf_pass_info")
            out.append(dict(kind=("col", "row", "switch_tc", "col_tc")[kind.value], l0=l0.value, k=k.value,
                            init=bool(fl.value & 1), switch=bool(fl.value & 2), final=bool(fl.value & 4)))
        return out

    def info(self) -> dict:
        i32, i64 = ctypes.c_int, ctypes.c_int64
        d, q, m, k, nl = i32(), i32(), i32(), i32(), i32()
        N, ws = i64(), i64()
        _check(load().bf_plan_info(self._h, ctypes.byref(d), ctypes.byref(N), ctypes.byref(q), ctypes.byref(m),
                                   ctypes.byref(k), ctypes.byref(nl), ctypes.byref(ws)), "bf_plan_info")
        return dict(d=d.value, N=N.value, q=q.value, m=m.value, fuse_levels=k.value, launches=nl.value,
                    workspace_bytes=ws.value)

    def selfcheck_phase(self, n: int = 1 << 20) -> float:
        """Largest error (cycles, mod 1) of the double-float phase against FP64 on the same features."""
        e = ctypes.c_double()
        _check(load().bf_selfcheck_phase(self._h, n, ctypes.byref(e)), "bf_selfcheck_phase", self._h)
        return e.value

    def phase_rate(self, paired: bool = False) -> float:
        """Measured phase factors per second (10^9) of this plan's phase, one or two per instruction stream."""
        e = ctypes.c_double()
        _check(load().bf_measure_phase_rate(self._h, 1 if paired else 0, ctypes.byref(e)), "bf_measure_phase_rate",
               self._h)
        return e.value

    def last_cuda_error(self) -> int:
        e = ctypes.c_int()
        _check(load().bf_last_cuda_error(self._h, ctypes.byref(e)), "bf_last_cuda_error")
        return e.value

    def close(self):
        if getattr(self, "_h", None) is not None and self._h.value:
            load().bf_destroy(self._h)
            self._h = ctypes.c_void_p()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


def selfcheck_sincos(n: int = 1 << 22) -> float:
    """Largest |error| of the mixed path's FP32 sin/cos of 2 pi f against FP64 sincospi."""
    e = ctypes.c_double()
    _check(load().bf_selfcheck_sincos(n, ctypes.byref(e)), "bf_selfcheck_sincos")
    return e.value


def selfcheck_umma(split: bool = False, fmt: str = "bf16") -> tuple[float, bool]:
    """Tensor-core GEMM self-check (128 x 32 x 64 with BF16 operands, or 128 x 32 x 32 with
    TF32 operands (fmt="tf32"); FP32 accumulator): the largest error relative to max |D|
    (0 expected without the split), and whether the completion wait gave up."""
    e, t = ctypes.c_double(), ctypes.c_int()
    if fmt not in ("bf16", "tf32"):
        raise ValueError(fmt)
    fn = "bf_selfcheck_umma" if fmt == "bf16" else "bf_selfcheck_umma_tf32"
    _check(getattr(load(), fn)(1 if split else 0, ctypes.byref(e), ctypes.byref(t)), fn)
    return e.value, bool(t.value)


def measure_fma_rate(fp64: bool = False, packed: bool = False) -> float:
    """Measured FMA rate of the current device, TFLOP/s: FP32, FP64 (fp64=True) or FP32 in
    packed pairs (packed=True)."""
    e = ctypes.c_double()
    mode = 1 if fp64 else (2 if packed else 0)
    _check(load().bf_measure_fma_rate(mode, ctypes.byref(e)), "bf_measure_fma_rate")
    return e.value


def apply_batched(plans, gs, fs, nrhs, stream=None) -> None:
    """Independent problems in order on one stream (device tensors)."""
    n = len(plans)
    vp = ctypes.c_void_p
    P = (vp * n)(*[p.handle for p in plans])
    G = (vp * n)(*[g.data_ptr() for g in gs])
    F = (vp * n)(*[f.data_ptr() for f in fs])
    R = (ctypes.c_int * n)(*nrhs)
    _check(load().bf_apply_batched(P, G, F, R, n, _stream_ptr(stream)), "bf_apply_batched")


class Batch:
    """Persistent batch: every pass of every problem in one kernel launch (bf_batch_*)."""

    def __init__(self, plans, nrhs):
        vp = ctypes.c_void_p
        n = len(plans)
        self.plans = list(plans)          # keep the plans alive
        self.nrhs = list(nrhs)
        P = (vp * n)(*[p.handle for p in plans])
        R = (ctypes.c_int * n)(*nrhs)
        h = vp()
        _check(load().bf_batch_create(P, R, n, ctypes.byref(h)), "bf_batch_create")
        self._h = h

    def _ptrs(self, gs, fs):
        vp = ctypes.c_void_p
        n = len(self.plans)
        if len(gs) != n or len(fs) != n:
            raise ValueError("one g and one f per problem")
        return (vp * n)(*[g.data_ptr() for g in gs]), (vp * n)(*[f.data_ptr() for f in fs])

    def apply(self, gs, fs, stream=None) -> None:
        G, F = self._ptrs(gs, fs)
        _check(load().bf_batch_apply(self._h, G, F, _stream_ptr(stream)), "bf_batch_apply")

    def status(self) -> bool:
        """True if a wait of the last apply timed out (synchronises the device)."""
        t = ctypes.c_int()
        _check(load().bf_batch_status(self._h, ctypes.byref(t)), "bf_batch_status")
        return bool(t.value)

    def selftest_timeout(self, gs, fs, stream=None) -> bool:
        G, F = self._ptrs(gs, fs)
        t = ctypes.c_int()
        _check(load().bf_batch_selftest_timeout(self._h, G, F, _stream_ptr(stream), ctypes.byref(t)),
               "bf_batch_selftest_timeout")
        return bool(t.value)

    def info(self) -> dict:
        i32, i64 = ctypes.c_int, ctypes.c_int64
        j, u, g, sm = i32(), i32(), i32(), i64()
        _check(load().bf_batch_info(self._h, ctypes.byref(j), ctypes.byref(u), ctypes.byref(g), ctypes.byref(sm)),
               "bf_batch_info")
        return dict(jobs=j.value, units=u.value, grid=g.value, smem_bytes=sm.value)

    def wait_stats(self) -> dict:
        """Dependency waits of the last apply: total CTA-milliseconds and count (synchronises)."""
        ms, n = ctypes.c_double(), ctypes.c_int64()
        _check(load().bf_batch_wait_stats(self._h, ctypes.byref(ms), ctypes.byref(n)), "bf_batch_wait_stats")
        return dict(wait_ms_total=ms.value, waits=n.value)

    def close(self) -> None:
        if getattr(self, "_h", None):
            load().bf_batch_destroy(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


def apply_noalloc(d: int, N: int, q: int, phase: str, g, f, precision: str = "mixed", scale: float = 1.0,
                  x_lo=None, x_w=None, y_lo=None, y_w=None, tgt_off: float = 0.0, src_off: float = 0.0,
                  switch_level: int = -1, node_kind: int = 0, fuse_levels: int = 0, stream=None) -> None:
    """bf_apply_noalloc: forward apply whose tables and workspace live in the library's
    static device array (no device allocation).  g, f: CUDA tensors of nrhs x N^d values."""
    lib = load()
    fn = lib.bf_apply_noalloc
    fn.argtypes = [ctypes.c_int, ctypes.c_int64, ctypes.c_int, ctypes.c_int, ctypes.POINTER(BfParams),
                   ctypes.c_void_p, ctypes.c_void_p, ctypes.c_int, ctypes.c_void_p]
    fn.restype = ctypes.c_int
    p = BfParams()
    _check(lib.bf_params_default(d, N, ctypes.byref(p)), "bf_params_default")
    for name, val in (("x_lo", x_lo), ("x_w", x_w), ("y_lo", y_lo), ("y_w", y_w)):
        if val is not None:
            arr = getattr(p, name)
            for k, v in enumerate(list(val)[:3]):
                arr[k] = float(v)
    p.phase_scale = scale
    p.tgt_off, p.src_off = tgt_off, src_off
    p.precision = PREC[precision]
    p.switch_level = switch_level
    p.node_kind = node_kind
    p.fuse_levels = fuse_levels
    npts = N ** d
    if g.numel() % npts or g.numel() != f.numel():
        raise ValueError("g and f must hold nrhs x N^d values each")
    _check(fn(d, N, q, PHASE[phase], ctypes.byref(p), g.data_ptr(), f.data_ptr(), g.numel() // npts,
              _stream_ptr(stream)), "bf_apply_noalloc")
