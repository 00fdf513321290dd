"""C ABI checks that need no GPU: the library loads, exports every entry point
declared in include/bf.h, and rejects invalid arguments before touching CUDA."""
import ctypes
import os
import re
import subprocess

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module")
def lib():
    from paper_1305_4650_gb300 import build, bf
    build.build()
    return bf.load()


def declared_functions():
    src = open(os.path.join(ROOT, "include", "bf.h")).read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    return sorted(set(re.findall(r"\b(bf_[a-z_]+)\s*\(", src)))


def test_header_declares_the_abi():
    names = declared_functions()
    for n in ["bf_plan_create", "bf_apply", "bf_apply_adjoint", "bf_destroy", "bf_apply_batched",
              "bf_status_string", "bf_last_cuda_error", "bf_apply_host", "bf_params_default", "bf_plan_info"]:
        assert n in names


def test_library_exports_every_declared_symbol(lib):
    from paper_1305_4650_gb300 import bf
    out = subprocess.run(["nm", "-D", "--defined-only", bf.LIB_PATH], capture_output=True, text=True, check=True).stdout
    exported = set(re.findall(r"\bT (bf_[a-z_]+)\b", out))
    missing = [n for n in declared_functions() if n not in exported]
    assert not missing, missing
    for n in declared_functions():
        assert hasattr(lib, n)


def test_status_strings(lib):
    assert lib.bf_status_string(0) == b"BF_OK"
    assert lib.bf_status_string(1) == b"BF_ERR_INVALID_ARG"
    assert lib.bf_status_string(99) == b"BF_ERR_UNKNOWN"


def test_invalid_arguments_rejected_without_gpu(lib):
    from paper_1305_4650_gb300.bf import BfParams
    p = BfParams()
    assert lib.bf_params_default(2, 64, ctypes.byref(p)) == 0
    assert p.y_lo[0] == -32.0 and p.y_w[1] == 64.0 and p.switch_level == -1
    h = ctypes.c_void_p()
    create = lambda d, N, q, ph, pp: lib.bf_plan_create(d, N, q, ph, ctypes.byref(pp), ctypes.byref(h))
    assert create(2, 63, 5, 1, p) == 1           # N not a power of two
    assert create(2, 1, 5, 1, p) == 1            # L = 0
    assert create(4, 64, 5, 1, p) == 1           # d out of range
    assert create(1, 64, 5, 1, p) == 2           # d = 1 not compiled
    assert create(2, 64, 1, 1, p) == 1           # q < 2
    assert create(2, 64, 7, 1, p) == 2           # q = 7 not compiled
    assert create(3, 64, 2, 2, p) == 1           # hyperbolic Radon is 2-D
    assert create(2, 64, 5, 9, p) == 1           # unknown phase
    assert create(2, 1 << 16, 5, 1, p) == 1      # N^d > 2^30
    for field, val in [("switch_level", 6), ("switch_level", -2), ("max_nrhs", 0), ("node_kind", 2),
                       ("precision", 5), ("tgt_off", 1.0), ("src_off", -0.1), ("fuse_levels", 9)]:
        q = BfParams()
        lib.bf_params_default(2, 64, ctypes.byref(q))
        setattr(q, field, val)
        assert create(2, 64, 5, 1, q) == 1, field
    q = BfParams()
    lib.bf_params_default(2, 64, ctypes.byref(q))
    q.x_w[0] = 0.0
    assert create(2, 64, 5, 1, q) == 1
    q = BfParams()
    lib.bf_params_default(2, 64, ctypes.byref(q))
    q.reserved[3] = 1
    assert create(2, 64, 5, 1, q) == 1
    # the mixed path needs |Phi| < 2^21 cycles: the separable test phase reaches y^2/2 = 8.4e6 at N = 4096
    q = BfParams()
    lib.bf_params_default(2, 4096, ctypes.byref(q))
    assert create(2, 4096, 3, 3, q) == 2
    assert h.value is None
    assert lib.bf_destroy(None) == 0
    assert lib.bf_apply(None, None, None, 1, None) == 1
    assert lib.bf_apply_adjoint(None, None, None, 1, None) == 1
    assert lib.bf_apply_batched(None, None, None, None, -1, None) == 1
    assert lib.bf_apply_batched(None, None, None, None, 0, None) == 0
    e = ctypes.c_int()
    assert lib.bf_last_cuda_error(None, ctypes.byref(e)) == 1
