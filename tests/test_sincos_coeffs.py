"""The FP32 sincos of the mixed path (sincos2pi in bf_device.cuh; sincos2pi2 in bf_pair.cuh
performs the same operations per lane): its coefficients are the minimax fits that
csrc/sincos_fit.py derives, and the polynomial evaluated in FP32 with the kernels' operation
order stays within the error bound the GPU self-check asserts.  CPU only: the FP32 steps are
emulated with NumPy (an FMA rounded once from the exact product plus the addend)."""
import importlib.util
import os
import re

import numpy as np

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
CSRC = os.path.join(ROOT, "paper_1305_4650_gb300", "csrc")


def _fit_module():
    spec = importlib.util.spec_from_file_location("sincos_fit", os.path.join(CSRC, "sincos_fit.py"))
    mod = importlib.util.module_from_spec(spec)
    spec.loader.exec_module(mod)
    return mod


def _header_constants():
    src = open(os.path.join(CSRC, "bf_device.cuh")).read()
    return {k: np.float32(float(v)) for k, v in re.findall(r"(SC_[SC]\d) = (-?[0-9.eE+-]+)f", src)}


def _fma(a, b, c):
    return np.float32(a.astype(np.float64) * b.astype(np.float64) + c.astype(np.float64))


def _sincos2pi_fp32(f, k):
    """The kernels' steps on float32 arrays."""
    f32 = np.float32
    M = f32(12582912.0)
    t = _fma(np.full_like(f, 4.0), f, np.full_like(f, M))
    q = t.view(np.int32)
    r = _fma(np.full_like(f, -0.25), (t - M).astype(np.float32), f)
    u = (r * r).astype(np.float32)
    c = lambda name: np.full_like(f, k[name])
    ps = _fma(u, c("SC_S3"), c("SC_S2"))
    ps = _fma(u, ps, c("SC_S1"))
    ps = _fma(u, ps, c("SC_S0"))
    sn = (r * ps).astype(np.float32)
    pc = _fma(u, c("SC_C3"), c("SC_C2"))
    pc = _fma(u, pc, c("SC_C1"))
    cs = _fma(u, pc, np.ones_like(f))
    s1, c1 = np.where(q & 1, cs, sn), np.where(q & 1, sn, cs)
    return np.where(q & 2, -s1, s1), np.where((q + 1) & 2, -c1, c1)


def test_header_coefficients_are_the_minimax_fit():
    s, c, es, ec = _fit_module().fit()
    k = _header_constants()
    assert sorted(k) == ["SC_C1", "SC_C2", "SC_C3", "SC_S0", "SC_S1", "SC_S2", "SC_S3"]
    for i, v in enumerate(s):
        assert abs(float(k[f"SC_S{i}"]) - v) <= 2 * abs(float(np.spacing(np.float32(v)))), (i, v)
    for i, v in enumerate(c):
        assert abs(float(k[f"SC_C{i + 1}"]) - v) <= 2 * abs(float(np.spacing(np.float32(v)))), (i, v)
    # the truncation errors of the polynomials, far below an FP32 ulp of 1 (1.2e-7)
    assert es < 2e-9 and ec < 4e-8, (es, ec)
    # the leading coefficients are the Taylor ones of sin(2 pi r) and cos(2 pi r) to a few digits
    assert abs(s[0] - 2 * np.pi) < 1e-6 and abs(c[0] + 2 * np.pi ** 2) < 1e-4


def test_fp32_evaluation_error():
    # quadrant boundaries, their neighbours and random phases in (-2, 2): the reduced phase
    # the kernels pass in is below 2 in magnitude
    k = _header_constants()
    rng = np.random.default_rng(5)
    grid = np.arange(-64, 65) / 32.0
    f = np.concatenate([rng.uniform(-2.0, 2.0, 400000), grid, grid + 1e-7, grid - 1e-7,
                        rng.uniform(-1e-3, 1e-3, 1000)]).astype(np.float32)
    s, c = _sincos2pi_fp32(f, k)
    x = 2 * np.pi * f.astype(np.float64)
    err = max(np.max(np.abs(s - np.sin(x))), np.max(np.abs(c - np.cos(x))))
    assert err < 1.5e-7, err                     # the bound of the GPU self-check
    assert np.all(np.abs(s) <= 1.0) and np.all(np.abs(c) <= 1.0 + 1e-7)


def test_a_wrong_coefficient_is_caught():
    # a sign slip or a 1% change in any one coefficient breaks the error bound
    k = _header_constants()
    f = np.random.default_rng(6).uniform(-2.0, 2.0, 100000).astype(np.float32)
    x = 2 * np.pi * f.astype(np.float64)
    for name in k:
        for bad in (-k[name], np.float32(k[name] * 1.01)):
            kk = dict(k)
            kk[name] = bad
            s, c = _sincos2pi_fp32(f, kk)
            err = max(np.max(np.abs(s - np.sin(x))), np.max(np.abs(c - np.cos(x))))
            assert err > 1.5e-7, (name, bad)
