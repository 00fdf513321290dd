"""Pins of the oracle's arbitrary-point butterfly (sources and targets anywhere in their
domains: the evaluation-anywhere property of Section 1.4 and the sparse point sets of
the paper's closing discussion).  CPU only."""
import numpy as np
import pytest

import oracle


def _prob(**kw):
    base = dict(d=2, L=4, q=5, phase="dot")
    base.update(kw)
    return oracle.Problem(**base)


def _rel(a, b):
    return float(np.linalg.norm(a - b) / np.linalg.norm(b))


def _random_points(rng, P, n, is_src, clustered=False):
    N = 1 << P.L
    lo = (np.array(P.y_lo[:P.d]) if P.y_lo is not None else np.full(P.d, -N / 2)) if is_src else np.array(P.x_lo[:P.d])
    w = (np.array(P.y_w[:P.d]) if P.y_w is not None else np.full(P.d, float(N))) if is_src else np.array(P.x_w[:P.d])
    u = rng.random((n, P.d))
    if clustered:                       # most points in one corner: many empty boxes, some crowded
        u = np.where(rng.random((n, 1)) < 0.8, 0.2 * u, u)
    return lo + u * w


def test_grid_points_in_any_order_reproduce_the_grid_butterfly():
    rng = np.random.default_rng(5)
    for kw in (dict(phase="genradon", L=5, q=4), dict(phase="dot", L=4, q=6, tgt_off=0.3, src_off=0.7),
               dict(d=3, L=2, q=3, phase="genradon")):
        P = _prob(**kw)
        y, x = oracle.grid_points(P, True), oracle.grid_points(P, False)
        g = rng.standard_normal(P.npts) + 1j * rng.standard_normal(P.npts)
        ps, pt = rng.permutation(P.npts), rng.permutation(P.npts)
        ref = oracle.butterfly(P, g)[pt]
        out = oracle.butterfly_points(P, y[ps], g[ps], x[pt])
        assert _rel(out, ref) < 1e-13, kw


def test_direct_sum_points_is_the_fourier_matrix():
    rng = np.random.default_rng(6)
    P = _prob(L=3)
    y, x = _random_points(rng, P, 37, True), _random_points(rng, P, 29, False)
    g = rng.standard_normal(37) + 1j * rng.standard_normal(37)
    K = np.exp(2j * np.pi * (x @ y.T))
    assert _rel(oracle.direct_sum_points(P, y, g, x), K @ g) < 1e-13


def test_separable_phase_is_exact_for_any_points():
    # every interpolated function is constant for Phi = a(x) + b(y): no approximation error
    rng = np.random.default_rng(7)
    P = _prob(phase="separable", L=4, q=3, scale=7.0)
    for clustered in (False, True):
        y, x = _random_points(rng, P, 500, True, clustered), _random_points(rng, P, 300, False, clustered)
        g = rng.standard_normal(500) + 1j * rng.standard_normal(500)
        assert _rel(oracle.butterfly_points(P, y, g, x), oracle.direct_sum_points(P, y, g, x)) < 1e-12


def test_error_falls_with_q_for_random_points():
    rng = np.random.default_rng(8)
    P0 = _prob(L=4)
    y, x = _random_points(rng, P0, 400, True, True), _random_points(rng, P0, 250, False)
    g = rng.standard_normal(400) + 1j * rng.standard_normal(400)
    ref = oracle.direct_sum_points(P0, y, g, x)
    errs = [_rel(oracle.butterfly_points(_prob(L=4, q=q), y, g, x), ref) for q in range(3, 10)]
    assert all(b < a for a, b in zip(errs, errs[1:])), errs
    assert errs[-1] < 1e-6, errs


def test_boundary_points_and_empty_sets():
    rng = np.random.default_rng(9)
    # points on the faces of the domains belong to the outermost boxes (q = 10: error ~2e-7)
    P = _prob(phase="hypradon", L=3, q=10, scale=8.0, x_lo=(1.0, 0.0, 0.0), y_lo=(1.0, 0.0, 0.0),
              y_w=(1.0, 1.0, 1.0))
    y = np.array([[1.0, 0.0], [2.0, 1.0], [1.5, 0.25], [2.0, 0.0]])     # corners and faces of Y
    x = np.array([[2.0, 1.0], [1.0, 0.0], [1.3, 0.9]])
    g = rng.standard_normal(4) + 1j * rng.standard_normal(4)
    assert _rel(oracle.butterfly_points(P, y, g, x), oracle.direct_sum_points(P, y, g, x)) < 1e-6
    assert np.all(oracle.butterfly_points(P, y[:0], g[:0], x) == 0)
    assert oracle.butterfly_points(P, y, g, x[:0]).shape == (0,)
