"""Pins for the FP64 CPU oracle (no GPU).

Each test ties the oracle to something other than itself: a library routine
(numpy.fft, numpy's Chebyshev points, scipy's barycentric interpolator), a
closed form (plane wave, Dirichlet kernel, Parseval), an exactness property of
the method (additively separable phase), brute force on tiny inputs, linear
algebra identities of the adjoint, and the paper's accuracy statement.
"""
import json
import os

import numpy as np
import pytest

import oracle
from paper_1305_4650_gb300 import workloads as wl

rng = np.random.default_rng(12345)
GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


def cgauss(n):
    return rng.standard_normal(n) + 1j * rng.standard_normal(n)


def rel(a, b):
    return np.linalg.norm(a - b) / np.linalg.norm(b)


# ----------------------------------------------------------- nodes / Lagrange

@pytest.mark.parametrize("q", [2, 3, 5, 8, 12])
def test_nodes_match_numpy_chebyshev_points(q):
    # Lobatto nodes = Chebyshev points of the second kind (numpy, ascending) / 2
    z = oracle.cheb_nodes(q, 0)
    np.testing.assert_allclose(np.sort(z), np.polynomial.chebyshev.chebpts2(q) / 2, atol=1e-15)
    assert z[0] == 0.5 and z[-1] == -0.5
    z1 = oracle.cheb_nodes(q, 1)
    np.testing.assert_allclose(np.sort(z1), np.polynomial.chebyshev.chebpts1(q) / 2, atol=1e-15)


@pytest.mark.parametrize("q,kind", [(2, 0), (4, 0), (5, 0), (7, 1), (9, 0)])
def test_lagrange_basis(q, kind):
    from scipy.interpolate import BarycentricInterpolator
    z = oracle.cheb_nodes(q, kind)
    xi = np.linspace(-0.5, 0.5, 13)
    for t in range(q):
        # cardinal property
        for s in range(q):
            assert abs(oracle.lagrange1(z, t, z[s]) - (1.0 if s == t else 0.0)) < 1e-14
        # scipy's barycentric interpolant of the unit vector e_t is l_t
        e = np.zeros(q)
        e[t] = 1.0
        ref = BarycentricInterpolator(z, e)(xi)
        got = np.array([oracle.lagrange1(z, t, x) for x in xi])
        np.testing.assert_allclose(got, ref, atol=1e-12)
    # partition of unity and reproduction of monomials of degree < q
    for p in range(q):
        for x in xi:
            v = sum(z[t] ** p * oracle.lagrange1(z, t, x) for t in range(q))
            assert abs(v - x ** p) < 1e-12


# ------------------------------------------------------------------ direct sum

def _dft_ref(g, N, d, off=0.0):
    """f(x_j) = sum_p e^{2 pi i x.p} g_p with x = (j+off)/N, p in [-N/2,N/2)^d, via numpy.fft."""
    G = g.reshape((N,) * d)
    f = N ** d * np.fft.ifftn(G)
    j = np.indices((N,) * d).sum(axis=0)
    return (f * (-1.0) ** j).ravel()


@pytest.mark.parametrize("d,L", [(1, 4), (2, 3), (2, 4), (3, 2)])
def test_direct_sum_is_the_dft(d, L):
    P = oracle.Problem(d=d, L=L, q=3, phase="dot")
    g = cgauss(P.npts)
    f = oracle.direct_sum(P, g)
    ref = _dft_ref(g, P.N, d)
    assert np.abs(f - ref).max() <= 1e-12 * np.abs(ref).max()
    # Parseval: ||f||^2 = N^d ||g||^2
    assert abs(np.vdot(f, f).real - P.npts * np.vdot(g, g).real) <= 1e-10 * P.npts * np.vdot(g, g).real


def test_direct_sum_plane_wave_and_dirichlet():
    P = oracle.Problem(d=2, L=4, q=3, phase="dot", tgt_off=0.3)
    N = P.N
    k0 = (3, 11)                             # p0 = k0 - N/2
    g = np.zeros(P.npts, complex)
    g[k0[0] * N + k0[1]] = 1.0
    f = oracle.direct_sum(P, g)
    x = (np.indices((N, N)).reshape(2, -1).T + 0.3) / N
    p0 = np.array(k0) - N / 2
    np.testing.assert_allclose(f, np.exp(2j * np.pi * x @ p0), atol=1e-13)
    # all-ones source: product of 1-D geometric sums (Dirichlet kernel)
    f1 = oracle.direct_sum(P, np.ones(P.npts, complex))
    p = np.arange(-N // 2, N // 2)
    D = lambda t: np.exp(2j * np.pi * np.outer(t, p)).sum(axis=1)
    closed = lambda t: np.exp(-1j * np.pi * t * N) * (1 - np.exp(2j * np.pi * t * N)) / (1 - np.exp(2j * np.pi * t))
    np.testing.assert_allclose(D(x[:, 0]), closed(x[:, 0]), atol=1e-11)
    np.testing.assert_allclose(f1, closed(x[:, 0]) * closed(x[:, 1]), atol=1e-10)


# ------------------------------------------------------------------- butterfly

@pytest.mark.parametrize("d,L,q,off", [(2, 1, 2, 0.0), (2, 3, 2, 0.25), (2, 4, 3, 0.0), (2, 5, 5, 0.7),
                                       (3, 2, 3, 0.0), (3, 3, 2, 0.4), (1, 6, 4, 0.1)])
def test_butterfly_exact_for_separable_phase(d, L, q, off):
    # Phi = a(x) + b(y): every interpolated function is constant, so the
    # approximate operator equals the direct sum up to rounding.
    P = oracle.Problem(d=d, L=L, q=q, phase="separable", tgt_off=off, src_off=1 - off if off else 0.0)
    g = cgauss(P.npts)
    fb = oracle.butterfly(P, g)
    fd = oracle.direct_sum(P, g)
    assert rel(fb, fd) < 1e-12


def test_butterfly_zero_phase_sums_sources():
    P = oracle.Problem(d=2, L=4, q=3, phase="separable", scale=0.0)
    g = cgauss(P.npts)
    np.testing.assert_allclose(oracle.butterfly(P, g), np.full(P.npts, g.sum()), rtol=1e-12)


def test_butterfly_dft_error_falls_with_q():
    P0 = oracle.Problem(d=2, L=5, q=3, phase="dot")
    g = cgauss(P0.npts)
    ref = _dft_ref(g, P0.N, 2)
    errs = []
    for q in range(3, 10):
        P = oracle.Problem(d=2, L=5, q=q, phase="dot")
        errs.append(rel(oracle.butterfly(P, g), ref))
    assert all(b < a for a, b in zip(errs, errs[1:])), errs
    assert errs[-1] < 1e-5 and errs[0] > 1e-2


def test_butterfly_hypradon_error_falls_with_q():
    # smooth phase (tau >= 1): hyperbolic Radon, Section 3.1
    errs = []
    for q in (3, 5, 7, 9, 11):
        s = wl.hypradon(5).with_(q=q)
        P = oracle.Problem(**s.oracle_kwargs())
        g = wl.source_values(s, 1, np.complex128)[0]
        errs.append(rel(oracle.butterfly(P, g), oracle.direct_sum(P, g)))
    assert all(b < a for a, b in zip(errs, errs[1:])), errs
    assert errs[-1] < 1e-6


def test_butterfly_first_kind_nodes_converge():
    errs = []
    for q in (4, 6, 8):
        P = oracle.Problem(d=2, L=5, q=q, phase="dot", node_kind=1)
        g = cgauss(P.npts)
        errs.append(rel(oracle.butterfly(P, g), _dft_ref(g, P.N, 2)))
    assert errs[0] > errs[1] > errs[2] and errs[2] < 1e-3


@pytest.mark.parametrize("m", [0, 1, 2, 3, 4])
def test_butterfly_every_switch_level(m):
    P = oracle.Problem(d=2, L=4, q=9, phase="dot", m=m, tgt_off=0.5, src_off=0.5)
    g = cgauss(P.npts)
    assert rel(oracle.butterfly(P, g), oracle.direct_sum(P, g)) < 1e-5


@pytest.mark.parametrize("d,L,q,ph", [(2, 1, 12, "dot"), (2, 2, 12, "dot"), (3, 1, 10, "dot"),
                                      (1, 3, 14, "dot"), (2, 2, 12, "hypradon")])
def test_butterfly_tiny_bruteforce(d, L, q, ph):
    # N = 2, 4, 8 with many nodes: the approximate operator reaches the direct sum
    kw = {}
    if ph == "hypradon":
        kw = dict(x_lo=(1, 0, 0), y_lo=(1, 0, 0), y_w=(1, 1, 1), scale=float(1 << L))
    P = oracle.Problem(d=d, L=L, q=q, phase=ph, tgt_off=0.3, src_off=0.6, **kw)
    g = cgauss(P.npts)
    assert rel(oracle.butterfly(P, g), oracle.direct_sum(P, g)) < 1e-8


def test_restricted_butterfly_equals_full():
    s = wl.genradon2d(L=5).with_(q=4)
    P = oracle.Problem(**s.oracle_kwargs())
    g = cgauss(P.npts)
    full = oracle.butterfly(P, g)
    for lvl, box in [(2, 7), (3, 40), (5, 1000), (0, 0)]:
        fr = oracle.butterfly(P, g, restrict=(lvl, box))
        tg = oracle.restricted_targets(P, lvl, box)
        assert np.array_equal(fr[tg], full[tg])
        mask = np.ones(P.npts, bool)
        mask[tg] = False
        assert not np.any(fr[mask])


# -------------------------------------------------------------------- adjoint

@pytest.mark.parametrize("d,L,q,ph", [(2, 4, 4, "genradon"), (3, 3, 3, "genradon"), (2, 5, 3, "dot"),
                                      (2, 1, 3, "dot"), (2, 3, 5, "separable")])
def test_adjoint_dot_product(d, L, q, ph):
    P = oracle.Problem(d=d, L=L, q=q, phase=ph, tgt_off=0.2)
    g, h = cgauss(P.npts), cgauss(P.npts)
    Bg = oracle.butterfly(P, g)
    BHh = oracle.butterfly_adjoint(P, h)
    assert abs(np.vdot(h, Bg) - np.vdot(BHh, g)) <= 1e-13 * np.linalg.norm(Bg) * np.linalg.norm(h)


def test_adjoint_is_dense_conjugate_transpose():
    P = oracle.Problem(d=2, L=2, q=3, phase="genradon")
    n = P.npts
    E = np.eye(n, dtype=complex)
    B = np.stack([oracle.butterfly(P, E[j]) for j in range(n)], axis=1)
    BH = np.stack([oracle.butterfly_adjoint(P, E[j]) for j in range(n)], axis=1)
    np.testing.assert_allclose(BH, B.conj().T, atol=1e-13)


# ---------------------------------------------------------- paper's accuracy

def test_paper_generalized_radon_accuracy():
    # Section 3.2: r = 5^3 gives roughly one percent relative sup-norm error for
    # Phi = pi (x.p + sqrt(gamma^2 + kappa^2)); K = e^{2 pi i Phi'} with Phi' = Phi / (2 pi).
    with open(os.path.join(GOLDEN, "paper_accuracy.json")) as fh:
        claim = json.load(fh)["genradon3d_r125"]
    P = oracle.Problem(d=3, L=4, q=claim["q"], phase="genradon_paper", scale=claim["scale"])
    g = cgauss(P.npts)
    fb, fd = oracle.butterfly(P, g), oracle.direct_sum(P, g)
    sup = np.abs(fb - fd).max() / np.abs(fd).max()
    lo, hi = claim["rel_sup_err_band"]
    assert lo <= sup <= hi, sup


# ------------------------------------------------------------- phase values

def test_phase_point_values():
    # Hand-computed values of every phase formula (Sections 3.1, 3.2) at points where
    # the trigonometric factors are 0, 1/2 or 1 and the square root is whole.
    import phase_pins
    assert phase_pins.failures() == []
