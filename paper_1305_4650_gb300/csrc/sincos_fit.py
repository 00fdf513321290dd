"""Coefficients of the FP32 sincos polynomials in bf_device.cuh (sincos2pi, SC_S*, SC_C*).

After the quadrant reduction f = j/4 + r, |r| <= 1/8, the kernels evaluate

    sin(2 pi r) = r (S0 + S1 u + S2 u^2 + S3 u^3),   cos(2 pi r) = 1 + C1 u + C2 u^2 + C3 u^3,   u = r^2,

with 2 pi folded into the coefficients.  Each polynomial minimises the largest absolute
error on |r| <= 1/8 (for the sine, the error of r S(u)), found by the Remez exchange
algorithm on u in [0, 1/64]; the cosine keeps its constant term at exactly 1.  Run as a
script to print the constants in the form the header holds them.
"""
import numpy as np

U_MAX = 1.0 / 64.0          # (1/8)^2


def _remez(f, w, lo, hi, powers, iters=40, grid=200001):
    """min over c of max_{x in [lo, hi]} |w(x) (f(x) - sum_k c_k x^powers[k])| (Remez exchange)."""
    n = len(powers)
    m = n + 1
    x = (lo + hi) / 2 - (hi - lo) / 2 * np.cos(np.pi * np.arange(m) / (m - 1))
    g = np.linspace(lo, hi, grid)
    for _ in range(iters):
        A = np.empty((m, m))
        for i in range(m):
            A[i, :n] = x[i] ** np.asarray(powers, dtype=float)
            A[i, n] = (-1) ** i / w(x[i])
        c = np.linalg.solve(A, f(x))[:n]
        err = w(g) * (f(g) - sum(ck * g ** pk for ck, pk in zip(c, powers)))
        # one extremum per run of equal sign
        starts = np.concatenate([[0], np.nonzero(np.diff(np.sign(err)))[0] + 1])
        ends = np.concatenate([starts[1:], [grid]])
        ext = [int(a + np.argmax(np.abs(err[a:b]))) for a, b in zip(starts, ends)]
        if len(ext) > m:
            ext = sorted(sorted(ext, key=lambda k: -abs(err[k]))[:m])
        if len(ext) < m:
            break
        x = g[ext]
    return c, float(np.max(np.abs(err)))


def fit():
    """(S0..S3, C1..C3, max abs error of the sine, of the cosine) in exact arithmetic."""
    root = lambda u: np.sqrt(np.maximum(u, 0.0))
    f_s = lambda u: np.where(u > 0, np.sin(2 * np.pi * root(u)) / np.maximum(root(u), 1e-300), 2 * np.pi)
    s, es = _remez(f_s, lambda u: root(u) + 1e-30, 0.0, U_MAX, [0, 1, 2, 3])
    f_c = lambda u: np.cos(2 * np.pi * root(u)) - 1.0
    c, ec = _remez(f_c, lambda u: np.ones_like(u), 0.0, U_MAX, [1, 2, 3])
    return tuple(s), tuple(c), es, ec


if __name__ == "__main__":
    s, c, es, ec = fit()
    f32 = lambda v: float(np.float32(v))
    print("constexpr float " + ", ".join(f"SC_S{k} = {f32(v):.18g}f" for k, v in enumerate(s)) + ";")
    print("constexpr float " + ", ".join(f"SC_C{k + 1} = {f32(v):.18g}f" for k, v in enumerate(c)) + ";")
    print(f"truncation error: sin {es:.3g}, cos {ec:.3g}")
