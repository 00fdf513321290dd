"""Hand-computed values of the phase functions, for pinning ``oracle.phi``.

Each case picks a target x where the sines and cosines inside the phase take
the values 0, 1/2 or 1, and a source y for which the square root is a whole
number, so the expected value is exact arithmetic done by hand (derivation in
the comment).  Phases (kernel exp(2 pi i Phi)):

* Fourier (Section 3): Phi = s x.y;
* generalized Radon analogue (Section 3.2, written with 2 pi outside Phi):
  Phi = s (x.y + sqrt(sum_k a_k(x)^2 y_k^2)) with, for d = 2,
  a_0 = (2 + sin 2pi x0 sin 2pi x1)/3, a_1 = (2 + cos 2pi x0 cos 2pi x1)/3, and for
  d = 3, a_k = (2 + sin 2pi x_k cos 2pi x_{k+1 mod 3})/3;
* the same as printed in Section 3.2 (gamma, kappa from x0, x1, p0, p1 only);
* hyperbolic Radon (Section 3.1): Phi = s w sqrt(tau^2 + p^2 h^2), x = (w, h), y = (tau, p);
* the separable test phase Phi = s (sum_k sin 2pi(x_k + (k+1)/7) + sum_k y_k^2/(k+2)).

A slip in any coefficient formula (sin for cos, the wrong neighbour index, a
swapped coordinate) changes at least one of these values by far more than
the tolerance.
"""
import oracle

TOL = 1e-13

# (phase, d, scale, x, y, expected Phi, derivation)
CASES = [
    ("dot", 2, 1.0, (0.5, 0.25), (6.0, -8.0), 1.0, "3 - 2"),
    ("dot", 3, 2.0, (0.5, 0.25, 0.125), (2.0, 4.0, 8.0), 6.0, "2 (1 + 1 + 1)"),
    # d = 2 at x = 0: a0 = (2 + 0)/3 = 2/3, a1 = (2 + 1)/3 = 1; (a0 y0, a1 y1) = (3, 4) -> 5
    ("genradon", 2, 1.0, (0.0, 0.0), (4.5, 4.0), 5.0, "0 + 5"),
    # x = (1/4, 1/4): sin(pi/2)^2 = 1 -> a0 = 1; cos(pi/2)^2 = 0 -> a1 = 2/3; (3, 4) -> 5; x.y = 9/4
    ("genradon", 2, 1.0, (0.25, 0.25), (3.0, 6.0), 7.25, "9/4 + 5"),
    # x = (1/12, 1/4): sin(pi/6) sin(pi/2) = 1/2 -> a0 = 5/6; cos(pi/6) cos(pi/2) = 0 -> a1 = 2/3;
    # (a0 y0, a1 y1) = (-5, 12) -> 13; x.y = -1/2 + 9/2 = 4
    ("genradon", 2, 1.0, (1.0 / 12, 0.25), (-6.0, 18.0), 17.0, "4 + 13"),
    # x = (1/4, 0): sin(pi/2) sin 0 = 0 -> a0 = 2/3; cos(pi/2) cos 0 = 0 -> a1 = 2/3;
    # (a0 y0, a1 y1) = (4, 3) -> 5; x.y = 3/2; scale 2
    ("genradon", 2, 2.0, (0.25, 0.0), (6.0, 4.5), 13.0, "2 (3/2 + 5)"),
    # d = 3, x = (1/4, 0, 0): a0 = (2 + sin(pi/2) cos 0)/3 = 1, a1 = (2 + sin 0 cos 0)/3 = 2/3,
    # a2 = (2 + sin 0 cos(pi/2))/3 = 2/3; (a_k y_k) = (2, 3, 6) -> 7; x.y = 1/2
    ("genradon", 3, 1.0, (0.25, 0.0, 0.0), (2.0, 4.5, 9.0), 7.5, "1/2 + 7"),
    # x = (0, 1/4, 1/4): a0 = (2 + 0)/3 = 2/3, a1 = (2 + sin(pi/2) cos(pi/2))/3 = 2/3,
    # a2 = (2 + sin(pi/2) cos 0)/3 = 1; (2, 3, 6) -> 7; x.y = 9/8 + 3/2 = 21/8
    ("genradon", 3, 1.0, (0.0, 0.25, 0.25), (3.0, 4.5, 6.0), 9.625, "21/8 + 7"),
    # x = (1/4, 1/6, 1/4): a0 = (2 + sin(pi/2) cos(pi/3))/3 = 5/6, a1 = (2 + sin(pi/3) cos(pi/2))/3 = 2/3,
    # a2 = (2 + sin(pi/2) cos(pi/2))/3 = 2/3; (a_k y_k) = (4, 4, 7) -> 9; x.y = 1.2 + 1 + 2.625
    ("genradon", 3, 1.0, (0.25, 1.0 / 6, 0.25), (4.8, 6.0, 10.5), 13.825, "4.825 + 9"),
    # Section 3.2 as printed, d = 3: gamma = 3 (2 + 1)/3 = 3, kappa = 6 (2 + 0)/3 = 4 -> 5;
    # x.y = 3/4 + 3/2 + 1 (the third coordinate enters x.y only)
    ("genradon_paper", 3, 1.0, (0.25, 0.25, 0.5), (3.0, 6.0, 2.0), 8.25, "13/4 + 5"),
    # hyperbolic: w = 1.5, h = 0.625, tau = 1.2, p = 0.8: tau^2 + p^2 h^2 = 1.44 + 0.25 = 1.69 -> 1.3
    ("hypradon", 2, 1.0, (1.5, 0.625), (1.2, 0.8), 1.95, "1.5 * 1.3"),
    # scale N = 512, w = 1, h = 0.75, tau = 1.6, p = 1.6: 2.56 + 1.44 = 4 -> 2
    ("hypradon", 2, 512.0, (1.0, 0.75), (1.6, 1.6), 1024.0, "512 * 1 * 2"),
    # separable: x_k + (k+1)/7 = 1/4 -> each sine is 1; y = (2, 3): 4/2 + 9/3 = 5
    ("separable", 2, 1.0, (0.25 - 1.0 / 7, 0.25 - 2.0 / 7), (2.0, 3.0), 7.0, "2 + 5"),
]


def failures():
    """The cases the current oracle build gets wrong, as (case, got) pairs."""
    bad = []
    for phase, d, s, x, y, want, why in CASES:
        P = oracle.Problem(d=d, L=2, q=2, phase=phase, scale=s)
        got = oracle.phi(P, x, y)
        if not abs(got - want) <= TOL * max(1.0, abs(want)):
            bad.append(((phase, d, s, x, y, want, why), got))
    return bad


def hold() -> bool:
    return not failures()
