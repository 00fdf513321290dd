"""The oracle's pins must catch plausible mistakes.

Each case copies bf_oracle.c, plants one mistake (a dropped conjugate, a
transposed Lagrange factor, a wrong sign, a misplaced switch, a wrong child
box), compiles the copy and checks that at least one pin fails.  The real
oracle is never modified.
"""
import os
import subprocess

import numpy as np
import pytest

import oracle

SRC = os.path.join(os.path.dirname(oracle.__file__), "bf_oracle.c")

MUTATIONS = {
    "demod_not_conjugated": ("wo[t] += conj(kern(P, cac, pt)) * acc;", "wo[t] += kern(P, cac, pt) * acc;"),
    "lagrange_transposed": ("acc += lagtab(d, q, l1, t, tp) * u[tp];", "acc += lagtab(d, q, l1, tp, t) * u[tp];"),
    "row_premod_sign": ("u[t] = conj(kern(P, pt, cb)) * w[t];", "u[t] = kern(P, pt, cb) * w[t];"),
    "switch_one_level_late": ("if (l == m) { /* switch to row-space", "if (l == m + 1) { /* switch to row-space"),
    "row_uses_parent_box": ("lag1tab(d, q, z, ca, wa, cac, wac, l1);", "lag1tab(d, q, z, ca, wa, ca, wa, l1);"),
    "final_drops_modulation": ("f[j] = kern(P, x, y0) * acc;", "f[j] = acc;"),
    "init_wrong_node": ("W[B * r + t] = conj(kern(P, x0, yt)) * lag(d, q, z, cb, wb, t, y) * src;",
                        "W[B * r + t] = conj(kern(P, x0, y)) * lag(d, q, z, cb, wb, t, y) * src;"),
    # phase formulas (Sections 3.1, 3.2)
    "genradon2d_a1_sin_for_cos": ("double a1 = (2.0 + cos(TWO_PI * x[0]) * cos(TWO_PI * x[1])) / 3.0;",
                                  "double a1 = (2.0 + sin(TWO_PI * x[0]) * cos(TWO_PI * x[1])) / 3.0;"),
    "genradon3d_wrong_neighbour": ("cos(TWO_PI * x[(k + 1) % d])", "cos(TWO_PI * x[k % d])"),
    "genradon2d_a0_cos_for_sin": ("double a0 = (2.0 + sin(TWO_PI * x[0]) * sin(TWO_PI * x[1])) / 3.0;",
                                  "double a0 = (2.0 + sin(TWO_PI * x[0]) * cos(TWO_PI * x[1])) / 3.0;"),
    "genradon_drops_linear_term": ("        s = xy + sqrt(q2);", "        s = sqrt(q2);"),
    "hypradon_wrong_slowness": ("s = x[0] * sqrt(y[0] * y[0] + y[1] * y[1] * x[1] * x[1]);",
                                "s = x[0] * sqrt(y[0] * y[0] + y[1] * y[1] * x[0] * x[0]);"),
    "separable_wrong_shift": ("a += sin(TWO_PI * (x[k] + (k + 1) / 7.0));", "a += sin(TWO_PI * (x[k] + k / 7.0));"),
}


def _pins_pass(rng) -> bool:
    """The phase point values, and two whole-pipeline pins: exactness for a separable
    phase, DFT accuracy at q = 8."""
    import phase_pins
    ok = phase_pins.hold()
    P = oracle.Problem(d=2, L=4, q=3, phase="separable", tgt_off=0.25, src_off=0.3)
    g = rng.standard_normal(P.npts) + 1j * rng.standard_normal(P.npts)
    fb, fd = oracle.butterfly(P, g), oracle.direct_sum(P, g)
    ok &= np.linalg.norm(fb - fd) < 1e-12 * np.linalg.norm(fd)
    P = oracle.Problem(d=2, L=5, q=8, phase="dot")
    g = rng.standard_normal(P.npts) + 1j * rng.standard_normal(P.npts)
    fb, fd = oracle.butterfly(P, g), oracle.direct_sum(P, g)
    ok &= np.linalg.norm(fb - fd) < 1e-4 * np.linalg.norm(fd)
    return bool(ok)


@pytest.mark.parametrize("name", sorted(MUTATIONS))
def test_pins_catch_planted_mistake(name, tmp_path):
    old, new = MUTATIONS[name]
    src = open(SRC).read()
    assert src.count(old) >= 1, f"mutation anchor for {name} not found"
    mutated = tmp_path / "mut.c"
    mutated.write_text(src.replace(old, new, 1))
    so = tmp_path / "libmut.so"
    subprocess.run(["gcc", "-std=gnu99", "-O1", "-fPIC", "-shared", "-fopenmp", str(mutated), "-o", str(so), "-lm"],
                   check=True)
    try:
        oracle.use_library(str(so))
        assert not _pins_pass(np.random.default_rng(7)), f"pins did not catch: {name}"
    finally:
        oracle.use_library(None)


def test_unmutated_oracle_passes_the_same_pins():
    assert _pins_pass(np.random.default_rng(7))
