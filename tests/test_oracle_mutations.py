"""The oracle's pins must catch plausible mistakes (no GPU).

Each case copies ``oracle/ich_oracle.cpp``, plants one mistake by a text substitution,
compiles the copy into a temporary directory and checks that at least one pin (brute
force, closed form, filter-off agreement) rejects it.  The committed oracle is untouched.
"""
import ctypes
import functools
import os
import subprocess
import tempfile

import numpy as np
import pytest

import bruteforce as bf
import oracle
from paper_1305_1293_gb300 import meshgen as mg

SRC = os.path.join(os.path.dirname(oracle.__file__), "ich_oracle.cpp")

MUTATIONS = {
    "loser_keeps_wrong_child": (
        "if (xs < aX[h] - tol) left = true;\n                else if (xs > aX[h] + tol) right = true;",
        "if (xs < aX[h] - tol) right = true;\n                else if (xs > aX[h] + tol) left = true;"),
    "third_test_either_end": ("dominated(d + IA, g[third] + dA_third) && dominated",
                              "dominated(d + IA, g[third] + dA_third) || dominated"),
    "no_pseudo_sources": ("m.pseudo[v] = boundary[v] || theta[v] > kTwoPi - 1e-9;", "m.pseudo[v] = 0;"),
    "no_boundary_pseudo_sources": ("m.pseudo[v] = boundary[v] || theta[v] > kTwoPi - 1e-9;",
                                   "m.pseudo[v] = theta[v] > kTwoPi - 1e-9;"),
    "child_d0_d1_swapped": ("Window{w.d, ta, tb, Iv2, w.d1, c}", "Window{w.d, ta, tb, w.d1, Iv2, c}"),
    "endpoint_test_wrong_end": ("dominated(w.d + IB, g[v0] + w.B)", "dominated(w.d + IA, g[v0] + w.A)"),
    "occupancy_sign": ("double xs = px + (xc - px) * (-py) / (yc - py);",
                       "double xs = px + (xc - px) * (py) / (yc - py);"),
    "dropped_v2_event": ("            vertex_event(v2, D2, w, work);\n", "\n"),
    "pseudo_source_above_edge": ("    py = -std::sqrt(t > 0 ? t : 0.0);", "    py = std::sqrt(t > 0 ? t : 0.0);"),
    "apex_frame_swapped": ("    xc = ((a - b) * (a + b) + L * L) / (2 * L);", "    xc = ((b - a) * (b + a) + L * L) / (2 * L);"),
    "dominance_without_margin_sign": ("return lhs > rhs * (1.0 + kDomRel);", "return lhs * (1.0 + 1e-3) > rhs;"),
    "no_fan_at_v0_event": ("if (w.A <= tol) vertex_event(v0, w.d + w.d0, w, work);", "if (w.A <= tol) {}"),
}

TINY = [mg.octahedron(0.1, 2, 1), mg.torus(6, 4, seed=6), mg.terrain(5, 4, seed=9, amp_range=(1.0, 3.0)),
        mg.cube(2), mg.geodesic_sphere(2, 0.05, 3)]


@functools.lru_cache(maxsize=None)
def _brute(i, s):
    m = TINY[i]
    return bf.geodesic(m.vertices, m.faces, s)


def _compile(tmp, name, old, new):
    text = open(SRC).read()
    assert old in text, name
    path = os.path.join(tmp, f"mut_{name}.cpp")
    with open(path, "w") as fh:
        fh.write(text.replace(old, new, 1))
    so = os.path.join(tmp, f"mut_{name}.so")
    subprocess.check_call(["g++", "-O1", "-std=c++17", "-shared", "-fPIC", "-o", so, path])
    return oracle.load_library(so)


def _pins_fail(lib):
    """True as soon as one pin rejects the (mutated) oracle."""
    def run(m, s, **kw):
        try:
            return oracle.geodesic(m.vertices, m.faces, s, lib=lib, max_windows=3_000_000, **kw)[0]
        except oracle.OracleError:
            return None
    for i, m in enumerate(TINY):
        for s in range(0, m.nv, max(1, m.nv // 3)):
            d = run(m, s)
            if d is None or not np.allclose(d, _brute(i, s), rtol=1e-9, atol=1e-12):
                return True
    flat = mg.flat_patch(9, jitter=0.3, seed=2)
    d = run(flat, 40)
    if d is None or not np.allclose(d, np.linalg.norm(flat.vertices - flat.vertices[40], axis=1), rtol=1e-9):
        return True
    m = mg.icosphere(3, 0.02, seed=7)
    a, b = run(m, 5), run(m, 5, flags=oracle.NO_CH | oracle.ORDER_FIFO)
    if a is None or b is None or not np.allclose(a, b, rtol=1e-9):
        return True
    return False


def test_unmutated_oracle_passes_the_same_pins():
    assert not _pins_fail(oracle._load())


@pytest.mark.parametrize("name", sorted(MUTATIONS))
def test_pins_catch_planted_mistake(name):
    old, new = MUTATIONS[name]
    with tempfile.TemporaryDirectory() as tmp:
        lib = _compile(tmp, name, old, new)
        assert _pins_fail(lib), f"planted mistake '{name}' passed every pin"
