"""Pins of the oracle's geodesic paths (no GPU).

The oracle traces a path back along the window sequence that gave the target its
distance (Section 4.4) as straight unfolded segments between pseudo-sources (Section 3).
Pinned here by what fixes a geodesic independently of that code:

* on a convex plane patch the path is the straight chord from the source, and on a
  prism tube unrolled onto its periodic strip a straight segment of the closed-form
  length;
* on brute-force meshes (exhaustive unfolding, tests/bruteforce.py) its length is the
  brute-force distance;
* on every mesh it passes the geometric checks of tests/pathcheck.py (starts at the
  target, ends at a source, consecutive points on a common face, no bend across an edge,
  length = the target's distance, the remainder after each vertex = that vertex's
  distance);
* multi-source paths end at a nearest source, a face-point source's paths end at the
  point, an unreachable target has no path;
* planted mistakes in the tracer (a copy of the oracle) are caught by these checks.
"""
import os
import subprocess
import tempfile

import numpy as np
import pytest

import bruteforce as bf
import oracle
import pathcheck as pc
from paper_1305_1293_gb300 import meshgen as mg


def _line_dev(p, a, b):
    u = (b - a) / np.linalg.norm(b - a)
    r = p - a
    return np.linalg.norm(r - np.outer(r @ u, u), axis=1)


@pytest.mark.parametrize("n,seed,src", [(8, 1, 0), (10, 2, 40), (12, 3, 84)])
def test_plane_paths_are_chords(oracle_lib, n, seed, src):
    m = mg.flat_patch(n, jitter=0.3, seed=seed)
    tg = np.arange(m.nv)
    d, paths = oracle_lib.trace_paths(m.vertices, m.faces, src, targets=tg)
    for t, p in zip(tg, paths):
        pc.check_path(m.vertices, m.faces, d, t, p, sources=[src])
        if t == src:
            assert len(p[0]) == 1
            continue
        xyz = pc.path_xyz(m.vertices, m.faces, p)
        assert np.max(_line_dev(xyz, m.vertices[src], m.vertices[t])) < 1e-12
        # the points run monotonically from the target to the source
        s = (xyz - m.vertices[t]) @ (m.vertices[src] - m.vertices[t])
        assert np.all(np.diff(s) >= -1e-12)


def test_plane_face_point_paths(oracle_lib):
    m = mg.flat_patch(8, jitter=0.25, seed=11)
    face, bary = 40, np.array([0.2, 0.3, 0.5])
    p0 = sum(b * m.vertices[m.faces[face, k]] for k, b in enumerate(bary))
    tg = np.arange(m.nv)
    d, paths = oracle_lib.trace_paths(m.vertices, m.faces, face=face, bary=bary, targets=tg)
    for t, p in zip(tg, paths):
        pc.check_path(m.vertices, m.faces, d, t, p, face_source=(face, bary))
        xyz = pc.path_xyz(m.vertices, m.faces, p)
        assert np.linalg.norm(xyz[-1] - p0) < 1e-12
        assert np.max(_line_dev(xyz, p0, m.vertices[t])) < 1e-12


def _prism_unroll(m, sides, perim, xyz):
    """Unrolled (s, z) of points on a prism tube's lateral surface, continuous along the
    sequence (a jump across the seam adds or removes the perimeter)."""
    c = m.vertices[:sides, :2]
    nxt = np.roll(c, -1, axis=0)
    seg = np.linalg.norm(nxt - c, axis=1)
    s0 = np.concatenate([[0.0], np.cumsum(seg)[:-1]])
    out, prev = [], None
    for p in xyz:
        best = None
        for k in range(sides):
            u = (nxt[k] - c[k]) / seg[k]
            r = p[:2] - c[k]
            along = float(r @ u)
            off = abs(float(r[0] * u[1] - r[1] * u[0]))
            if -1e-12 <= along <= seg[k] + 1e-12 and (best is None or off < best[0]):
                best = (off, s0[k] + along)
        assert best is not None and best[0] < 1e-9
        sv = best[1]
        if prev is not None:
            sv += perim * round((prev - sv) / perim)
        out.append((sv, p[2]))
        prev = sv
    return np.array(out)


@pytest.mark.parametrize("sides,rings,seed,src", [(7, 4, 0, 0), (11, 6, 1, 30), (5, 9, 2, 24)])
def test_prism_paths_are_straight_unrolled(oracle_lib, sides, rings, seed, src):
    """Unrolled onto the periodic strip, every path is one straight segment whose length
    is the closed-form distance (the wrap-around copy of the source it ends at)."""
    m, s, z, perim = mg.prism_tube(sides, rings, height=1.5, seed=seed)
    tg = np.arange(m.nv)
    d, paths = oracle_lib.trace_paths(m.vertices, m.faces, src, targets=tg)
    ds, dz = s - s[src], z - z[src]
    ex = np.min([np.hypot(ds + k * perim, dz) for k in (-1, 0, 1)], axis=0)
    for t, p in zip(tg, paths):
        pc.check_path(m.vertices, m.faces, d, t, p, sources=[src])
        if t == src:
            continue
        uv = _prism_unroll(m, sides, perim, pc.path_xyz(m.vertices, m.faces, p))
        a, b = uv[0], uv[-1]
        assert abs(np.linalg.norm(b - a) - ex[t]) <= 1e-12 * max(ex[t], 1.0)
        # crossing points within 1e-10 of the segment: the oracle's (d0, d1) windows give the
        # pseudo-source's height through d0^2 - px^2, which loses digits when the source is
        # far from a short edge (a wrong crossing would be off by a face's size)
        u = (b - a) / np.linalg.norm(b - a)
        dev = np.abs((uv - a) @ np.array([-u[1], u[0]]))
        assert np.max(dev) <= 1e-10 * max(ex[t], 1.0), (t, np.max(dev))


TINY = [
    ("octa1", lambda: mg.octahedron(0.1, 2, 1)),
    ("terrain5x4", lambda: mg.terrain(5, 4, seed=9, amp_range=(1.0, 3.0))),
    ("torus6x4", lambda: mg.torus(6, 4, seed=6)),
    ("cube2", lambda: mg.cube(2)),
    ("pyramid", lambda: mg.pyramid(5, 2)[0]),
    ("geosphere2", lambda: mg.geodesic_sphere(2, 0.05, 3)),
]


@pytest.mark.parametrize("name,make", TINY, ids=[t[0] for t in TINY])
def test_path_lengths_match_bruteforce(oracle_lib, name, make):
    m = make()
    tg = np.arange(m.nv)
    for s in range(0, m.nv, max(1, m.nv // 3)):
        b = bf.geodesic(m.vertices, m.faces, s)
        d, paths = oracle_lib.trace_paths(m.vertices, m.faces, s, targets=tg)
        for t, p in zip(tg, paths):
            length = pc.check_path(m.vertices, m.faces, d, t, p, sources=[s])
            assert abs(length - b[t]) <= 1e-12 * max(b[t], 1.0), (name, s, t)


SMALL = [
    ("icosphere3", lambda: mg.icosphere(3, 0.02, seed=7), 0),
    ("terrain24", lambda: mg.terrain(24, 24, seed=8), 300),
    ("torus40x14", lambda: mg.torus(40, 14, seed=9), 11),
    ("octsphere3", lambda: mg.multi_octave_sphere(3, 0.05, seed=11), 5),
    ("cube6", lambda: mg.cube(6), 0),
]


@pytest.mark.parametrize("name,make,src", SMALL, ids=[t[0] for t in SMALL])
def test_paths_valid_everywhere(oracle_lib, name, make, src):
    m = make()
    tg = np.arange(m.nv)
    d, paths = oracle_lib.trace_paths(m.vertices, m.faces, src, targets=tg)
    ref, _ = oracle_lib.geodesic(m.vertices, m.faces, src)
    assert np.array_equal(d, ref)
    for t, p in zip(tg, paths):
        assert p is not None, (name, t)
        pc.check_path(m.vertices, m.faces, d, t, p, sources=[src])


def test_multi_source_paths_end_at_nearest(oracle_lib):
    m = mg.icosphere(3, 0.02, seed=7)
    srcs = [0, 77, 300, 501]
    tg = np.arange(m.nv)
    d, paths = oracle_lib.trace_paths(m.vertices, m.faces, sources=srcs, targets=tg)
    single = np.stack([oracle_lib.geodesic(m.vertices, m.faces, s)[0] for s in srcs])
    for t, p in zip(tg, paths):
        pc.check_path(m.vertices, m.faces, d, t, p, sources=srcs)
        end = srcs.index(int(p[1][-1]))
        assert abs(single[end, t] - d[t]) <= 1e-12 * max(d[t], 1.0)


def test_unreachable_target_has_no_path(oracle_lib):
    a = mg.icosphere(1, 0.0, seed=0)
    v = np.concatenate([a.vertices, a.vertices + 5.0])
    f = np.concatenate([a.faces, a.faces + a.nv]).astype(np.int32)
    d, paths = oracle_lib.trace_paths(v, f, 0, targets=[3, a.nv + 3])
    assert np.isfinite(d[3]) and np.isinf(d[a.nv + 3])
    assert len(paths[0][0]) >= 2 and len(paths[1][0]) == 0


SRC = os.path.join(os.path.dirname(oracle.__file__), "ich_oracle.cpp")
TRACE_MUTATIONS = {
    "child_side_swapped": ("if (w->e == m.twin[prv(hp)]) {", "if (w->e == m.twin[nxt(hp)]) {"),
    "crossing_sign": ("x = std::min(std::max(ppx + (qx - ppx) * (-ppy) / (qy - ppy), 0.0), Lp);",
                      "x = std::min(std::max(ppx + (qx - ppx) * (ppy) / (qy - ppy), 0.0), Lp);"),
    "right_child_from_v0": ("qx = xc + f * (Lp - xc);", "qx = f * (Lp - xc);"),
    "v2_crossing_skipped": ("out.push_back(Pt{1, h, x / L, 0.0});", "(void)0;"),
    "fan_edge_event_skips_vertex": ("                v = ev.src;\n                out.push_back(Pt{0, v, 0.0, 0.0});\n"
                                    "                continue;",
                                    "                v = ev.src;\n                continue;"),
    "edge_fraction_from_end": ("out.push_back(Pt{1, hp, x / Lp, 0.0});", "out.push_back(Pt{1, hp, 1.0 - x / Lp, 0.0});"),
}


def _path_pins_fail(lib):
    cases = [(mg.flat_patch(8, jitter=0.3, seed=1), 0), (mg.torus(6, 4, seed=6), 0),
             (mg.terrain(6, 5, seed=3, amp_range=(1.0, 3.0)), 0), (mg.icosphere(2, 0.02, seed=1), 0)]
    for m, s in cases:
        tg = np.arange(m.nv)
        try:
            d, paths = oracle.trace_paths(m.vertices, m.faces, s, targets=tg, lib=lib)
        except oracle.OracleError:
            return True
        for t, p in zip(tg, paths):
            if p is None:
                return True
            try:
                pc.check_path(m.vertices, m.faces, d, t, p, sources=[s])
            except (AssertionError, IndexError, KeyError):
                return True
    return False


def test_unmutated_tracer_passes_path_pins():
    assert not _path_pins_fail(oracle._load())


@pytest.mark.parametrize("name", sorted(TRACE_MUTATIONS))
def test_path_pins_catch_planted_mistake(name):
    old, new = TRACE_MUTATIONS[name]
    text = open(SRC).read()
    assert old in text, name
    with tempfile.TemporaryDirectory() as tmp:
        path = os.path.join(tmp, f"mut_{name}.cpp")
        with open(path, "w") as fh:
            fh.write(text.replace(old, new, 1))
        so = os.path.join(tmp, f"mut_{name}.so")
        subprocess.check_call(["g++", "-O1", "-std=c++17", "-shared", "-fPIC", "-o", so, path])
        lib = oracle.load_library(so)
        assert _path_pins_fail(lib), f"planted mistake '{name}' passed every path pin"
