"""Pins of the CPU oracle against brute-force unfolding and against invariants (no GPU).

* brute force: Dijkstra over exhaustive straight-line visibility (tests/bruteforce.py),
  on meshes of at most ~80 faces;
* invariants that any exact distance field obeys: chord <= g <= edge-graph distance,
  1-Lipschitz along every edge, g(source) = 0, symmetry g_s(t) = g_t(s);
* order invariance (the paper's correctness argument, Section 4.3 and Remark 2): the
  priority queue, FIFO order and a random order give the same distances;
* filter soundness (Section 4.3: the filters remove only useless windows): switching the
  "one angle one split" rule off does not change the distances;
* multi-source (Section 4.2, source set S): the field equals the minimum of the
  single-source fields.
"""
import numpy as np
import pytest

import bruteforce as bf
from paper_1305_1293_gb300 import meshgen as mg

TINY = [
    ("octa", lambda: mg.octahedron(0.15, 1, 0)),
    ("octa1", lambda: mg.octahedron(0.1, 2, 1)),
    ("ico0", lambda: mg.icosphere(0, 0.1, 3)),
    ("terrain3x3", lambda: mg.terrain(3, 3, seed=4, amp_range=(0.2, 0.8))),
    ("terrain5x4", lambda: mg.terrain(5, 4, seed=9, amp_range=(1.0, 3.0))),
    ("torus6x4", lambda: mg.torus(6, 4, seed=6)),
    ("cube2", lambda: mg.cube(2)),
    ("tetra2", lambda: mg.tetrahedron(2)),
    ("pyramid", lambda: mg.pyramid(5, 2)[0]),
    ("prism", lambda: mg.prism_tube(5, 2)[0]),
    ("geosphere2", lambda: mg.geodesic_sphere(2, 0.05, 3)),
]


def _rel(a, b):
    return np.max(np.abs(a - b) / np.maximum(np.abs(b), 1e-300))


@pytest.mark.parametrize("name,make", TINY, ids=[t[0] for t in TINY])
def test_oracle_matches_bruteforce(oracle_lib, name, make):
    m = make()
    assert m.nf <= 80
    for s in range(0, m.nv, max(1, m.nv // 3)):
        b = bf.geodesic(m.vertices, m.faces, s)
        o, _ = oracle_lib.geodesic(m.vertices, m.faces, s)
        assert _rel(o, b) < 1e-12, (name, s)


SMALL = [
    ("icosphere3", lambda: mg.icosphere(3, 0.02, seed=7)),
    ("terrain24", lambda: mg.terrain(24, 24, seed=8)),
    ("torus40x14", lambda: mg.torus(40, 14, seed=9)),
    ("geosphere6", lambda: mg.geodesic_sphere(6, 0.02, seed=10)),
    ("octsphere3", lambda: mg.multi_octave_sphere(3, 0.05, seed=11)),
]


def _edges(m):
    f = m.faces
    e = np.concatenate([f[:, [0, 1]], f[:, [1, 2]], f[:, [2, 0]]])
    return e


@pytest.mark.parametrize("name,make", SMALL, ids=[t[0] for t in SMALL])
def test_invariants(oracle_lib, name, make):
    m = make()
    src = m.nv // 3
    d, _ = oracle_lib.geodesic(m.vertices, m.faces, src)
    assert d[src] == 0.0
    assert np.all(np.isfinite(d)) and np.all(d >= 0)
    chord = np.linalg.norm(m.vertices - m.vertices[src], axis=1)
    assert np.all(d >= chord * (1 - 1e-12))
    up = bf.edge_graph_dijkstra(m.vertices, m.faces, src)
    assert np.all(d <= up * (1 + 1e-12))
    e = _edges(m)
    le = np.linalg.norm(m.vertices[e[:, 0]] - m.vertices[e[:, 1]], axis=1)
    assert np.all(np.abs(d[e[:, 0]] - d[e[:, 1]]) <= le * (1 + 1e-12) + 1e-14)
    # symmetry of the metric
    for t in (0, m.nv // 2, m.nv - 1):
        dt, _ = oracle_lib.geodesic(m.vertices, m.faces, t)
        assert abs(dt[src] - d[t]) <= 1e-12 * max(d[t], 1e-300)


@pytest.mark.parametrize("name,make", SMALL[:3], ids=[t[0] for t in SMALL[:3]])
def test_order_invariance_and_filter_soundness(oracle_lib, name, make):
    m = make()
    src = 5
    ref, st = oracle_lib.geodesic(m.vertices, m.faces, src)
    for fl in (oracle_lib.ORDER_FIFO, oracle_lib.ORDER_RANDOM, oracle_lib.NO_CH,
               oracle_lib.NO_CH | oracle_lib.ORDER_FIFO):
        d, st2 = oracle_lib.geodesic(m.vertices, m.faces, src, flags=fl)
        assert _rel(d, ref) < 1e-12, fl
    # the priority queue is the ordering that keeps the window count down (Section 5.2)
    _, fifo = oracle_lib.geodesic(m.vertices, m.faces, src, flags=oracle_lib.ORDER_FIFO)
    assert st["created"] <= fifo["created"]


@pytest.mark.parametrize("name,make", SMALL[:3], ids=[t[0] for t in SMALL[:3]])
def test_cpu_pch_rounds_exact(oracle_lib, name, make):
    """Section 6's CPU PCH (rounds of the k nearest windows, quickselect, no order inside
    a round) gives the same field as the priority queue (Remark 2); with k = 1 a round is
    exactly one priority-queue pop, so it creates exactly the same windows; larger rounds
    cost extra windows."""
    m = make()
    src = 5
    ref, st = oracle_lib.geodesic(m.vertices, m.faces, src)
    d1, s1 = oracle_lib.cpu_pch(m.vertices, m.faces, src, 1)
    assert np.array_equal(d1, ref)
    assert s1["created"] == st["created"] and s1["rounds"] == s1["created"]
    for k in (7, 64, 1024):
        d, sk = oracle_lib.cpu_pch(m.vertices, m.faces, src, k)
        assert _rel(d, ref) < 1e-12, k
        assert sk["created"] >= st["created"] and sk["rounds"] < s1["rounds"]


def test_ich_filter_off_tiny(oracle_lib):
    """With the Xin-Wang filter off (CH rule only) the distances are unchanged."""
    for name, make in TINY[:5]:
        m = make()
        ref, st = oracle_lib.geodesic(m.vertices, m.faces, 0)
        d, st2 = oracle_lib.geodesic(m.vertices, m.faces, 0, flags=oracle_lib.NO_ICH, max_windows=2_000_000)
        assert _rel(d, ref) < 1e-12, name
        assert st2["created"] >= st["created"]


def test_multi_source_is_min(oracle_lib):
    m = mg.icosphere(3, 0.02, seed=12)
    srcs = [3, 200, 511]
    d, _ = oracle_lib.geodesic(m.vertices, m.faces, sources=srcs)
    single = np.min([oracle_lib.geodesic(m.vertices, m.faces, s)[0] for s in srcs], axis=0)
    assert _rel(d, single) < 1e-12


def test_early_stop_targets_final(oracle_lib):
    """Keys never decrease (a child is farther than its parent), so once the smallest
    pending key passes g(t), g(t) is final: the early-stopped values equal the full run."""
    m = mg.terrain(32, 32, seed=13)
    src = mg.terrain_center(32, 32)
    full, st = oracle_lib.geodesic(m.vertices, m.faces, src)
    near = np.argsort(full)[1:40]
    part, st2 = oracle_lib.geodesic(m.vertices, m.faces, src, targets=near)
    assert np.array_equal(part[near], full[near])
    assert st2["propagated"] < st["propagated"]


def test_angle_sums_classify(oracle_lib):
    """Total angle (Section 3): 2 pi on a flat interior vertex, < 2 pi at a cube corner."""
    m = mg.flat_patch(5, jitter=0.2, seed=3)
    th, ps = oracle_lib.vertex_angles(m.vertices, m.faces)
    i = np.arange(m.nv)
    inner = (i % 6 > 0) & (i % 6 < 5) & (i // 6 > 0) & (i // 6 < 5)
    assert np.allclose(th[inner], 2 * np.pi, atol=1e-12)
    c = mg.cube(2)
    th, ps = oracle_lib.vertex_angles(c.vertices, c.faces)
    corner = np.all((c.vertices == 0) | (c.vertices == 1), axis=1)
    assert np.allclose(th[corner], 1.5 * np.pi, atol=1e-12)
    assert not ps[corner].any()
