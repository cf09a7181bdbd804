"""Golden fixtures: small meshes with their stored exact geodesic fields.

The fields were written by ``tests/golden/make_golden.py``, which calls only the CPU
oracle.  The CPU tests keep the oracle from drifting away from the stored fields and
check each stored field against properties every exact polyhedral geodesic distance
has (zero at the source, at least the straight-line distance, 1-Lipschitz along edges,
at most the shortest path along edges); the GPU test compares the library with the
stored fields at the parity bar (max relative error 1e-9)."""
import glob
import heapq
import os

import numpy as np
import pytest

HERE = os.path.dirname(os.path.abspath(__file__))
FIXTURES = sorted(glob.glob(os.path.join(HERE, "golden", "*.txt")))
REL = 1e-12  # oracle rebuilt with another compiler / fma contraction: rounding order only


def read_fixture(path):
    with open(path) as f:
        lines = [l for l in f.read().splitlines() if l and not l.startswith("#")]
    nv, nf, s = (int(x) for x in lines[0].split())
    v = np.array([[float(x) for x in l.split()] for l in lines[1:1 + nv]])
    t = np.array([[int(x) for x in l.split()] for l in lines[1 + nv:1 + nv + nf]], dtype=np.int32)
    d = np.array([float(l) for l in lines[1 + nv + nf:1 + 2 * nv + nf]])
    assert v.shape == (nv, 3) and t.shape == (nf, 3) and d.shape == (nv,)
    return v, t, s, d


def edge_graph(v, t):
    adj = [dict() for _ in range(len(v))]
    for tri in t:
        for a, b in ((tri[0], tri[1]), (tri[1], tri[2]), (tri[2], tri[0])):
            w = float(np.linalg.norm(v[a] - v[b]))
            adj[a][b] = w
            adj[b][a] = w
    return adj


def dijkstra(adj, s):
    d = np.full(len(adj), np.inf)
    d[s] = 0.0
    pq = [(0.0, s)]
    while pq:
        du, u = heapq.heappop(pq)
        if du > d[u]:
            continue
        for w, l in adj[u].items():
            if du + l < d[w]:
                d[w] = du + l
                heapq.heappush(pq, (d[w], w))
    return d


def test_fixtures_present():
    assert len(FIXTURES) >= 4


@pytest.mark.parametrize("path", FIXTURES, ids=lambda p: os.path.basename(p)[:-4])
def test_golden_field_properties(path):
    v, t, s, d = read_fixture(path)
    assert d[s] == 0.0 and np.all(np.isfinite(d))
    chord = np.linalg.norm(v - v[s], axis=1)
    assert np.all(d >= chord * (1 - 1e-12))
    adj = edge_graph(v, t)
    for a in range(len(v)):
        for b, l in adj[a].items():
            assert abs(d[a] - d[b]) <= l * (1 + 1e-12)
    assert np.all(d <= dijkstra(adj, s) * (1 + 1e-12))


@pytest.mark.parametrize("path", FIXTURES, ids=lambda p: os.path.basename(p)[:-4])
def test_oracle_reproduces_golden(oracle_lib, path):
    v, t, s, d = read_fixture(path)
    got, _ = oracle_lib.geodesic(v, t, s)
    r = np.abs(got - d) / np.maximum(d, 1e-300)
    r[s] = abs(got[s])
    assert float(r.max()) <= REL


@pytest.mark.gpu
@pytest.mark.parametrize("path", FIXTURES, ids=lambda p: os.path.basename(p)[:-4])
def test_library_matches_golden(path):
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("needs a GPU")
    import __graft_entry__
    __graft_entry__.build()
    from paper_1305_1293_gb300 import pch
    v, t, s, d = read_fixture(path)
    mesh = pch.Mesh(v, t)
    try:
        got = pch.solve(mesh, s)
    finally:
        mesh.close()
    assert got[s] == 0.0
    fin = np.isfinite(d)
    assert np.array_equal(np.isfinite(got), fin)
    assert float(np.max(np.abs(got - d) / np.maximum(d, 1e-300))) <= 1e-9
