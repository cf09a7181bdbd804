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


# ------------------------------------------------------------------ full-size fixtures
FULL = ["terrain512_centre", "torus1250x400_src0"]


@pytest.mark.parametrize("name", FULL)
def test_full_field_fixture(oracle_lib, name):
    """The stored full fields of the full-size terrain and torus (written by
    make_fullfield.py from the oracle): they belong to the generator's current mesh, have
    the properties of an exact geodesic field on every vertex and edge, and the oracle
    reproduces them on the vertices nearest the source (an early-stopped run)."""
    import make_fullfield as mf
    from paper_1305_1293_gb300 import meshgen as mg
    assert os.path.exists(mf.path_of(name)), f"{name}.npz missing: run tests/golden/make_fullfield.py"
    d, s, fsha, probe, wl = mf.load(name)
    m = mg.workload(wl, "full")[0][0]
    assert mf.same_mesh(m, fsha, probe)
    v, f = m.vertices, m.faces
    assert d.shape == (m.nv,) and d[s] == 0.0 and np.all(np.isfinite(d))
    q = 2.0 ** -37                       # relative rounding of the stored values
    chord = np.linalg.norm(v - v[s], axis=1)
    assert np.all(d >= chord * (1 - 1e-12 - q))
    e = np.concatenate([f[:, [0, 1]], f[:, [1, 2]], f[:, [2, 0]]])
    le = np.linalg.norm(v[e[:, 0]] - v[e[:, 1]], axis=1)
    # each end carries its own rounding: up to 2 q of the larger distance on the difference
    assert np.all(np.abs(d[e[:, 0]] - d[e[:, 1]]) <= le * (1 + 1e-12) + 2 * q * np.maximum(d[e[:, 0]], d[e[:, 1]]))
    from scipy.sparse import coo_matrix
    from scipy.sparse.csgraph import dijkstra as sp_dijkstra
    g = coo_matrix((le, (e[:, 0], e[:, 1])), shape=(m.nv, m.nv)).tocsr()
    assert np.all(d <= sp_dijkstra(g, directed=False, indices=s) * (1 + 1e-12 + q))
    near = np.argsort(chord)[:3000].astype(np.int32)
    ref, _ = oracle_lib.geodesic(v, f, s, targets=near)
    r = np.abs(d[near] - ref[near]) / np.maximum(ref[near], 1e-300)
    assert float(r.max()) <= 1e-11
