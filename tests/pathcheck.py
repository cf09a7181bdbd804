"""Geometric checks of a traced geodesic path (shared by the oracle and GPU path tests).

A path is (kind, id, t0, t1) arrays, target first: kind 0 a vertex, 1 a point on
half-edge id (3 f + i runs from corner i to corner i + 1 of face f) at fraction t0 from
its start, 2 the face-point source in face id with barycentric weights t0, t1 of corners
1 and 2.  The checks use only the mesh and Section 3's characterisation of a geodesic
(straight inside a face and straight in the unfolding across an edge):

* it starts at the target and ends at a source (distance 0) or at the face-point source;
* consecutive points lie on a common face;
* its length equals the exact distance of the target, and the length that remains after
  each vertex on it equals that vertex's distance;
* at every edge crossing the incoming and outgoing segments make the same angle with the
  edge (the two faces unfolded into one plane, the path does not bend).
"""
import numpy as np


def point_xyz(vertices, faces, kind, pid, t0, t1):
    if kind == 0:
        return vertices[pid]
    if kind == 1:
        f, i = divmod(int(pid), 3)
        a, b = vertices[faces[f, i]], vertices[faces[f, (i + 1) % 3]]
        return a + t0 * (b - a)
    c = faces[int(pid)]
    return (1.0 - t0 - t1) * vertices[c[0]] + t0 * vertices[c[1]] + t1 * vertices[c[2]]


def path_xyz(vertices, faces, path):
    kinds, ids, t0, t1 = path
    return np.array([point_xyz(vertices, faces, k, i, a, b) for k, i, a, b in zip(kinds, ids, t0, t1)])


_MAPS = {}


def _maps(faces):
    """Vertex -> faces and edge -> faces of a face array (cached per array content)."""
    key = (faces.shape, hash(np.ascontiguousarray(faces).tobytes()))
    if key not in _MAPS:
        if len(_MAPS) > 16:
            _MAPS.clear()
        _MAPS[key] = (vertex_faces(faces), edge_faces(faces))
    return _MAPS[key]


def vertex_faces(faces):
    vf = {}
    for f, tri in enumerate(faces):
        for v in tri:
            vf.setdefault(int(v), set()).add(f)
    return vf


def edge_faces(faces):
    ef = {}
    for f, tri in enumerate(faces):
        for i in range(3):
            a, b = int(tri[i]), int(tri[(i + 1) % 3])
            ef.setdefault((min(a, b), max(a, b)), set()).add(f)
    return ef


def faces_of(faces, vf, ef, kind, pid, t0):
    if kind == 0:
        return vf.get(int(pid), set())
    if kind == 1:
        f, i = divmod(int(pid), 3)
        a, b = int(faces[f, i]), int(faces[f, (i + 1) % 3])
        s = set(ef[(min(a, b), max(a, b))])
        # a crossing at an end of the edge is that vertex
        if t0 <= 1e-12:
            s |= vf[a]
        if t0 >= 1 - 1e-12:
            s |= vf[b]
        return s
    return {int(pid)}


def check_path(vertices, faces, dist, target, path, sources=None, face_source=None, rel=1e-9,
               straight_tol=1e-7):
    """Assert that `path` is a geodesic from the source(s) to `target` of length
    dist[target].  Returns the path's 3D length."""
    kinds, ids, t0, t1 = path
    n = len(kinds)
    if not np.isfinite(dist[target]):
        assert n == 0, "an unreachable target has an empty path"
        return np.inf
    assert n >= 1
    assert kinds[0] == 0 and ids[0] == target, "the path starts at its target"
    if kinds[-1] == 0:
        assert dist[ids[-1]] == 0.0, "the path ends at a source"
        if sources is not None:
            assert int(ids[-1]) in set(int(s) for s in sources)
    else:
        assert kinds[-1] == 2 and face_source is not None
        f, bary = face_source
        assert ids[-1] == f
        assert abs(t0[-1] - bary[1]) < 1e-9 and abs(t1[-1] - bary[2]) < 1e-9
    assert np.all((kinds >= 0) & (kinds <= 2))
    assert np.all((t0 >= 0.0) & (t0 <= 1.0))
    p = path_xyz(vertices, faces, path)
    seg = np.linalg.norm(np.diff(p, axis=0), axis=1)
    length = float(seg.sum())
    scale = max(float(dist[target]), 1e-300)
    assert abs(length - dist[target]) <= rel * scale, (length, dist[target])
    # remaining length at every vertex on the path equals its distance
    rem = np.concatenate([np.cumsum(seg[::-1])[::-1], [0.0]])
    for j in range(n):
        if kinds[j] == 0:
            assert abs(rem[j] - dist[ids[j]]) <= rel * scale, (j, rem[j], dist[ids[j]])
    vf, ef = _maps(faces)
    for j in range(n - 1):
        a = faces_of(faces, vf, ef, kinds[j], ids[j], t0[j])
        b = faces_of(faces, vf, ef, kinds[j + 1], ids[j + 1], t0[j + 1])
        assert a & b, f"points {j} and {j + 1} share no face"
    # straightness across edges (skip zero-length neighbours)
    lmin = 1e-9 * scale
    for j in range(1, n - 1):
        if kinds[j] != 1 or seg[j - 1] < lmin or seg[j] < lmin:
            continue
        f, i = divmod(int(ids[j]), 3)
        u = vertices[faces[f, (i + 1) % 3]] - vertices[faces[f, i]]
        u = u / np.linalg.norm(u)
        c_in = float(np.dot(p[j] - p[j - 1], u)) / seg[j - 1]
        c_out = float(np.dot(p[j + 1] - p[j], u)) / seg[j]
        assert abs(c_in - c_out) <= straight_tol, (j, c_in, c_out)
    return length


def dedup_xyz(p, tol):
    """Drop consecutive points closer than tol (a crossing at a vertex repeats it)."""
    keep = [0]
    for j in range(1, len(p)):
        if np.linalg.norm(p[j] - p[keep[-1]]) > tol:
            keep.append(j)
    return p[keep]
