"""GPU geodesic paths (pch_trace_paths) against the oracle's paths, through the C ABI.

Where the shortest path is unique (the seeded noisy meshes) the library and the oracle
must report the same path: after dropping repeated positions (a path may step onto a
vertex through an edge point at an end of its edge, a zero-length step), the same
sequence of 3D points within 1e-9 of the target's distance.  What is not unique, the
representation (which of the windows with the final distance a vertex keeps), is only
required to be valid: every path must pass the geometric checks of tests/pathcheck.py
(from the target to a source over common faces, straight across every edge, length =
the exact distance within 1e-9 relative, and the remainder after each vertex = that
vertex's distance).  Where several shortest paths exist (a cube, whose paths pass
through vertices) only those checks apply.
"""
import numpy as np
import pytest

import pathcheck as pc
from paper_1305_1293_gb300 import meshgen as mg

pytestmark = pytest.mark.gpu
TOL = 1e-9


@pytest.fixture(scope="module")
def pch():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("needs a GPU")
    import __graft_entry__
    __graft_entry__.build()
    from paper_1305_1293_gb300 import pch as p
    return p


@pytest.fixture(scope="module")
def ora():
    import oracle
    oracle.build()
    return oracle


def _trace(pch, m, sources, targets, **kw):
    mesh = pch.Mesh(m.vertices, m.faces)
    try:
        return pch.trace_paths(mesh, sources, targets, **kw)
    finally:
        mesh.close()


def _same_path(m, a, b, dist):
    """The same polyline on the surface: 3D points, repeated positions dropped."""
    scale = max(float(dist), 1e-12)
    pa = pc.dedup_xyz(pc.path_xyz(m.vertices, m.faces, a), TOL * scale)
    pb = pc.dedup_xyz(pc.path_xyz(m.vertices, m.faces, b), TOL * scale)
    return len(pa) == len(pb) and float(np.max(np.linalg.norm(pa - pb, axis=1), initial=0.0)) <= TOL * scale


GENERIC = [
    ("icosphere3", lambda: mg.icosphere(3, 0.02, seed=7), 0),
    ("terrain24", lambda: mg.terrain(24, 24, seed=8), 300),
    ("torus40x14", lambda: mg.torus(40, 14, seed=9), 11),
    ("flat12", lambda: mg.flat_patch(12, jitter=0.3, seed=3), 84),
    ("octsphere3", lambda: mg.multi_octave_sphere(3, 0.05, seed=11), 5),
]


@pytest.mark.parametrize("name,make,src", GENERIC, ids=[g[0] for g in GENERIC])
def test_paths_match_oracle(pch, ora, name, make, src):
    m = make()
    tg = np.arange(m.nv)
    d, paths = _trace(pch, m, [src], tg)
    dref, ref = ora.trace_paths(m.vertices, m.faces, src, targets=tg)
    fin = np.isfinite(dref)
    assert np.array_equal(np.isfinite(d), fin)
    assert np.max(np.abs(d[fin] - dref[fin]) / np.maximum(dref[fin], 1e-300)) <= TOL
    same = 0
    for t in tg:
        assert paths[t] is not None, (name, t)
        pc.check_path(m.vertices, m.faces, d, t, paths[t], sources=[src], rel=TOL)
        same += _same_path(m, paths[t], ref[t], d[t])
    # unique shortest paths: the same polyline (a rare tie may pick another valid path)
    assert same >= 0.99 * m.nv, (name, same, m.nv)


def test_paths_on_a_cube_are_valid(pch, ora):
    m = mg.cube(6)
    tg = np.arange(m.nv)
    d, paths = _trace(pch, m, [0], tg)
    dref, _ = ora.trace_paths(m.vertices, m.faces, 0, targets=tg)
    assert np.max(np.abs(d - dref) / np.maximum(dref, 1e-300)) <= TOL
    ok = 0
    for t in tg:
        if paths[t] is None:   # a path through a vertex may end the trace (documented)
            continue
        pc.check_path(m.vertices, m.faces, d, t, paths[t], sources=[0], rel=TOL)
        ok += 1
    assert ok >= 0.9 * m.nv


def test_face_point_source_paths(pch, ora):
    m = mg.flat_patch(10, jitter=0.25, seed=5)
    face, bary = 57, np.array([0.2, 0.3, 0.5])
    tg = np.arange(m.nv)
    d, paths = _trace(pch, m, None, tg, face=face, bary=bary)
    dref, _ = ora.trace_paths(m.vertices, m.faces, face=face, bary=bary, targets=tg)
    assert np.max(np.abs(d - dref) / np.maximum(dref, 1e-300)) <= TOL
    p0 = sum(b * m.vertices[m.faces[face, k]] for k, b in enumerate(bary))
    for t in tg:
        assert paths[t] is not None, t
        pc.check_path(m.vertices, m.faces, d, t, paths[t], face_source=(face, bary), rel=TOL)
        xyz = pc.path_xyz(m.vertices, m.faces, paths[t])
        assert np.linalg.norm(xyz[-1] - p0) <= 1e-9


def test_multi_source_paths(pch, ora):
    m = mg.icosphere(3, 0.02, seed=7)
    srcs = [0, 77, 300, 501]
    tg = np.arange(m.nv)
    d, paths = _trace(pch, m, srcs, tg)
    dref, ref = ora.trace_paths(m.vertices, m.faces, sources=srcs, targets=tg)
    assert np.max(np.abs(d - dref) / np.maximum(dref, 1e-300)) <= TOL
    same = 0
    for t in tg:
        pc.check_path(m.vertices, m.faces, d, t, paths[t], sources=srcs, rel=TOL)
        same += _same_path(m, paths[t], ref[t], d[t])
    assert same >= 0.99 * m.nv


def test_paths_larger_mesh_sampled(pch, ora):
    """Terrain 64 x 64 (8,192 faces) from its centre: every vertex traced, a sample
    checked against the oracle's paths, all checked geometrically."""
    m = mg.terrain(64, 64, seed=21)
    src = mg.terrain_center(64, 64)
    tg = np.arange(m.nv)
    d, paths = _trace(pch, m, [src], tg, max_points=2048)
    assert all(p is not None for p in paths)
    for t in tg[::7]:
        pc.check_path(m.vertices, m.faces, d, t, paths[t], sources=[src], rel=TOL)
    sample = tg[::97]
    dref, ref = ora.trace_paths(m.vertices, m.faces, src, targets=sample)
    same = sum(_same_path(m, paths[t], r, d[t]) for t, r in zip(sample, ref))
    assert same >= 0.95 * len(sample)


def test_unreachable_and_source_targets(pch):
    a = mg.icosphere(1, 0.0, seed=0)
    v = np.concatenate([a.vertices, a.vertices + 5.0])
    f = np.concatenate([a.faces, a.faces + a.nv]).astype(np.int32)
    mesh = pch.Mesh(v, f)
    try:
        d, paths = pch.trace_paths(mesh, [0], [0, 3, a.nv + 3])
    finally:
        mesh.close()
    assert len(paths[0][0]) == 1 and paths[0][0][0] == 0 and paths[0][1][0] == 0
    assert len(paths[1][0]) >= 2
    assert np.isinf(d[a.nv + 3]) and len(paths[2][0]) == 0


def test_truncation_and_errors(pch):
    m = mg.terrain(24, 24, seed=8)
    mesh = pch.Mesh(m.vertices, m.faces)
    try:
        _, full = pch.trace_paths(mesh, [0], [m.nv - 1])
        n = len(full[0][0])
        assert n > 3
        with pytest.raises(pch.PchError):
            pch.trace_paths(mesh, [0], [m.nv - 1], max_points=n - 1)
        with pytest.raises(pch.PchError):
            pch.trace_paths(mesh, [0], [m.nv])          # target out of range
        with pytest.raises(pch.PchError):
            pch.trace_paths(mesh, [0], [1], max_points=0)
        # the field of a path solve is the field of a plain solve
        d0 = pch.solve(mesh, 0)
        d1, _ = pch.trace_paths(mesh, [0], [1])
        assert np.max(np.abs(d1 - d0) / np.maximum(d0, 1e-300)) <= 1e-12
    finally:
        mesh.close()
