"""Pins of the CPU oracle against closed-form geodesic distances (no GPU).

Each surface here unfolds isometrically onto a plane region where the shortest path is a
straight segment, so its exact distance is a formula that shares nothing with the
oracle's window propagation (Section 3: a geodesic is straight in the unfolding)."""
import math

import numpy as np
import pytest

from paper_1305_1293_gb300 import meshgen as mg

TOL = 1e-12


def _rel(a, b):
    return np.max(np.abs(a - b) / np.maximum(np.abs(b), 1e-300))


@pytest.mark.parametrize("n,seed,src", [(6, 1, 0), (9, 2, 40), (12, 3, 84), (10, 4, 120)])
def test_plane_is_euclidean(oracle_lib, n, seed, src):
    m = mg.flat_patch(n, jitter=0.3, seed=seed)
    d, _ = oracle_lib.geodesic(m.vertices, m.faces, src)
    ex = np.linalg.norm(m.vertices - m.vertices[src], axis=1)
    assert d[src] == 0.0
    assert np.max(np.abs(d - ex)) < TOL


@pytest.mark.parametrize("face,bary", [(7, (0.2, 0.3, 0.5)), (30, (1 / 3, 1 / 3, 1 / 3)), (55, (0.9, 0.05, 0.05))])
def test_plane_face_point_source(oracle_lib, face, bary):
    m = mg.flat_patch(7, jitter=0.25, seed=11)
    p = sum(b * m.vertices[m.faces[face, k]] for k, b in enumerate(bary))
    d, _ = oracle_lib.geodesic(m.vertices, m.faces, face=face, bary=np.array(bary))
    ex = np.linalg.norm(m.vertices - p, axis=1)
    assert np.max(np.abs(d - ex)) < TOL


@pytest.mark.parametrize("sides,rings,seed", [(7, 4, 0), (11, 6, 1), (5, 9, 2)])
def test_prism_tube_unrolls(oracle_lib, sides, rings, seed):
    """Lateral surface of a prism: periodic strip [0,P) x [0,H]; wrap k in {-1,0,1}."""
    m, s, z, perim = mg.prism_tube(sides, rings, height=1.5, seed=seed)
    for src in (0, m.nv // 2, m.nv - 1):
        d, _ = oracle_lib.geodesic(m.vertices, m.faces, src)
        ds = s - s[src]
        dz = z - z[src]
        ex = np.min([np.hypot(ds + k * perim, dz) for k in (-1, 0, 1)], axis=0)
        assert _rel(d, ex) < TOL


@pytest.mark.parametrize("sides,sub", [(5, 3), (6, 4), (4, 5)])
def test_pyramid_cone_unrolls(oracle_lib, sides, sub):
    """Pyramid lateral surface unrolls to a sector of angle Theta < 2 pi around the apex:
    g = sqrt(r1^2 + r2^2 - 2 r1 r2 cos(phi)), phi the shorter angular separation."""
    m, r, th, Theta = mg.pyramid(sides, sub, height=1.0)
    assert Theta < 2 * math.pi
    d, _ = oracle_lib.geodesic(m.vertices, m.faces, 0)          # apex source
    assert _rel(d[1:], r[1:]) < TOL
    for src in (1, m.nv // 2, m.nv - 1):
        d, _ = oracle_lib.geodesic(m.vertices, m.faces, src)
        dphi = np.abs(th - th[src]) % Theta
        phi = np.minimum(dphi, Theta - dphi)
        ex = np.sqrt(np.maximum(r ** 2 + r[src] ** 2 - 2 * r * r[src] * np.cos(phi), 0.0))
        mask = np.arange(m.nv) != src
        assert _rel(d[mask], ex[mask]) < 1e-11


def _cube_corner_distance(p):
    """Distance on the unit cube surface from corner (0,0,0) to surface point p."""
    x, y, z = p
    if min(x, y, z) < 1e-12:
        return float(np.linalg.norm(p))       # p on a face through the corner: straight segment
    best = math.inf
    for a in range(3):                         # p on a far face {coordinate a = 1}
        if abs(p[a] - 1.0) < 1e-12:
            u, w = [p[k] for k in range(3) if k != a]
            # unfold the far face onto one of the two near faces sharing an edge with it
            best = min(best, math.hypot(1 + u, w), math.hypot(1 + w, u))
    return best


@pytest.mark.parametrize("m_", [2, 3, 4])
def test_cube_from_corner(oracle_lib, m_):
    m = mg.cube(m_)
    src = int(np.argmin(np.linalg.norm(m.vertices, axis=1)))
    d, _ = oracle_lib.geodesic(m.vertices, m.faces, src)
    ex = np.array([_cube_corner_distance(p) for p in m.vertices])
    assert _rel(d, ex) < TOL


def _tet_distance(corners, faces_c, src_c, p):
    """Regular tetrahedron: from corner src_c to p, straight on a face through src_c, or
    through exactly one edge of the opposite face (min over the three unfoldings)."""
    c0 = corners[src_c]
    if np.linalg.norm(p - c0) < 1e-14:
        return 0.0
    opp = [k for k in range(4) if k != src_c]
    # is p on a face containing src_c?  (barycentric weight of the opposite corner)
    n = np.cross(corners[opp[1]] - corners[opp[0]], corners[opp[2]] - corners[opp[0]])
    on_opposite = abs(np.dot(p - corners[opp[0]], n)) < 1e-12
    if not on_opposite:
        return float(np.linalg.norm(p - c0))
    best = math.inf
    for i in range(3):
        a, b = corners[opp[i]], corners[opp[(i + 1) % 3]]
        # 2D frame: a at origin, b on +x; c0 above, unfolded p below
        L = np.linalg.norm(b - a)
        ex = (b - a) / L

        def place(q, sign):
            x = np.dot(q - a, ex)
            y = math.sqrt(max(np.linalg.norm(q - a) ** 2 - x * x, 0.0))
            return np.array([x, sign * y])
        C = place(c0, 1.0)
        P = place(p, -1.0)
        t = C[1] / (C[1] - P[1]) if C[1] != P[1] else -1
        xcross = C[0] + t * (P[0] - C[0])
        if -1e-12 <= xcross <= L + 1e-12:
            best = min(best, float(np.linalg.norm(C - P)))
    return best


@pytest.mark.parametrize("m_", [2, 3, 5])
def test_tetrahedron_from_corner(oracle_lib, m_):
    m = mg.tetrahedron(m_)
    corners = np.array([[1, 1, 1], [1, -1, -1], [-1, 1, -1], [-1, -1, 1]], dtype=np.float64) / math.sqrt(8.0)
    for src_c in range(4):
        src = int(np.argmin(np.linalg.norm(m.vertices - corners[src_c], axis=1)))
        d, _ = oracle_lib.geodesic(m.vertices, m.faces, src)
        ex = np.array([_tet_distance(corners, None, src_c, p) for p in m.vertices])
        assert _rel(d, ex) < TOL


def test_flat_grid_corner_source_rows(oracle_lib):
    """Special case: unjittered flat grid, source at a corner: distance along the first
    row equals the edge-path distance (collinear vertices, Section 3 pass-through)."""
    m = mg.flat_patch(8, jitter=0.0, seed=0)
    d, _ = oracle_lib.geodesic(m.vertices, m.faces, 0)
    row = np.arange(9)
    assert np.max(np.abs(d[row] - row / 8.0)) < TOL
    assert np.max(np.abs(d - np.linalg.norm(m.vertices, axis=1))) < TOL
