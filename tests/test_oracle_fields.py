"""Pins of the oracle's geodesic Voronoi labels and iso-contours (oracle/fields.py), no GPU.

Voronoi: on a convex planar patch the exact field is Euclidean, so the labels are the
Euclidean nearest sites; on tiny meshes they are the argmin of the brute-force fields;
each source labels itself; the multiple-source field of the oracle equals the labelled
source's distance.  Iso-contours: on the plane every contour point lies on the edge
between the exact circle of radius L and its linear-interpolation error bound
(the distance along a line is convex, so the interpolant overestimates it by at most
h^2 / (8 r)); on closed meshes every crossed edge is shared by exactly two segments with
the same crossing point, and the oriented segments close into loops; the segment count
equals the number of faces whose vertices straddle the level.  Planted mistakes in copies
of the oracle's functions are each caught."""
import math

import numpy as np
import pytest

import bruteforce as bf
from oracle import fields
from paper_1305_1293_gb300 import meshgen as mg


# ------------------------------------------------------------------ Voronoi
def _plane_case():
    m = mg.flat_patch(16, jitter=0.3, seed=61)
    sources = [0, 40, 150, 200, m.nv - 1]
    return m, sources


def _euclid_labels(m, sources):
    E = np.vstack([np.linalg.norm(m.vertices - m.vertices[s], axis=1) for s in sources])
    o = np.argsort(E, axis=0)
    gap = np.take_along_axis(E, o[1:2], 0)[0] - np.take_along_axis(E, o[:1], 0)[0]
    return o[0], gap


def test_voronoi_plane_is_euclidean_nearest(oracle_lib):
    m, sources = _plane_case()
    lab, D, gap = fields.voronoi(m.vertices, m.faces, sources)
    el, egap = _euclid_labels(m, sources)
    ok = egap > 1e-9
    assert ok.sum() > 0.95 * m.nv
    assert np.array_equal(lab[ok], el[ok])
    assert np.all(lab[sources] == np.arange(len(sources)))


@pytest.mark.parametrize("make", [lambda: mg.octahedron(0.1, 2, 1), lambda: mg.cube(2), lambda: mg.torus(6, 4, seed=6)],
                         ids=["octa1", "cube2", "torus6x4"])
def test_voronoi_matches_bruteforce(oracle_lib, make):
    m = make()
    sources = [0, m.nv // 3, (2 * m.nv) // 3]
    lab, _, gap = fields.voronoi(m.vertices, m.faces, sources)
    B = np.vstack([bf.geodesic(m.vertices, m.faces, s) for s in sources])
    ok = gap > 1e-9 * np.max(B)
    assert np.array_equal(lab[ok], np.argmin(B, axis=0)[ok])


def test_voronoi_consistent_with_multi_source_field(oracle_lib):
    m = mg.torus(30, 12, seed=62)
    sources = [1, 100, 250, 333]
    lab, D, _ = fields.voronoi(m.vertices, m.faces, sources)
    multi, _ = oracle_lib.geodesic(m.vertices, m.faces, sources=sources)
    np.testing.assert_array_equal(D[lab, np.arange(m.nv)], multi)
    # a face-point source labelled after the vertex sources
    lab2, D2, _ = fields.voronoi(m.vertices, m.faces, sources[:2], face_points=[(17, (0.2, 0.3, 0.5))])
    assert set(np.unique(lab2)) == {0, 1, 2}


def test_voronoi_disconnected_is_unlabelled(oracle_lib):
    v = np.array([[0, 0, 0], [1, 0, 0], [0, 1, 0], [5, 5, 0], [6, 5, 0], [5, 6, 0]], dtype=np.float64)
    f = np.array([[0, 1, 2], [3, 4, 5]], dtype=np.int32)
    lab, _, _ = fields.voronoi(v, f, [0, 1])
    assert list(lab[3:]) == [-1, -1, -1] and lab[0] == 0 and lab[1] == 1


def test_voronoi_pin_catches_planted_mistakes(oracle_lib, monkeypatch):
    m, sources = _plane_case()
    el, egap = _euclid_labels(m, sources)
    ok = egap > 1e-9
    real = np.argsort

    def second_nearest(a, axis=-1, kind=None):        # labels from the wrong end of the order
        return real(a, axis=axis, kind=kind)[::-1]

    monkeypatch.setattr(fields.np, "argsort", second_nearest)
    lab, _, _ = fields.voronoi(m.vertices, m.faces, sources)
    assert not np.array_equal(lab[ok], el[ok])
    monkeypatch.setattr(fields.np, "argsort", real)
    lab, _, _ = fields.voronoi(m.vertices, m.faces, sources[::-1])   # labels of a permuted list
    assert not np.array_equal(lab[ok], el[ok])


# ------------------------------------------------------------------ iso-contours
def _seg_points(m, segs):
    P = []
    for li, f, (h0, t0), (h1, t1) in segs:
        pts = []
        for h, t in ((h0, t0), (h1, t1)):
            ff, i = divmod(h, 3)
            a, b = m.vertices[m.faces[ff, i]], m.vertices[m.faces[ff, (i + 1) % 3]]
            pts.append(a + t * (b - a))
        P.append(pts)
    return P


def _plane_contour_check(iso, m, s, dist, levels):
    segs = iso(m.faces, dist, levels)
    assert len(segs) > 20
    e = np.concatenate([m.faces[:, [0, 1]], m.faces[:, [1, 2]], m.faces[:, [2, 0]]])
    h = np.max(np.linalg.norm(m.vertices[e[:, 0]] - m.vertices[e[:, 1]], axis=1))
    worst = 0.0
    for (li, f, *_), pts in zip(segs, _seg_points(m, segs)):
        L = levels[li]
        for p in pts:
            r = float(np.linalg.norm(p - m.vertices[s]))
            lo = L - h * h / (8 * (L - h))
            assert lo - 1e-12 <= r <= L + 1e-12, (L, r, lo)
            worst = max(worst, L - r)
    return worst


def test_contours_plane_within_interpolation_bound():
    m = mg.flat_patch(30, jitter=0.3, seed=63)
    s = 465
    dist = np.linalg.norm(m.vertices - m.vertices[s], axis=1)      # the exact field on the plane
    _plane_contour_check(fields.iso_contours, m, s, dist, [0.2, 0.35, 0.45])


def _closed_mesh_checks(iso, m, dist, levels):
    segs = iso(m.faces, dist, levels)
    # count: faces whose vertices straddle the level
    for li, L in enumerate(levels):
        below = dist[m.faces] < L
        straddle = int(np.sum(below.any(1) & ~below.all(1)))
        assert sum(1 for sg in segs if sg[0] == li) == straddle
    # every crossed edge is shared by the two faces around it, at the same point
    key = {}
    for li, f, a, b in segs:
        for h, t in (a, b):
            ff, i = divmod(h, 3)
            u, w = int(m.faces[ff, i]), int(m.faces[ff, (i + 1) % 3])
            k = (li, min(u, w), max(u, w))
            tt = t if u < w else 1.0 - t
            key.setdefault(k, []).append(tt)
    for k, ts in key.items():
        assert len(ts) == 2 and abs(ts[0] - ts[1]) < 1e-12, (k, ts)
    # the region below the level lies to the left of each segment, seen from the face's
    # front side (corners counter-clockwise)
    for (li, f, a, b), (P, Q) in zip(segs, _seg_points(m, segs)):
        A, B, C = m.vertices[m.faces[f]]
        n = np.cross(B - A, C - A)
        for c in m.faces[f]:
            if dist[c] < levels[li]:
                assert np.dot(n, np.cross(Q - P, m.vertices[c] - P)) > 0, (li, f)
    # oriented segments close into loops: every point starts one segment and ends another
    starts, ends = {}, {}
    for li, f, a, b in segs:
        for pt, dct in ((a, starts), (b, ends)):
            ff, i = divmod(pt[0], 3)
            u, w = int(m.faces[ff, i]), int(m.faces[ff, (i + 1) % 3])
            k = (li, min(u, w), max(u, w))
            dct[k] = dct.get(k, 0) + 1
    assert starts.keys() == ends.keys() and all(v == 1 for v in starts.values()) and all(v == 1 for v in ends.values())


def test_contours_close_into_oriented_loops(oracle_lib):
    m = mg.icosphere(3, 0.02, seed=64)
    dist, _ = oracle_lib.geodesic(m.vertices, m.faces, 0)
    _closed_mesh_checks(fields.iso_contours, m, dist, [0.3, 1.0, 2.0, 2.9])


def test_contours_pin_catches_planted_mistakes(oracle_lib):
    m = mg.flat_patch(30, jitter=0.3, seed=63)
    s = 465
    dist = np.linalg.norm(m.vertices - m.vertices[s], axis=1)
    levels = [0.2, 0.35, 0.45]
    ms = mg.icosphere(3, 0.02, seed=64)
    dsph, _ = oracle_lib.geodesic(ms.vertices, ms.faces, 0)

    def complement_t(faces, d, lv):                  # t measured from the other end
        return [(li, f, (h0, 1 - t0), (h1, 1 - t1)) for li, f, (h0, t0), (h1, t1) in fields.iso_contours(faces, d, lv)]

    def reversed_orientation(faces, d, lv):
        return [(li, f, b, a) for li, f, a, b in fields.iso_contours(faces, d, lv)]

    def dropped_edge(faces, d, lv):                  # the segment ends at the face's first crossing twice
        return [(li, f, a, a) for li, f, a, b in fields.iso_contours(faces, d, lv)]

    with pytest.raises(AssertionError):
        _plane_contour_check(complement_t, m, s, dist, levels)
    with pytest.raises(AssertionError):
        _closed_mesh_checks(reversed_orientation, ms, dsph, [0.3, 1.0])
    with pytest.raises(AssertionError):
        _closed_mesh_checks(dropped_edge, ms, dsph, [0.3, 1.0])


def test_contours_edge_cases():
    m = mg.icosphere(2, 0.0, seed=0)
    d = np.linalg.norm(m.vertices - m.vertices[0], axis=1)
    assert fields.iso_contours(m.faces, d, [-1.0, 10.0]) == []          # no level crosses
    d2 = d.copy()
    d2[5] = np.inf                                                      # faces at vertex 5 are skipped
    segs = fields.iso_contours(m.faces, d2, [float(np.median(d))])
    assert all(5 not in m.faces[f] for _, f, _, _ in segs)
