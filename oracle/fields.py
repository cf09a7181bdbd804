"""Geodesic Voronoi labels and iso-contours from the oracle's exact fields - TEST
INFRASTRUCTURE ONLY (the tests call it; the product path never does).

Both are plain definitions written out, on top of the pinned sequential oracle
(``oracle.geodesic``):

* ``voronoi`` - the geodesic Voronoi diagram of a source set (the use of the multiple-
  source field named in Section 7): each vertex takes the index of its nearest source,
  the argmin over the single-source exact fields.  The gap to the second-nearest source
  is returned too, so that comparisons can skip vertices where two sources tie.
* ``iso_contours`` - the iso-contours of a field (Section 2 cites iso-contours of the
  exact geodesic distance): on each face the field is the linear interpolation of its
  vertex values; a vertex is below level L when its value is < L; the contour crosses
  each edge whose ends are on different sides at t = (L - d_start) / (d_end - d_start),
  one segment per face and level, from the crossing on the edge whose start is below L
  to the crossing on the edge whose start is not.  Plain loops over faces and levels.
"""
from __future__ import annotations

import numpy as np


def voronoi(vertices, faces, sources=(), face_points=(), lib=None):
    """Labels (index into sources, then face_points) of the nearest source of every vertex
    (-1 where no source reaches), the single-source fields stacked (S, V), and the gap
    between the second-nearest and the nearest distance (inf with one source)."""
    from . import geodesic
    fields = [geodesic(vertices, faces, int(s), lib=lib)[0] for s in sources]
    fields += [geodesic(vertices, faces, face=int(f), bary=np.asarray(b, dtype=np.float64), lib=lib)[0]
               for f, b in face_points]
    D = np.vstack(fields)
    order = np.argsort(D, axis=0, kind="stable")
    labels = order[0].astype(np.int32)
    best = np.take_along_axis(D, order[:1], axis=0)[0]
    if D.shape[0] > 1:
        second = np.take_along_axis(D, order[1:2], axis=0)[0]
        with np.errstate(invalid="ignore"):
            gap = np.where(np.isfinite(best), second - best, np.inf)
    else:
        gap = np.full(D.shape[1], np.inf)
    labels[~np.isfinite(best)] = -1
    return labels, D, gap


def iso_contours(faces, dist, levels):
    """List of (level index, face, (h0, t0), (h1, t1)) in face order, then level order;
    half-edge 3 f + i runs from corner i to corner (i + 1) % 3 of face f."""
    out = []
    for f, tri in enumerate(np.asarray(faces)):
        d = [float(dist[int(tri[0])]), float(dist[int(tri[1])]), float(dist[int(tri[2])])]
        if not all(np.isfinite(d)):
            continue
        for li, L in enumerate(levels):
            L = float(L)
            crossed = [i for i in range(3) if (d[i] < L) != (d[(i + 1) % 3] < L)]
            if not crossed:
                continue
            leaving = [i for i in crossed if d[i] < L]        # start corner below L
            entering = [i for i in crossed if not d[i] < L]
            assert len(leaving) == 1 and len(entering) == 1
            pts = []
            for i in (leaving[0], entering[0]):
                a, b = d[i], d[(i + 1) % 3]
                pts.append((3 * f + i, (L - a) / (b - a)))
            out.append((li, f, pts[0], pts[1]))
    return out
