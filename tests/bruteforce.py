"""Brute-force exact geodesic distance on tiny meshes: an independent pin for the oracle.

By the structure theorem the paper quotes from Mitchell, Mount and Papadimitriou
(Section 3, "Theorem"), a shortest path is an alternating sequence of vertices and
straight segments, each straight in the unfolding of the faces it crosses, and it crosses
every face at most once.  So the exact distance is Dijkstra's shortest path over the
graph whose arcs join two vertices that "see" each other along a straight unfolded
segment, weighted by the length of the shortest such segment.

Visibility is found by exhaustive search: from every vertex u and every face around it,
unfold face after face (each at most once per sequence), keeping the cone of directions
from u that still passes through every crossed edge, and record every vertex that falls
strictly inside the cone.  Nothing here is shared with the oracle: its own half-edge
table, its own unfolding, no windows, no filters, no queue ordering.
"""
from __future__ import annotations

import heapq
import math

import numpy as np


def _cross(a, b):
    return a[0] * b[1] - a[1] * b[0]


class _Tri:
    def __init__(self, vertices, faces):
        self.v = np.asarray(vertices, dtype=np.float64)
        self.f = np.asarray(faces, dtype=np.int64)
        self.opp = {}      # directed edge (a, b) -> (face, third vertex) of the face holding a->b
        for fi, (a, b, c) in enumerate(self.f.tolist()):
            for x, y, z in ((a, b, c), (b, c, a), (c, a, b)):
                self.opp[(x, y)] = (fi, z)

    def d(self, a, b):
        return float(np.linalg.norm(self.v[a] - self.v[b]))


def _unfold_third(p, q, lp, lq):
    """Point at distances lp from p and lq from q, on the right of the directed line p->q."""
    ex, ey = q[0] - p[0], q[1] - p[1]
    L = math.hypot(ex, ey)
    ux, uy = ex / L, ey / L
    x = (L * L + lp * lp - lq * lq) / (2 * L)
    y = math.sqrt(max(lp * lp - x * x, 0.0))
    nx, ny = uy, -ux
    return (p[0] + x * ux + y * nx, p[1] + x * uy + y * ny)


def _more_ccw(a, b):
    return b if _cross(a, b) > 0 else a


def _more_cw(a, b):
    return b if _cross(a, b) < 0 else a


def visibility(mesh: _Tri, u: int, max_depth: int = 64):
    """dict vertex -> shortest straight unfolded distance from u (vertex-free segments)."""
    best = {}

    def see(w, dist):
        if dist < best.get(w, math.inf):
            best[w] = dist

    for (a0, b0), (fi, c0) in mesh.opp.items():
        if a0 != u:
            continue
        # face (u, b0, c0) in CCW order: u at origin, b0 on +x, c0 above
        a_, b_ = b0, c0
        pa = (mesh.d(u, a_), 0.0)
        # c0 on the left of u->b0: mirror of the right-side construction
        pr = _unfold_third((0.0, 0.0), pa, mesh.d(u, b_), mesh.d(a_, b_))
        pb = (pr[0], -pr[1])
        see(a_, mesh.d(u, a_))
        see(b_, mesh.d(u, b_))
        # cone from u: right boundary towards a_, left boundary towards b_
        stack = [(a_, b_, pa, pb, pa, pb, frozenset([fi]), 0)]
        while stack:
            p, q, P, Q, R, Lf, used, depth = stack.pop()
            if depth >= max_depth:
                continue
            nb = mesh.opp.get((q, p))
            if nb is None:
                continue
            f2, c = nb
            if f2 in used:
                continue
            C = _unfold_third(P, Q, mesh.d(p, c), mesh.d(q, c))
            if _cross(R, C) > 0 and _cross(C, Lf) > 0:
                see(c, math.hypot(C[0], C[1]))
            used2 = used | {f2}
            # sub-edge p -> c (p on the right, c on the left)
            R1, L1 = _more_ccw(R, P), _more_cw(Lf, C)
            if _cross(R1, L1) > 0:
                stack.append((p, c, P, C, R1, L1, used2, depth + 1))
            # sub-edge c -> q
            R2, L2 = _more_ccw(R, C), _more_cw(Lf, Q)
            if _cross(R2, L2) > 0:
                stack.append((c, q, C, Q, R2, L2, used2, depth + 1))
    return best


def geodesic(vertices, faces, source: int) -> np.ndarray:
    """Exact polyhedral distance from vertex ``source`` to every vertex (tiny meshes)."""
    mesh = _Tri(vertices, faces)
    n = mesh.v.shape[0]
    adj = [visibility(mesh, u) for u in range(n)]
    dist = [math.inf] * n
    dist[source] = 0.0
    pq = [(0.0, source)]
    while pq:
        dd, u = heapq.heappop(pq)
        if dd > dist[u]:
            continue
        for w, wgt in adj[u].items():
            nd = dd + wgt
            if nd < dist[w]:
                dist[w] = nd
                heapq.heappush(pq, (nd, w))
    return np.array(dist)


def edge_graph_dijkstra(vertices, faces, source: int) -> np.ndarray:
    """Shortest path along mesh edges: an upper bound of the geodesic distance."""
    v = np.asarray(vertices, dtype=np.float64)
    adj = {}
    for a, b, c in np.asarray(faces).tolist():
        for x, y in ((a, b), (b, c), (c, a)):
            w = float(np.linalg.norm(v[x] - v[y]))
            adj.setdefault(x, {})[y] = w
            adj.setdefault(y, {})[x] = w
    dist = np.full(v.shape[0], math.inf)
    dist[source] = 0.0
    pq = [(0.0, source)]
    while pq:
        dd, u = heapq.heappop(pq)
        if dd > dist[u]:
            continue
        for w, wgt in adj.get(u, {}).items():
            if dd + wgt < dist[w]:
                dist[w] = dd + wgt
                heapq.heappush(pq, (dd + wgt, w))
    return dist
