"""Seeded synthetic triangle meshes: the inputs of every test, bench line and smoke run.

This module builds meshes and picks source vertices; it holds none of the geodesic
arithmetic, so both the CPU oracle and the CUDA path can take their inputs from it.

Random numbers come from a vectorised splitmix64 counter generator (Steele, Lea and
Flood, "Fast splittable pseudorandom number generators", OOPSLA 2014), so the same seed
gives bit-identical meshes on x86 and on Arm, whatever the numpy version.

Workload recipes (sizes follow the paper's range of 144K-4M faces, Table `tab:speedup`):

* ``icosphere(levels, noise)`` - icosahedron, midpoint-subdivided ``levels`` times with
  projection to the unit sphere; each vertex radius scaled by ``1 + U(-noise, noise)``.
  levels=4 gives 2,562 vertices / 5,120 faces; levels=9 gives 5,242,880 faces.
* ``geodesic_sphere(nu, noise)`` - class-I geodesic sphere of frequency ``nu``
  (20*nu^2 faces), used for meshes of arbitrary size.
* ``terrain(nx, ny)`` - height field on the integer grid, z = sum of 8 random sines
  plus N(0, 0.01^2), every quad split along a random diagonal.
* ``torus(nu, nv, R, r, jitter)`` - torus grid with vertices moved tangentially (in the
  (u, v) parameter plane) by up to ``jitter`` of the local grid step: thin and obtuse
  triangles.
* ``multi_octave_sphere(levels, amp)`` - icosphere with multi-octave radial noise.
* closed-form solids for the oracle's pins: flat convex patch, prism tube, pyramid,
  cube and regular tetrahedron surfaces.
"""
from __future__ import annotations

import dataclasses
import math

import numpy as np

_MASK64 = (1 << 64) - 1
_GOLDEN = np.uint64(0x9E3779B97F4A7C15)


class SplitMix64:
    """Counter-based splitmix64 stream; ``sub(tag)`` derives an independent stream."""

    def __init__(self, seed: int):
        self.state = np.uint64(seed & _MASK64)

    def u64(self, n: int) -> np.ndarray:
        with np.errstate(over="ignore"):
            idx = np.arange(1, n + 1, dtype=np.uint64)
            z = self.state + idx * _GOLDEN
            self.state = np.uint64((int(self.state) + n * int(_GOLDEN)) & _MASK64)
            z = (z ^ (z >> np.uint64(30))) * np.uint64(0xBF58476D1CE4E5B9)
            z = (z ^ (z >> np.uint64(27))) * np.uint64(0x94D049BB133111EB)
            z = z ^ (z >> np.uint64(31))
        return z

    def uniform(self, n: int, lo: float = 0.0, hi: float = 1.0) -> np.ndarray:
        u = (self.u64(n) >> np.uint64(11)).astype(np.float64) * (2.0 ** -53)
        return lo + (hi - lo) * u

    def normal(self, n: int) -> np.ndarray:
        u1 = 1.0 - self.uniform(n)          # (0, 1]
        u2 = self.uniform(n)
        return np.sqrt(-2.0 * np.log(u1)) * np.cos(2.0 * math.pi * u2)

    def integers(self, n: int, hi: int) -> np.ndarray:
        return np.minimum((self.uniform(n) * hi).astype(np.int64), hi - 1)

    def sub(self, tag: int) -> "SplitMix64":
        z = SplitMix64((int(self.state) ^ ((tag * 0xD1B54A32D192ED03) & _MASK64)) & _MASK64)
        z.u64(3)
        return SplitMix64(int(z.u64(1)[0]))


@dataclasses.dataclass
class Mesh:
    vertices: np.ndarray        # (V, 3) float64
    faces: np.ndarray           # (F, 3) int32, consistently oriented
    name: str = "mesh"

    @property
    def nv(self) -> int:
        return int(self.vertices.shape[0])

    @property
    def nf(self) -> int:
        return int(self.faces.shape[0])

    def mean_edge_length(self) -> float:
        f = self.faces
        v = self.vertices
        e = np.concatenate([v[f[:, 1]] - v[f[:, 0]], v[f[:, 2]] - v[f[:, 1]], v[f[:, 0]] - v[f[:, 2]]])
        return float(np.sqrt((e * e).sum(1)).mean())


def _finish(v, f, name) -> Mesh:
    return Mesh(np.ascontiguousarray(v, dtype=np.float64), np.ascontiguousarray(f, dtype=np.int32), name)


# ----------------------------------------------------------------------------- spheres
def _icosahedron():
    p = (1.0 + math.sqrt(5.0)) / 2.0
    v = np.array([[-1, p, 0], [1, p, 0], [-1, -p, 0], [1, -p, 0],
                  [0, -1, p], [0, 1, p], [0, -1, -p], [0, 1, -p],
                  [p, 0, -1], [p, 0, 1], [-p, 0, -1], [-p, 0, 1]], dtype=np.float64)
    v /= np.linalg.norm(v, axis=1, keepdims=True)
    f = np.array([[0, 11, 5], [0, 5, 1], [0, 1, 7], [0, 7, 10], [0, 10, 11],
                  [1, 5, 9], [5, 11, 4], [11, 10, 2], [10, 7, 6], [7, 1, 8],
                  [3, 9, 4], [3, 4, 2], [3, 2, 6], [3, 6, 8], [3, 8, 9],
                  [4, 9, 5], [2, 4, 11], [6, 2, 10], [8, 6, 7], [9, 8, 1]], dtype=np.int64)
    return v, f


def _orient_outward(v, f):
    """Flip faces whose normal points towards the origin (meshes star-shaped about 0)."""
    a, b, c = v[f[:, 0]], v[f[:, 1]], v[f[:, 2]]
    n = np.cross(b - a, c - a)
    bad = (n * (a + b + c)).sum(1) < 0
    f = f.copy()
    f[bad] = f[bad][:, [0, 2, 1]]
    return f


def _midpoint_subdivide(v, f):
    nv = v.shape[0]
    e = np.concatenate([f[:, [0, 1]], f[:, [1, 2]], f[:, [2, 0]]])
    key = np.minimum(e[:, 0], e[:, 1]) * nv + np.maximum(e[:, 0], e[:, 1])
    uniq, inv = np.unique(key, return_inverse=True)
    a, b = uniq // nv, uniq % nv
    mid = 0.5 * (v[a] + v[b])
    mid /= np.linalg.norm(mid, axis=1, keepdims=True)
    nf = f.shape[0]
    m01, m12, m20 = nv + inv[:nf], nv + inv[nf:2 * nf], nv + inv[2 * nf:]
    f0, f1, f2 = f[:, 0], f[:, 1], f[:, 2]
    nfaces = np.concatenate([np.stack([f0, m01, m20], 1), np.stack([m01, f1, m12], 1),
                             np.stack([m20, m12, f2], 1), np.stack([m01, m12, m20], 1)])
    return np.concatenate([v, mid]), nfaces


def icosphere(levels: int, noise: float = 0.0, seed: int = 0) -> Mesh:
    """Icosahedron midpoint-subdivided ``levels`` times; radius 1 + U(-noise, noise)."""
    v, f = _icosahedron()
    for _ in range(levels):
        v, f = _midpoint_subdivide(v, f)
    if noise > 0.0:
        r = 1.0 + SplitMix64(seed).uniform(v.shape[0], -noise, noise)
        v = v * r[:, None]
    return _finish(v, f, f"icosphere{levels}")


def geodesic_sphere(nu: int, noise: float = 0.0, seed: int = 0) -> Mesh:
    """Class-I geodesic sphere of frequency ``nu`` (20 nu^2 faces, 10 nu^2 + 2 vertices).

    Every grid point is identified by its integer barycentric weights over the base
    icosahedron's corners, so points shared by two base faces get one id."""
    bv, bf = _icosahedron()
    ij = [(i, j) for i in range(nu + 1) for j in range(nu + 1 - i)]
    ij = np.array(ij, dtype=np.int64)
    keys, pos = [], []
    for fi in range(20):
        a, b, c = bf[fi]
        w = np.stack([nu - ij[:, 0] - ij[:, 1], ij[:, 0], ij[:, 1]], 1)
        # canonical key: the (corner id, weight) pairs sorted, a zero weight carrying id 15,
        # so a point on a shared edge or corner gets the same key from every base face
        cid = np.broadcast_to(np.array([a, b, c]), w.shape).copy()
        cid[w == 0] = 15
        pairs = np.stack([cid, w], 2)
        srt = np.argsort(pairs[:, :, 0] * 2048 + pairs[:, :, 1], axis=1)
        pairs = np.take_along_axis(pairs, srt[:, :, None], axis=1)
        k = ((pairs[:, 0, 0] * 1024 + pairs[:, 0, 1]) * 16 + pairs[:, 1, 0]) * 1024 + pairs[:, 1, 1]
        k = (k * 16 + pairs[:, 2, 0]) * 1024 + pairs[:, 2, 1]
        p = (w[:, 0:1] * bv[a] + w[:, 1:2] * bv[b] + w[:, 2:3] * bv[c]) / nu
        keys.append(k)
        pos.append(p)
    allk = np.concatenate(keys)
    allp = np.concatenate(pos)
    uk, first, inv = np.unique(allk, return_index=True, return_inverse=True)
    verts = allp[first]
    verts /= np.linalg.norm(verts, axis=1, keepdims=True)
    # local (i, j) -> index within a face's point list
    lid = -np.ones((nu + 1, nu + 1), dtype=np.int64)
    lid[ij[:, 0], ij[:, 1]] = np.arange(len(ij))
    tris = []
    npf = len(ij)
    for fi in range(20):
        g = inv[fi * npf:(fi + 1) * npf]
        for i in range(nu):
            j = np.arange(nu - i)
            t1 = np.stack([g[lid[i, j]], g[lid[i + 1, j]], g[lid[i, j + 1]]], 1)
            tris.append(t1)
            j2 = np.arange(nu - i - 1)
            if len(j2):
                t2 = np.stack([g[lid[i + 1, j2]], g[lid[i + 1, j2 + 1]], g[lid[i, j2 + 1]]], 1)
                tris.append(t2)
    f = np.concatenate(tris)
    f = _orient_outward(verts, f)
    if noise > 0.0:
        r = 1.0 + SplitMix64(seed).uniform(verts.shape[0], -noise, noise)
        verts = verts * r[:, None]
    return _finish(verts, f, f"geosphere{nu}")


def multi_octave_sphere(levels: int, amp: float = 0.05, seed: int = 0) -> Mesh:
    """Icosphere with radius 1 + amp * N(p)/max|N|, N a 5-octave sum of 8 random plane waves."""
    m = icosphere(levels, 0.0)
    rng = SplitMix64(seed)
    u = rng.normal(24).reshape(8, 3)
    u /= np.linalg.norm(u, axis=1, keepdims=True)
    kappa = rng.uniform(8, 2.0, 4.0)
    phi = rng.uniform(8, 0.0, 2 * math.pi)
    p = m.vertices
    n = np.zeros(p.shape[0])
    for o in range(5):
        for j in range(8):
            n += 2.0 ** (-o) * np.sin((2.0 ** o) * kappa[j] * (p @ u[j]) + phi[j])
    r = 1.0 + amp * n / np.abs(n).max()
    return _finish(p * r[:, None], m.faces, f"octsphere{levels}")


# ----------------------------------------------------------------------------- terrain
def terrain(nx: int, ny: int, seed: int = 0, n_sines: int = 8, sigma: float = 0.01,
            amp_range=(1.0, 8.0), freq_max: float = 6.0) -> Mesh:
    """(nx+1)(ny+1) grid vertices at integer (x, y); z = sum of sines + N(0, sigma^2)."""
    rng = SplitMix64(seed)
    s = float(max(nx, ny))
    a = rng.uniform(n_sines, *amp_range)
    fx = rng.uniform(n_sines, -freq_max, freq_max)
    fy = rng.uniform(n_sines, -freq_max, freq_max)
    ph = rng.uniform(n_sines, 0.0, 2 * math.pi)
    x, y = np.meshgrid(np.arange(nx + 1, dtype=np.float64), np.arange(ny + 1, dtype=np.float64), indexing="xy")
    x, y = x.ravel(), y.ravel()
    z = np.zeros_like(x)
    for i in range(n_sines):
        z += a[i] * np.sin(2 * math.pi * (fx[i] * x + fy[i] * y) / s + ph[i])
    z += sigma * rng.normal(x.shape[0])
    v = np.stack([x, y, z], 1)
    idx = lambda i, j: j * (nx + 1) + i
    i, j = np.meshgrid(np.arange(nx), np.arange(ny), indexing="xy")
    i, j = i.ravel(), j.ravel()
    v00, v10, v11, v01 = idx(i, j), idx(i + 1, j), idx(i + 1, j + 1), idx(i, j + 1)
    coin = rng.uniform(nx * ny) < 0.5
    fa = np.where(coin[:, None], np.stack([v00, v10, v11], 1), np.stack([v00, v10, v01], 1))
    fb = np.where(coin[:, None], np.stack([v00, v11, v01], 1), np.stack([v10, v11, v01], 1))
    f = np.stack([fa, fb], 1).reshape(-1, 3)
    return _finish(v, f, f"terrain{nx}x{ny}")


def terrain_center(nx: int, ny: int) -> int:
    return (ny // 2) * (nx + 1) + nx // 2


# ----------------------------------------------------------------------------- torus
def torus(nu: int, nv: int, R: float = 1.0, r: float = 0.3, jitter: float = 0.4, seed: int = 0) -> Mesh:
    """Torus grid (nu around the axis, nv around the tube), vertices jittered in the
    (u, v) parameter plane by a point drawn uniformly in a disk of radius
    ``jitter`` grid steps; vertices of inverted or near-degenerate faces are redrawn."""
    rng = SplitMix64(seed)
    du, dv = 2 * math.pi / nu, 2 * math.pi / nv
    ui, vi = np.meshgrid(np.arange(nu), np.arange(nv), indexing="ij")
    ui, vi = ui.ravel(), vi.ravel()
    n = nu * nv

    def draw(k):
        rho = np.sqrt(rng.uniform(k)) * jitter
        th = rng.uniform(k, 0.0, 2 * math.pi)
        return rho * np.cos(th), rho * np.sin(th)

    ju, jv = draw(n)
    idx = lambda a, b: (a % nu) * nv + (b % nv)
    a, b = np.meshgrid(np.arange(nu), np.arange(nv), indexing="ij")
    a, b = a.ravel(), b.ravel()
    v00, v10, v11, v01 = idx(a, b), idx(a + 1, b), idx(a + 1, b + 1), idx(a, b + 1)
    f = np.concatenate([np.stack([v00, v10, v11], 1), np.stack([v00, v11, v01], 1)])
    # parameter-plane positions in grid-step units, unwrapped per face
    base_u = np.stack([a, a + 1, a + 1], 1), np.stack([a, a + 1, a], 1)
    base_v = np.stack([b, b, b + 1], 1), np.stack([b, b + 1, b + 1], 1)
    bu = np.concatenate(base_u).astype(np.float64)
    bvv = np.concatenate(base_v).astype(np.float64)
    for _ in range(64):
        pu = bu + ju[f]
        pv = bvv + jv[f]
        area2 = (pu[:, 1] - pu[:, 0]) * (pv[:, 2] - pv[:, 0]) - (pu[:, 2] - pu[:, 0]) * (pv[:, 1] - pv[:, 0])
        bad = area2 < 0.02
        if not bad.any():
            break
        redo = np.unique(f[bad].ravel())
        nu_, nv_ = draw(redo.shape[0])
        ju[redo], jv[redo] = nu_, nv_
    uu = (ui + ju) * du
    vv = (vi + jv) * dv
    x = (R + r * np.cos(vv)) * np.cos(uu)
    y = (R + r * np.cos(vv)) * np.sin(uu)
    z = r * np.sin(vv)
    verts = np.stack([x, y, z], 1)
    # orient outward: tube normal is the direction from the tube centre circle
    cen = np.stack([R * np.cos(uu), R * np.sin(uu), np.zeros_like(uu)], 1)
    pa, pb, pc = verts[f[:, 0]], verts[f[:, 1]], verts[f[:, 2]]
    nrm = np.cross(pb - pa, pc - pa)
    out = (pa + pb + pc) / 3 - cen[f[:, 0]]
    flip = (nrm * out).sum(1) < 0
    # the grid is consistently oriented; flip all faces if most normals point inward
    if 2 * int(flip.sum()) > flip.shape[0]:
        f = f[:, [0, 2, 1]]
    return _finish(verts, f, f"torus{nu}x{nv}")


# ----------------------------------------------------------------------------- closed-form solids
def flat_patch(n: int, jitter: float = 0.3, seed: int = 0, size: float = 1.0) -> Mesh:
    """Convex square [0,size]^2 in the plane z=0, n x n quads, interior vertices jittered,
    random diagonals, no folded triangle.  Geodesic distance = Euclidean distance."""
    rng = SplitMix64(seed)
    h = size / n
    x, y = np.meshgrid(np.arange(n + 1) * h, np.arange(n + 1) * h, indexing="xy")
    x, y = x.ravel().copy(), y.ravel().copy()
    i, j = np.meshgrid(np.arange(n + 1), np.arange(n + 1), indexing="xy")
    inner = ((i > 0) & (i < n) & (j > 0) & (j < n)).ravel()
    k = int(inner.sum())
    # jitter inside a disk of radius jitter*h: with jitter < 0.35 no triangle can fold
    # (each vertex-to-opposite-side height, >= h/sqrt(2), shrinks by at most 2*jitter*h)
    rho = np.sqrt(rng.uniform(k)) * jitter * h
    th = rng.uniform(k, 0.0, 2 * math.pi)
    x[inner] += rho * np.cos(th)
    y[inner] += rho * np.sin(th)
    v = np.stack([x, y, np.zeros_like(x)], 1)
    m = terrain(n, n, seed=seed + 1)  # reuse connectivity (random diagonals)
    return _finish(v, m.faces, f"flat{n}")


def prism_tube(sides: int, rings: int, height: float = 1.0, seed: int = 0, irregular: float = 0.3):
    """Lateral surface of a prism over a convex polygon, open at both ends.

    Returns (mesh, s, z, perimeter): s = arc-length position of each vertex along the
    polygon, z = height.  Unrolled, the surface is the periodic strip [0,P) x [0,H]."""
    rng = SplitMix64(seed)
    ang = (np.arange(sides) + rng.uniform(sides, -irregular, irregular)) * 2 * math.pi / sides
    ang = np.sort(ang)
    rad = 1.0
    px, py = rad * np.cos(ang), rad * np.sin(ang)
    seg = np.hypot(np.roll(px, -1) - px, np.roll(py, -1) - py)
    s_corner = np.concatenate([[0.0], np.cumsum(seg)[:-1]])
    perim = float(seg.sum())
    zr = np.sort(rng.uniform(rings - 1, 0.0, height))
    zr = np.concatenate([[0.0], zr, [height]])[: rings + 1]
    zr[-1] = height
    verts, s_all, z_all = [], [], []
    for r_ in range(rings + 1):
        for k in range(sides):
            verts.append([px[k], py[k], zr[r_]])
            s_all.append(s_corner[k])
            z_all.append(zr[r_])
    v = np.array(verts)
    idx = lambda r_, k: r_ * sides + (k % sides)
    f = []
    coin = rng.uniform(rings * sides) < 0.5
    c = 0
    for r_ in range(rings):
        for k in range(sides):
            a, b, cc, d = idx(r_, k), idx(r_, k + 1), idx(r_ + 1, k + 1), idx(r_ + 1, k)
            if coin[c]:
                f += [[a, b, cc], [a, cc, d]]
            else:
                f += [[a, b, d], [b, cc, d]]
            c += 1
    return _finish(v, np.array(f), f"prism{sides}x{rings}"), np.array(s_all), np.array(z_all), perim


def pyramid(sides: int, sub: int, height: float = 1.0, seed: int = 0):
    """Lateral surface of a regular pyramid (apex spherical), each lateral triangle split
    into sub^2 triangles.  Returns (mesh, r, theta, Theta): polar coordinates of every
    vertex in the unrolled sector of total angle Theta around the apex (vertex 0)."""
    ang = np.arange(sides) * 2 * math.pi / sides
    base = np.stack([np.cos(ang), np.sin(ang), np.zeros(sides)], 1)
    apex = np.array([0.0, 0.0, height])
    verts = [apex]
    key = {}

    def vid(face_k, i, j):
        # point = apex + (base_k - apex) * i/sub + (base_{k+1} - base_k) * j/sub, 0 <= j <= i
        if i == 0:
            return 0
        kk = face_k % sides
        if j == 0:
            kkey = ("e", kk, i)
        elif j == i:
            kkey = ("e", (kk + 1) % sides, i)
        else:
            kkey = ("f", kk, i, j)
        if kkey not in key:
            b0, b1 = base[kk], base[(kk + 1) % sides]
            p = apex + (b0 - apex) * i / sub + (b1 - b0) * j / sub
            key[kkey] = len(verts)
            verts.append(p)
        return key[kkey]

    f = []
    for k in range(sides):
        for i in range(sub):
            for j in range(i + 1):
                f.append([vid(k, i, j), vid(k, i + 1, j), vid(k, i + 1, j + 1)])
                if j < i:
                    f.append([vid(k, i, j), vid(k, i + 1, j + 1), vid(k, i, j + 1)])
    v = np.array(verts)
    f = np.array(f)
    # unrolled polar coordinates
    slant = np.linalg.norm(base[0] - apex)
    apex_angle = 2 * math.asin(np.linalg.norm(base[1] - base[0]) / 2 / slant)
    Theta = sides * apex_angle
    r = np.linalg.norm(v - apex, axis=1)
    theta = np.zeros(v.shape[0])
    for kkey, idx_ in key.items():
        kk = kkey[1]
        p = v[idx_]
        d0 = base[kk] - apex
        q = p - apex
        within = math.atan2(np.linalg.norm(np.cross(q, d0)), np.dot(q, d0))
        theta[idx_] = kk * apex_angle + within
    fm = _orient_outward(v - np.array([0, 0, height / 3]), f)
    return _finish(v, fm, f"pyramid{sides}x{sub}"), r, theta, Theta


def cube(m: int) -> Mesh:
    """Surface of the unit cube [0,1]^3, each face an m x m grid of split squares."""
    key = {}
    verts = []

    def vid(p):
        k = tuple(int(round(c * m)) for c in p)
        if k not in key:
            key[k] = len(verts)
            verts.append([c / m for c in k])
        return key[k]

    f = []
    for axis in range(3):
        for side in (0.0, 1.0):
            u_ax, v_ax = [a for a in range(3) if a != axis]
            for i in range(m):
                for j in range(m):
                    def P(a, b):
                        p = [0.0, 0.0, 0.0]
                        p[axis] = side
                        p[u_ax] = a / m
                        p[v_ax] = b / m
                        return vid(p)
                    a, b, c, d = P(i, j), P(i + 1, j), P(i + 1, j + 1), P(i, j + 1)
                    if (i + j) % 2 == 0:
                        f += [[a, b, c], [a, c, d]]
                    else:
                        f += [[a, b, d], [b, c, d]]
    v = np.array(verts, dtype=np.float64)
    f = _orient_outward(v - 0.5, np.array(f))
    return _finish(v, f, f"cube{m}")


def tetrahedron(m: int) -> Mesh:
    """Regular tetrahedron (edge 1), each face split into m^2 triangles."""
    c = np.array([[1, 1, 1], [1, -1, -1], [-1, 1, -1], [-1, -1, 1]], dtype=np.float64) / math.sqrt(8.0)
    faces = [(0, 1, 2), (0, 3, 1), (0, 2, 3), (1, 3, 2)]
    key = {}
    verts = []

    def vid(wts):
        k = tuple(sorted((ci, w) for ci, w in wts if w > 0))
        if k not in key:
            key[k] = len(verts)
            verts.append(sum(w * c[ci] for ci, w in wts) / m)
        return key[k]

    f = []
    for (a, b, cc) in faces:
        P = lambda i, j: vid([(a, m - i - j), (b, i), (cc, j)])
        for i in range(m):
            for j in range(m - i):
                f.append([P(i, j), P(i + 1, j), P(i, j + 1)])
                if i + j < m - 1:
                    f.append([P(i + 1, j), P(i + 1, j + 1), P(i, j + 1)])
    v = np.array(verts)
    f = _orient_outward(v, np.array(f))
    return _finish(v, f, f"tetra{m}")


def octahedron(noise: float = 0.0, seed: int = 0, levels: int = 0) -> Mesh:
    v = np.array([[1, 0, 0], [-1, 0, 0], [0, 1, 0], [0, -1, 0], [0, 0, 1], [0, 0, -1]], dtype=np.float64)
    f = np.array([[0, 2, 4], [2, 1, 4], [1, 3, 4], [3, 0, 4], [2, 0, 5], [1, 2, 5], [3, 1, 5], [0, 3, 5]])
    for _ in range(levels):
        v, f = _midpoint_subdivide(v, f)
    if noise > 0:
        rng = SplitMix64(seed)
        v = v * (1.0 + rng.uniform(v.shape[0], -noise, noise))[:, None]
        v = v + rng.uniform(v.size, -noise, noise).reshape(v.shape) * 0.5
    f = _orient_outward(v, f)
    return _finish(v, f, f"octa{levels}")


# ----------------------------------------------------------------------------- workloads
def pick_sources(mesh: Mesh, n: int, seed: int) -> np.ndarray:
    """``n`` distinct seeded vertex ids."""
    rng = SplitMix64(seed)
    out = []
    seen = set()
    while len(out) < n:
        c = int(rng.integers(1, mesh.nv)[0])
        if c not in seen:
            seen.add(c)
            out.append(c)
    return np.array(out, dtype=np.int32)


SEED_BASE = 0xC0FFEE


def workload(name: str, scale: str = "full"):
    """The five synthetic workloads: returns (list of meshes, list of per-mesh source arrays).

    ``scale='small'`` gives a reduced instance of the same family that the oracle solves
    in seconds (used by the parity tests)."""
    small = scale == "small"
    if name == "icosphere":          # single source, 5,120 faces
        m = icosphere(3 if small else 4, 0.02, seed=SEED_BASE + 0)
        return [m], [np.array([0], dtype=np.int32)]
    if name == "terrain":            # 512 x 512 height field, centre source
        n = 48 if small else 512
        m = terrain(n, n, seed=SEED_BASE + 1)
        return [m], [np.array([terrain_center(n, n)], dtype=np.int32)]
    if name == "torus":              # 1M-face jittered torus, 4 sources
        nu, nv = (60, 20) if small else (1250, 400)
        m = torus(nu, nv, seed=SEED_BASE + 2)
        return [m], [pick_sources(m, 4, SEED_BASE + 102)]
    if name == "batch":              # 256 uneven meshes, one source each
        rng = SplitMix64(SEED_BASE + 3)
        count = 12 if small else 256
        lo, hi = (200, 3000) if small else (2000, 200000)
        fstar = np.exp(rng.uniform(count, math.log(lo), math.log(hi)))
        coin = rng.uniform(count) < 0.5
        meshes, srcs = [], []
        for i in range(count):
            if coin[i]:
                nu = max(2, int(round(math.sqrt(fstar[i] / 20.0))))
                m = geodesic_sphere(nu, 0.02, seed=SEED_BASE + 1000 + i)
            else:
                side = max(2, int(round(math.sqrt(fstar[i] / 2.0))))
                m = terrain(side, side, seed=SEED_BASE + 1000 + i)
            meshes.append(m)
            srcs.append(pick_sources(m, 1, SEED_BASE + 2000 + i))
        return meshes, srcs
    if name == "multisrc":           # 64 sources on one 100,820-face geodesic sphere
        m = geodesic_sphere(12 if small else 71, 0.02, seed=SEED_BASE + 4)
        return [m], [pick_sources(m, 8 if small else 64, SEED_BASE + 104)]
    if name == "large":              # icosphere subdivided 9x (5,242,880 faces), 32 sources
        m = multi_octave_sphere(4 if small else 9, 0.05, seed=SEED_BASE + 5)
        return [m], [pick_sources(m, 4 if small else 32, SEED_BASE + 105)]
    raise KeyError(name)


WORKLOADS = ("icosphere", "terrain", "torus", "batch", "multisrc", "large")
