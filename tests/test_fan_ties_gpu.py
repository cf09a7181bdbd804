"""A saddle vertex on the symmetry line of a source, reached along two shortest paths of
equal length from two directions (the geometry of Fig. `fig:propagation`(c) met twice).

The mesh is a planar grid, mirror-symmetric about x = 0, with a square hole between the
source and a strong saddle vertex v on the axis (its one-ring lifted and lowered in
turn).  Every shortest path to v goes around one of the hole's upper corners, so v's
distance is reached from the left and from the right with the same length (bit for bit
or within rounding, depending on the order of the arithmetic); the region behind v is
the union of both directions' fanned areas.  The field must match the oracle (which fans
over the whole one-ring) at every vertex, for several selection sizes and orders."""
import numpy as np
import pytest

pytestmark = pytest.mark.gpu
TOL = 1e-9


def tie_mesh(h=0.4):
    xs = np.arange(-8, 9) * 0.5
    ys = np.arange(-12, 13) * 0.5
    nx, ny = xs.size, ys.size
    vid = lambda i, j: j * nx + i
    V = np.array([[x, y, 0.0] for y in ys for x in xs])
    F = []
    for j in range(ny - 1):
        for i in range(nx - 1):
            cx, cy = (xs[i] + xs[i + 1]) / 2, (ys[j] + ys[j + 1]) / 2
            if -1 < cx < 1 and -3 < cy < -1:
                continue                                     # the hole
            a, b, c, d = vid(i, j), vid(i + 1, j), vid(i + 1, j + 1), vid(i, j + 1)
            F += [[a, b, c], [a, c, d]] if cx > 0 else [[a, b, d], [b, c, d]]
    F = np.array(F, dtype=np.int32)
    v = vid(8, 14)                                           # (0, 1)
    assert np.allclose(V[v], [0, 1, 0])
    ring = {(0.0, 1.5): h, (0.5, 1.0): h, (-0.5, 1.0): h, (0.5, 1.5): -h, (-0.5, 1.5): -h, (0.0, 0.5): -h}
    for (x, y), z in ring.items():
        V[vid(int(round(x * 2)) + 8, int(round(y * 2)) + 12), 2] = z
    s = vid(8, 2)                                            # (0, -5)
    corners = (vid(6, 10), vid(10, 10))                      # (-1, -1), (1, -1)
    # drop the vertices inside the hole (no face uses them)
    used = np.unique(F)
    remap = -np.ones(len(V), dtype=np.int64)
    remap[used] = np.arange(used.size)
    return V[used], remap[F].astype(np.int32), int(remap[s]), int(remap[v]), tuple(int(remap[c]) for c in corners)


@pytest.fixture(scope="module")
def pch():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("needs a GPU")
    import __graft_entry__
    __graft_entry__.build()
    from paper_1305_1293_gb300 import pch as p
    return p


@pytest.mark.parametrize("k,hops", [(1, 1), (4, 1), (64, 4), (24576, 32)])
def test_tied_saddle_on_symmetry_line(pch, oracle_lib, k, hops):
    V, F, s, v, (corner_l, corner_r) = tie_mesh()
    th, pseudo = oracle_lib.vertex_angles(V, F)
    assert pseudo[v] and th[v] > 2 * np.pi + 0.1              # a strong saddle
    ref, _ = oracle_lib.geodesic(V, F, s)
    assert np.all(np.isfinite(ref))
    # the two paths to v around the hole's upper corners have equal length, and v's
    # distance is reached through them (not straight from the source)
    assert abs(ref[corner_l] - ref[corner_r]) <= 1e-12 * ref[corner_l]
    assert ref[v] > np.linalg.norm(V[v] - V[s]) + 0.1
    mesh = pch.Mesh(V, F)
    got, st = pch.solve(mesh, s, stats=True, k=k, hops=hops, max_iters=1 << 22)
    mesh.close()
    assert np.all(np.isfinite(got))
    err = float(np.max(np.abs(got - ref) / np.maximum(ref, 1e-300)))
    print(f"k={k} hops={hops}: max rel err {err:.2e}, fans {st['fans']}, tie fans {st['fan_ties']}")
    assert err < TOL
