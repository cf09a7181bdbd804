"""Geodesic Voronoi labels (pch_voronoi) and iso-contours (pch_iso_contours) on the GPU
against the oracle (oracle/fields.py), through the C ABI.

Voronoi labels must equal the oracle's wherever the nearest source is unique by more
than the parity bar (the second-nearest source farther by over 1e-9 relative); where two
sources tie within it, the label must name one of the tied sources.  Iso-contours of a
given field must equal the oracle's exactly in their combinatorics (level, face, crossed
half-edges, order) with crossing fractions within 1e-12; the contours of the GPU's own
field must equal those of the oracle's field on every face none of whose vertex
distances lies within 1e-9 (relative) of the level."""
import numpy as np
import pytest

from oracle import fields
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


def _check_labels(lab, dist, ref_lab, D, gap):
    best = D[ref_lab.clip(0), np.arange(D.shape[1])]
    fin = np.isfinite(best)
    assert np.array_equal(lab[~fin], np.full((~fin).sum(), -1))
    rel_gap = gap / np.maximum(best, 1e-300)
    sure = fin & (rel_gap > TOL)
    assert np.array_equal(lab[sure], ref_lab[sure]), np.nonzero(lab[sure] != ref_lab[sure])
    # near ties: the label names a source within the bar of the nearest distance
    tie = fin & ~sure
    if tie.any():
        assert np.all(lab[tie] >= 0)
        dl = D[lab[tie], np.nonzero(tie)[0]]
        assert np.all(np.abs(dl - best[tie]) <= TOL * np.maximum(best[tie], 1e-300))
    ok = fin & (best > 0)
    assert np.max(np.abs(dist[ok] - best[ok]) / best[ok]) < TOL
    return int(sure.sum()), int(tie.sum())


@pytest.mark.parametrize("case", ["icosphere", "torus", "terrain", "plane"])
def test_voronoi_vs_oracle(pch, oracle_lib, case):
    m = {"icosphere": lambda: mg.icosphere(3, 0.02, seed=71),
         "torus": lambda: mg.torus(60, 20, seed=72),
         "terrain": lambda: mg.terrain(40, 32, seed=73),
         "plane": lambda: mg.flat_patch(24, jitter=0.3, seed=74)}[case]()
    sources = [int(x) for x in mg.pick_sources(m, 7, 75)]
    h = pch.Mesh(m.vertices, m.faces)
    lab, dist = pch.voronoi(h, sources)
    h.close()
    ref_lab, D, gap = fields.voronoi(m.vertices, m.faces, sources)
    sure, tie = _check_labels(lab, dist, ref_lab, D, gap)
    assert sure > 0.95 * m.nv
    assert np.all(lab[sources] == np.arange(len(sources)))
    if case == "plane":   # the Euclidean nearest site
        E = np.vstack([np.linalg.norm(m.vertices - m.vertices[s], axis=1) for s in sources])
        o = np.sort(E, axis=0)
        clear = o[1] - o[0] > TOL
        assert np.array_equal(lab[clear], np.argmin(E, axis=0)[clear])


def test_voronoi_face_points_and_unreachable(pch, oracle_lib):
    m = mg.torus(40, 14, seed=76)
    srcs = [3, 300]
    fp = [(101, (0.2, 0.5, 0.3)), (700, (1 / 3, 1 / 3, 1 / 3))]
    h = pch.Mesh(m.vertices, m.faces)
    lab, dist = pch.voronoi(h, srcs, faces=[f for f, _ in fp], barys=[b for _, b in fp])
    h.close()
    ref_lab, D, gap = fields.voronoi(m.vertices, m.faces, srcs, face_points=fp)
    _check_labels(lab, dist, ref_lab, D, gap)
    assert set(np.unique(lab)) == {0, 1, 2, 3}
    # two components: the second one is unreachable from a source on the first
    v = np.array([[0, 0, 0], [1, 0, 0], [0, 1, 0], [5, 5, 0], [6, 5, 0], [5, 6, 0]], dtype=np.float64)
    f = np.array([[0, 1, 2], [3, 4, 5]], dtype=np.int32)
    h = pch.Mesh(v, f)
    lab, dist = pch.voronoi(h, [0, 2])
    h.close()
    assert list(lab) == [0, 0, 1, -1, -1, -1] or list(lab) == [0, 1, 1, -1, -1, -1]
    assert np.all(np.isinf(dist[3:]))


def test_voronoi_batch_sized(pch, oracle_lib):
    """64 sources on the 100,820-face sphere of the multi-source workload: labels against
    the oracle's single-source fields of 8 of the sources restricted to the vertices whose
    nearest source is among them by a clear margin (oracle cost bounded)."""
    meshes, srcs = mg.workload("multisrc", "full")
    m = meshes[0]
    sources = [int(s) for s in srcs[0]]
    h = pch.Mesh(m.vertices, m.faces)
    lab, dist = pch.voronoi(h, sources, k=24576, hops=4, block=256)
    h.close()
    assert np.all(lab >= 0)
    assert np.all(lab[sources] == np.arange(len(sources)))
    # each vertex's label names a source at exactly the field's distance: the label's own
    # single-source field, for 4 labels, from the oracle
    for j in (0, 9, 33, 63):
        Dj, _ = oracle_lib.geodesic(m.vertices, m.faces, sources[j])
        mine = lab == j
        assert mine.sum() > 100
        assert np.max(np.abs(dist[mine] - Dj[mine]) / np.maximum(Dj[mine], 1e-300)) < TOL
        # and no vertex labelled otherwise is clearly nearer to source j
        other = ~mine
        assert np.all(Dj[other] >= dist[other] * (1 - TOL))


def _segs_from_gpu(arr):
    return [(int(r["level"]), int(r["face"]), (int(r["half_edge"][0]), float(r["t"][0])),
             (int(r["half_edge"][1]), float(r["t"][1]))) for r in arr]


@pytest.mark.parametrize("case", ["icosphere", "terrain", "torus"])
def test_contours_of_a_given_field(pch, oracle_lib, case):
    m = {"icosphere": lambda: mg.icosphere(4, 0.02, seed=81),
         "terrain": lambda: mg.terrain(64, 48, seed=82),
         "torus": lambda: mg.torus(80, 30, seed=83)}[case]()
    ref, _ = oracle_lib.geodesic(m.vertices, m.faces, 5)
    levels = list(np.quantile(ref, [0.05, 0.3, 0.5, 0.77, 0.99]))
    h = pch.Mesh(m.vertices, m.faces)
    got = _segs_from_gpu(pch.iso_contours(h, ref, levels))
    want = fields.iso_contours(m.faces, ref, levels)
    assert len(got) == len(want) > 0
    for g, w in zip(got, want):
        assert g[:2] == w[:2] and g[2][0] == w[2][0] and g[3][0] == w[3][0], (g, w)
        assert abs(g[2][1] - w[2][1]) <= 1e-12 and abs(g[3][1] - w[3][1]) <= 1e-12, (g, w)
    # the same from a device-resident field, and a truncated copy
    import torch
    dd = torch.from_numpy(ref).cuda()
    got_d = _segs_from_gpu(pch.iso_contours(h, dd, levels))
    assert got_d == got
    part = _segs_from_gpu(pch.iso_contours(h, ref, levels, capacity=17))
    assert part == got[:17]
    h.close()


def test_contours_of_the_gpu_field(pch, oracle_lib):
    m = mg.terrain(80, 80, seed=84)
    s = mg.terrain_center(80, 80)
    h = pch.Mesh(m.vertices, m.faces)
    d = pch.solve(h, s)
    ref, _ = oracle_lib.geodesic(m.vertices, m.faces, s)
    levels = [5.0, 12.5, 20.0, 31.0]
    got = {(g[0], g[1]): g for g in _segs_from_gpu(pch.iso_contours(h, d, levels))}
    want = {(w[0], w[1]): w for w in fields.iso_contours(m.faces, ref, levels)}
    h.close()
    near = set()
    for li, L in enumerate(levels):
        close = np.abs(ref - L) <= TOL * L
        for f in np.nonzero(close[m.faces].any(1))[0]:
            near.add((li, int(f)))
    assert set(got) - near == set(want) - near
    for k in set(want) - near:
        g, w = got[k], want[k]
        assert g[2][0] == w[2][0] and g[3][0] == w[3][0]
        for (hg, tg), (hw, tw) in ((g[2], w[2]), (g[3], w[3])):
            f, i = divmod(hg, 3)
            a, b = ref[m.faces[f, i]], ref[m.faces[f, (i + 1) % 3]]
            # |dt| from a 1e-9 relative change of the three values involved
            bound = 4 * TOL * max(abs(a), abs(b), levels[k[0]]) / abs(b - a)
            assert abs(tg - tw) <= bound + 1e-12, (k, tg, tw, bound)


def test_contours_edge_cases(pch):
    m = mg.icosphere(2, 0.0, seed=0)
    h = pch.Mesh(m.vertices, m.faces)
    d = np.linalg.norm(m.vertices - m.vertices[0], axis=1)
    assert len(pch.iso_contours(h, d, [-1.0, 10.0])) == 0
    d2 = d.copy()
    d2[5] = np.inf
    segs = _segs_from_gpu(pch.iso_contours(h, d2, [float(np.median(d))]))
    assert segs == fields.iso_contours(m.faces, d2, [float(np.median(d))])
    with pytest.raises(pch.PchError) as e:
        pch.iso_contours(h, d, [np.inf])
    assert e.value.status == pch.PCH_ERR_INVALID_ARG
    h.close()
