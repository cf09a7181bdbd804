"""GPU parity: the CUDA path against the CPU oracle and closed forms, through the C ABI.

Tolerance: max relative error 1e-9 over vertices with finite distance, the source
exactly 0, infinities identical (the bar of the workload definition).  Both sides are
exact methods in FP64, so agreement is normally ~1e-13; 1e-9 leaves room for the
different rounding order of the (px, py) and (d0, d1) window representations.
"""
import math

import numpy as np
import pytest

import bruteforce as bf
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


def max_rel(got, ref):
    fin = np.isfinite(ref)
    assert np.array_equal(np.isfinite(got), fin), "finiteness differs"
    r = ref[fin]
    return float(np.max(np.abs(got[fin] - r) / np.maximum(r, 1e-300))) if r.size else 0.0


def gpu_solve(pch, m, src=None, **kw):
    mesh = pch.Mesh(m.vertices, m.faces)
    try:
        return pch.solve(mesh, src, stats=True, **kw)
    finally:
        mesh.close()


# ------------------------------------------------------------------ closed forms
def test_plane_euclidean(pch):
    m = mg.flat_patch(30, jitter=0.3, seed=21)
    for s in (0, 465, 960):
        d, _ = gpu_solve(pch, m, s)
        ex = np.linalg.norm(m.vertices - m.vertices[s], axis=1)
        assert d[s] == 0.0
        assert np.max(np.abs(d - ex)) < 1e-12


def test_plane_face_point(pch):
    m = mg.flat_patch(20, jitter=0.25, seed=22)
    for f, b in ((100, (0.2, 0.3, 0.5)), (401, (1 / 3, 1 / 3, 1 / 3))):
        p = sum(bb * m.vertices[m.faces[f, k]] for k, bb in enumerate(b))
        mesh = pch.Mesh(m.vertices, m.faces)
        d = pch.solve(mesh, face=f, bary=b)
        mesh.close()
        assert np.max(np.abs(d - np.linalg.norm(m.vertices - p, axis=1))) < 1e-12


def test_prism_and_pyramid(pch):
    m, s, z, perim = mg.prism_tube(13, 9, height=2.0, seed=3)
    for src in (0, m.nv // 2):
        d, _ = gpu_solve(pch, m, src)
        ex = np.min([np.hypot(s - s[src] + k * perim, z - z[src]) for k in (-1, 0, 1)], axis=0)
        assert max_rel(d, ex + (ex == 0)) < 1e-11 or np.max(np.abs(d - ex)) < 1e-12
    m, r, th, Theta = mg.pyramid(7, 6)
    d, _ = gpu_solve(pch, m, 0)
    assert np.max(np.abs(d[1:] - r[1:]) / r[1:]) < 1e-12


def test_cube_and_tetra_vs_bruteforce(pch):
    for m in (mg.cube(2), mg.tetrahedron(3), mg.torus(6, 4, seed=6), mg.octahedron(0.1, 2, 1)):
        for s in range(0, m.nv, max(1, m.nv // 3)):
            d, _ = gpu_solve(pch, m, s)
            assert max_rel(d, bf.geodesic(m.vertices, m.faces, s)) < TOL


# ------------------------------------------------------------------ oracle parity, reduced workloads
SMALL = ["icosphere", "terrain", "torus", "multisrc", "large"]


@pytest.mark.parametrize("name", SMALL)
def test_parity_reduced_workloads(pch, oracle_lib, name):
    meshes, srcs = mg.workload(name, "small")
    m = meshes[0]
    mesh = pch.Mesh(m.vertices, m.faces)
    for s in srcs[0][:3]:
        ref, ost = oracle_lib.geodesic(m.vertices, m.faces, int(s))
        got, st = pch.solve(mesh, int(s), stats=True)
        assert got[int(s)] == 0.0
        assert max_rel(got, ref) < TOL, (name, int(s))
        # window count sanity: the parallel method creates more windows than the
        # sequential priority-queue oracle, but not wildly more (Table `tab:speedup`)
        assert st["windows_propagated"] > 0
    mesh.close()


def test_parity_icosphere_full(pch, oracle_lib):
    meshes, srcs = mg.workload("icosphere", "full")
    m = meshes[0]
    ref, _ = oracle_lib.geodesic(m.vertices, m.faces, 0)
    for loop in (pch.LOOP_GRAPH, pch.LOOP_HOST):
        got, st = gpu_solve(pch, m, 0, loop=loop)
        assert max_rel(got, ref) < TOL
        assert st["iterations"] > 1


@pytest.mark.parametrize("k,hops", [(1, 1), (7, 1), (256, 1), (4096, 1), (1 << 22, 1), (1, 8), (64, 2),
                                    (4096, 4), (1 << 22, 16)])
def test_result_independent_of_k_and_hops(pch, oracle_lib, k, hops):
    """Section 4.3 / Remark 2: any selection order gives the exact field."""
    m = mg.terrain(24, 20, seed=31)
    s = mg.terrain_center(24, 20)
    ref, _ = oracle_lib.geodesic(m.vertices, m.faces, s)
    got, st = gpu_solve(pch, m, s, k=k, hops=hops, max_iters=1 << 22)
    assert max_rel(got, ref) < TOL
    if hops == 1:
        assert st["windows_chained"] == 0


@pytest.mark.parametrize("k", [3, 256, 24576])
def test_strided_selection_exact(pch, oracle_lib, k):
    """Section 5.1's approximate k-selection (Remark 2): the selection is approximate,
    the field is exact; every selected window propagates one hop."""
    m = mg.terrain(24, 20, seed=31)
    s = mg.terrain_center(24, 20)
    ref, _ = oracle_lib.geodesic(m.vertices, m.faces, s)
    got, st = gpu_solve(pch, m, s, k=k, control=pch.CONTROL_STRIDED, hops=8, max_iters=1 << 22)
    assert max_rel(got, ref) < TOL
    assert st["windows_chained"] == 0 and st["iterations"] > 1


def test_strided_selection_batch_and_host_loop(pch, oracle_lib):
    meshes, srcs = mg.workload("batch", "small")
    hs = [pch.Mesh(m.vertices, m.faces) for m in meshes]
    for loop in (pch.LOOP_GRAPH, pch.LOOP_HOST):
        outs = pch.solve_batch(hs, [int(s[0]) for s in srcs], control=pch.CONTROL_STRIDED, k=4096, loop=loop)
        for m, s, got in zip(meshes, srcs, outs):
            ref, _ = oracle_lib.geodesic(m.vertices, m.faces, int(s[0]))
            assert max_rel(got, ref) < TOL
    for x in hs:
        x.close()


def test_unknown_control_rejected(pch):
    m = mg.icosphere(1)
    mesh = pch.Mesh(m.vertices, m.faces)
    with pytest.raises(pch.PchError) as e:
        pch.solve(mesh, 0, control=7)
    assert e.value.status == pch.PCH_ERR_INVALID_ARG
    mesh.close()


@pytest.mark.parametrize("flags", ["EDGE_SORT", "EDGE_SORT|NO_TRIM", "FULL_FAN", "EDGE_SORT|FULL_FAN"])
def test_variants_same_result(pch, oracle_lib, flags):
    """Per-edge trimming (after the edge sort) and the fanned-area restriction remove only
    useless windows."""
    fl = 0
    for f in flags.split("|"):
        fl |= getattr(pch, "FLAG_" + f)
    for m, s in ((mg.geodesic_sphere(9, 0.02, seed=5), 3), (mg.terrain(20, 17, seed=6, amp_range=(1, 6)), 180)):
        ref, _ = oracle_lib.geodesic(m.vertices, m.faces, s)
        a, sa = gpu_solve(pch, m, s)
        b, sb = gpu_solve(pch, m, s, flags=fl)
        assert max_rel(a, ref) < TOL and max_rel(b, ref) < TOL


def test_face_point_source_vs_oracle(pch, oracle_lib):
    m = mg.icosphere(3, 0.02, seed=41)
    for f, b in ((17, (0.1, 0.6, 0.3)), (900, (0.5, 0.25, 0.25))):
        ref, _ = oracle_lib.geodesic(m.vertices, m.faces, face=f, bary=np.array(b))
        mesh = pch.Mesh(m.vertices, m.faces)
        got = pch.solve(mesh, face=f, bary=b)
        mesh.close()
        assert max_rel(got, ref) < TOL


def test_multi_source_vs_oracle(pch, oracle_lib):
    m = mg.torus(40, 14, seed=9)
    srcs = [3, 200, 511]
    ref, _ = oracle_lib.geodesic(m.vertices, m.faces, sources=srcs)
    mesh = pch.Mesh(m.vertices, m.faces)
    got = pch.solve_multi(mesh, srcs)
    mesh.close()
    assert max_rel(got, ref) < TOL
    assert np.all(got[srcs] == 0.0)


def test_batch_vs_oracle(pch, oracle_lib):
    meshes, srcs = mg.workload("batch", "small")
    hs = [pch.Mesh(m.vertices, m.faces) for m in meshes]
    outs, st = pch.solve_batch(hs, [int(s[0]) for s in srcs], stats=True)
    for m, s, got in zip(meshes, srcs, outs):
        ref, _ = oracle_lib.geodesic(m.vertices, m.faces, int(s[0]))
        assert max_rel(got, ref) < TOL
    # many sources on one mesh: instances share the mesh handle
    m = mg.geodesic_sphere(8, 0.02, seed=2)
    h = pch.Mesh(m.vertices, m.faces)
    srcv = [1, 50, 300, 600]
    outs = pch.solve_batch([h] * 4, srcv)
    for s, got in zip(srcv, outs):
        assert max_rel(got, oracle_lib.geodesic(m.vertices, m.faces, s)[0]) < TOL
    for x in hs + [h]:
        x.close()


def test_device_output_and_stream(pch, oracle_lib):
    import torch
    m = mg.icosphere(3, 0.02, seed=7)
    mesh = pch.Mesh(m.vertices, m.faces)
    s = torch.cuda.Stream()
    out = torch.full((m.nv,), -1.0, dtype=torch.float64, device="cuda")
    with torch.cuda.stream(s):
        pch.solve(mesh, 5, out=out, stream=s)
    s.synchronize()
    ref, _ = oracle_lib.geodesic(m.vertices, m.faces, 5)
    assert max_rel(out.cpu().numpy(), ref) < TOL
    mesh.close()


# ------------------------------------------------------------------ edge cases
def test_single_triangle_and_disconnected(pch):
    v = np.array([[0, 0, 0], [1, 0, 0], [0, 1, 0], [5, 5, 0], [6, 5, 0], [5, 6, 0]], dtype=np.float64)
    f = np.array([[0, 1, 2], [3, 4, 5]], dtype=np.int32)
    d, _ = gpu_solve(pch, mg.Mesh(v, f), 0)
    assert d[0] == 0.0 and abs(d[1] - 1) < 1e-15 and abs(d[2] - 1) < 1e-15
    assert np.all(np.isinf(d[3:]))


def test_boundary_source_and_concave_boundary(pch, oracle_lib):
    # an L-shaped flat patch: geodesics bend around the reflex boundary corner
    m = mg.flat_patch(12, jitter=0.2, seed=8)
    c = m.vertices[m.faces].mean(1)
    keep = ~((c[:, 0] > 0.5) & (c[:, 1] > 0.5))
    f = m.faces[keep]
    used = np.unique(f)
    remap = -np.ones(m.nv, dtype=np.int64)
    remap[used] = np.arange(used.size)
    mm = mg.Mesh(m.vertices[used], remap[f].astype(np.int32))
    for s in (0, mm.nv - 1):
        ref, _ = oracle_lib.geodesic(mm.vertices, mm.faces, s)
        got, _ = gpu_solve(pch, mm, s)
        assert max_rel(got, ref) < TOL


@pytest.mark.parametrize("bad", ["nonmanifold", "degenerate", "flipped"])
def test_invalid_meshes_rejected(pch, bad):
    m = mg.flat_patch(3, jitter=0.0)
    f = m.faces.copy()
    v = m.vertices.copy()
    if bad == "nonmanifold":
        f = np.concatenate([f, f[:1]])
        want = pch.PCH_ERR_NONMANIFOLD
    elif bad == "degenerate":
        v[5] = (v[4] + v[6]) / 2           # collapse: vertex 5 on the segment 4-6
        f = np.array([[4, 5, 6]], dtype=np.int32)
        want = pch.PCH_ERR_DEGENERATE
    else:
        f[0] = f[0][::-1]
        want = pch.PCH_ERR_NONMANIFOLD
    with pytest.raises(pch.PchError) as e:
        pch.Mesh(v, f)
    assert e.value.status == want


def test_iteration_cap_reports_timeout(pch):
    m = mg.icosphere(3, 0.02, seed=7)
    mesh = pch.Mesh(m.vertices, m.faces)
    with pytest.raises(pch.PchError) as e:
        pch.solve(mesh, 0, k=8, max_iters=3)
    assert e.value.status == pch.PCH_ERR_TIMEOUT
    got = pch.solve(mesh, 0)          # the handle stays usable
    assert got[0] == 0.0
    mesh.close()


def test_mesh_info(pch):
    m = mg.terrain(10, 8, seed=1)
    mesh = pch.Mesh(m.vertices, m.faces)
    info = mesh.info()
    assert info["n_vertices"] == m.nv and info["n_faces"] == m.nf
    assert info["n_boundary_half_edges"] == 2 * (10 + 8)
    mesh.close()


# ------------------------------------------------------------------ full-size workloads
def _edge_graph_upper(m, s):
    from scipy.sparse import coo_matrix
    from scipy.sparse.csgraph import dijkstra
    f = m.faces
    e = np.concatenate([f[:, [0, 1]], f[:, [1, 2]], f[:, [2, 0]]])
    w = np.linalg.norm(m.vertices[e[:, 0]] - m.vertices[e[:, 1]], axis=1)
    g = coo_matrix((w, (e[:, 0], e[:, 1])), shape=(m.nv, m.nv)).tocsr()
    return dijkstra(g, directed=False, indices=s)


def _full_size_checks(pch, oracle_lib, m, s, n_near=64, fixture=None, **opts):
    """Invariants on every vertex, then parity: against the stored full field of the
    oracle on every vertex when a fixture is given, else on the n_near vertices nearest
    the source (which the oracle finalises early: its keys never decrease)."""
    mesh = pch.Mesh(m.vertices, m.faces)
    got, st = pch.solve(mesh, s, stats=True, **opts)
    mesh.close()
    assert got[s] == 0.0 and np.all(np.isfinite(got))
    chord = np.linalg.norm(m.vertices - m.vertices[s], axis=1)
    assert np.all(got >= chord * (1 - 1e-12))
    assert np.all(got <= _edge_graph_upper(m, s) * (1 + 1e-12))
    e = np.concatenate([m.faces[:, [0, 1]], m.faces[:, [1, 2]]])
    le = np.linalg.norm(m.vertices[e[:, 0]] - m.vertices[e[:, 1]], axis=1)
    assert np.all(np.abs(got[e[:, 0]] - got[e[:, 1]]) <= le * (1 + 1e-12) + 1e-14)
    if fixture is not None:
        import make_fullfield as mf
        ref, src, fsha, probe, _ = mf.load(fixture)
        assert src == s and mf.same_mesh(m, fsha, probe), "the stored field belongs to another mesh"
        # stored values carry a relative rounding of at most 2^-37 (about 7e-12)
        err = max_rel(got, ref)
        print(f"{fixture}: full-field max relative error {err:.3e} over {m.nv} vertices")
        assert err < TOL
        return st
    order = np.argsort(got)
    near = order[1:1 + n_near]
    ref, _ = oracle_lib.geodesic(m.vertices, m.faces, s, targets=near)
    assert max_rel(got[near], ref[near]) < TOL
    return st


BENCH_OPTS = {"k": 393216, "hops": 32, "block": 64}     # the terrain's tuned configuration


@pytest.mark.parametrize("opts", [{}, BENCH_OPTS], ids=["defaults", "tuned"])
def test_full_terrain_512(pch, oracle_lib, opts):
    """The 512 x 512 terrain, every vertex against the oracle's stored full field."""
    meshes, srcs = mg.workload("terrain", "full")
    st = _full_size_checks(pch, oracle_lib, meshes[0], int(srcs[0][0]), fixture="terrain512_centre", **opts)
    assert st["windows_propagated"] > meshes[0].nf


def test_full_torus_sources(pch, oracle_lib):
    """The 1M-face torus from its first source, every vertex against the stored field."""
    meshes, srcs = mg.workload("torus", "full")
    _full_size_checks(pch, oracle_lib, meshes[0], int(srcs[0][0]), fixture="torus1250x400_src0")


def test_fast_reciprocal_and_sqrt_within_few_ulp(pch):
    """The Newton-Raphson 1/x and sqrt used by the propagation kernel stay within a few
    ulp of CUDA's IEEE operations over 1e-30..1e30 and both signs (reciprocal)."""
    import torch
    rng = np.random.default_rng(5)
    e = rng.uniform(-30, 30, 200000)
    x = (10.0 ** e) * rng.choice([-1.0, 1.0], e.size)
    x = np.concatenate([x, [1.0, 2.0, 0.5, 3.0, 1e-31, 1e31, 7.0e-300]])
    ur, us = pch.selftest_math(torch.from_numpy(x).cuda())
    assert ur <= 2 and us <= 2, (ur, us)


def _sampled_batch_checks(pch, oracle_lib, meshes, inst, outs, n_near, n_oracle, upper_every=0):
    """Invariants on every vertex of every instance of a batched solve, at the parity bar
    (1e-9 relative: the bound the workload sets for every distance), and the oracle on
    the n_near vertices nearest the source of n_oracle instances spread over the batch."""
    step = max(1, len(inst) // max(1, n_oracle))
    worst_chord = worst_lip = 0.0
    for j, ((mi, s), got) in enumerate(zip(inst, outs)):
        m = meshes[mi]
        assert got[s] == 0.0 and np.all(np.isfinite(got)), (j, int(np.sum(~np.isfinite(got))))
        chord = np.linalg.norm(m.vertices - m.vertices[s], axis=1)
        assert np.all(got >= chord * (1 - TOL)), (j, float(np.min(got / np.maximum(chord, 1e-300))))
        worst_chord = max(worst_chord, float(np.max(1.0 - got[chord > 0] / chord[chord > 0])))
        e = np.concatenate([m.faces[:, [0, 1]], m.faces[:, [1, 2]]])
        le = np.linalg.norm(m.vertices[e[:, 0]] - m.vertices[e[:, 1]], axis=1)
        ratio = np.abs(got[e[:, 0]] - got[e[:, 1]]) / le
        assert np.all(ratio <= 1 + TOL), (j, float(np.max(ratio)))
        worst_lip = max(worst_lip, float(np.max(ratio)) - 1.0)
        if upper_every and j % upper_every == 0:
            assert np.all(got <= _edge_graph_upper(m, s) * (1 + TOL))
        if j % step == 0:
            near = np.argsort(got)[1:1 + n_near].astype(np.int32)
            ref, _ = oracle_lib.geodesic(m.vertices, m.faces, s, targets=near)
            assert max_rel(got[near], ref[near]) < TOL, (j, s)
    print(f"{len(inst)} instances: largest chord excess {worst_chord:.2e}, largest edge Lipschitz excess "
          f"{worst_lip:.2e} (relative)")


def test_full_batch_256_meshes(pch, oracle_lib):
    """The 256-mesh workload at full size in one batched solve (plain control with the
    tuned chaining): every vertex of the 16 smallest instances against the oracle's full
    field, invariants on every instance, sampled oracle parity on 16 more."""
    meshes, srcs = mg.workload("batch", "full")
    hs = [pch.Mesh(m.vertices, m.faces) for m in meshes]
    inst = [(i, int(s[0])) for i, s in enumerate(srcs)]
    outs = pch.solve_batch([hs[i] for i, _ in inst], [s for _, s in inst], k=24576, hops=16, block=128)
    _sampled_batch_checks(pch, oracle_lib, meshes, inst, outs, n_near=150, n_oracle=16, upper_every=32)
    smallest = sorted(range(len(inst)), key=lambda j: meshes[inst[j][0]].nf)[:16]
    worst = 0.0
    for j in smallest:
        mi, s = inst[j]
        ref, _ = oracle_lib.geodesic(meshes[mi].vertices, meshes[mi].faces, s)
        worst = max(worst, max_rel(outs[j], ref))
    print(f"batch: full-field max relative error {worst:.3e} on the 16 smallest instances "
          f"({min(meshes[inst[j][0]].nf for j in smallest)}-{max(meshes[inst[j][0]].nf for j in smallest)} faces)")
    assert worst < TOL
    for h in hs:
        h.close()


def test_full_multisrc_64_sources(pch, oracle_lib):
    """64 sources on the 100,820-face sphere as one batched solve, every field checked by
    invariants and 8 of them against the oracle."""
    meshes, srcs = mg.workload("multisrc", "full")
    m = meshes[0]
    h = pch.Mesh(m.vertices, m.faces)
    inst = [(0, int(s)) for s in srcs[0]]
    outs = pch.solve_batch([h] * len(inst), [s for _, s in inst], k=24576, hops=4, block=256)
    _sampled_batch_checks(pch, oracle_lib, meshes, inst, outs, n_near=300, n_oracle=8, upper_every=16)
    h.close()


def test_full_large_32_sources(pch, oracle_lib):
    """The 5,242,880-face sphere with 32 sources in one batched solve (the largest
    workload), every field checked by invariants and 4 against the oracle."""
    meshes, srcs = mg.workload("large", "full")
    m = meshes[0]
    h = pch.Mesh(m.vertices, m.faces)
    inst = [(0, int(s)) for s in srcs[0]]
    outs = pch.solve_batch([h] * len(inst), [s for _, s in inst], k=1 << 22, hops=64, block=64)
    _sampled_batch_checks(pch, oracle_lib, meshes, inst, outs, n_near=200, n_oracle=4, upper_every=0)
    h.close()
