"""The selection controller as the solver runs it (rows a8 and a9 of the hot path).

k_tau computes the frontier features of every instance at every iteration and, under
PCH_CONTROL_LEARNED, runs the network on them to pick the iteration's window count k.
PCH_FLAG_TRACE records both; pch_trace_fetch returns them.  These tests check

* the features of the first iteration after the source's fan against a CPU restatement
  of their definition from the mesh geometry (the pool then holds exactly the source's
  fan windows, whose keys are the distances from the source to the opposite edges);
* properties every trace row must have (constant mesh features, the iteration counter,
  a cumulative histogram ending at 1, pending counts consistent between two features);
* the k every learned iteration used against the FP64 network of oracle/mlp_oracle.py
  evaluated on the same features: k = floor(2^(24 y)) for an output y in [8/24, 26/24],
  else the plain k;
* that a learned solve without installed weights runs the plain control (in a fresh
  process), and that learned solves give the exact field.
"""
import math
import os
import subprocess
import sys

import numpy as np
import pytest

from oracle import mlp_oracle as mo
from paper_1305_1293_gb300 import meshgen as mg

pytestmark = pytest.mark.gpu
ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module")
def pch():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("needs a GPU")
    import __graft_entry__
    __graft_entry__.build()
    from paper_1305_1293_gb300 import pch as p
    yield p
    p.load_controller()           # leave the trained weights installed for later tests


def _mean_half_edge_length(m):
    v, f = m.vertices, m.faces
    return float(np.mean(np.concatenate([np.linalg.norm(v[f[:, (i + 1) % 3]] - v[f[:, i]], axis=1)
                                         for i in range(3)])))


def _point_segment_distance(p, a, b):
    ab = b - a
    t = np.clip(np.dot(p - a, ab) / np.dot(ab, ab), 0.0, 1.0)
    return float(np.linalg.norm(p - (a + t * ab)))


def _expected_first_features(m, s):
    """The 24 features at the first iteration with a non-empty pool, from their
    definition: the pool holds one window per face around the (interior) source s, on
    the edge opposite s, with key = distance from s to that edge; the histogram
    reference is 0; the previous iteration selected nothing."""
    keys = []
    for f in m.faces[np.any(m.faces == s, axis=1)]:
        i = int(np.nonzero(f == s)[0][0])
        a, b = m.vertices[f[(i + 1) % 3]], m.vertices[f[(i + 2) % 3]]
        keys.append(_point_segment_distance(m.vertices[s], a, b))
    keys = np.array(keys)
    n = keys.size
    lbar = _mean_half_edge_length(m)
    t = keys / lbar
    x = np.zeros(24)
    x[0] = math.log2(1 + n) / 20
    # group j of the 16-bin octaves: (key - ref) / lbar below (2^(j+1) - 1) / 4
    edges = (2.0 ** np.arange(1, 17) - 1.0) / 4.0
    x[1:17] = [(t < e).sum() / n for e in edges]
    x[17] = math.log2(m.nf) / 24
    x[18] = math.log2(lbar) / 8
    x[19] = math.log2(1 + 1) / 16
    x[20] = 0.0
    x[21] = 0.0
    x[22] = math.log2(1 + n / m.nf) / 8
    x[23] = 1.0
    # no key may sit on a group boundary, where FP32 rounding could move it across
    margin = float(np.min(np.abs(t[:, None] / edges[None, :] - 1.0)))
    return x, margin


@pytest.mark.parametrize("case", ["icosphere", "geosphere", "torus"])
def test_first_iteration_features(pch, case):
    m = {"icosphere": lambda: mg.icosphere(3, 0.02, seed=41),
         "geosphere": lambda: mg.geodesic_sphere(13, 0.02, seed=42),
         "torus": lambda: mg.torus(40, 14, seed=43)}[case]()
    mesh = pch.Mesh(m.vertices, m.faces)
    checked = 0
    for s in mg.pick_sources(m, 6, 77):
        want, margin = _expected_first_features(m, int(s))
        if margin < 1e-5:
            continue
        pch.solve(mesh, int(s), flags=pch.FLAG_TRACE)
        feats, _ = pch.trace_fetch(mesh)
        assert feats.shape[0] >= 2
        np.testing.assert_allclose(feats[0].astype(np.float64), want, rtol=2e-6, atol=2e-6)
        checked += 1
    mesh.close()
    assert checked >= 3


def _check_trace_rows(m, feats):
    lbar = _mean_half_edge_length(m)
    n = feats.shape[0]
    assert n >= 3
    np.testing.assert_allclose(feats[:, 17], math.log2(m.nf) / 24, rtol=1e-6)
    np.testing.assert_allclose(feats[:, 18], math.log2(lbar) / 8, rtol=1e-5, atol=1e-6)
    assert np.all(feats[:, 23] == 1.0)
    it = 2.0 ** (16 * feats[:, 19].astype(np.float64)) - 1
    assert np.allclose(it, np.round(it), atol=1e-3 * np.maximum(1, it))
    assert np.all(np.diff(np.round(it)) >= 1) and round(it[0]) == 1
    cum = feats[:, 1:17]
    assert np.all(np.diff(cum, axis=1) >= 0) and np.all(cum >= 0)
    assert np.all(cum[:, -1] == 1.0)                  # every pending window in some bin
    npend = 2.0 ** (20 * feats[:, 0].astype(np.float64)) - 1
    np.testing.assert_allclose(feats[:, 22], np.log2(1 + npend / m.nf) / 8, rtol=1e-4, atol=1e-6)
    assert np.all(feats[:, 20] >= 0) and np.all(feats[:, 21] >= 0)
    assert np.all(np.diff(feats[:, 21]) >= -1e-6)    # the reference (nearest key) never falls


def test_trace_row_properties(pch):
    m = mg.terrain(40, 36, seed=44)
    mesh = pch.Mesh(m.vertices, m.faces)
    pch.solve(mesh, mg.terrain_center(40, 36), k=512, hops=4, flags=pch.FLAG_TRACE)
    feats, chosen = pch.trace_fetch(mesh)
    mesh.close()
    _check_trace_rows(m, feats)
    assert np.allclose(chosen, math.log2(512) / 24, rtol=1e-6)


def _random_controller(seed):
    """Weights whose outputs stay mostly inside the controller's range [12/24, 1], so that
    most iterations take the network's k unclamped."""
    from paper_1305_1293_gb300.meshgen import SplitMix64
    p = mo.init_params(seed) * 0.5
    q = mo.unpack(p)
    q["W4"] = SplitMix64(seed + 1).normal(mo.N_HIDDEN) * 0.2
    q["b1"] = np.full(mo.N_HIDDEN, 0.05)
    q["b4"] = np.array([0.7])
    return mo.pack(q).astype(np.float32)


def _check_learned_choices(feats, chosen, params, plain_k):
    """Every row's k against the FP64 network on the same features."""
    y = mo.forward(params.astype(np.float64), feats.astype(np.float64))[0]
    lk = 24.0 * chosen.astype(np.float64)             # log2 of the k used
    used_net = 0
    delta = 24 * 1e-4                                 # FP32 network vs FP64: |dy| <= 1e-4
    for j in range(len(y)):
        a = 24.0 * y[j]
        if not math.isfinite(a):
            assert abs(lk[j] - math.log2(plain_k)) < 1e-5, (j, a, lk[j])
        elif 12 + delta <= a <= 24 - delta:
            # k = floor(2^(24 y)) with y within delta of the FP64 value
            assert math.log2(2.0 ** (a - delta) - 1) - 1e-5 <= lk[j] <= a + delta + 1e-5, (j, a, lk[j])
            used_net += 1
        elif a < 12 - delta or a > 24 + delta:
            # clamped to the trained range: exactly 2^12 or 2^24
            assert abs(lk[j] - (12.0 if a < 12 else 24.0)) < 1e-5, (j, a, lk[j])
            used_net += 1
    return used_net


@pytest.mark.parametrize("seed", [3, 8])
def test_in_solve_inference_matches_oracle(pch, oracle_lib, seed):
    """The MLP inference inside k_tau (block-cooperative, FP32) against the FP64 network."""
    params = _random_controller(seed)
    pch.mlp_set_weights(params)
    for m, s in ((mg.torus(90, 30, seed=45), 17), (mg.terrain(48, 40, seed=46), mg.terrain_center(48, 40))):
        mesh = pch.Mesh(m.vertices, m.faces)
        d = pch.solve(mesh, s, control=pch.CONTROL_LEARNED, flags=pch.FLAG_TRACE)
        feats, chosen = pch.trace_fetch(mesh)
        mesh.close()
        _check_trace_rows(m, feats)
        assert _check_learned_choices(feats, chosen, params, 24576) >= 0.8 * len(chosen)
        ref, _ = oracle_lib.geodesic(m.vertices, m.faces, s)
        assert np.max(np.abs(d - ref) / np.maximum(ref, 1e-300)) < 1e-9


def test_trained_controller_inference_matches_oracle(pch):
    """The shipped weights, in solve, against the FP64 network."""
    path = os.path.join(ROOT, "paper_1305_1293_gb300", "controller_weights.npy")
    if not os.path.exists(path):
        pytest.skip("no trained weights")
    params = np.load(path).astype(np.float32)
    pch.mlp_set_weights(params)
    m = mg.torus(200, 60, seed=47)
    mesh = pch.Mesh(m.vertices, m.faces)
    pch.solve(mesh, 5, control=pch.CONTROL_LEARNED, flags=pch.FLAG_TRACE)
    feats, chosen = pch.trace_fetch(mesh)
    mesh.close()
    _check_trace_rows(m, feats)
    _check_learned_choices(feats, chosen, params, 24576)


def test_learned_without_weights_runs_plain():
    """In a fresh process no weights are installed: a learned solve runs the plain control
    (every iteration uses the plain k) and gives the same exact field."""
    code = (
        "import sys, math, numpy as np; sys.path.insert(0, %r)\n"
        "from paper_1305_1293_gb300 import pch, meshgen as mg\n"
        "m = mg.icosphere(3, 0.02, seed=7); h = pch.Mesh(m.vertices, m.faces)\n"
        "a = pch.solve(h, 3, control=pch.CONTROL_LEARNED, k=1000, flags=pch.FLAG_TRACE)\n"
        "f, c = pch.trace_fetch(h)\n"
        "b = pch.solve(h, 3, k=1000)\n"
        "assert len(c) > 2 and np.allclose(c, math.log2(1000) / 24, rtol=1e-6), c\n"
        "assert np.array_equal(a, b)\n"
        "print('plain fallback ok', len(c))\n" % ROOT)
    r = subprocess.run([sys.executable, "-c", code], capture_output=True, text=True, timeout=300)
    assert r.returncode == 0, r.stdout + r.stderr
    assert "plain fallback ok" in r.stdout
