"""Train the learned selection controller on the GPU from the plain method's own traces.

Recipe (build-side; the paper fixes k by hand, Section 5.2):
  1. Training meshes: icospheres, geodesic spheres, terrains, jittered tori and
     multi-octave spheres of 5K-1.3M faces, seeds disjoint from every benchmark
     workload (``TRAIN_SEED``), one or two random sources each.
  2. Threshold sweep: solve each with the plain control at k in ``SWEEP_K`` and record
     every iteration's frontier features (PCH_FLAG_TRACE) and the solve time.
  3. Labels: every recorded state (from every k) gets y = log2(k_best) / 24, the best k of
     that mesh: the largest one within 3% of the fastest solve (the time-vs-k curve has a
     cliff below a plateau; labels on the far side are robust to prediction error).
  4. Fit: 3 x 64 ReLU MLP, loss 0.5 mean (y_hat - y)^2, Adam with a cosine learning-rate
     decay, keeping the lowest-loss weights, using the library's pch_mlp_backward /
     pch_mlp_adam kernels (no autograd).
The weights are written to ``controller_weights.npy`` next to this file.
"""
from __future__ import annotations

import math
import os
import sys
import time

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
WEIGHTS = os.path.join(HERE, "controller_weights.npy")
TRAIN_SEED = 0x7A1E5
SWEEP_K = (4096, 16384, 65536, 262144, 1048576, 4194304, 16777216)


def training_set():
    from . import meshgen as mg
    out = []
    for i in range(3):
        s = TRAIN_SEED + i
        out += [mg.icosphere(4 + i % 2, 0.02, seed=s), mg.geodesic_sphere(40 + 30 * i, 0.02, seed=s),
                mg.terrain(96 + 64 * i, 96 + 48 * i, seed=s), mg.torus(200 + 150 * i, 60 + 40 * i, seed=s),
                mg.multi_octave_sphere(5 + i % 2, 0.05, seed=s)]
    s = TRAIN_SEED + 10
    out += [mg.terrain(320, 320, seed=s), mg.terrain(400, 360, seed=s + 1), mg.torus(700, 200, seed=s + 2),
            mg.multi_octave_sphere(7, 0.05, seed=s + 3), mg.geodesic_sphere(120, 0.02, seed=s + 4),
            mg.torus(900, 250, seed=s + 5), mg.geodesic_sphere(90, 0.05, seed=s + 6),
            mg.torus(400, 130, jitter=0.2, seed=s + 7)]
    # large meshes (0.8M-1.3M faces): where a small k multiplies the iterations
    s = TRAIN_SEED + 20
    out += [mg.multi_octave_sphere(8, 0.05, seed=s), mg.geodesic_sphere(200, 0.02, seed=s + 1),
            mg.terrain(640, 640, seed=s + 2), mg.torus(1100, 380, seed=s + 3)]
    return out


def sweep(pch, mesh_np, sources, ks=SWEEP_K):
    """Features, labels and per-k solve times of one training mesh."""
    if mesh_np.nf > 500000:
        ks = tuple(k for k in ks if k >= 262144)     # smaller k are far from best there, and slow
    elif mesh_np.nf > 100000:
        ks = tuple(k for k in ks if k >= 16384)      # k = 4096 is far from best there, and slow
    mesh = pch.Mesh(mesh_np.vertices, mesh_np.faces)
    feats, labels, times = [], [], {}
    traces = {}
    for k in ks:
        t = 0.0
        for s in sources:
            pch.solve(mesh, int(s), k=k)                      # warm the graph for this k
            _, st = pch.solve(mesh, int(s), k=k, stats=True, flags=pch.FLAG_TRACE)
            t += st["ms_total"]
            f, _ = pch.trace_fetch(mesh)
            traces.setdefault(k, []).append(f)
        times[k] = t
    mesh.close()
    t_best = min(times.values())
    k_best = max(k for k, t in times.items() if t <= 1.03 * t_best)
    for k, fl in traces.items():
        for f in fl:
            feats.append(f)
            labels.append(np.full(f.shape[0], math.log2(k_best) / 24.0, dtype=np.float32))
    return np.concatenate(feats), np.concatenate(labels), times, k_best


def init_params(pch, seed: int = 1) -> np.ndarray:
    """He initialisation (seeded splitmix stream), layer layout of include/pch.h."""
    from .meshgen import SplitMix64
    rng = SplitMix64(seed)
    nf, nh = pch.mlp_num_features(), 64
    parts = []
    for fan_in, fan_out, scale in ((nf, nh, 1.0), (nh, nh, 1.0), (nh, nh, 1.0), (nh, 1, 0.1)):
        parts.append(rng.normal(fan_in * fan_out) * math.sqrt(2.0 / fan_in) * scale)
        parts.append(np.zeros(fan_out))
    p = np.concatenate(parts).astype(np.float32)
    assert p.size == pch.mlp_num_params()
    return p


def fit(pch, X, y, epochs=3000, lr=3e-3, seed=1, log=None):
    """Full-batch Adam on the GPU with the library's kernels.  Returns (params, losses)."""
    import torch
    p = torch.from_numpy(init_params(pch, seed)).cuda()
    m = torch.zeros_like(p)
    v = torch.zeros_like(p)
    g = torch.empty_like(p)
    loss = torch.empty(1, dtype=torch.float32, device="cuda")
    xd = torch.from_numpy(np.ascontiguousarray(X, dtype=np.float32)).cuda()
    yd = torch.from_numpy(np.ascontiguousarray(y, dtype=np.float32)).cuda()
    losses = []
    best = float("inf")
    best_p = p.clone()
    for t in range(1, epochs + 1):
        pch.mlp_backward(p, xd, yd, g, loss)          # loss of the current parameters
        lt = float(loss.item())
        if lt < best:
            best = lt
            best_p.copy_(p)
        pch.mlp_adam(p, g, m, v, t, lr * 0.5 * (1.0 + math.cos(math.pi * t / epochs)))
        if t % 250 == 0 or t == 1:
            losses.append((t, lt))
            if log:
                log(f"epoch {t} loss {lt:.6f} best {best:.6f}")
    losses.append((epochs, best))
    return best_p.cpu().numpy(), losses


def main():
    sys.path.insert(0, os.path.dirname(HERE))
    import __graft_entry__
    __graft_entry__.build()
    from paper_1305_1293_gb300 import meshgen as mg, pch
    t0 = time.time()
    Xs, ys = [], []
    for mesh in training_set():
        srcs = mg.pick_sources(mesh, 2 if mesh.nf <= 100000 else 1, TRAIN_SEED + mesh.nv)
        X, y, times, kb = sweep(pch, mesh, srcs)
        print(f"{mesh.name:>18s} F={mesh.nf:8d} best k={kb:8d} " +
              " ".join(f"{k}:{t:.1f}ms" for k, t in times.items()), flush=True)
        Xs.append(X)
        ys.append(y)
    X = np.concatenate(Xs)
    y = np.concatenate(ys)
    print(f"dataset {X.shape[0]} states, sweep {time.time() - t0:.1f}s", flush=True)
    params, losses = fit(pch, X, y, log=lambda s: print(s, flush=True))
    np.save(WEIGHTS, params.astype(np.float32))
    print(f"saved {WEIGHTS}; final loss {losses[-1][1]:.5f}", flush=True)


if __name__ == "__main__":
    main()
