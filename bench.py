"""Benchmark: exact geodesic solves on the 512 x 512 synthetic terrain (524,288 faces).

One step = one complete solve (selection, propagation, organisation, events, until no
window is pending) from the centre vertex, mesh resident on the device.  Prints one
JSON line (rank 0).  `--impl reference` times the sequential CPU oracle instead, on a
bounded sample of the same workload (the oracle stops once a fixed set of vertices
nearest the source is final).

Multi-GPU (torchrun): a single solve does not shard, so every rank runs the same
workload as an independent replica ("replicas only"); value = total windows
propagated per second over all ranks, time = max over ranks.
"""
from __future__ import annotations

import argparse
import json
import os
import statistics
import subprocess
import sys
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "solve ms & windows/s vs plain PCH on same GB300 at max rel err ≤1e-9"
UNIT = "windows/s"
WORKLOAD = "terrain512: 512x512 height-field grid (263,169 V, 524,288 F), 8 sines + N(0,0.01^2), random diagonals, source = centre vertex, fp64"
# oracle samples: stop once the n vertices nearest the source are final.  The reference
# arm times one per step (about 1 s on the GPU machine's host); the bench line's cpu_baseline
# times one larger sample once (about 10-30 s of CPU work)
NEAR_SAMPLE = 8000
NEAR_SAMPLE_BASELINE = 30000
FP64_PEAK_DERIVED = 152 * 4 * 2.07e9 / 1e12   # SMs x FP64 flops/clk/SM x max clock (TFLOP/s)


def _dist_env():
    ws = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return ws, rank, local


class ClockSampler:
    """nvidia-smi clock / throttle sampling during the timed region."""
    QUERY = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,clocks_event_reasons.hw_slowdown,"
             "clocks_event_reasons.hw_thermal_slowdown,clocks_event_reasons.sw_thermal_slowdown,"
             "clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_index: int):
        self.gpu = gpu_index
        self.proc = None
        import tempfile
        self.path = os.path.join(tempfile.gettempdir(), f"pch_bench_clocks_rank{gpu_index}.csv")

    def __enter__(self):
        os.makedirs(os.path.dirname(self.path), exist_ok=True)
        try:
            self.fh = open(self.path, "w")
            self.proc = subprocess.Popen(["nvidia-smi", f"--id={self.gpu}", f"--query-gpu={self.QUERY}",
                                          "--format=csv,noheader,nounits", "-lms", "200"], stdout=self.fh,
                                         stderr=subprocess.DEVNULL)
        except Exception:
            self.proc = None
        return self

    def __exit__(self, *a):
        if self.proc:
            self.proc.terminate()
            try:
                self.proc.wait(5)
            except Exception:
                self.proc.kill()
            self.fh.close()

    def summary(self):
        try:
            rows = [r.split(",") for r in open(self.path).read().strip().splitlines() if r.strip()]
        except Exception:
            rows = []
        if not rows:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["unsampled"]}
        sm = [float(r[1]) for r in rows if r[1].strip().replace(".", "").isdigit()]
        mx = [float(r[2]) for r in rows if r[2].strip().replace(".", "").isdigit()]
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        reasons = sorted({names[i] for r in rows for i in range(4) if len(r) > 5 + i and r[5 + i].strip() == "Active"})
        return {"sm_mhz": statistics.median(sm) if sm else None, "sm_max_mhz": max(mx) if mx else None,
                "reasons": reasons, "samples": len(rows)}


def oracle_sample(m, s, n_near: int = NEAR_SAMPLE):
    """Time the CPU oracle on a bounded sample: stop once the n_near nearest vertices
    (by Euclidean distance) are final.  Returns windows/s, seconds, windows."""
    import oracle
    near = np.argsort(np.linalg.norm(m.vertices - m.vertices[s], axis=1))[:n_near]
    t = time.perf_counter()
    _, st = oracle.geodesic(m.vertices, m.faces, s, targets=near.astype(np.int32))
    dt = time.perf_counter() - t
    return st["propagated"] / dt, dt, st["propagated"]


def cpu_pch_sample(k: int = 24576):
    """The paper's CPU PCH (Section 6: rounds of the k nearest windows, unordered) against
    the sequential priority-queue oracle on the reduced terrain of the same family (48 x 48,
    4,608 faces, whole field): the window overhead of unordered rounds, which the GPU path
    shares, and the CPU rate."""
    import oracle
    from paper_1305_1293_gb300 import meshgen as mg
    meshes, srcs = mg.workload("terrain", "small")
    m, s = meshes[0], int(srcs[0][0])
    t = time.perf_counter()
    ref, st_ich = oracle.geodesic(m.vertices, m.faces, s)
    t_ich = time.perf_counter() - t
    t = time.perf_counter()
    d, st_pch = oracle.cpu_pch(m.vertices, m.faces, s, k)
    t_pch = time.perf_counter() - t
    return {"mesh": "terrain 48 x 48 (4,608 F), whole field", "k": k, "cores": 1,
            "ich_windows": st_ich["propagated"], "cpu_pch_windows": st_pch["propagated"],
            "window_ratio": st_pch["propagated"] / max(1, st_ich["propagated"]), "rounds": st_pch["rounds"],
            "ich_s": t_ich, "cpu_pch_s": t_pch, "cpu_pch_windows_per_s": st_pch["propagated"] / max(t_pch, 1e-9),
            "max_rel_diff": float(np.max(np.abs(d - ref) / np.maximum(ref, 1e-300)))}


def run_reference(args):
    ws, rank, _ = _dist_env()
    if rank != 0:
        return
    from paper_1305_1293_gb300 import meshgen as mg
    import oracle
    oracle.build()
    meshes, srcs = mg.workload("terrain", "full")
    m, s = meshes[0], int(srcs[0][0])
    for _ in range(args.warmup):
        oracle_sample(m, s)
    vals, times, wins = [], [], []
    for _ in range(args.steps):
        v, dt, w = oracle_sample(m, s)
        vals.append(v)
        times.append(dt)
        wins.append(w)
    value = sum(wins) / sum(times)
    sample = f"oracle stops once the {NEAR_SAMPLE} vertices nearest the source are final ({wins[0]} windows per step)"
    line = {"impl": "reference", "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": args.gpus,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1e3 * sum(times) / len(times),
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
            "config": {"workload": WORKLOAD + "; " + sample, "parallelism": "1 host core (sequential oracle)"},
            "cpu_baseline": {"value": value, "unit": UNIT, "cores": 1, "kind": "oracle", "sample": sample},
            "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)


def run_gpu(args):
    import torch
    ws, rank, local = _dist_env()
    torch.cuda.set_device(local)
    if ws > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl", device_id=torch.device("cuda", local))
    import __graft_entry__
    if rank == 0 or ws == 1:
        __graft_entry__.build()
    if ws > 1:
        import torch.distributed as dist
        dist.barrier()
    from paper_1305_1293_gb300 import meshgen as mg, pch

    meshes, srcs = mg.workload("terrain", "full")
    m, s = meshes[0], int(srcs[0][0])
    mesh = pch.Mesh(m.vertices, m.faces)
    stream = torch.cuda.current_stream()
    out = torch.empty(m.nv, dtype=torch.float64, device="cuda")
    flush = torch.empty(256 * 1024 * 1024 // 4, dtype=torch.float32, device="cuda")   # > L2 (129 MB)
    # plain control with the autotuned fixed k, block and hops (cache keyed by GPU and mesh)
    if args.k:
        tuned = {"k": args.k, "block": 0, "hops": args.hops}
    else:
        tuned = pch.autotune(mesh, s, cache_path=os.path.join(ROOT, "paper_1305_1293_gb300", "autotune_cache.txt"))
    sopts = {"k": tuned["k"], "block": tuned["block"], "hops": tuned["hops"],
             "loop": pch.LOOP_HOST if args.loop == "host" else pch.LOOP_GRAPH}
    opts = dict(stream=stream, **sopts)

    def step():
        return pch.solve(mesh, s, out=out, stats=True, **opts)[1]

    for _ in range(args.warmup):
        step()
    torch.cuda.synchronize()
    if ws > 1:
        torch.distributed.barrier()
    per_step, stats = [], []
    with ClockSampler(local) as clk:
        torch.cuda.synchronize()
        for _ in range(args.steps):
            flush.fill_(1.0)                       # evict L2 between timed steps
            a = torch.cuda.Event(enable_timing=True)
            b = torch.cuda.Event(enable_timing=True)
            a.record(stream)
            st = step()
            b.record(stream)
            b.synchronize()
            per_step.append(a.elapsed_time(b))
            stats.append(st)
        torch.cuda.synchronize()
    total_ms = sum(per_step)
    wins = sum(st["windows_propagated"] for st in stats)
    if ws > 1:
        import torch.distributed as dist
        t = torch.tensor([total_ms], device="cuda")
        dist.all_reduce(t, op=dist.ReduceOp.MAX)
        total_ms = float(t.item())
        w = torch.tensor([float(wins)], device="cuda")
        dist.all_reduce(w, op=dist.ReduceOp.SUM)
        wins = float(w.item())
    value = wins / (total_ms / 1e3)

    # parity of the benchmarked field on sampled vertices (oracle early stop)
    got = out.cpu().numpy()

    # per-phase device time (one profiled solve, events around every phase)
    _, pst = pch.solve(mesh, s, stats=True, flags=pch.FLAG_PROFILE, **{k: v for k, v in sopts.items() if k != "loop"})
    ph = pst["ms_phase"]
    prop_ms = ph["propagate"]
    prop_launches = pst["iterations"]
    # the paper's own setting on the same GPU and kernels: k = 24 * 2^10, one hop, chosen
    # by the histogram threshold, and by the paper's strided approximate selection
    _, paper_st = pch.solve(mesh, s, stats=True, k=24576, hops=1)
    _, strided_st = pch.solve(mesh, s, stats=True, k=24576, control=pch.CONTROL_STRIDED)
    achieved_tf = pst["prop_fp64_ops"] / (prop_ms / 1e3) / 1e12
    fp64_meas = pch.measure_fp64_peak()

    # end to end through the C ABI with host buffers (mesh upload + solve + download)
    vh = torch.from_numpy(m.vertices).pin_memory().numpy()
    fh = torch.from_numpy(m.faces).pin_memory().numpy()
    res = torch.empty(m.nv, dtype=torch.float64).pin_memory().numpy()
    e2e_ms, e2e_w = [], 0
    for i in range(max(1, args.steps // 2)):
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        mm = pch.Mesh(vh, fh)
        _, st = pch.solve(mm, s, out=res, stats=True, **sopts)
        mm.close()
        e2e_ms.append(1e3 * (time.perf_counter() - t0))
        e2e_w += st["windows_propagated"]
    e2e_value = e2e_w / (sum(e2e_ms) / 1e3)

    line = None
    if rank == 0:
        import oracle
        oracle.build()
        near = np.argsort(got)[1:201]
        ref, _ = oracle.geodesic(m.vertices, m.faces, s, targets=near.astype(np.int32))
        parity = float(np.max(np.abs(got[near] - ref[near]) / ref[near]))
        cpu_v, cpu_dt, cpu_w = oracle_sample(m, s, NEAR_SAMPLE_BASELINE)
        cpu_pch = cpu_pch_sample()
        clocks = clk.summary()
        st0 = stats[-1]
        line = {
            "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": ws, "steps": args.steps, "warmup": args.warmup,
            "ms_per_step": total_ms / args.steps, "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
            "dtype": "f64", "data": "synthetic",
            "config": {"workload": WORKLOAD, "control": "plain (fixed k)", "k": sopts["k"], "hops": sopts["hops"],
                       "block": sopts["block"], "loop": args.loop,
                       "parallelism": "replicas" if ws > 1 else "single GPU",
                       "l2": "flushed between timed steps (256 MB write); working set > L2",
                       "windows_per_solve": st0["windows_propagated"], "iterations": st0["iterations"],
                       "peak_pending": st0["peak_pending"]},
            "solve_ms": total_ms / args.steps,
            "paper_setting_solve_ms": paper_st["ms_total"],
            "paper_setting_windows": paper_st["windows_propagated"],
            "paper_strided_solve_ms": strided_st["ms_total"],
            "paper_strided_windows": strided_st["windows_propagated"],
            "parity_max_rel_err_sampled": parity,
            "roofline": {"bound": "alu", "kernel": "k_propagate", "achieved": achieved_tf,
                         "peak": FP64_PEAK_DERIVED, "unit": "TFLOP/s", "frac": achieved_tf / FP64_PEAK_DERIVED,
                         "traffic": prop_traffic(), "fp64_microbench_tflops": fp64_meas,
                         "fp64_ops_per_launch": pst["prop_fp64_ops"] / max(1, prop_launches),
                         "fp64_ops_per_window": pst["prop_fp64_ops"] / max(1, pst["windows_propagated"]),
                         "launches": prop_launches,
                         "avg_launch_us": 1e3 * prop_ms / max(1, prop_launches),
                         "phase_ms": ph, "memory_phases": phase_rooflines(pst, pst["sort_passes"])},
            "cpu_baseline": {"value": cpu_v, "unit": UNIT, "cores": 1, "kind": "oracle",
                             "sample": f"sequential oracle on the same terrain, stopped once the "
                                       f"{NEAR_SAMPLE_BASELINE} nearest vertices are final ({cpu_w} windows, "
                                       f"{cpu_dt:.1f} s)"},
            "e2e": {"value": e2e_value, "unit": UNIT, "ms_per_step": sum(e2e_ms) / len(e2e_ms),
                    "h2d_bytes_per_step": int(m.vertices.nbytes + m.faces.nbytes),
                    "d2h_bytes_per_step": int(8 * m.nv)},
            "cpu_pch_baseline": cpu_pch,
            "gpu_launches": int(sum(st["kernel_launches"] for st in stats)),
            "clocks": clocks,
        }
        print(json.dumps(line), flush=True)
    mesh.close()
    if ws > 1:
        import torch.distributed as dist
        dist.barrier()
        dist.destroy_process_group()


HBM_PEAK_GBS = 6699.8   # measured STREAM-style copy bandwidth of a GB300 (MEASURED_PEAKS.json hbm_gbs)

# DRAM bytes (read + write) per k_propagate launch on this workload, from the ncu launch
# list in profiles/terrain512_launch_list.md, valid only for the kernel sources it was
# taken on (their hash); any change of them reports null until the list is taken again.
PROP_TRAFFIC = {"sources_sha256_16": "0d616c4973624cd2", "bytes_per_launch": 26.80e6}
PROP_SOURCES = ("paper_1305_1293_gb300/csrc/solver.cu", "paper_1305_1293_gb300/csrc/pch_common.cuh",
                "paper_1305_1293_gb300/csrc/fastmath.cuh")


def prop_traffic():
    import hashlib
    h = hashlib.sha256()
    for f in PROP_SOURCES:
        with open(os.path.join(ROOT, f), "rb") as fh:
            h.update(fh.read())
    return PROP_TRAFFIC["bytes_per_launch"] if h.hexdigest()[:16] == PROP_TRAFFIC["sources_sha256_16"] else None


def phase_rooflines(pst, passes):
    """Achieved FP64 rate of k_propagate and HBM rates of the memory-bound phases from the
    algorithmic work counted in one profiled solve (bytes per window as in the comments below)."""
    ph = pst["ms_phase"]
    out = {"propagate_fp64_tflops": pst["prop_fp64_ops"] / max(ph["propagate"], 1e-9) / 1e9}
    sel_bytes = 128 * pst["windows_scanned"]                        # 60 B in + 60 B out + 8 B gather
    sort_bytes = pst["windows_sorted"] * (8 + 20 * passes)          # pass 0 reads he/inst; 4+8+8 B a pass
    app_bytes = 240 * pst["windows_sorted"]                         # key/index 8, window 60, record 96, g 16, out 60
    for name, b, ms in (("select", sel_bytes, ph["select"]), ("sort", sort_bytes, ph["sort"]),
                        ("append", app_bytes, ph["append"])):
        gbs = b / max(ms, 1e-9) / 1e6
        out[name + "_gbs"] = gbs
        out[name + "_hbm_frac"] = gbs / HBM_PEAK_GBS
    out["propagate_fp64_frac"] = out["propagate_fp64_tflops"] / FP64_PEAK_DERIVED
    return out


def run_workload(args):
    """Per-workload report line (not the default bench): plain with the paper's k, plain
    with a tuned fixed k, the learned controller, and for multi-instance workloads one
    batched launch against sequential solves; parity sampled against the oracle."""
    import torch
    torch.cuda.set_device(0)
    import __graft_entry__
    __graft_entry__.build()
    import oracle
    from paper_1305_1293_gb300 import meshgen as mg, pch
    pch.load_controller()
    meshes, srcs = mg.workload(args.workload, "full")
    handles = [pch.Mesh(m.vertices, m.faces) for m in meshes]
    inst = [(i, int(s)) for i, ss in enumerate(srcs) for s in ss]
    if args.workload == "torus":
        inst = inst[:4]
    hmesh = [handles[i] for i, _ in inst]
    hsrc = [s for _, s in inst]

    def seq(**kw):
        t = w = 0
        outs = []
        for h, s in zip(hmesh, hsrc):
            pch.solve(h, s, **kw)                                  # warm the graph
            d, st = pch.solve(h, s, stats=True, **kw)
            t += st["ms_total"]
            w += st["windows_propagated"]
            outs.append(d)
        return t, w, outs

    res = {}
    single = len(inst) == 1
    big = sum(m.nf for m in meshes) * len(inst) / len(meshes) > 3e7

    def batched(**kw):
        if not big:                                                # warm the graph
            pch.solve_batch(hmesh, hsrc, **kw)
        outs, st = pch.solve_batch(hmesh, hsrc, stats=True, **kw)
        return st["ms_total"], st["windows_propagated"], outs, st

    if not big:
        res["plain_paper_k24576_hops1"] = seq(k=24576, hops=1)[:2]
        res["strided_paper_k24576"] = seq(k=24576, control=pch.CONTROL_STRIDED)[:2]
    tuned = pch.autotune(handles[0], hsrc[0], cache_path=os.path.join(ROOT, "paper_1305_1293_gb300", "autotune_cache.txt"))
    tk = {"k": tuned["k"], "block": tuned["block"], "hops": tuned["hops"]}
    if not big:
        res["plain_tuned"] = seq(**tk)[:2]
        res["learned"] = seq(control=pch.CONTROL_LEARNED)[:2]
    final = None
    if not single:
        t, w, outs, st = batched(control=pch.CONTROL_LEARNED, block=tk["block"], hops=tk["hops"])
        res["batched_learned"] = (t, w)
        t2, w2, outs2, st2 = batched(**tk)
        res["batched_tuned"] = (t2, w2)
        final = outs2 if t2 < t else outs
    else:
        final = seq(**tk)[2]
    # parity on sampled vertices of every instance (oracle early stop), at most 8 instances
    worst = 0.0
    for (i, s), d in list(zip(inst, final))[:8]:
        m = meshes[i]
        near = np.argsort(d)[1:151].astype(np.int32)
        ref, _ = oracle.geodesic(m.vertices, m.faces, s, targets=near)
        worst = max(worst, float(np.max(np.abs(d[near] - ref[near]) / ref[near])))
    # profiled run of the tuned configuration on the first instance (roofline)
    _, pst = pch.solve(hmesh[0], hsrc[0], stats=True, flags=pch.FLAG_PROFILE, **tk)
    roof = phase_rooflines(pst, pst["sort_passes"])
    best_name = min(res, key=lambda k: res[k][0])
    t, w = res[best_name]
    line = {"workload": args.workload, "metric": METRIC, "value": w / (t / 1e3), "unit": UNIT,
            "ms_per_step": t, "best_form": best_name, "instances": len(inst),
            "faces_total": int(sum(meshes[i].nf for i, _ in inst)),
            "forms_ms_windows": {k: [round(v[0], 2), int(v[1])] for k, v in res.items()},
            "tuned": tk, "parity_max_rel_err_sampled": worst, "roofline_first_instance": roof}
    print(json.dumps(line), flush=True)
    for h in handles:
        h.close()


def run_paths(args):
    """Report line for geodesic paths on the benchmark terrain (512 x 512 quads, source at
    the centre): the solve with distance events recorded against the plain solve (same
    tuned configuration), and the paths of 4,096 seeded target vertices traced on the
    device.  Times: the solves' device time (CUDA events inside the library) and the wall
    time of the whole pch_trace_paths call (target upload, solve, event pick, trace,
    download of the points).  Check: the 3D length of every traced path against the
    target's distance (a property of an exact geodesic at any size)."""
    import time
    import torch
    torch.cuda.set_device(0)
    import __graft_entry__
    __graft_entry__.build()
    from paper_1305_1293_gb300 import meshgen as mg, pch
    meshes, srcs = mg.workload("terrain", "full")
    m, src = meshes[0], int(srcs[0][0])
    h = pch.Mesh(m.vertices, m.faces)
    tuned = pch.autotune(h, src, cache_path=os.path.join(ROOT, "paper_1305_1293_gb300", "autotune_cache.txt"))
    tk = {"k": tuned["k"], "block": tuned["block"], "hops": tuned["hops"]}
    rng = np.random.default_rng(0xC0FFEE + 1)
    targets = rng.choice(m.nv, size=4096, replace=False).astype(np.int32)
    pch.solve(h, src, **tk)                                           # warm the graph
    _, st_plain = pch.solve(h, src, stats=True, **tk)
    pch.trace_paths(h, [src], targets[:8], max_points=4096, **tk)     # warm the recording graph
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    d, paths, st = pch.trace_paths(h, [src], targets, max_points=4096, stats=True, **tk)
    wall_ms = (time.perf_counter() - t0) * 1e3
    failed = sum(p is None for p in paths)
    npts, worst = [], 0.0
    for t, p in zip(targets, paths):
        if p is None:
            continue
        kind, pid, a, b = p
        xyz = np.empty((len(kind), 3))
        for j in range(len(kind)):
            if kind[j] == 0:
                xyz[j] = m.vertices[pid[j]]
            elif kind[j] == 1:
                f, i = divmod(int(pid[j]), 3)
                u, w = m.vertices[m.faces[f, i]], m.vertices[m.faces[f, (i + 1) % 3]]
                xyz[j] = u + a[j] * (w - u)
            else:
                c = m.faces[int(pid[j])]
                xyz[j] = (1 - a[j] - b[j]) * m.vertices[c[0]] + a[j] * m.vertices[c[1]] + b[j] * m.vertices[c[2]]
        length = float(np.linalg.norm(np.diff(xyz, axis=0), axis=1).sum())
        if d[t] > 0:
            worst = max(worst, abs(length - d[t]) / d[t])
        npts.append(len(kind))
    line = {"workload": "paths", "mesh": "terrain 512x512 (524,288 faces), centre source",
            "targets": int(len(targets)), "failed_traces": int(failed),
            "mean_points_per_path": float(np.mean(npts)), "max_points_per_path": int(np.max(npts)),
            "plain_solve_ms": st_plain["ms_total"], "recording_solve_ms": st["ms_total"],
            "recording_overhead": st["ms_total"] / st_plain["ms_total"],
            "trace_call_wall_ms": wall_ms, "paths_per_s_wall": len(targets) / (wall_ms / 1e3),
            "length_vs_distance_max_rel_err": worst, "tuned": tk}
    print(json.dumps(line), flush=True)
    h.close()


NCU_CASES = {
    # name: (mesh builder, sources, solve options) - one solve each, host-driven loop, so
    # that every phase kernel is its own launch and the k-th k_propagate launch is the
    # k-th iteration's
    "terrain256": (lambda mg: mg.terrain(256, 256, seed=mg.SEED_BASE + 1), lambda mg, m: [mg.terrain_center(256, 256)],
                   {"k": 393216, "hops": 32, "block": 64}),
    "terrain512": (lambda mg: mg.workload("terrain", "full")[0][0], lambda mg, m: [mg.terrain_center(512, 512)],
                   {"k": 393216, "hops": 32, "block": 64}),
    "sphere7x8": (lambda mg: mg.multi_octave_sphere(7, 0.05, seed=mg.SEED_BASE + 5),
                  lambda mg, m: [int(x) for x in mg.pick_sources(m, 8, mg.SEED_BASE + 105)],
                  {"k": 1 << 20, "hops": 64, "block": 64}),
}


def run_ncu_case(args):
    """One solve of a small named case with the host-driven loop, for ncu captures (never
    a bench value: nothing is timed here)."""
    import torch
    torch.cuda.set_device(0)
    import __graft_entry__
    __graft_entry__.build()
    from paper_1305_1293_gb300 import meshgen as mg, pch
    make, srcs, opts = NCU_CASES[args.ncu_case]
    m = make(mg)
    sv = srcs(mg, m)
    h = pch.Mesh(m.vertices, m.faces)
    if len(sv) == 1:
        _, st = pch.solve(h, sv[0], stats=True, loop=pch.LOOP_HOST, **opts)
    else:
        _, st = pch.solve_batch([h] * len(sv), sv, stats=True, loop=pch.LOOP_HOST, **opts)
    print(json.dumps({"ncu_case": args.ncu_case, "faces": m.nf, "sources": len(sv), "opts": opts,
                      "iterations": st["iterations"], "windows_propagated": st["windows_propagated"],
                      "kernel_launches": st["kernel_launches"], "prop_fp64_ops": st["prop_fp64_ops"]}), flush=True)
    h.close()


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=20)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--k", type=int, default=0, help="windows per iteration (0 = autotuned)")
    ap.add_argument("--hops", type=int, default=0, help="with --k: propagation hops (0 = library default)")
    ap.add_argument("--workload", default="terrain",
                    choices=["terrain", "icosphere", "torus", "batch", "multisrc", "large", "paths"],
                    help="terrain = the benchmark line; others print a per-workload report line")
    ap.add_argument("--loop", default="graph", choices=["graph", "host"],
                    help="iteration driver: CUDA graph with device-side termination, or host-driven (for ncu)")
    ap.add_argument("--ncu-case", default=None, choices=sorted(NCU_CASES),
                    help="run one untimed solve of a small case for an ncu capture")
    args = ap.parse_args()
    if args.ncu_case:
        run_ncu_case(args)
    elif args.impl == "reference":
        run_reference(args)
    elif args.workload == "paths":
        run_paths(args)
    elif args.workload != "terrain":
        run_workload(args)
    else:
        run_gpu(args)


if __name__ == "__main__":
    main()
