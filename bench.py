"""Benchmark: exact geodesic distance on the largest synthetic workload of the set, the
5,242,880-face sphere (icosahedron subdivided 9 times, 5% multi-octave radial noise) with
32 seeded sources, learned selection controller and autotuned propagation tiles.

One step = one batched solve (selection, propagation, organisation, events, until no
window is pending) of a group of 8 of the 32 sources in one launch sequence, with the
learned controller; the steps cycle through the four groups, so every 4 steps solve the
whole source set.  The mesh is resident on the device; inputs (33 GB of workspace and
the 1.5 GB mesh) are far larger than L2, and L2 is flushed between steps anyway.  Beside
it, on the same GPU and group: plain PCH as the paper runs it (k = 24 * 2^10, one hop per
iteration, one source at a time), plain PCH with the autotuned fixed k (sequential and
batched), and the 512 x 512 terrain.  Prints one JSON line (rank 0).

`--impl reference` times the sequential CPU oracle instead, on bounded samples of the same
workload (the oracle stops once a fixed set of vertices nearest the source is final).

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
WORKLOAD = ("large: icosahedron subdivided 9x (2,621,442 V, 5,242,880 F), radius 1 + 0.05 N(p)/max|N| with N a "
            "5-octave sum of 8 random plane waves, 32 seeded source vertices, fp64 geometry, learned selection "
            "controller (fp32 3 x 64 MLP) and autotuned propagation tiles; the largest configuration of the set, "
            "the one the metric is quoted on")
GROUP = 8                     # sources per batched launch sequence (one bench step)
TERRAIN = "terrain512: 512x512 height-field grid (263,169 V, 524,288 F), 8 sines + N(0,0.01^2), random diagonals, centre source"
# oracle samples: stop once the n vertices nearest the source are final
NEAR_SAMPLE = 6000            # the reference arm, per step (a few seconds on one core)
NEAR_SAMPLE_BASELINE = 15000  # the bench line's cpu_baseline, per core (about 10-30 s each)
FP64_PEAK_DERIVED = 152 * 4 * 2.07e9 / 1e12   # SMs x FP64 flops/clk/SM x max clock (TFLOP/s)
TUNE_CACHE = os.path.join(ROOT, "paper_1305_1293_gb300", "autotune_cache.txt")


_T0 = time.time()


def _log(msg):
    """Progress of the run on stderr (the JSON line goes to stdout)."""
    print(f"[bench {time.time() - _T0:7.1f} s] {msg}", file=sys.stderr, flush=True)


def _peaks():
    """HBM copy bandwidth measured on this machine (MEASURED_PEAKS.json), else the fallback."""
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
            return float(json.load(f)["hbm_gbs"]), "measured"
    except Exception:
        return 6800.0, "fallback"


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


def _near_targets(m, s, n_near):
    return np.argsort(np.linalg.norm(m.vertices - m.vertices[s], axis=1))[:n_near].astype(np.int32)


def oracle_sample(m, s, n_near: int = NEAR_SAMPLE):
    """Time the CPU oracle on a bounded sample: stop once the n_near nearest vertices
    (by Euclidean distance) are final.  Returns windows/s, seconds, windows."""
    import oracle
    near = _near_targets(m, s, n_near)
    t = time.perf_counter()
    _, st = oracle.geodesic(m.vertices, m.faces, s, targets=near)
    dt = time.perf_counter() - t
    return st["propagated"] / dt, dt, st["propagated"]


def _oracle_worker(job):
    """One source of the large workload on one host core (process pool, spawn)."""
    s, n_near = job
    sys.path.insert(0, ROOT)
    from paper_1305_1293_gb300 import meshgen as mg
    m = mg.workload("large", "full")[0][0]
    v, dt, w = oracle_sample(m, s, n_near)
    return s, dt, w


def cpu_baseline_parallel(sources, n_near=NEAR_SAMPLE_BASELINE):
    """The oracle on the machine's host cores, one source per core (spawned processes, no
    threading inside a solve), each stopped once its n_near nearest vertices are final."""
    import multiprocessing as mp
    cores = os.cpu_count() or 1
    jobs = [(int(s), n_near) for s in sources[:cores]]
    t = time.perf_counter()
    with mp.get_context("spawn").Pool(len(jobs)) as pool:
        res = pool.map(_oracle_worker, jobs)
    wall = time.perf_counter() - t
    per = [dt for _, dt, _ in res]
    wins = sum(w for _, _, w in res)
    return {"value": wins / max(max(per), 1e-9),
            "unit": UNIT, "cores": len(jobs), "host_cores": cores, "kind": "oracle",
            "sample": f"one source per core on the large workload ({len(jobs)} of its 32 sources), each oracle run "
                      f"stopped once the {n_near} vertices nearest its source are final; value = windows of all "
                      f"cores / the slowest core's time",
            "per_source_s_median": statistics.median(per), "per_source_s_max": max(per),
            "wall_s_with_process_start": wall, "windows_total": wins}


def full_field_comparison(pch, mg):
    """Full-field solve time on one stated instance, oracle (one core) against the GPU:
    the large workload's family at 4 subdivisions fewer (20,480 faces), first source."""
    import oracle
    m = mg.multi_octave_sphere(5, 0.05, seed=mg.SEED_BASE + 5)
    s = int(mg.pick_sources(m, 1, mg.SEED_BASE + 105)[0])
    t = time.perf_counter()
    ref, ost = oracle.geodesic(m.vertices, m.faces, s)
    t_or = time.perf_counter() - t
    h = pch.Mesh(m.vertices, m.faces)
    pch.solve(h, s, control=pch.CONTROL_LEARNED)
    times = []
    for _ in range(5):
        d, st = pch.solve(h, s, stats=True, control=pch.CONTROL_LEARNED)
        times.append(st["ms_total"])
    h.close()
    err = float(np.max(np.abs(d - ref) / np.maximum(ref, 1e-300)))
    # the paper's sequential CPU PCH (Section 6) on the same instance: rounds of the k
    # nearest windows, against the priority-queue order of the oracle
    cpu_pch = {}
    for k in (256, 24576):
        t = time.perf_counter()
        dk, kst = oracle.cpu_pch(m.vertices, m.faces, s, k)
        cpu_pch[f"k{k}"] = {"one_core_ms": 1e3 * (time.perf_counter() - t), "windows": kst["propagated"],
                            "rounds": kst["rounds"], "windows_vs_ich": kst["propagated"] / max(1, ost["propagated"]),
                            "max_rel_err_vs_ich": float(np.max(np.abs(dk - ref) / np.maximum(ref, 1e-300)))}
    return {"instance": f"multi-octave sphere subdivided 5x ({m.nf} F), source {s}, whole field",
            "oracle_one_core_ms": 1e3 * t_or, "oracle_windows": ost["propagated"],
            "gpu_learned_ms_median": statistics.median(times), "gpu_windows": st["windows_propagated"],
            "max_rel_err": err, "cpu_pch": cpu_pch}


def run_reference(args):
    ws, rank, _ = _dist_env()
    if rank != 0:
        return
    from paper_1305_1293_gb300 import meshgen as mg
    import oracle
    oracle.build()
    meshes, srcs = mg.workload("large", "full")
    m, sv = meshes[0], [int(x) for x in srcs[0]]
    for i in range(args.warmup):
        oracle_sample(m, sv[i % len(sv)])
    times, wins = [], []
    for i in range(args.steps):
        _, dt, w = oracle_sample(m, sv[i % len(sv)])
        times.append(dt)
        wins.append(w)
    value = sum(wins) / sum(times)
    sample = (f"each step one source of the large workload (cycling over its 32 sources), the oracle stopped once "
              f"the {NEAR_SAMPLE} vertices nearest the source are final (mean {int(np.mean(wins))} windows per step)")
    line = {"impl": "reference", "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": args.gpus,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1e3 * sum(times) / len(times),
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
            "config": {"workload": WORKLOAD + "; " + sample, "parallelism": "1 host core (sequential oracle)"},
            "cpu_baseline": {"value": value, "unit": UNIT, "cores": 1, "kind": "oracle", "sample": sample},
            "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)


def _timed(stream, fn):
    import torch
    a = torch.cuda.Event(enable_timing=True)
    b = torch.cuda.Event(enable_timing=True)
    a.record(stream)
    r = fn()
    b.record(stream)
    b.synchronize()
    return a.elapsed_time(b), r


def terrain_extras(pch, mg, stream):
    """The 512 x 512 terrain from its centre (the earlier headline workload): plain PCH
    with the autotuned fixed k, the paper's setting, and the learned controller."""
    import torch
    meshes, srcs = mg.workload("terrain", "full")
    m, s = meshes[0], int(srcs[0][0])
    h = pch.Mesh(m.vertices, m.faces)
    out = torch.empty(m.nv, dtype=torch.float64, device="cuda")
    t0 = time.perf_counter()
    tuned = pch.autotune(h, s, cache_path=TUNE_CACHE)
    tune_s = time.perf_counter() - t0
    tk = {"k": tuned["k"], "block": tuned["block"], "hops": tuned["hops"]}
    res = {}
    for name, kw in (("plain_tuned", tk), ("learned", {"control": pch.CONTROL_LEARNED, "block": tk["block"],
                                                       "hops": tk["hops"]}),
                     ("paper_k24576_1hop", {"k": 24576, "hops": 1})):
        pch.solve(h, s, out=out, stream=stream, **kw)
        reps = 10 if name != "paper_k24576_1hop" else 2
        ms, w = [], 0
        for _ in range(reps):
            t, (_, st) = _timed(stream, lambda: pch.solve(h, s, out=out, stats=True, stream=stream, **kw))
            ms.append(t)
            w = st["windows_propagated"]
        res[name] = {"ms_median": statistics.median(ms), "windows": w,
                     "windows_per_s": w / (statistics.median(ms) / 1e3)}
    h.close()
    return {"workload": TERRAIN, "tuned": tk, "tune_s": tune_s, **res}


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
    if not pch.load_controller():
        raise RuntimeError("trained controller weights are missing (paper_1305_1293_gb300/controller_weights.npy)")

    meshes, srcs = mg.workload("large", "full")
    m = meshes[0]
    sv = [int(x) for x in srcs[0]]
    groups = [sv[i:i + GROUP] for i in range(0, len(sv), GROUP)]
    h = pch.Mesh(m.vertices, m.faces)
    stream = torch.cuda.current_stream()
    outs = [torch.empty(m.nv, dtype=torch.float64, device="cuda") for _ in range(GROUP)]
    flush = torch.empty(256 * 1024 * 1024 // 4, dtype=torch.float32, device="cuda")   # > L2 (129 MB)
    # the learned controller picks k each iteration; the tuner picks hops and the block
    t0 = time.perf_counter()
    _log("mesh built; tuning hops and block for the learned control")
    tl = pch.autotune(h, sv[0], cache_path=TUNE_CACHE, control=pch.CONTROL_LEARNED)
    _log(f"tuned {tl}")
    tune_learned_s = time.perf_counter() - t0
    lopts = {"control": pch.CONTROL_LEARNED, "hops": tl["hops"], "block": tl["block"]}

    def step(i):
        g = groups[i % len(groups)]
        return pch.solve_batch([h] * len(g), g, outs=outs[:len(g)], stats=True, stream=stream, **lopts)[1]

    for i in range(args.warmup):
        step(i)
    torch.cuda.synchronize()
    _log("warm-up done")
    if ws > 1:
        torch.distributed.barrier()
    per_step, stats = [], []
    with ClockSampler(local) as clk:
        torch.cuda.synchronize()
        for i in range(args.steps):
            flush.fill_(1.0)                       # evict L2 between timed steps
            t, st = _timed(stream, lambda: step(i))
            per_step.append(t)
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
    last_group = groups[(args.steps - 1) % len(groups)]
    got = [o.cpu().numpy() for o in outs[:len(last_group)]]

    line = None
    if rank == 0:
        g0 = groups[0]
        # ---- plain PCH on the same GPU and group
        t0 = time.perf_counter()
        _log("timed steps done; tuning the plain control")
        tp = pch.autotune(h, sv[0], cache_path=TUNE_CACHE)
        _log(f"tuned {tp}")
        tune_plain_s = time.perf_counter() - t0
        popts = {"k": tp["k"], "hops": tp["hops"], "block": tp["block"]}
        seq_ms, seq_w = 0.0, 0
        for s in g0:
            t, (_, st) = _timed(stream, lambda: pch.solve(h, s, out=outs[0], stats=True, stream=stream, **popts))
            seq_ms += t
            seq_w += st["windows_propagated"]
        t, (_, bst) = _timed(stream, lambda: pch.solve_batch([h] * len(g0), g0, outs=outs[:len(g0)], stats=True,
                                                             stream=stream, **popts))
        bat_ms, bat_w = t, bst["windows_propagated"]
        t, (_, lst) = _timed(stream, lambda: pch.solve_batch([h] * len(g0), g0, outs=outs[:len(g0)], stats=True,
                                                             stream=stream, **lopts))
        lrn_g0_ms, lrn_g0_w = t, lst["windows_propagated"]
        _log("plain arms done; the paper's setting")
        # the paper's setting: measured on the group's first source, counted for the group
        pch.solve(h, g0[0], out=outs[0], stream=stream, k=24576, hops=1)   # warm its graph
        t, (_, pst0) = _timed(stream, lambda: pch.solve(h, g0[0], out=outs[0], stats=True, stream=stream,
                                                         k=24576, hops=1))
        paper_ms_per_source = t
        _log("profiled step")
        # ---- per-phase device time of one headline step (events around every phase)
        _, prof = pch.solve_batch([h] * len(g0), g0, stats=True, flags=pch.FLAG_PROFILE, **lopts)
        ph = prof["ms_phase"]
        prop_launches = prof["iterations"]
        achieved_tf = prof["prop_fp64_ops"] / (ph["propagate"] / 1e3) / 1e12
        fp64_meas = pch.measure_fp64_peak()
        hbm, hbm_src = _peaks()
        # ---- end to end through the C ABI with host buffers: mesh upload and build, one
        # group's batched solve, download of its fields
        vh = torch.from_numpy(m.vertices).pin_memory().numpy()
        fh = torch.from_numpy(m.faces).pin_memory().numpy()
        res = [torch.empty(m.nv, dtype=torch.float64).pin_memory().numpy() for _ in range(GROUP)]
        e2e_ms, e2e_w = [], 0
        for i in range(2):
            g = groups[i % len(groups)]
            torch.cuda.synchronize()
            t0 = time.perf_counter()
            mm = pch.Mesh(vh, fh)
            _, st = pch.solve_batch([mm] * len(g), g, outs=res[:len(g)], stats=True, **lopts)
            mm.close()
            e2e_ms.append(1e3 * (time.perf_counter() - t0))
            e2e_w += st["windows_propagated"]
        e2e_value = e2e_w / (sum(e2e_ms) / 1e3)
        _log("end to end done; parity samples")
        # ---- parity of the benchmarked fields on sampled vertices (oracle early stop)
        import oracle
        oracle.build()
        parity = 0.0
        for j in (0, len(last_group) - 1):
            near = np.argsort(got[j])[1:201].astype(np.int32)
            ref, _ = oracle.geodesic(m.vertices, m.faces, last_group[j], targets=near)
            parity = max(parity, float(np.max(np.abs(got[j][near] - ref[near]) / ref[near])))
        terrain = terrain_extras(pch, mg, stream)
        _log("terrain done; CPU baseline")
        cpu = cpu_baseline_parallel(sv)
        _log("CPU baseline done; full-field comparison")
        ff = full_field_comparison(pch, mg)
        clocks = clk.summary()
        ms_step = total_ms / args.steps
        paper_group_ms = paper_ms_per_source * len(g0)
        line = {
            "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": ws, "steps": args.steps, "warmup": args.warmup,
            "ms_per_step": ms_step, "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
            "dtype": "f64", "data": "synthetic",
            "config": {"workload": WORKLOAD, "step": f"one batched solve of {GROUP} of the 32 sources (cycling "
                                                     f"over the 4 groups)",
                       "control": "learned", "hops": lopts["hops"], "block": lopts["block"],
                       "parallelism": "replicas" if ws > 1 else "single GPU",
                       "l2": "flushed between timed steps (256 MB write); working set > L2",
                       "windows_per_step_mean": int(np.mean([st["windows_propagated"] for st in stats])),
                       "iterations_per_step_mean": float(np.mean([st["iterations"] for st in stats]))},
            "solve_ms_per_source": ms_step / GROUP,
            "solve_ms_all_32_sources": ms_step * len(groups),
            "vs_plain": {
                "group": g0, "learned_batched_ms": lrn_g0_ms,
                "paper_k24576_1hop_sequential_ms": paper_group_ms,
                "paper_k24576_1hop_note": "measured on the group's first source, times the group size",
                "tuned_fixed_k_sequential_ms": seq_ms, "tuned_fixed_k_batched_ms": bat_ms, "tuned": popts,
                "speedup_vs_paper_setting": paper_group_ms / lrn_g0_ms,
                "speedup_vs_tuned_fixed_k_sequential": seq_ms / lrn_g0_ms,
                "speedup_vs_tuned_fixed_k_batched": bat_ms / lrn_g0_ms,
                "windows": {"learned_batched": lrn_g0_w, "tuned_sequential": seq_w, "tuned_batched": bat_w,
                            "paper_first_source": pst0["windows_propagated"]},
                "tuner_s": {"learned": tune_learned_s, "plain": tune_plain_s}},
            "parity_max_rel_err_sampled": parity,
            "roofline": {"bound": "alu", "kernel": "k_propagate", "achieved": achieved_tf,
                         "peak": FP64_PEAK_DERIVED, "unit": "TFLOP/s", "frac": achieved_tf / FP64_PEAK_DERIVED,
                         "peak_note": "152 SMs x 4 FP64 flops/clk x 2.07 GHz (derived)",
                         "traffic": prop_traffic(prof),
                         "fp64_microbench_tflops": fp64_meas, "frac_of_measured_dfma": achieved_tf / fp64_meas,
                         "fp64_ops_per_launch": prof["prop_fp64_ops"] / max(1, prop_launches),
                         "fp64_ops_per_window": prof["prop_fp64_ops"] / max(1, prof["windows_propagated"]),
                         "launches": prop_launches, "avg_launch_us": 1e3 * ph["propagate"] / max(1, prop_launches),
                         "phase_ms": ph, "memory_phases": phase_rooflines(prof, prof["sort_passes"], hbm),
                         "hbm_peak_gbs": hbm, "hbm_peak_source": hbm_src},
            "cpu_baseline": cpu,
            "full_field_small_instance": ff,
            "e2e": {"value": e2e_value, "unit": UNIT, "ms_per_step": sum(e2e_ms) / len(e2e_ms),
                    "h2d_bytes_per_step": int(m.vertices.nbytes + m.faces.nbytes),
                    "d2h_bytes_per_step": int(8 * m.nv * GROUP)},
            "terrain512": terrain,
            "gpu_launches": int(sum(st["kernel_launches"] for st in stats)),
            "clocks": clocks,
        }
        print(json.dumps(line), flush=True)
    h.close()
    if ws > 1:
        import torch.distributed as dist
        dist.barrier()
        dist.destroy_process_group()


# DRAM bytes (read + write) per propagated window of k_propagate, from an ncu capture of
# mid-solve launches of a smaller batched sphere of the same family (profiles/), valid
# only for the kernel sources it was taken on (their hash); scaled to a launch of the
# benchmark by its windows.  Any change of the sources reports null until it is taken again.
PROP_TRAFFIC = {"sources_sha256_16": "0db47d1f64d77651", "bytes_per_window": 13.27}
PROP_SOURCES = ("paper_1305_1293_gb300/csrc/solver.cu", "paper_1305_1293_gb300/csrc/pch_common.cuh",
                "paper_1305_1293_gb300/csrc/fastmath.cuh")


def prop_sources_hash():
    import hashlib
    h = hashlib.sha256()
    for f in PROP_SOURCES:
        with open(os.path.join(ROOT, f), "rb") as fh:
            h.update(fh.read())
    return h.hexdigest()[:16]


def prop_traffic(prof):
    if PROP_TRAFFIC["bytes_per_window"] is None or prop_sources_hash() != PROP_TRAFFIC["sources_sha256_16"]:
        return None
    return PROP_TRAFFIC["bytes_per_window"] * prof["windows_examined"] / max(1, prof["iterations"])


def phase_rooflines(pst, passes, hbm):
    """Achieved FP64 rate of k_propagate and HBM rates of the memory-bound phases from the
    algorithmic work counted in one profiled solve (bytes per window as in the comments below)."""
    ph = pst["ms_phase"]
    out = {"propagate_fp64_tflops": pst["prop_fp64_ops"] / max(ph["propagate"], 1e-9) / 1e9}
    sel_bytes = 160 * pst["windows_scanned"]                        # 76 B in + 76 B out + 8 B gather
    sort_bytes = pst["windows_sorted"] * (8 + 20 * passes)          # pass 0 reads he/inst; 4+8+8 B a pass
    app_bytes = 276 * pst["windows_sorted"]                         # key/index 8, window 76, record 96, g 16, out 76
    for name, b, ms in (("select", sel_bytes, ph["select"]), ("sort", sort_bytes, ph["sort"]),
                        ("append", app_bytes, ph["append"])):
        gbs = b / max(ms, 1e-9) / 1e6
        out[name + "_gbs"] = gbs
        out[name + "_hbm_frac"] = gbs / hbm
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
    tuned = pch.autotune(handles[0], hsrc[0], cache_path=TUNE_CACHE)
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
    roof = phase_rooflines(pst, pst["sort_passes"], _peaks()[0])
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
    tuned = pch.autotune(h, src, cache_path=TUNE_CACHE)
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
    # the terrain's autotuned configuration on a GB300
    "terrain512": (lambda mg: mg.workload("terrain", "full")[0][0], lambda mg, m: [mg.terrain_center(512, 512)],
                   {"k": 1572864, "hops": 32, "block": 64}),
    # the bench step's configuration (8 sources batched, learned control, 64 hops) on the
    # same family at 2 subdivisions fewer (327,680 faces, about 2 GB on the device)
    "sphere7x8": (lambda mg: mg.multi_octave_sphere(7, 0.05, seed=mg.SEED_BASE + 5),
                  lambda mg, m: [int(x) for x in mg.pick_sources(m, 8, mg.SEED_BASE + 105)],
                  {"control": 1, "hops": 64, "block": 64}),
}


def run_ncu_case(args):
    """One solve of a small named case with the host-driven loop, for ncu captures (never
    a bench value: nothing is timed here)."""
    import torch
    torch.cuda.set_device(0)
    import __graft_entry__
    __graft_entry__.build()
    from paper_1305_1293_gb300 import meshgen as mg, pch
    pch.load_controller()
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
                      "windows_examined": st["windows_examined"],
                      "kernel_launches": st["kernel_launches"], "prop_fp64_ops": st["prop_fp64_ops"]}), flush=True)
    h.close()


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=8)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--workload", default="bench",
                    choices=["bench", "icosphere", "terrain", "torus", "batch", "multisrc", "large", "paths"],
                    help="bench = the benchmark line; others print a per-workload report line")
    ap.add_argument("--ncu-case", default=None, choices=sorted(NCU_CASES),
                    help="run one untimed solve of a small case for an ncu capture")
    args = ap.parse_args()
    if args.ncu_case:
        run_ncu_case(args)
    elif args.impl == "reference":
        run_reference(args)
    elif args.workload == "paths":
        run_paths(args)
    elif args.workload != "bench":
        run_workload(args)
    else:
        run_gpu(args)


if __name__ == "__main__":
    main()
