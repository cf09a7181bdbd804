"""CPU oracle for exact polyhedral geodesic distance - TEST INFRASTRUCTURE ONLY.

Only ``tests/``, ``__graft_entry__.smoke()`` and ``bench.py``'s CPU-baseline leg may
import this package.  It wraps ``ich_oracle.cpp`` (sequential FP64 Chen-Han/Xin-Wang,
Algorithm 2 of the paper, the sequential CPU PCH variant of Section 6, and geodesic paths
traced back along the window sequence of Section 4.4) and ``mlp_oracle.py`` (FP64
reference of the selection controller's network).  It shares no code with the CUDA path.
"""
from __future__ import annotations

import ctypes
import os
import subprocess

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SO = os.path.join(_HERE, "liboracle.so")
_lib = None

ORDER_PQ, ORDER_FIFO, ORDER_RANDOM, ORDER_BATCH = 0, 1, 2, 3
NO_CH, NO_ICH = 4, 8


def build(force: bool = False) -> str:
    """Compile the oracle shared library in-tree (plain g++, portable flags)."""
    src = os.path.join(_HERE, "ich_oracle.cpp")
    if force or not os.path.exists(_SO) or os.path.getmtime(_SO) < os.path.getmtime(src):
        subprocess.check_call(["g++", "-O2", "-std=c++17", "-shared", "-fPIC", "-o", _SO, src])
    return _SO


def load_library(path: str):
    """Load an oracle build from ``path`` (the tests also load mutated copies)."""
    lib = ctypes.CDLL(path)
    _declare(lib)
    return lib


def _declare(lib):
    lib.oracle_geodesic.restype = ctypes.c_int
    lib.oracle_geodesic.argtypes = [
        ctypes.c_int, ctypes.c_void_p, ctypes.c_int, ctypes.c_void_p, ctypes.c_int, ctypes.c_int,
        ctypes.c_int, ctypes.c_void_p, ctypes.c_int, ctypes.c_void_p, ctypes.c_int,
        ctypes.c_longlong, ctypes.c_int, ctypes.c_void_p, ctypes.c_void_p, ctypes.c_void_p]
    lib.oracle_cpu_pch.restype = ctypes.c_int
    lib.oracle_cpu_pch.argtypes = [ctypes.c_int, ctypes.c_void_p, ctypes.c_int, ctypes.c_void_p, ctypes.c_int,
                                   ctypes.c_longlong, ctypes.c_int, ctypes.c_void_p, ctypes.c_void_p]
    lib.oracle_trace_paths.restype = ctypes.c_int
    lib.oracle_trace_paths.argtypes = [
        ctypes.c_int, ctypes.c_void_p, ctypes.c_int, ctypes.c_void_p, ctypes.c_int, ctypes.c_int, ctypes.c_int,
        ctypes.c_void_p, ctypes.c_int, ctypes.c_void_p, ctypes.c_int, ctypes.c_void_p, ctypes.c_int,
        ctypes.c_void_p, ctypes.c_void_p, ctypes.c_void_p, ctypes.c_void_p, ctypes.c_void_p, ctypes.c_void_p]
    lib.oracle_vertex_angles.restype = ctypes.c_int
    lib.oracle_vertex_angles.argtypes = [ctypes.c_int, ctypes.c_void_p, ctypes.c_int, ctypes.c_void_p,
                                         ctypes.c_void_p, ctypes.c_void_p]


def _load():
    global _lib
    if _lib is None:
        build()
        lib = ctypes.CDLL(_SO)
        _declare(lib)
        _lib = lib
    return _lib


class OracleError(RuntimeError):
    pass


def geodesic(vertices, faces, source=None, *, face=None, bary=None, sources=None, flags: int = 0,
             targets=None, max_windows: int = 0, lib=None):
    """Exact geodesic distance to every vertex.  Returns (dist[V], stats dict).

    source: vertex id; or face/bary for a point inside a face; or sources (list) for the
    multi-source field (distance to the nearest source)."""
    lib = lib or _load()
    v = np.ascontiguousarray(vertices, dtype=np.float64)
    f = np.ascontiguousarray(faces, dtype=np.int32)
    out = np.empty(v.shape[0], dtype=np.float64)
    stats = np.zeros(5, dtype=np.int64)
    b = np.zeros(3, dtype=np.float64)
    srcs = np.zeros(1, dtype=np.int32)
    if sources is not None:
        kind, sv, sf = 2, 0, 0
        srcs = np.ascontiguousarray(sources, dtype=np.int32)
    elif face is not None:
        kind, sv, sf = 1, 0, int(face)
        b = np.ascontiguousarray(bary, dtype=np.float64)
    else:
        kind, sv, sf = 0, int(source), 0
    t = np.zeros(1, dtype=np.int32) if targets is None else np.ascontiguousarray(targets, dtype=np.int32)
    nt = 0 if targets is None else int(t.shape[0])
    rc = lib.oracle_geodesic(v.shape[0], v.ctypes.data, f.shape[0], f.ctypes.data, kind, sv, sf,
                             b.ctypes.data, int(srcs.shape[0]), srcs.ctypes.data, int(flags),
                             int(max_windows), nt, t.ctypes.data, out.ctypes.data, stats.ctypes.data)
    if rc != 0:
        raise OracleError(f"oracle_geodesic failed with code {rc}")
    return out, _stats(stats)


def _stats(stats):
    return {"created": int(stats[0]), "propagated": int(stats[1]), "peak": int(stats[2]),
            "events": int(stats[3]), "rounds": int(stats[4])}


def cpu_pch(vertices, faces, source: int, k: int, *, flags: int = 0, lib=None):
    """The CPU PCH algorithm of Section 6 (a sequential baseline of the parallel method):
    rounds of the k nearest pending windows chosen by quickselect and propagated one by
    one in no particular order.  Returns (dist[V], stats dict with "rounds")."""
    lib = lib or _load()
    v = np.ascontiguousarray(vertices, dtype=np.float64)
    f = np.ascontiguousarray(faces, dtype=np.int32)
    out = np.empty(v.shape[0], dtype=np.float64)
    stats = np.zeros(5, dtype=np.int64)
    rc = lib.oracle_cpu_pch(v.shape[0], v.ctypes.data, f.shape[0], f.ctypes.data, int(source), int(k), int(flags),
                            out.ctypes.data, stats.ctypes.data)
    if rc != 0:
        raise OracleError(f"oracle_cpu_pch failed with code {rc}")
    return out, _stats(stats)


def trace_paths(vertices, faces, source=None, *, targets, face=None, bary=None, sources=None,
                max_points: int = 1 << 16, lib=None):
    """Geodesic paths from the source(s) to each target, from the window sequence that
    gave the target its distance (Section 4.4) and the straight unfolded segments of
    Section 3's path structure.  Returns (dist[V], paths): paths[i] is None if the chain
    was broken, else a tuple (kind, id, t0, t1) of arrays, target first: kind 0 a vertex,
    1 a point on half-edge id (3 f + i, corner i to corner i + 1 of face f) at fraction
    t0 from its start, 2 the face-point source in face id (barycentric t0, t1 of corners
    1 and 2).  An unreachable target has an empty path."""
    lib = lib or _load()
    v = np.ascontiguousarray(vertices, dtype=np.float64)
    f = np.ascontiguousarray(faces, dtype=np.int32)
    t = np.ascontiguousarray(targets, dtype=np.int32)
    nt = int(t.shape[0])
    out = np.empty(v.shape[0], dtype=np.float64)
    b = np.zeros(3, dtype=np.float64)
    srcs = np.zeros(1, dtype=np.int32)
    if sources is not None:
        kind, sv, sf = 2, 0, 0
        srcs = np.ascontiguousarray(sources, dtype=np.int32)
    elif face is not None:
        kind, sv, sf = 1, 0, int(face)
        b = np.ascontiguousarray(bary, dtype=np.float64)
    else:
        kind, sv, sf = 0, int(source), 0
    kinds = np.zeros((max(nt, 1), max_points), dtype=np.int32)
    ids = np.zeros_like(kinds)
    t0 = np.zeros((max(nt, 1), max_points), dtype=np.float64)
    t1 = np.zeros_like(t0)
    n = np.zeros(max(nt, 1), dtype=np.int32)
    rc = lib.oracle_trace_paths(v.shape[0], v.ctypes.data, f.shape[0], f.ctypes.data, kind, sv, sf, b.ctypes.data,
                                int(srcs.shape[0]), srcs.ctypes.data, nt, t.ctypes.data, int(max_points),
                                kinds.ctypes.data, ids.ctypes.data, t0.ctypes.data, t1.ctypes.data, n.ctypes.data,
                                out.ctypes.data)
    if rc != 0:
        raise OracleError(f"oracle_trace_paths failed with code {rc}")
    paths = []
    for i in range(nt):
        k = int(n[i])
        if k < 0:
            paths.append(None)
            continue
        if k > max_points:
            raise OracleError(f"path {i} has {k} points, more than max_points={max_points}")
        paths.append((kinds[i, :k].copy(), ids[i, :k].copy(), t0[i, :k].copy(), t1[i, :k].copy()))
    return out, paths


def vertex_angles(vertices, faces):
    lib = _load()
    v = np.ascontiguousarray(vertices, dtype=np.float64)
    f = np.ascontiguousarray(faces, dtype=np.int32)
    th = np.empty(v.shape[0])
    ps = np.empty(v.shape[0], dtype=np.uint8)
    rc = lib.oracle_vertex_angles(v.shape[0], v.ctypes.data, f.shape[0], f.ctypes.data, th.ctypes.data,
                                  ps.ctypes.data)
    if rc != 0:
        raise OracleError(f"oracle_vertex_angles failed with code {rc}")
    return th, ps.astype(bool)
