"""Thin ctypes binding of libpch.so (include/pch.h): argument marshalling only.

Every step of the geodesic computation runs in the library's CUDA kernels; this module
converts numpy / torch arguments into pointers and status codes into exceptions.  It
raises at import time if the in-tree library is missing (no CPU fallback exists).
"""
from __future__ import annotations

import ctypes
import os

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "libpch.so")

PCH_OK, PCH_ERR_INVALID_ARG, PCH_ERR_NONMANIFOLD, PCH_ERR_DEGENERATE = 0, 1, 2, 3
PCH_ERR_OOM, PCH_ERR_CUDA, PCH_ERR_CAPACITY, PCH_ERR_TIMEOUT = 4, 5, 6, 7
CONTROL_PLAIN, CONTROL_LEARNED, CONTROL_STRIDED = 0, 1, 2
LOOP_GRAPH, LOOP_HOST = 0, 1
FLAG_NO_TRIM, FLAG_FULL_FAN, FLAG_TRACE, FLAG_PROFILE, FLAG_EDGE_SORT = 1, 2, 4, 8, 16
PHASES = ("select", "propagate", "fan", "sort", "append", "control")

_STATUS = {1: "INVALID_ARG", 2: "NONMANIFOLD", 3: "DEGENERATE", 4: "OOM", 5: "CUDA", 6: "CAPACITY", 7: "TIMEOUT"}


class PchError(RuntimeError):
    def __init__(self, status: int, msg: str):
        super().__init__(f"PCH_ERR_{_STATUS.get(status, status)}: {msg}")
        self.status = status


class Source(ctypes.Structure):
    _fields_ = [("kind", ctypes.c_int32), ("vertex", ctypes.c_int32), ("face", ctypes.c_int32),
                ("reserved", ctypes.c_int32), ("bary", ctypes.c_double * 3)]


class PathPoint(ctypes.Structure):
    _fields_ = [("kind", ctypes.c_int32), ("id", ctypes.c_int32), ("t0", ctypes.c_double), ("t1", ctypes.c_double)]


PATH_POINT_DTYPE = np.dtype([("kind", np.int32), ("id", np.int32), ("t0", np.float64), ("t1", np.float64)])
POINT_VERTEX, POINT_EDGE, POINT_FACE = 0, 1, 2


class Options(ctypes.Structure):
    _fields_ = [("control", ctypes.c_int32), ("loop", ctypes.c_int32), ("k", ctypes.c_int64),
                ("max_iters", ctypes.c_int64), ("stream", ctypes.c_void_p), ("out_on_device", ctypes.c_int32),
                ("block", ctypes.c_int32), ("flags", ctypes.c_int32), ("hops", ctypes.c_int32)]


class Stats(ctypes.Structure):
    _fields_ = [("iterations", ctypes.c_int64), ("windows_created", ctypes.c_int64),
                ("windows_propagated", ctypes.c_int64), ("peak_pending", ctypes.c_int64),
                ("ms_total", ctypes.c_double), ("ms_setup", ctypes.c_double), ("bytes_workspace", ctypes.c_int64),
                ("kernel_launches", ctypes.c_int64), ("ms_phase", ctypes.c_double * 6), ("fans", ctypes.c_int64),
                ("fan_windows", ctypes.c_int64), ("fan_candidates", ctypes.c_int64), ("windows_chained", ctypes.c_int64),
                ("prop_fp64_ops", ctypes.c_int64), ("windows_scanned", ctypes.c_int64),
                ("windows_sorted", ctypes.c_int64), ("sort_passes", ctypes.c_int64),
                ("windows_examined", ctypes.c_int64), ("windows_occupied", ctypes.c_int64),
                ("children_computed", ctypes.c_int64), ("fan_ties", ctypes.c_int64)]

    def as_dict(self):
        d = {f[0]: getattr(self, f[0]) for f in self._fields_ if f[0] != "ms_phase"}
        d["ms_phase"] = dict(zip(PHASES, list(self.ms_phase)))
        return d


def _load():
    if not os.path.exists(LIB_PATH):
        raise ImportError(f"{LIB_PATH} is missing: build it with __graft_entry__.build() (no CPU fallback exists)")
    lib = ctypes.CDLL(LIB_PATH)
    P, I32, I64, D = ctypes.c_void_p, ctypes.c_int32, ctypes.c_int64, ctypes.c_double
    sig = {
        "pch_create_mesh": (I32, [P, I32, P, I32, P]),
        "pch_mesh_info": (I32, [P, P, P, P, P]),
        "pch_solve": (I32, [P, P, P, P, P]),
        "pch_solve_multi": (I32, [P, P, I32, P, P, P]),
        "pch_solve_batch": (I32, [P, P, I32, P, P, P]),
        "pch_destroy": (None, [P]),
        "pch_last_error": (ctypes.c_char_p, []),
        "pch_mlp_num_features": (I32, []),
        "pch_mlp_num_params": (I32, []),
        "pch_mlp_set_weights": (I32, [P, I32]),
        "pch_mlp_forward": (I32, [P, P, I32, P, P]),
        "pch_mlp_backward": (I32, [P, P, P, I32, P, P, P]),
        "pch_mlp_backward_noalloc": (I32, [P, P, P, I32, P, P, P]),
        "pch_mlp_adam": (I32, [P, P, P, P, I32, ctypes.c_float, P]),
        "pch_trace_fetch": (I32, [P, I32, P, P, P]),
        "pch_measure_fp64_peak": (I32, [P]),
        "pch_autotune": (I32, [P, P, P, ctypes.c_char_p, P]),
        "pch_build_id": (ctypes.c_char_p, []),
        "pch_selftest_math": (I32, [P, I32, P]),
        "pch_trace_paths": (I32, [P, P, I32, P, P, I32, I32, P, P, P, P]),
        "pch_voronoi": (I32, [P, P, I32, P, P, P, P]),
        "pch_iso_contours": (I32, [P, P, I32, P, I32, P, I64, P]),
    }
    for name, (res, args) in sig.items():
        fn = getattr(lib, name)
        fn.restype = res
        fn.argtypes = args
    return lib


lib = _load()


def _check(st: int):
    if st != PCH_OK:
        raise PchError(st, lib.pch_last_error().decode())


def _ptr(a) -> int:
    """Address of a contiguous numpy array or torch tensor (host or device)."""
    if isinstance(a, np.ndarray):
        return a.ctypes.data
    return a.data_ptr()


def _stream_of(stream):
    if stream is None:
        return None
    if hasattr(stream, "cuda_stream"):
        return stream.cuda_stream
    return int(stream)


def make_options(control=CONTROL_PLAIN, loop=LOOP_GRAPH, k=0, max_iters=0, stream=None, out_on_device=False,
                 block=0, flags=0, hops=0) -> Options:
    o = Options()
    o.control, o.loop, o.k, o.max_iters = control, loop, k, max_iters
    o.stream = _stream_of(stream)
    o.out_on_device, o.block, o.flags, o.hops = int(bool(out_on_device)), block, flags, hops
    return o


def make_source(vertex=None, face=None, bary=None) -> Source:
    s = Source()
    if face is not None:
        s.kind, s.face = 1, int(face)
        for k in range(3):
            s.bary[k] = float(bary[k])
    else:
        s.kind, s.vertex = 0, int(vertex)
    return s


class Mesh:
    """A pch_mesh handle built from host arrays (vertices (V,3) f64, faces (F,3) i32)."""

    def __init__(self, vertices, faces):
        v = np.ascontiguousarray(vertices, dtype=np.float64)
        f = np.ascontiguousarray(faces, dtype=np.int32)
        h = ctypes.c_void_p()
        _check(lib.pch_create_mesh(v.ctypes.data, v.shape[0], f.ctypes.data, f.shape[0], ctypes.byref(h)))
        self.handle = h
        self.nv, self.nf = int(v.shape[0]), int(f.shape[0])

    def info(self):
        a = [ctypes.c_int32() for _ in range(4)]
        _check(lib.pch_mesh_info(self.handle, *[ctypes.byref(x) for x in a]))
        return {"n_vertices": a[0].value, "n_faces": a[1].value, "n_boundary_half_edges": a[2].value,
                "n_pseudo_vertices": a[3].value}

    def close(self):
        if getattr(self, "handle", None):
            lib.pch_destroy(self.handle)
            self.handle = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


def solve(mesh: Mesh, source=None, *, face=None, bary=None, out=None, stats=False, **opts):
    """Geodesic distance from one source.  ``out``: optional torch CUDA tensor (V,) f64
    to fill on the device; otherwise a numpy array is returned."""
    src = make_source(source, face, bary)
    dev = out is not None and not isinstance(out, np.ndarray)
    o = make_options(out_on_device=dev, **opts)
    res = out if out is not None else np.empty(mesh.nv, dtype=np.float64)
    st = Stats()
    _check(lib.pch_solve(mesh.handle, ctypes.byref(src), ctypes.byref(o), _ptr(res), ctypes.byref(st)))
    return (res, st.as_dict()) if stats else res


def solve_multi(mesh: Mesh, sources, *, out=None, stats=False, **opts):
    srcs = (Source * len(sources))(*[make_source(s) for s in sources])
    dev = out is not None and not isinstance(out, np.ndarray)
    o = make_options(out_on_device=dev, **opts)
    res = out if out is not None else np.empty(mesh.nv, dtype=np.float64)
    st = Stats()
    _check(lib.pch_solve_multi(mesh.handle, srcs, len(sources), ctypes.byref(o), _ptr(res), ctypes.byref(st)))
    return (res, st.as_dict()) if stats else res


def solve_batch(meshes, sources, *, outs=None, stats=False, **opts):
    """Instance i: meshes[i] from vertex sources[i].  Returns a list of arrays."""
    n = len(meshes)
    handles = (ctypes.c_void_p * n)(*[m.handle for m in meshes])
    srcs = (Source * n)(*[make_source(s) for s in sources])
    dev = outs is not None and not isinstance(outs[0], np.ndarray)
    res = outs if outs is not None else [np.empty(m.nv, dtype=np.float64) for m in meshes]
    ptrs = (ctypes.c_void_p * n)(*[_ptr(r) for r in res])
    o = make_options(out_on_device=dev, **opts)
    st = Stats()
    _check(lib.pch_solve_batch(handles, srcs, n, ctypes.byref(o), ptrs, ctypes.byref(st)))
    return (res, st.as_dict()) if stats else res


def trace_paths(mesh: Mesh, sources, targets, *, face=None, bary=None, max_points: int = 4096, stats=False, **opts):
    """Exact geodesic paths (pch_trace_paths) from vertex ``sources`` (a list), or from
    the point of ``face`` with barycentric ``bary`` when sources is None, to each vertex of
    ``targets``.  Returns (dist, paths): paths[i] is None when the trace failed, else a
    tuple (kind, id, t0, t1) of arrays, target first (an empty path for an unreachable
    target).  Raises if a path has more than max_points points."""
    if sources is None:
        src_list = [make_source(face=face, bary=bary)]
    else:
        src_list = [make_source(s) for s in sources]
    srcs = (Source * len(src_list))(*src_list)
    tg = np.ascontiguousarray(targets, dtype=np.int32)
    nt = int(tg.shape[0])
    pts = np.zeros((max(nt, 1), max_points), dtype=PATH_POINT_DTYPE)
    n = np.zeros(max(nt, 1), dtype=np.int32)
    dist = np.empty(mesh.nv, dtype=np.float64)
    o = make_options(**opts)
    st = Stats()
    _check(lib.pch_trace_paths(mesh.handle, srcs, len(src_list), ctypes.byref(o), tg.ctypes.data, nt, max_points,
                               pts.ctypes.data, n.ctypes.data, dist.ctypes.data, ctypes.byref(st)))
    paths = []
    for i in range(nt):
        k = int(n[i])
        if k < 0:
            paths.append(None)
            continue
        if k > max_points:
            raise PchError(PCH_ERR_CAPACITY, f"path {i} has {k} points, more than max_points={max_points}")
        p = pts[i, :k]
        paths.append((p["kind"].copy(), p["id"].copy(), p["t0"].copy(), p["t1"].copy()))
    return (dist, paths, st.as_dict()) if stats else (dist, paths)


def voronoi(mesh: Mesh, sources, *, faces=None, barys=None, stats=False, **opts):
    """Geodesic Voronoi labels (pch_voronoi): index of the nearest of ``sources`` (vertex
    ids), then of the face points ``faces``/``barys``, for every vertex (-1 unreachable).
    Returns (labels, dist) or (labels, dist, stats)."""
    src_list = [make_source(s) for s in (sources or [])]
    src_list += [make_source(face=f, bary=b) for f, b in zip(faces or [], barys or [])]
    srcs = (Source * len(src_list))(*src_list)
    labels = np.empty(mesh.nv, dtype=np.int32)
    dist = np.empty(mesh.nv, dtype=np.float64)
    o = make_options(**opts)
    st = Stats()
    _check(lib.pch_voronoi(mesh.handle, srcs, len(src_list), ctypes.byref(o), labels.ctypes.data, dist.ctypes.data,
                           ctypes.byref(st)))
    return (labels, dist, st.as_dict()) if stats else (labels, dist)


CONTOUR_DTYPE = np.dtype([("level", np.int32), ("face", np.int32), ("half_edge", np.int32, 2), ("t", np.float64, 2)])


def iso_contours(mesh: Mesh, dist, levels, capacity: int | None = None):
    """Iso-contour segments (pch_iso_contours) of the field ``dist`` (numpy array, or a
    torch CUDA tensor) at ``levels``: a structured array with fields level, face,
    half_edge[2], t[2], ordered by face then level."""
    lev = np.ascontiguousarray(levels, dtype=np.float64)
    on_dev = not isinstance(dist, np.ndarray)
    d = dist if on_dev else np.ascontiguousarray(dist, dtype=np.float64)
    n = ctypes.c_int64()
    if capacity is None:
        _check(lib.pch_iso_contours(mesh.handle, _ptr(d), int(on_dev), lev.ctypes.data, lev.size, None, 0,
                                    ctypes.byref(n)))
        capacity = n.value
    out = np.zeros(max(int(capacity), 1), dtype=CONTOUR_DTYPE)
    _check(lib.pch_iso_contours(mesh.handle, _ptr(d), int(on_dev), lev.ctypes.data, lev.size, out.ctypes.data,
                                int(capacity), ctypes.byref(n)))
    return out[:min(n.value, int(capacity))]


def mlp_num_features() -> int:
    return lib.pch_mlp_num_features()


def mlp_num_params() -> int:
    return lib.pch_mlp_num_params()


def mlp_set_weights(params: np.ndarray):
    p = np.ascontiguousarray(params, dtype=np.float32)
    _check(lib.pch_mlp_set_weights(p.ctypes.data, p.shape[0]))


def mlp_forward(params_dev, x_dev, y_dev, stream=None):
    _check(lib.pch_mlp_forward(_ptr(params_dev), _ptr(x_dev), int(x_dev.shape[0]), _ptr(y_dev), _stream_of(stream)))


def mlp_backward(params_dev, x_dev, target_dev, grad_dev, loss_dev, stream=None):
    _check(lib.pch_mlp_backward(_ptr(params_dev), _ptr(x_dev), _ptr(target_dev), int(x_dev.shape[0]),
                                _ptr(grad_dev), _ptr(loss_dev), _stream_of(stream)))


def mlp_backward_noalloc(params_dev, x_dev, target_dev, grad_dev, loss_dev, stream=None):
    """pch_mlp_backward without any allocation (at most 4096 samples)."""
    _check(lib.pch_mlp_backward_noalloc(_ptr(params_dev), _ptr(x_dev), _ptr(target_dev), int(x_dev.shape[0]),
                                        _ptr(grad_dev), _ptr(loss_dev), _stream_of(stream)))


def mlp_adam(params_dev, grad_dev, m_dev, v_dev, t: int, lr: float, stream=None):
    _check(lib.pch_mlp_adam(_ptr(params_dev), _ptr(grad_dev), _ptr(m_dev), _ptr(v_dev), int(t), ctypes.c_float(lr),
                            _stream_of(stream)))


def trace_fetch(mesh: Mesh, max_rows: int = 1 << 18):
    nf = mlp_num_features()
    feats = np.empty((max_rows, nf), dtype=np.float32)
    chosen = np.empty(max_rows, dtype=np.float32)
    n = ctypes.c_int32()
    _check(lib.pch_trace_fetch(mesh.handle, max_rows, feats.ctypes.data, chosen.ctypes.data, ctypes.byref(n)))
    return feats[: n.value].copy(), chosen[: n.value].copy()


def measure_fp64_peak() -> float:
    t = ctypes.c_double()
    _check(lib.pch_measure_fp64_peak(ctypes.byref(t)))
    return t.value


def autotune(mesh: Mesh, source: int, cache_path: str | None = None, **opts):
    """Fastest (k, block, hops) for this mesh and source; returns a dict with the time."""
    src = make_source(source)
    o = make_options(**opts)
    ms = ctypes.c_double()
    _check(lib.pch_autotune(mesh.handle, ctypes.byref(src), ctypes.byref(o),
                            cache_path.encode() if cache_path else None, ctypes.byref(ms)))
    return {"k": int(o.k), "block": int(o.block), "hops": int(o.hops), "ms": ms.value}


def build_id() -> str:
    """SHA-256 prefix of the library's sources (keys the autotuner's cache)."""
    return lib.pch_build_id().decode()


def load_controller(path: str | None = None) -> bool:
    """Install trained controller weights (default: controller_weights.npy next to this
    module).  Returns False if the file does not exist."""
    path = path or os.path.join(_HERE, "controller_weights.npy")
    if not os.path.exists(path):
        return False
    mlp_set_weights(np.load(path))
    return True


def selftest_math(x_dev):
    """Largest ulp distance of the library's reciprocal and square root from IEEE."""
    out = (ctypes.c_ulonglong * 2)()
    _check(lib.pch_selftest_math(_ptr(x_dev), int(x_dev.shape[0]), out))
    return int(out[0]), int(out[1])
