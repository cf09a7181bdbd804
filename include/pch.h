/*
 * pch.h - C ABI of the GB300 (sm_103a) Parallel Chen-Han exact-geodesic library.
 *
 * Computes exact single-source-all-destination geodesic distance on a triangle mesh
 * with the iterated four-phase loop of Ying, Xin and He, "Parallel Chen-Han (PCH)
 * Algorithm for Discrete Geodesics": window selection, window propagation, data
 * organisation and events processing (Section 4.2, Algorithm 1), every phase a CUDA
 * kernel.  Plain C types only: pointers, sizes and status codes.
 *
 * Conventions for every entry point:
 *  - Host pointers unless an argument says "device".  The library copies what it keeps;
 *    the caller may free its inputs as soon as a call returns.
 *  - Results are written only on success (PCH_OK).  On error nothing the caller owns is
 *    modified, the status is returned and pch_last_error() describes it.
 *  - No exceptions cross the ABI.  Calls are synchronous with respect to the host
 *    unless pch_options.out_on_device is set, in which case results are complete when
 *    pch_options.stream (or the legacy default stream) reaches the end of the call.
 *  - Calls that share a pch_mesh (it carries the solver workspace) must not run
 *    concurrently from several host threads.
 *
 * Environment variables (read each time a solve sets up its configuration; defaults in
 * brackets; invalid values are ignored).  They change speed, never the distances:
 *  - PCH_DEFAULT_K [24576]: windows selected per iteration when pch_options.k <= 0.
 *  - PCH_DEFAULT_HOPS [32]: chained propagation hops when pch_options.hops <= 0.
 *  - PCH_TAKE_MIN [1, range 1..32]: fresh windows a propagation warp takes at once, at
 *    least (a short selected list is spread over every resident warp above this floor).
 *  - PCH_TAIL_CUT [0]: once the selected list is exhausted, a warp keeps chaining only
 *    while it holds at least this many queued windows.
 *  - PCH_PROP_BLOCKS_PER_SM [384 / block threads, range 1..32]: resident propagation
 *    blocks per SM (the grid is this times the SM count).
 */
#ifndef PCH_H_
#define PCH_H_

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

/* Opaque mesh handle: the half-edge structure of Section 4.1 plus per-half-edge
 * unfolding frames, resident in device memory, and the solver workspace.  Owned by
 * the library; release it with pch_destroy(). */
typedef struct pch_mesh pch_mesh;

typedef enum {
    PCH_OK = 0,
    PCH_ERR_INVALID_ARG = 1,   /* null pointer, index out of range, non-finite coordinate */
    PCH_ERR_NONMANIFOLD = 2,   /* an oriented edge used twice, or a vertex whose faces do not form one fan */
    PCH_ERR_DEGENERATE = 3,    /* a face with (near) zero area or a repeated vertex */
    PCH_ERR_OOM = 4,           /* device memory allocation failed */
    PCH_ERR_CUDA = 5,          /* a CUDA runtime call failed (message in pch_last_error) */
    PCH_ERR_CAPACITY = 6,      /* a size limit was exceeded (see the entry point) */
    PCH_ERR_TIMEOUT = 7        /* the iteration cap (pch_options.max_iters) was reached */
} pch_status;

/* A source: a mesh vertex (kind 0), or a point inside face `face` with barycentric
 * weights `bary` over that face's three corners in their stored order (kind 1).
 * Algorithm 1 takes sources in V; the face point is the same initialisation applied
 * to the three edges of the face. */
typedef struct {
    int32_t kind;
    int32_t vertex;
    int32_t face;
    int32_t reserved;
    double bary[3];
} pch_source;

/* Selection control (Step 1 of Section 4.2). */
enum {
    PCH_CONTROL_PLAIN = 0,    /* fixed window count k per iteration (the paper's k) */
    PCH_CONTROL_LEARNED = 1,  /* MLP controller maps frontier statistics to log2 of the
                                 number of windows to select, clamped to the trained range
                                 [2^12, 2^24]; falls back to PLAIN on a non-finite output,
                                 and runs PLAIN when no weights were installed
                                 (pch_mlp_set_weights) on the current device since its
                                 CUDA context was created */
    PCH_CONTROL_STRIDED = 2   /* the paper's approximate k-selection of Section 5.1: T threads
                                 each take every T-th pending window and select their
                                 ceil(k / T) nearest, about k windows per instance in total.
                                 T is 2048 threads per SM; the per-thread count is rounded up
                                 to a power of two (at most 16, T grows beyond that).  Each
                                 selected window propagates one hop (hops is ignored) */
};

/* Iteration driver. */
enum {
    PCH_LOOP_GRAPH = 0,       /* iterations replayed from a CUDA graph with a device-side
                                 termination condition (default) */
    PCH_LOOP_HOST = 1         /* host launches every iteration and reads the pending count */
};

/* Solve options.  Pass NULL for the defaults; a zero field also means "default". */
typedef struct {
    int32_t control;          /* PCH_CONTROL_* */
    int32_t loop;             /* PCH_LOOP_* */
    int64_t k;                /* PLAIN/STRIDED: windows selected per instance per iteration
                                 (default 24576, the paper's 24 * 2^10) */
    int64_t max_iters;        /* iteration cap; exceeded -> PCH_ERR_TIMEOUT (default 2^31) */
    void* stream;             /* cudaStream_t to run on (NULL = legacy default stream) */
    int32_t out_on_device;    /* nonzero: output pointers are device pointers */
    int32_t block;            /* threads per block of the propagation kernel, a multiple of 32
                                 in [32, 256] (0 = default 64) */
    int32_t flags;            /* PCH_FLAG_* */
    int32_t hops;             /* windows one propagation lane may chain within an iteration's
                                 band (1 = the paper's one hop per iteration; 0 = default 32) */
} pch_options;

enum {
    PCH_FLAG_NO_TRIM = 1,     /* with PCH_FLAG_EDGE_SORT: skip the per-edge trimming of Step 4 */
    PCH_FLAG_FULL_FAN = 2,    /* pseudo-source fans over the whole one-ring instead of the
                                 fanned area of Fig. `fig:propagation`(c) */
    PCH_FLAG_TRACE = 4,       /* record per-iteration controller features (pch_trace_fetch) */
    PCH_FLAG_PROFILE = 8,     /* host-driven loop with CUDA events around every phase
                                 (pch_stats.ms_phase); slower, for measurement only */
    PCH_FLAG_EDGE_SORT = 16   /* organise new windows by (instance, half-edge) with a radix
                                 sort and drop windows another window on the same edge
                                 dominates (per-edge trimming); by default they are only
                                 grouped by instance (Algorithm 3's gap-free copy) */
};

/* Per-call statistics (the columns of Table `tab:speedup`: time, windows, peak windows). */
typedef struct {
    int64_t iterations;
    int64_t windows_created;      /* windows written to the pool (children + fans) */
    int64_t windows_propagated;   /* selected windows that passed the filter and were propagated */
    int64_t peak_pending;         /* largest pending pool seen */
    double ms_total;              /* device time of the solve loop (CUDA events) */
    double ms_setup;              /* device time of initialisation */
    int64_t bytes_workspace;      /* device bytes held by the solver workspace */
    int64_t kernel_launches;      /* CUDA kernels this call launched */
    double ms_phase[6];           /* PCH_FLAG_PROFILE: selection (tau + compaction), propagation,
                                     fans, sort, append, loop control; else 0 */
    int64_t fans;                 /* pseudo-source fans built */
    int64_t fan_windows;          /* windows those fans created */
    int64_t fan_candidates;       /* distance events at pseudo-source vertices examined */
    int64_t windows_chained;      /* children propagated in the same iteration (hops > 1) */
    int64_t prop_fp64_ops;        /* algorithmic FP64 operations of the propagation kernel */
    int64_t windows_scanned;      /* pending windows read by the selection compaction */
    int64_t windows_sorted;       /* new windows sorted by the organisation step */
    int64_t sort_passes;          /* 8-bit radix passes per sort */
    int64_t windows_examined;     /* windows the propagation kernel tested (selected + chained) */
    int64_t windows_occupied;     /* of those, windows whose rays reach the opposite vertex */
    int64_t children_computed;    /* child windows whose geometry was computed (before the filter) */
    int64_t fan_ties;             /* fans made for a tie: a pseudo-source vertex reached at its
                                     final distance (within the filters' margin) from a second
                                     direction */
} pch_stats;

/* Build a mesh: host arrays `vertices` (n_vertices x 3 doubles, xyz) and `faces`
 * (n_faces x 3 int32 vertex ids, one consistent orientation).  The half-edge table,
 * edge lengths, per-half-edge unfolding frames, vertex total angles and the
 * saddle/boundary classification of Section 3 are computed on the device (Section 4.1:
 * the method needs only the metric).  Errors: INVALID_ARG, NONMANIFOLD, DEGENERATE,
 * OOM, CUDA.  On success *out owns the device data. */
pch_status pch_create_mesh(const double* vertices, int32_t n_vertices, const int32_t* faces,
                           int32_t n_faces, pch_mesh** out);

/* Counts of a mesh: vertices, faces, boundary half-edges, pseudo-source vertices. */
pch_status pch_mesh_info(const pch_mesh* m, int32_t* n_vertices, int32_t* n_faces,
                         int32_t* n_boundary_half_edges, int32_t* n_pseudo_vertices);

/* Single-source-all-destination exact geodesic distance (Algorithm 1).  out_dist:
 * n_vertices doubles (host, or device if opt->out_on_device), caller-owned.  The
 * source vertex gets exactly 0; vertices unreachable from the source get +inf.
 * stats may be NULL.  Errors: INVALID_ARG, OOM, CUDA, CAPACITY, TIMEOUT. */
pch_status pch_solve(pch_mesh* m, const pch_source* src, const pch_options* opt, double* out_dist,
                     pch_stats* stats);

/* Multiple-source-all-destination field (Section 4.2, source set S; Table
 * `tab:multiple`): distance to the nearest of the n_sources sources. */
pch_status pch_solve_multi(pch_mesh* m, const pch_source* srcs, int32_t n_sources,
                           const pch_options* opt, double* out_dist, pch_stats* stats);

/* Many independent solves in one launch sequence: instance i solves meshes[i] from
 * srcs[i] into out_dists[i] (n_vertices of meshes[i] doubles each).  Instances may
 * share a mesh (many sources on one mesh) or use different meshes of any size.  All
 * meshes must live on the current device.  The workspace is held by meshes[0]. */
pch_status pch_solve_batch(pch_mesh* const* meshes, const pch_source* srcs, int32_t n_instances,
                           const pch_options* opt, double* const* out_dists, pch_stats* stats);

/* ---- geodesic paths (Section 4.4, Section 3) ---------------------------------------- */
enum {
    PCH_POINT_VERTEX = 0,     /* mesh vertex `id` */
    PCH_POINT_EDGE = 1,       /* on half-edge `id` (3 f + i runs from corner i to corner (i + 1) % 3
                                 of face f) at fraction t0 of its length from its start; the
                                 path crosses the edge into (or out of) face f */
    PCH_POINT_FACE = 2        /* the face-point source inside face `id`: barycentric weights t0,
                                 t1 of corners 1 and 2 (corner 0 has 1 - t0 - t1) */
};

/* A point of a geodesic path on the surface. */
typedef struct {
    int32_t kind;             /* PCH_POINT_* */
    int32_t id;
    double t0, t1;
} pch_path_point;

/* Exact geodesic paths from the source(s) to the vertices targets[0 .. n_targets-1].
 * Solves the field as pch_solve_multi does while recording every distance event that
 * lowered a vertex's distance, with its window (edge, pseudo-source position, pseudo-
 * source vertex).  The event whose distance is the vertex's final one comes from the
 * last window of the window sequence that carries its shortest path (Section 4.4).  A
 * device kernel then walks each path back from its target: a straight segment through
 * the faces unfolded along that window's strip to the window's pseudo-source (Section 3:
 * a geodesic is straight in every unfolding and bends only at saddle or boundary
 * vertices), then on from that vertex's own event, until a source.
 * points (host): n_targets x max_points entries; path i starts at points[i * max_points],
 * target first, source (or the face-point source) last, with every edge crossing and
 * every vertex it passes.  Consecutive points may coincide where the recorded window
 * chain touches a vertex (an edge point at an end of its edge, next to that vertex):
 * zero-length steps of the same path.  n_points (host, n_targets entries): the path's point count;
 * when it exceeds max_points only its first max_points points are stored; 0 for an
 * unreachable target; -1 if a trace failed numerically (it left the mesh, met a vertex
 * without a recorded event, found no edge to cross where a path passes exactly through a
 * vertex that is not its pseudo-source, or exceeded 2^22 steps).  out_dist (host, n_vertices) may be
 * NULL.  opt is used as by pch_solve_multi except that out_on_device is ignored (all
 * outputs are host arrays).  Errors: as pch_solve_multi, and INVALID_ARG for a target
 * out of range or max_points < 1. */
pch_status pch_trace_paths(pch_mesh* m, const pch_source* srcs, int32_t n_sources, const pch_options* opt,
                           const int32_t* targets, int32_t n_targets, int32_t max_points,
                           pch_path_point* points, int32_t* n_points, double* out_dist, pch_stats* stats);

/* ---- geodesic Voronoi diagram (Section 7: the multiple-source field applied to the
 * geodesic Voronoi diagram) ------------------------------------------------------------
 * Labels every vertex with the index (into srcs) of its nearest source.  Solves the field
 * as pch_solve_multi does while recording the distance events (as pch_trace_paths does);
 * a vertex's final event names the last pseudo-source vertex of its shortest path
 * (Section 3: geodesics bend only at saddle or boundary vertices), or the face-point
 * source itself, and the chain of those vertices, whose distances strictly decrease,
 * ends at the source that labels the vertex.  Where two sources are equally near (within
 * rounding) either label may be returned.  labels (host, n_vertices): the source index,
 * -1 for a vertex no source reaches, -2 if a vertex's chain could not be followed (no
 * recorded event carries its final distance; not expected).  out_dist (host, n_vertices)
 * may be NULL.  opt as for pch_solve_multi, except that out_on_device is ignored.
 * Errors: as pch_solve_multi. */
pch_status pch_voronoi(pch_mesh* m, const pch_source* srcs, int32_t n_sources, const pch_options* opt,
                       int32_t* labels, double* out_dist, pch_stats* stats);

/* ---- iso-contours ----------------------------------------------------------------------
 * A segment of the iso-contour of level levels[level] inside face `face`: from the point
 * at fraction t[0] along half-edge half_edge[0] to the point at fraction t[1] along
 * half_edge[1] (half-edge 3 f + i runs from corner i to corner (i + 1) % 3 of face f; the
 * fraction is measured from its start).  Seen from the face's front side (corners
 * counter-clockwise) the region below the level lies to the left of the segment. */
typedef struct {
    int32_t level;
    int32_t face;
    int32_t half_edge[2];
    double t[2];
} pch_contour_segment;

/* Iso-contours of a distance field (the iso-contours of geodesic distance that Section 2
 * cites as a use of exact distances), one straight segment per face and level.  On each
 * face the field is the linear interpolation of its three vertex distances: a vertex is
 * below a level L when its distance is < L, and the contour crosses every edge whose two
 * ends are on different sides at the interpolated point t = (L - d_start) / (d_end -
 * d_start).  Faces with a non-finite vertex distance have no segment.  dist: n_vertices
 * doubles (a field from pch_solve), a device pointer if dist_on_device else host; levels:
 * n_levels finite doubles (host).  Segments are ordered by face, then by level index.
 * *n_segments gets the total count; the first min(total, capacity) segments are written
 * to segments (host), so a call with capacity 0 only counts.  Errors: INVALID_ARG,
 * CAPACITY (more than 2^31 - 1 segments), OOM, CUDA. */
pch_status pch_iso_contours(const pch_mesh* m, const double* dist, int32_t dist_on_device, const double* levels,
                            int32_t n_levels, pch_contour_segment* segments, int64_t capacity, int64_t* n_segments);

/* Release a mesh and its workspace (NULL is a no-op). */
void pch_destroy(pch_mesh* m);

/* Message of the last error on the calling host thread ("" if none). */
const char* pch_last_error(void);

/* ---- learned selection controller (build-only; no counterpart in the paper) -----------
 * A 3 x 64 hidden-layer fp32 MLP maps per-iteration frontier statistics to the number of
 * windows the next selection takes (output log2(k) / 24, k in [2^8, 2^26]).  Weights are a flat fp32 array of pch_mlp_num_params() values
 * (layer by layer: W then b, W row-major [out][in]). */
int32_t pch_mlp_num_features(void);
int32_t pch_mlp_num_params(void);
/* Install weights used by PCH_CONTROL_LEARNED on the current device (host array, copied
 * to a device buffer the library keeps for that device's current CUDA context; call it on
 * every device that runs learned solves, and again after a device reset). */
pch_status pch_mlp_set_weights(const float* params, int32_t n_params);
/* Forward pass on the device: x (n x num_features), y (n) device pointers. */
pch_status pch_mlp_forward(const float* params_dev, const float* x_dev, int32_t n, float* y_dev,
                           void* stream);
/* Gradient of 0.5 * mean((y - target)^2) w.r.t. the parameters (device pointers);
 * grad_dev gets num_params floats, loss_dev one float.  Deterministic reduction. */
pch_status pch_mlp_backward(const float* params_dev, const float* x_dev, const float* target_dev,
                            int32_t n, float* grad_dev, float* loss_dev, void* stream);
/* Same result as pch_mlp_backward, without allocating: for callers that cannot call
 * cudaMalloc, such as a host application whose own memory manager owns all device
 * memory, or a training loop that must not stall on or fail an allocation mid-run.
 * There is no counterpart in the paper.  Its scratch is one fixed device array of the
 * library (6.3 MB, held on every GPU that loads the library until exit), so n is
 * limited to 4096 samples; a larger n returns PCH_ERR_CAPACITY and computes nothing.
 * The first call on a device (and the first after its CUDA context was replaced, e.g. by
 * cudaDeviceReset) looks the array up for that device; make that first call before any
 * stream capture.  All calls share the array: calls whose work overlaps on
 * the GPU (other threads, other streams) race and must be serialised by the caller.
 * Nothing in the array needs clearing between calls. */
pch_status pch_mlp_backward_noalloc(const float* params_dev, const float* x_dev, const float* target_dev,
                                    int32_t n, float* grad_dev, float* loss_dev, void* stream);
/* One Adam step in place (device pointers; m_dev, v_dev: moment buffers; t >= 1). */
pch_status pch_mlp_adam(float* params_dev, const float* grad_dev, float* m_dev, float* v_dev,
                        int32_t t, float lr, void* stream);
/* Per-iteration features and choices of the last solve on this mesh's workspace (the
 * controller's training traces): up to max_rows rows of num_features floats into
 * features (host), log2(k) / 24 of the k used into chosen (host). */
pch_status pch_trace_fetch(pch_mesh* m, int32_t max_rows, float* features, float* chosen,
                           int32_t* n_rows);

/* ---- autotuner (build-only) ------------------------------------------------------------
 * Times full solves of `src` on `m`: first the library defaults (k 24576, block 64, 32
 * hops), then a coordinate search over windows-per-iteration k (24576 times powers of 4,
 * up to 8x the face count, from the largest down until one is twice as slow as the best)
 * at block 128 and 16 hops, then hops (64, 32, 16, 8, 4, from the most down until one is
 * twice as slow as the best), then propagation block sizes (64, 128, 256); under
 * PCH_CONTROL_LEARNED (the network picks k every iteration) only hops and the block size
 * are searched.  Each trial is timed on its second solve (the first builds its graph),
 * unless its first solve was already twice as slow as the best.
 * Writes the fastest into opt->k, opt->block and opt->hops (the other fields of *opt are
 * kept and used for every trial) and its time into *best_ms (may be NULL).  If
 * cache_path is not NULL the result is looked up first in, and then appended to, that
 * text file, keyed by GPU name, library build id (pch_build_id), mesh size, control and
 * flags, so a second call with the same library does no timing.  Errors: as pch_solve. */
pch_status pch_autotune(pch_mesh* m, const pch_source* src, pch_options* opt, const char* cache_path,
                        double* best_ms);

/* ---- measurement helpers ---------------------------------------------------------- */
/* Build id of the library: the first 16 hex digits of the SHA-256 of its sources (a
 * static string owned by the library). */
const char* pch_build_id(void);

/* Accuracy check of the library's FP64 reciprocal and square root (Newton-Raphson from a
 * single-precision estimate) against IEEE 1/x and sqrt(|x|) on n device doubles x_dev:
 * max_ulp_host[0], [1] get the largest distance in units in the last place. */
pch_status pch_selftest_math(const double* x_dev, int32_t n, unsigned long long* max_ulp_host);

/* Sustained FP64 FMA rate of this GPU (TFLOP/s, 2 flops per FMA) from a
 * register-resident DFMA loop; the roofline denominator for the propagation kernel. */
pch_status pch_measure_fp64_peak(double* tflops);

#ifdef __cplusplus
}
#endif
#endif /* PCH_H_ */
