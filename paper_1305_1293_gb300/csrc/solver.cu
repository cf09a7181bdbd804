// The four-phase PCH iteration (Section 4.2, Algorithm 1) on sm_103a.
//
// One iteration, every phase a kernel over device-resident counts (fixed grids, so the
// whole iteration can be replayed from a CUDA graph):
//   k_tau        Step 1a: per-instance selection threshold from the key histogram
//                (plain: the k-th nearest window, the paper's k; learned: MLP controller)
//   k_compact    Step 1b: windows with key <= tau -> work list, the rest -> next pool
//                (warp ballot / prefix compaction, structure-of-arrays copies)
//   k_propagate  Step 2, Algorithm 2: FP64 unfolding, endpoint / occupancy events,
//                one angle one split, children, Xin-Wang filter
//   k_fan        Step 2, Fig. `fig:propagation`(c): windows from improved pseudo-sources
//   sort         Step 3, Algorithm 3: radix sort of the new windows by edge (radix.cu)
//   k_append     Step 3/4: gap-free append in edge order with per-edge trimming and a
//                re-filter against the updated distances
//   k_finish     loop control (Algorithm 1's "until all windows are processed")
// Events of Algorithm 4 are applied as they are produced: the vertex distance is an
// atomicMin on the ordered 64-bit image of the nonnegative double, which keeps exactly
// the first event of Algorithm 4's (key, value) order; angle_split is one packed 64-bit
// word per half-edge (rounded-up distance | crossing position), also updated by atomicMin.
#include <algorithm>
#include <cmath>
#include <cstring>
#include <vector>

#include "fastmath.cuh"
#include "pch_host.h"
#include "radix.cuh"
#include "solver.cuh"

namespace pch {

// ====================================================================== device helpers
__device__ __forceinline__ int he_next(int h) { return 3 * (h / 3) + (h % 3 + 1) % 3; }

__device__ __forceinline__ double ldg_dist(const unsigned long long* g, unsigned v) {
    return bitsd(__ldcg(g + v));
}

// Pack a (distance to v2, crossing position on the edge) pair for angle_split: the
// distance is rounded UP to 40 significant bits (so a stored value never understates the
// window's distance) and the crossing position, given as xq = 2^24 x / L, floored to 24
// bits.
// Crossing position in angle_split units: floor(xq) clamped to [0, 2^24 - 1].
__device__ __forceinline__ long long angle_pos(double xq) {
    const long long q = __double2ll_rd(xq);
    return q < 0 ? 0 : (q > (long long)kAngleXMask ? (long long)kAngleXMask : q);
}
__device__ __forceinline__ unsigned long long pack_angle(double D, double xq) {
    unsigned long long b = dbits(D);
    if (b & kAngleXMask) b = (b | kAngleXMask) + 1ull;
    return (b & ~kAngleXMask) | (unsigned long long)angle_pos(xq);
}
// kEpsSnap in angle_split units (the snap tolerance kEpsSnap * L times 2^24 / L).
constexpr double kSplitTol = kEpsSnap * (double)(1 << kAngleXBits);

struct WarpScan {
    int excl, total;
};
__device__ __forceinline__ WarpScan warp_scan(int x) {
    const int lane = threadIdx.x & 31;
    int incl = x;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        int t = __shfl_up_sync(0xffffffffu, incl, o);
        if (lane >= o) incl += t;
    }
    return {incl - x, __shfl_sync(0xffffffffu, incl, 31)};
}

// Warp-aggregated reservation of `x` slots per lane on counter `c`; returns the lane's
// base.  With `fill`, a warp that reserved anything gets the counter's value after its
// reservation there (unchanged otherwise).
__device__ __forceinline__ int warp_reserve(int* c, int x, int* fill = nullptr) {
    WarpScan s = warp_scan(x);
    int base = 0;
    if ((threadIdx.x & 31) == 31 && s.total) base = atomicAdd(c, s.total);
    base = __shfl_sync(0xffffffffu, base, 31);
    if (fill && s.total) *fill = base + s.total;
    return base + s.excl;
}

__device__ __forceinline__ void warp_add_ull(unsigned long long* c, int x) {
    int t = warp_scan(x).total;
    if ((threadIdx.x & 31) == 0 && t) atomicAdd(c, (unsigned long long)t);
}

// Where a distance event came from (kept only for geodesic paths): the window's half-edge
// h, its pseudo-source vertex src and position (px, py) in h's frame (kind 0); a fan's
// event along a boundary edge from src (kind 1); a corner of the face-point source's face
// with the point at (px, py) in h's frame (kind 2).
struct EvSrc {
    int inst, h, src, kind;
    double px, py;
};

__device__ __forceinline__ unsigned sm_id() {
    unsigned r;
    asm volatile("mov.u32 %0, %%smid;" : "=r"(r));
    return r;
}

// Record one distance event.  The lanes of the warp that record at the same time reserve
// their slots with one atomic (opportunistic warp aggregation over the active lanes), on
// the counter of the shard of the SM the warp runs on; shard r owns records
// [r * per, (r + 1) * per), per = plog_cap / kPlogShards.
__device__ __forceinline__ void log_event(const Work& w, const EvSrc& es, unsigned v, unsigned long long db) {
    const unsigned mask = __activemask();
    const int lane = threadIdx.x & 31;
    const int leader = __ffs(mask) - 1;
    const int rank = __popc(mask & ((1u << lane) - 1u));
    const int shard = (int)(sm_id() & (kPlogShards - 1));
    int base = 0;
    if (lane == leader) base = atomicAdd(&w.cnt->n_plog_shard[shard], __popc(mask));
    base = __shfl_sync(mask, base, leader);
    const int slot = base + rank;
    const int per = w.plog_cap / kPlogShards;
    if (slot < per) {
        ProvRec r;
        r.db = db; r.inst = es.inst; r.v = (int)v; r.h = es.h; r.src = es.src; r.kind = es.kind; r.pad = 0;
        r.px = es.px; r.py = es.py;
        w.plog[(size_t)shard * per + slot] = r;
    } else {
        atomicOr(&w.cnt->error, kErrProvFull);
    }
}

// Distance event (Algorithm 2, Algorithm 4): min into geod_dist.  Returns true when the
// event lowered the distance of a pseudo-source vertex, or tied with it (equal within the
// filters' relative margin): the caller then files a fan candidate carrying the event's
// incoming direction.  A tie matters where a saddle is reached along two shortest paths
// from different directions: the region behind it is the union of both directions'
// fanned areas.  With PROV an event that lowered the distance is also recorded with its
// origin `es` (geodesic paths).
// Return values, also the kinds of fan candidates (FanReq.tie): kEvNone; kReqLowered (the
// event lowered the distance: a candidate for this iteration's fan of the vertex);
// kReqTie (it tied with the distance: a candidate compared, an iteration later, with the
// direction of the vertex's fan); kReqDeferredTie is a tie so deferred.
enum : int { kEvNone = 0, kReqLowered = 1, kReqTie = 2, kReqDeferredTie = 3 };
template <bool PROV = false>
__device__ __forceinline__ int vertex_event(const Inst& I, unsigned vf, double D, double& gcache,
                                            const Work* w = nullptr, const EvSrc* es = nullptr) {
    const bool pseudo = (vf & kPseudoBit) != 0;
    if (!lt_s(D, gcache)) return pseudo && dbits(D) <= dbits(gcache) + kDomUlps ? kReqTie : kEvNone;
    unsigned v = vf & ~kPseudoBit;
    unsigned long long nb = dbits(D);
    unsigned long long old = atomicMin(I.g + v, nb);
    if (nb < old) {
        if constexpr (PROV) log_event(*w, *es, v, nb);
        gcache = D;
        return pseudo ? kReqLowered : kEvNone;
    }
    gcache = bitsd(old);
    return pseudo && nb <= old + kDomUlps ? kReqTie : kEvNone;
}

// A fan candidate carries the incoming ray as a direction (dx, dy), of any length, in
// the frame of a reference half-edge href leaving v (href < 0: every direction).
__device__ __forceinline__ void push_fan(FanReq* req, int* n, int cap, int* err, int inst, unsigned v, double D,
                                         int href, double dx, double dy, int tie = kReqLowered) {
    int slot = atomicAdd(n, 1);
    if (slot < cap) {
        FanReq r;
        r.inst = inst; r.v = v; r.href = href; r.tie = tie; r.D = D; r.dx = dx; r.dy = dy;
        req[slot] = r;
    } else {
        atomicOr(err, kErrReqFull);
    }
}

__device__ __forceinline__ int hist_bin(double key, double ref, double ilbar) {
    float t = (float)((key - ref) * ilbar);
    t = fmaxf(t, 0.f);
    float b = kBinsPerOctave * __log2f(1.f + kBinScale * t);
    int bi = (int)b;
    return bi < 0 ? 0 : (bi >= kBins ? kBins - 1 : bi);
}

__device__ __forceinline__ double bin_upper(int b, double ref, double lbar) {
    return ref + lbar * (exp2((double)(b + 1) / (double)kBinsPerOctave) - 1.0) / (double)kBinScale;
}

// Writes of windows into the next pool also feed the next iteration's selection
// statistics: per-instance histogram (relative to ctl.ref), minimum key and count.
struct PoolStats {
    unsigned* sh_hist;   // shared-memory histogram (n_inst <= kShHistInst) or nullptr
    unsigned* g_hist;
    int n_inst;
};
constexpr int kShHistInst = 32;      // 32 KB of shared memory per block

__device__ __forceinline__ void pool_stat(const Work& w, const PoolStats& ps, int inst, double key, bool on) {
    // minimum key per instance: warp-reduce when the warp holds a single instance
    const unsigned full = 0xffffffffu;
    unsigned long long kb = on ? dbits(key) : ~0ull;
    int inst0 = __shfl_sync(full, inst, 0);
    bool uniform = __all_sync(full, !on || inst == inst0);
    if (uniform) {
        unsigned long long m = kb;
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) {
            unsigned long long t = __shfl_xor_sync(full, m, o);
            m = t < m ? t : m;
        }
        int cntw = __popc(__ballot_sync(full, on));
        if ((threadIdx.x & 31) == 0 && cntw) {
            atomicMin(&w.ctl[inst0].kmin, m);
            atomicAdd(&w.ctl[inst0].n_next, cntw);
        }
    } else if (on) {
        atomicMin(&w.ctl[inst].kmin, kb);
        atomicAdd(&w.ctl[inst].n_next, 1);
    }
    if (on) {
        const InstCtl& c = w.ctl[inst];
        int b = hist_bin(key, c.ref, w.inst[inst].ilbar);
        if (ps.sh_hist) {
            atomicAdd(&ps.sh_hist[inst * kBins + b], 1u);
        } else {
            // many instances: lanes that hit the same global bin add together
            const int slot = inst * kBins + b;
            const unsigned peers = __match_any_sync(__activemask(), slot);
            if ((threadIdx.x & 31) == __ffs(peers) - 1) atomicAdd(&ps.g_hist[slot], (unsigned)__popc(peers));
        }
    }
}

__device__ __forceinline__ void load_win(const WinSoA& s, int i, int& he, int& inst, double& d, double& A, double& B,
                                         double& px, double& py, double& key, int& src, double& IA, double& IB) {
    he = s.he[i]; inst = s.inst[i]; d = s.d[i]; A = s.A[i]; B = s.B[i]; px = s.px[i]; py = s.py[i]; key = s.key[i];
    src = s.src[i]; IA = s.IA[i]; IB = s.IB[i];
}
__device__ __forceinline__ void store_win(const WinSoA& s, int i, int he, int inst, double d, double A, double B,
                                          double px, double py, double key, int src, double IA, double IB) {
    s.he[i] = he; s.inst[i] = inst; s.d[i] = d; s.A[i] = A; s.B[i] = B; s.px[i] = px; s.py[i] = py; s.key[i] = key;
    s.src[i] = src; s.IA[i] = IA; s.IB[i] = IB;
}

// A window whose pseudo-source vertex has since been reached by a shorter path is
// useless: the same straight segment from that vertex, after the shorter path, is a
// real path of smaller length (build-side filter; the paper's filters are in Fig.
// `fig:filter`).
__device__ __forceinline__ bool stale_source(const Inst& I, int src, double d) {
    return src >= 0 && dominated(d, bitsd(__ldcg(I.g + src)));
}

// ====================================================================== init
__global__ void k_fill_inf(unsigned long long* g, long long n) {
    const unsigned long long inf = 0x7FF0000000000000ull;
    for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x)
        g[i] = inf;
}

// Algorithm 1, initialisation: geod_dist = 0 at the sources; a window on every edge
// opposite a source (issued as the source's fan request); for a point inside a face,
// one window on each edge of the face and the three corner distances.
__global__ void k_init_sources(Work w, const SrcDev* __restrict__ srcs, int n_src) {
    Counters* cnt = w.cnt;
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n_src; i += gridDim.x * blockDim.x) {
        SrcDev s = srcs[i];
        const Inst& I = w.inst[s.inst];
        if (s.kind == 0) {
            I.g[s.vertex] = 0ull;
            // the source's fan covers every direction
            push_fan(w.req[0], &cnt->n_req, w.req_cap, &cnt->error, s.inst, (unsigned)s.vertex, 0.0, -1, 0.0, 0.0);
        }
    }
}

// Face-point sources (one thread each, after k_init_sources): corner distances and the
// three windows, written to the child arena of iteration 0.
__global__ void k_init_face_sources(Work w, const SrcDev* __restrict__ srcs, int n_src) {
    Counters* cnt = w.cnt;
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n_src; i += gridDim.x * blockDim.x) {
        SrcDev s = srcs[i];
        if (s.kind != 1) continue;
        const Inst& I = w.inst[s.inst];
        for (int k = 0; k < 3; ++k) {
            int h = 3 * s.face + k;
            HERec R = I.rec[h];
            // barycentric weights of h's end vertex and apex (its start vertex sits at 0)
            double b1 = s.bary[(k + 1) % 3], b2 = s.bary[(k + 2) % 3];
            double x = b1 * R.L + b2 * R.xc, y = b2 * R.yc;        // point in h's frame
            double dstart = sqrt(x * x + y * y);
            double gc = ldg_dist(I.g, R.v0 & ~kPseudoBit);
            const EvSrc es{s.inst, h, -1 - s.label, 2, x, y};
            if (const int ev = w.plog ? vertex_event<true>(I, R.v0, dstart, gc, &w, &es) : vertex_event(I, R.v0, dstart, gc)) {
                // incoming direction: from the corner towards the point, inside face(h)
                push_fan(w.req[0], &cnt->n_req, w.req_cap, &cnt->error, s.inst, R.v0 & ~kPseudoBit, dstart, h, x, y, ev);
            }
            if (R.twin < 0) continue;
            // window on twin(h) = (v1 -> v0): point at (L - x, -y), interval [0, L]
            double px = R.L - x, py = -y;
            const double IA = sqrt(px * px + py * py), IB = sqrt((px - R.L) * (px - R.L) + py * py);
            double key = px < 0 ? IA : (px > R.L ? IB : -py);
            int slot = atomicAdd(&cnt->n_child, 1);
            if (slot < w.arena_cap) store_win(w.arena, slot, R.twin, s.inst, 0.0, 0.0, R.L, px, py, key, -1 - s.label, IA, IB);
        }
    }
}

// ====================================================================== Step 1: selection
// Per instance: the plain control selects the k nearest windows (Section 4.2, Step 1)
// through the key histogram: tau = upper edge of the first bin where the cumulative
// count reaches k.  Also rolls the histogram reference and the running minimum.
__global__ void k_tau(Work w, int control, const float* __restrict__ mlp) {
    __shared__ unsigned sh[kBins];
    __shared__ float feat[kFeatures];
    __shared__ float hb0[kHidden], hb1[kHidden];
    __shared__ float y;
    Counters* cnt = w.cnt;
    if (cnt->halt) return;
    const int it = cnt->iter;
    const unsigned* hist = w.hist[it & 1];
    unsigned* hist_nx = w.hist[(it + 1) & 1];
    for (int inst = blockIdx.x; inst < w.n_inst; inst += gridDim.x) {
        InstCtl& c = w.ctl[inst];
        const int np = c.n_next;
        for (int b = threadIdx.x; b < kBins; b += blockDim.x) sh[b] = hist[inst * kBins + b];
        __syncthreads();
        const bool learned = control == PCH_CONTROL_LEARNED && mlp != nullptr && np > 0;
        if ((learned || w.trace) && threadIdx.x == 0) controller_features(c, w.inst[inst], sh, np, it, feat);
        __syncthreads();
        if (learned) mlp_forward_block(mlp, feat, hb0, hb1, &y);
        if (threadIdx.x == 0) {
            double tau;
            const double ref = c.ref;
            const double lbar = w.inst[inst].lbar;
            long long k = c.k_target;
            if (learned) {
                c.ctl_out = y;
                // y = log2(windows to select) / 24, clamped to the range of k the network
                // was trained on (2^12 to 2^24); the plain k only when it is not finite.
                // (Falling back to the plain k for a finite output beyond that range, a
                // small k under this control, made late iterations select few windows.)
                if (isfinite(y)) k = (long long)exp2(24.0 * (double)fminf(fmaxf(y, 12.f / 24.f), 1.f));
            }
            if (np == 0) {
                tau = -INFINITY;
            } else if ((long long)np <= k) {
                tau = INFINITY;
            } else {
                long long run = 0;
                int b = 0;
                for (; b < kBins; ++b) {
                    run += sh[b];
                    if (run >= k) break;
                }
                tau = b >= kBins - 1 ? INFINITY : bin_upper(b, ref, lbar);
            }
            if (w.trace && np > 0) {
                int row = atomicAdd(w.trace_rows, 1);
                if (row < w.trace_cap) {
                    float* f = w.trace + (size_t)row * (kFeatures + 2);
                    for (int j = 0; j < kFeatures; ++j) f[j] = feat[j];
                    f[kFeatures] = (float)(log2((double)k) / 24.0);
                    f[kFeatures + 1] = (float)inst;
                }
            }
            // the strided selection decides by per-thread thresholds instead; tau = -inf
            // also turns chaining off (the paper propagates each selected window one hop)
            c.tau = control == PCH_CONTROL_STRIDED ? -INFINITY : tau;
            c.n_pending = np;
            c.n_next = 0;
            if (c.kmin != ~0ull) c.ref = bitsd(c.kmin);   // min key of the current pool
            c.kmin = ~0ull;
        }
        for (int b = threadIdx.x; b < kBins; b += blockDim.x) hist_nx[inst * kBins + b] = 0u;
        __syncthreads();
    }
}

// Section 5.1's approximate k-selection: virtual thread t of T scans the pool positions
// t, t + T, t + 2T, ... and keeps its M nearest windows (by key, ties to the earlier
// position); the M-th of them is the thread's threshold (all ones when it owns fewer than
// M windows: it selects all of them).  k_compact then selects position i when
// (key bits, i) <= the threshold of thread i mod T, so T * M windows are selected in
// total (every window when the pool holds fewer).  The scan is coalesced: neighbouring
// threads read neighbouring positions.
template <int M>
__global__ void __launch_bounds__(256) k_strided(Work w) {
    Counters* cnt = w.cnt;
    if (cnt->halt) return;
    const int T = w.stride_T;
    const double* __restrict__ key = w.pool[cnt->iter & 1].key;
    const int n = min(cnt->n_pending, w.pool_cap);
    for (int t = blockIdx.x * blockDim.x + threadIdx.x; t < T; t += gridDim.x * blockDim.x) {
        unsigned long long bk[M];
        int bi[M];
#pragma unroll
        for (int j = 0; j < M; ++j) { bk[j] = ~0ull; bi[j] = 0x7fffffff; }
        for (int i = t; i < n; i += T) {
            const unsigned long long kb = dbits(__ldcs(key + i));
            if (kb < bk[M - 1]) {      // positions increase: an equal key keeps the earlier one
                bk[M - 1] = kb;
                bi[M - 1] = i;
#pragma unroll
                for (int j = M - 1; j > 0; --j) {
                    if (bk[j] < bk[j - 1]) {
                        const unsigned long long tk = bk[j]; bk[j] = bk[j - 1]; bk[j - 1] = tk;
                        const int ti = bi[j]; bi[j] = bi[j - 1]; bi[j - 1] = ti;
                    }
                }
            }
        }
        w.sthr_key[t] = bk[M - 1];
        w.sthr_idx[t] = bi[M - 1];
    }
}

// Compaction: selected windows to the work list, the rest to the next pool.
__global__ void __launch_bounds__(256) k_compact(Work w) {
    __shared__ unsigned sh_hist[kShHistInst * kBins];
    Counters* cnt = w.cnt;
    if (cnt->halt) return;
    const int it = cnt->iter;
    const WinSoA cur = w.pool[it & 1], nxt = w.pool[(it + 1) & 1];
    const int n = min(cnt->n_pending, w.pool_cap);
    PoolStats ps{w.n_inst <= kShHistInst ? sh_hist : nullptr, w.hist[(it + 1) & 1], w.n_inst};
    if (ps.sh_hist) {
        for (int j = threadIdx.x; j < w.n_inst * kBins; j += blockDim.x) sh_hist[j] = 0u;
        __syncthreads();
    }
    for (int base = blockIdx.x * blockDim.x; base < n; base += gridDim.x * blockDim.x) {
        int i = base + threadIdx.x;
        bool valid = i < n;
        int he = 0, inst = 0, src = -1;
        double d = 0, A = 0, B = 0, px = 0, py = 0, key = 0, IA = 0, IB = 0;
        if (valid) {
            load_win(cur, i, he, inst, d, A, B, px, py, key, src, IA, IB);
            if (stale_source(w.inst[inst], src, d)) valid = false;   // dropped from the pool
        }
        bool sel;
        if (w.stride_T > 0) {           // strided selection: the owning thread's threshold
            const int t = i % w.stride_T;
            const unsigned long long kb = dbits(key), tk = w.sthr_key[t];
            sel = valid && (kb < tk || (kb == tk && i <= w.sthr_idx[t]));
        } else {
            sel = valid && key <= w.ctl[inst].tau;
        }
        int slot = warp_reserve(&cnt->n_sel, sel ? 1 : 0);
        if (sel && slot >= w.sel_cap) sel = false;   // work list full: stays pending
        if (sel) store_win(w.sel, slot, he, inst, d, A, B, px, py, key, src, IA, IB);
        bool rest = valid && !sel;
        int rslot = warp_reserve(&cnt->n_rest, rest ? 1 : 0);
        if (rest) store_win(nxt, rslot, he, inst, d, A, B, px, py, key, src, IA, IB);
        pool_stat(w, ps, inst, key, rest);
    }
    if (ps.sh_hist) {
        __syncthreads();
        for (int j = threadIdx.x; j < w.n_inst * kBins; j += blockDim.x)
            if (sh_hist[j]) atomicAdd(&ps.g_hist[j], sh_hist[j]);
    }
}

// ====================================================================== Step 2: propagation
struct ChildOut {
    int he;
    double A, B, px, py, key;
    double IA, IB;          // |I A|, |I B| (reused when the child is propagated at once)
};

// The ray from I along D = P - I (P a window endpoint on the parent edge, D = (dx, -py)
// in the parent frame) meets the child's line O + s u where
//   s = cross(I - O, D) / cross(u, D),   I + t D with t = cross(I - O, u) / cross(u, D),
// and cross(I - O, u) = -Ipy.  Inputs: upy = ux py, rpy = rx py, (rx, ry) = I - O.
// Returns s and |I X| = t |D|.  A hit within 2^-40 Lc beyond an end (rounding, for a
// parent window that ends on a vertex) is clamped to that end with |I X| kept; a hit
// further outside [0, Lc] (or a ray that does not cross) is clamped to the nearer end
// with |I X| recomputed there.
__device__ __forceinline__ void ray_hit(double dx, double ID, double ux, double uy, double ry, double upy, double rpy,
                                        double py, double Ipx, double Ipy, double Lc, double& xh, double& IX) {
    const double den = -fma(uy, dx, upy);   // cross(u, D)
    const double r = rcp_nr(den);           // full precision: |I X| compounds along a lineage
    xh = -fma(ry, dx, rpy) * r;             // cross(I - O, D) / cross(u, D)
    IX = (-Ipy * r) * ID;
    if (!gt0_s(den) || !(ge0_s(xh) && le_s(xh, Lc))) {
        const long long xb = sbits(xh);
        if (gt0_s(den) && xb < 0 && (xb & 0x7fffffffffffffffll) <= sbits(times_eps(Lc))) {
            xh = 0.0;
            return;
        }
        if (gt0_s(den) && xb > sbits(Lc) && xb - sbits(Lc) <= kSnapUlps) {
            xh = Lc;
            return;
        }
        xh = gt0_s(den) ? (lt_s(xh, 0.0) ? 0.0 : (lt_s(Lc, xh) ? Lc : xh))
                        : (gt0_s(fma(ux, dx, -uy * py)) ? Lc : 0.0);   // dot(u, D) > 0: towards Lc
        if (!(xh == xh)) xh = 0.0;
        const double ex = xh - Ipx;
        IX = sqrt_nr(fma(ex, ex, Ipy * Ipy));
    }
}

__device__ __forceinline__ double child_key(double d, double a, double b, double Ipx, double Ipy, double IA,
                                            double IB) {
    return d + (lt_s(Ipx, a) ? IA : (lt_s(b, Ipx) ? IB : -Ipy));
}

// dominated(lhs, rhs) with rhs = g + sqrt(q): compares squares, no square root.
constexpr double kInvDom = 1.0 / (1.0 + kDomRel);
__device__ __forceinline__ bool dominated_sq(double lhs, double g, double q) {
    const double t = lhs * kInvDom - g;
    return gt0_s(t) && gt0_s(fma(t, t, -q));
}

// The round's write side of the propagation kernel's shared-memory queue: the second
// child of a window whose rays reach v2 is deferred there as a task, so that each lane
// computes one child per round.
struct TaskQueue {
    double *d, *A, *B, *px, *py, *IA, *IB;
    int *he, *inst, *src, *hop;
    int* count;   // entries reserved this round
    int cap;      // entries the next round can take
};
constexpr int kHopTask = 1 << 30;   // hop-field flag of a queue entry: a deferred left child

// Algorithm 2 for one window: events, one angle one split, children with the Xin-Wang
// filter.  Returns whether the window passed the filter; children in c0, c1 (nch).  When
// both children exist the left one is deferred to q as a task (if q has room).  A task
// (task = true) skips the window's own part, done in an earlier round, and computes the
// left child only; IB_in then holds |I v2|.
template <bool PROV>
__device__ __forceinline__ bool propagate_window(const Work& w, Counters* cnt, FanReq* req, int inst,
                                                 int src, double d, int h, double A, double B, double px, double py,
                                                 bool task, int hop, const TaskQueue& q, ChildOut& c0, ChildOut& c1,
                                                 int& nch, int& occ_out, int& ncomp, int& nray, double IA_in,
                                                 double IB_in) {
    bool prop = false;
    nch = 0;
    occ_out = 0;
    ncomp = 0;
    nray = 0;
    {
        const Inst& I = w.inst[inst];
        const HERec R = I.rec[h];
        const double L = R.L;
        double g0 = ldg_dist(I.g, R.v0 & ~kPseudoBit);
        double g1 = ldg_dist(I.g, R.v1 & ~kPseudoBit);
        double g2 = ldg_dist(I.g, R.v2 & ~kPseudoBit);
        const double ax = A - px, bx = B - px;
        // |IA|, |IB|: carried over from the parent when the window was chained
        const double IA = ge0_s(IA_in) ? IA_in : sqrt_nr(fma(ax, ax, py * py));
        const double IB = ge0_s(IB_in) ? IB_in : sqrt_nr(fma(bx, bx, py * py));
        const double xc = R.xc, yc = R.yc;
        bool left = false, right = false, occ = false;
        double Iv2 = IB;
        if (task) {
            occ = true;
            left = R.tw2 >= 0;
        } else if ((hop > 0 || !(dominated(d + IB, g0 + B) || dominated(d + IA, g1 + (L - A)))) &&
                   !stale_source(I, src, d)) {
            // Xin-Wang endpoint tests against the current distances passed: the window is
            // useless if the path via v0 beats it at B, or the path via v1 at A.  A chained
            // window (hop > 0) passed the same two tests when its parent created it a round
            // ago; distances only fall, so repeating them could only prune more, never keep
            // a window that must go, and they are skipped.
            prop = true;
            const EvSrc es{inst, h, src, 0, px, py};   // event origin, recorded with PROV only
            const double py2 = py * py;
            const double tol = times_eps(L);
            const double tiny = tol;
            // Algorithm 2: endpoint events at v0 (A = v0) and v1 (B = v1)
            if (le_s(A, tol)) {
                double D0 = d + (sbits(A) == 0 ? IA : sqrt_nr(fma(px, px, py2)));
                if (const int ev = vertex_event<PROV>(I, R.v0, D0, g0, &w, &es))   // the ray arrives at v0 from I (h's frame)
                    push_fan(req, &cnt->n_req, w.req_cap, &cnt->error, inst, R.v0 & ~kPseudoBit, D0, h, px, py, ev);
            }
            if (sbits(L) - sbits(B) <= kSnapUlps) {
                double q = L - px;
                double D1 = d + (sbits(B) == sbits(L) ? IB : sqrt_nr(fma(q, q, py2)));
                if (const int ev = vertex_event<PROV>(I, R.v1, D1, g1, &w, &es))   // at v1, in the frame of twin(h) = (v1 -> v0)
                    push_fan(req, &cnt->n_req, w.req_cap, &cnt->error, inst, R.v1 & ~kPseudoBit, D1, R.twin, q, -py, ev);
            }
            // occupancy of v2: the ray I -> v2 crosses e at xs = px + num / den;
            // decided without the division (den > 0), by the signs of fused residuals
            const double den = yc - py, num = (xc - px) * (-py);
            const bool before_A = gt0_s(fma(ax - tol, den, -num));
            occ = !before_A && ge0_s(fma(bx + tol, den, -num));
            occ_out = occ;
            if (occ) {
                const double xs = px + num * rcp_nr(den);
                const double xcl = lt_s(xs, A) ? A : (lt_s(B, xs) ? B : xs);
                // angle_split position: xs in units of 2^-24 |e| (only the order of positions
                // on one edge matters, so any fixed scale per edge will do)
                const double xq = xs * (rcp_nr(L) * (double)(1 << kAngleXBits));
                const double dx = xc - px, dy = yc - py;
                Iv2 = sqrt_nr(dx * dx + dy * dy);
                const double D2 = d + Iv2;
                // one angle one split (Fig. `fig:filter`(a)) against angle_split[h]
                unsigned long long* ap = I.ang + h;
                const unsigned long long aw = __ldcg(ap);
                bool win = aw == kEmptyAngle || dbits(D2) < (aw & ~kAngleXMask);
                if (win) {
                    left = right = true;
                    atomicMin(ap, pack_angle(D2, xq));
                } else {
                    // loser: keep the child on its own side of the winner's ray, which
                    // crosses e in [q, q + 1] (angle_split units), widened by the snap
                    // tolerance
                    // (positions compared after the same clamping the stored one had)
                    const long long q = (long long)(aw & kAngleXMask);
                    left = angle_pos(xq + kSplitTol) < q;
                    right = angle_pos(xq - kSplitTol) > q;
                    if (!left && !right) left = right = true;
                }
                if (const int ev = vertex_event<PROV>(I, R.v2, D2, g2, &w, &es)) {
                    // the ray arrives at v2 inside face(h); direction to I in the frame of
                    // prev(h) = (v2 -> v0), whose axis is (-xc, -yc) / L2
                    const int hp = 3 * (h / 3) + (h % 3 + 2) % 3;
                    const double ux = -R.u2x, uy = -R.u2y, ex = px - xc, ey = py - yc;
                    push_fan(req, &cnt->n_req, w.req_cap, &cnt->error, inst, R.v2 & ~kPseudoBit, D2, hp,
                             ex * ux + ey * uy, ux * ey - uy * ex, ev);
                }
                if (le_s(B - xcl, tiny)) right = false;
                if (le_s(xcl - A, tiny)) left = false;
            } else {
                right = before_A;
                left = !right;
            }
            right = right && R.tw1 >= 0;
            left = left && R.tw2 >= 0;
        }
        {
            // Children, one code path in child order (right first): the right child
            // lies on edge v2 -> v1 (frame origin v2), the left on v0 -> v2 (origin v0).
            // When v2 is occupied the child's endpoint at v2 is exact.
#pragma unroll 1
            for (int j = 0; j < 2; ++j) {
                if (!(j == 0 ? (right || left) : (right && left))) break;
                if (j == 1) {   // defer the left child: one child per lane and round
                    const int ts = atomicAdd(q.count, 1);
                    if (ts < q.cap) {
                        q.he[ts] = h; q.inst[ts] = inst; q.src[ts] = src; q.hop[ts] = hop | kHopTask;
                        q.d[ts] = d; q.A[ts] = A; q.B[ts] = B; q.px[ts] = px; q.py[ts] = py;
                        q.IA[ts] = IA; q.IB[ts] = Iv2;
                        break;
                    }
                }
                const bool rt = j == 0 && right;
                ++ncomp;
                nray += occ ? 1 : 2;
                {   // the child's record, needed when it is propagated (next round when chained)
                    const char* cr = reinterpret_cast<const char*>(I.rec + (rt ? R.tw1 : R.tw2));
                    asm volatile("prefetch.global.L1 [%0];" ::"l"(cr));
                    asm volatile("prefetch.global.L1 [%0];" ::"l"(cr + sizeof(HERec) - 8));
                }
                // both sides as one select-driven path (a warp holds left and right children)
                const double Lc = rt ? R.L1 : R.L2;
                const double ox = rt ? xc : 0.0, oy = rt ? yc : 0.0;
                const double ux = rt ? R.u1x : R.u2x;
                const double uy = rt ? R.u1y : R.u2y;
                const double rx = px - ox, ry = py - oy;
                const double Ipx = fma(rx, ux, ry * uy), Ipy = fma(ux, ry, -(uy * rx));
                const double upy = ux * py, rpy = rx * py;
                // rays through A and B; at v2 (occupied) the right child starts at 0,
                // the left child ends at Lc
                double a, IAc, b, IBc;
                if (occ && rt) {
                    a = 0.0;
                    IAc = Iv2;
                } else {
                    ray_hit(ax, IA, ux, uy, ry, upy, rpy, py, Ipx, Ipy, Lc, a, IAc);
                }
                if (occ && !rt) {
                    b = Lc;
                    IBc = Iv2;
                } else {
                    ray_hit(bx, IB, ux, uy, ry, upy, rpy, py, Ipx, Ipy, Lc, b, IBc);
                }
                if (!lt_s(times_eps(Lc), b - a)) continue;
                // Xin-Wang filter (Fig. `fig:filter`(b)) on the new window: against its
                // start and end vertices (right child: v2, v1; left child: v0, v2), and
                // against the vertex T of the parent edge off the child's edge (right: v0;
                // left: v1), at both ends of the child.  d + |I x| - |T x| is smallest at
                // the end nearer the vertex shared with the parent edge (the end the paper
                // tests); requiring both ends is the same decision in exact arithmetic and
                // keeps the child when rounding puts one end's test on the wrong side of
                // the margin.
                const double gS = rt ? g2 : g0, gE = rt ? g1 : g2, gT = rt ? g0 : g1;
                const double dA = d + IAc, dB = d + IBc;
                const double Tx = rt ? xc : -L;           // the child's origin relative to T
                const double Xax = fma(a, ux, Tx), Xay = fma(a, uy, oy);
                const double Xbx = fma(b, ux, Tx), Xby = fma(b, uy, oy);
                const bool useless = dominated(dB, gS + b) || dominated(dA, gE + (Lc - a)) ||
                                     (dominated_sq(dA, gT, fma(Xax, Xax, Xay * Xay)) &&
                                      dominated_sq(dB, gT, fma(Xbx, Xbx, Xby * Xby)));
                if (useless) continue;
                const ChildOut co{rt ? R.tw1 : R.tw2, a, b, Ipx, Ipy, child_key(d, a, b, Ipx, Ipy, IAc, IBc), IAc, IBc};
                if (nch == 0) c0 = co;
                else c1 = co;
                ++nch;
            }
        }
    }
    return prop;
}

// Windows in flight per warp: the shared-memory queue of chained children holds at most
// one window per lane, in two buffers (read / written by alternate rounds) of 7 doubles
// and 4 ints per entry (blocks of at most 256 threads: 36 KB).
constexpr int kPropQueueBytesPerThread = 2 * (7 * 8 + 4 * 4);
constexpr int kPropMaxWarps = 8;      // warps per block at most (256 threads)

// Step 3 of the iteration (Algorithm 2 over the selected windows), persistent.  Every
// warp advances on its own in rounds: in each round lane t takes entry t of the warp's
// queue (a child chained from the warp's previous round, key <= tau, at most `hops` hops
// from its selected ancestor) or else a fresh selected window; children that continue
// are pushed back into the warp's queue (chaining stops while the child arena is half
// full).  Repacking the chains onto the warp's lowest lanes every round keeps the lanes
// that issue FP64 work together; no warp waits for another (only __syncwarp between
// rounds), and a warp leaves once the selected list is exhausted and its queue is empty.
// A warp takes at most ceil(selected / resident warps) fresh windows at once (take_min
// at least), so that a short list (the first iterations, a ring-shaped frontier) keeps
// every resident warp busy and the chains' deferred children fill the free lanes.
// 168 registers a thread at most (164 used, no spills): 6 blocks of 64 threads per SM.
// PROV: also record the distance events (geodesic paths).
template <bool PROV>
__global__ void __maxnreg__(168) k_propagate(Work w, int hops, int tail_cut, int take_min) {
    extern __shared__ double q_mem[];   // blockDim.x * kPropQueueBytesPerThread bytes
    const int QB = 2 * blockDim.x;
    double* q_d = q_mem;
    double* q_A = q_d + QB;
    double* q_B = q_A + QB;
    double* q_px = q_B + QB;
    double* q_py = q_px + QB;
    double* q_IA = q_py + QB;
    double* q_IB = q_IA + QB;
    int* q_he = reinterpret_cast<int*>(q_IB + QB);
    int* q_inst = q_he + QB;
    int* q_src = q_inst + QB;
    int* q_hop = q_src + QB;
    // per warp and buffer: entries written (by the round that writes that buffer)
    __shared__ int s_cnt[kPropMaxWarps][2];
    Counters* cnt = w.cnt;
    if (cnt->halt) return;
    const unsigned full = 0xffffffffu;
    const int lane = threadIdx.x & 31;
    const int wid = threadIdx.x >> 5;
    const unsigned lt = (1u << lane) - 1u;
    const int it = cnt->iter;
    const int n = min(cnt->n_sel, w.sel_cap);
    FanReq* req = w.req[it & 1];
    const int room = w.arena_cap / 2 - 2 * (int)(gridDim.x * blockDim.x);
    // Fresh windows a warp holds at once: a short selected list is spread over all
    // resident warps (take_min a warp at least), so that the lanes left free take the
    // deferred children of the chains instead of the arena; a list of a warp's width per
    // resident warp or more fills whole warps.
    const int nwarps = (int)(gridDim.x * (blockDim.x >> 5));
    const int quota = max(take_min, min(32, (n + nwarps - 1) / max(nwarps, 1)));
    const unsigned take_mask = quota >= 32 ? 0xffffffffu : (1u << quota) - 1u;
    // the arena fill this warp last saw (updated whenever it reserves arena slots): a
    // warp overshoots the room by at most one round of its own writes
    int seen_child = *(volatile int*)&cnt->n_child;
    // statistics, kept per thread and added to the counters once when the warp ends
    unsigned n_prop = 0, n_chain = 0, n_exam = 0, n_occ = 0, n_comp = 0, n_ray = 0;
    if (lane == 0) s_cnt[wid][0] = s_cnt[wid][1] = 0;
    bool dry = false;          // uniform over the warp: the selected list is exhausted
    for (int r = 0;; ++r) {
        const int rb = r & 1, wb = rb ^ 1;
        __syncwarp();          // last round's queue writes are visible, its reads are done
        const int nq = min(s_cnt[wid][rb], 32);
        __syncwarp();          // every lane has read the count before it is reused
        if (lane == 0) s_cnt[wid][wb] = 0;
        __syncwarp();
        const int qr = rb * blockDim.x + wid * 32 + lane;   // this lane's entry in the read buffer
        bool have = lane < nq, task = false;
        int h = 0, inst = 0, src = -1, hop = 0;
        double d = 0.0, A = 0.0, B = 0.0, px = 0.0, py = 0.0, cIA = -1.0, cIB = -1.0;
        if (have) {
            h = q_he[qr]; inst = q_inst[qr]; src = q_src[qr]; hop = q_hop[qr];
            task = (hop & kHopTask) != 0;
            hop &= ~kHopTask;
            d = q_d[qr]; A = q_A[qr]; B = q_B[qr]; px = q_px[qr]; py = q_py[qr];
            cIA = q_IA[qr]; cIB = q_IB[qr];
        }
        const unsigned need = __ballot_sync(full, !have) & take_mask;   // lanes nq.. below the quota
        if (need && !dry) {
            int base = 0;
            if (lane == 0) base = atomicAdd(&cnt->work_next, __popc(need));
            base = __shfl_sync(full, base, 0);
            if (base + __popc(need) >= n) dry = true;
            if ((need >> lane) & 1u) {
                const int idx = base + __popc(need & lt);
                if (idx < n) {
                    h = w.sel.he[idx]; inst = w.sel.inst[idx]; d = w.sel.d[idx]; src = w.sel.src[idx];
                    A = w.sel.A[idx]; B = w.sel.B[idx]; px = w.sel.px[idx]; py = w.sel.py[idx];
                    cIA = w.sel.IA[idx]; cIB = w.sel.IB[idx];
                    have = true;
                }
            }
        }
        if (!__any_sync(full, have)) {             // nothing queued and nothing left to take
            const unsigned sums[6] = {__reduce_add_sync(full, n_prop), __reduce_add_sync(full, n_chain),
                                      __reduce_add_sync(full, n_exam), __reduce_add_sync(full, n_occ),
                                      __reduce_add_sync(full, n_comp), __reduce_add_sync(full, n_ray)};
            unsigned long long* dst[6] = {&cnt->propagated, &cnt->chained, &cnt->examined, &cnt->occupied,
                                          &cnt->children, &cnt->rays};
            if (lane < 6 && sums[lane]) atomicAdd(dst[lane], (unsigned long long)sums[lane]);
            break;
        }
        ChildOut c0, c1;
        int nch = 0, occ = 0, ncomp = 0, nray = 0;
        bool prop = false;
        const int wo = wb * blockDim.x + wid * 32;  // the warp's region of the write buffer
        const TaskQueue tq{q_d + wo, q_A + wo, q_B + wo, q_px + wo, q_py + wo, q_IA + wo, q_IB + wo,
                           q_he + wo, q_inst + wo, q_src + wo, q_hop + wo, &s_cnt[wid][wb], 32};
        if (have)
            prop = propagate_window<PROV>(w, cnt, req, inst, src, d, h, A, B, px, py, task, hop, tq, c0, c1, nch,
                                          occ, ncomp, nray, cIA, cIB);
        bool cont = have && nch > 0 && hop + 1 < hops && le_s(c0.key, w.ctl[inst].tau) &&
                    (!dry || nq >= tail_cut) && seen_child < room;
        // the continuing child goes to the queue while it has room, every other child to
        // the arena
        const int qs = warp_reserve(&s_cnt[wid][wb], cont ? 1 : 0);
        if (cont && qs >= 32) cont = false;
        if (cont) {
            const int q = wo + qs;
            q_he[q] = c0.he; q_inst[q] = inst; q_src[q] = src; q_hop[q] = hop + 1;
            q_d[q] = d; q_A[q] = c0.A; q_B[q] = c0.B; q_px[q] = c0.px; q_py[q] = c0.py;
            q_IA[q] = c0.IA; q_IB[q] = c0.IB;
        }
        const int nwrite = have ? (cont ? nch - 1 : nch) : 0;
        int fill = -1;
        const int slot = warp_reserve(&cnt->n_child, nwrite, &fill);
        if (fill >= 0) seen_child = fill;
        if (nwrite > 0) {
            const ChildOut& cf = cont ? c1 : c0;
            if (slot < w.arena_cap)
                store_win(w.arena, slot, cf.he, inst, d, cf.A, cf.B, cf.px, cf.py, cf.key, src, cf.IA, cf.IB);
            else atomicOr(&cnt->error, kErrPoolFull);
        }
        if (nwrite > 1) {
            if (slot + 1 < w.arena_cap)
                store_win(w.arena, slot + 1, c1.he, inst, d, c1.A, c1.B, c1.px, c1.py, c1.key, src, c1.IA, c1.IB);
            else atomicOr(&cnt->error, kErrPoolFull);
        }
        n_prop += prop ? 1u : 0u;
        n_chain += cont ? 1u : 0u;
        n_exam += have && !task ? 1u : 0u;
        n_occ += (unsigned)occ;
        n_comp += (unsigned)ncomp;
        n_ray += (unsigned)nray;
    }
}

// Pseudo-source fans (Fig. `fig:propagation`(c)).  For each fan candidate whose distance
// is still the vertex's distance (one per vertex per iteration): windows with I = the
// vertex and d = its distance on the edges opposite it, restricted to the fanned area:
// the directions at least pi away from the incoming ray on both sides (a wedge of width
// total angle - 2 pi at an interior saddle; at a boundary vertex the directions that
// wrap around it).  Boundary edges get their endpoint events instead of a window.
//
// No trigonometry at fan time: the mesh keeps, for every half-edge leaving a vertex, the
// unit complex number of its angular position, and for every vertex that of its total
// angle.  The incoming direction times its reference half-edge's number is the incoming
// ray in the vertex's angular frame; the wedge boundaries are that ray turned by pi (and
// by the total angle), and turned back into a corner's own frame by the conjugate of the
// corner's number: a few FP64 products, then one division for the point on the opposite
// edge.  FP32 angles (good to about 1e-6 radians) only pick the corners a boundary may
// fall in, with a margin; a boundary that proves to lie outside its corner clamps to the
// corner's end, so the choice never changes a window.
constexpr float kPiF = 3.14159265358979f;
constexpr float kFanPickMargin = 1e-4f;   // radians: corners within this of a wedge boundary are computed exactly
// interval widening for FP64 rounding, relative to the edge length: the fanned area's
// boundary and the children of windows passing the vertex are computed from different
// unfoldings, whose pseudo-source coordinates carry rounding accumulated over long
// lineages (up to about 1e-10 of the edge on the 5.2M-face sphere)
constexpr double kFanWiden = 1e-7;
constexpr int kFanLanes = 8;              // lanes per fan candidate (corners handled in turn)
// Ties: a fan candidate whose distance equals the vertex's final one within the filters'
// margin but that did not make the iteration's fan (another candidate did) is deferred to
// the next iteration and fanned there when its incoming direction differs from that of
// the vertex's last fan: on another sheet of the angular coordinate (more than
// kTieSheet apart in FP32) or, on the same sheet, by more than kTieDir radians (FP64 unit
// directions; below that the fanned areas differ by less than the fan intervals'
// widening kFanWiden).  Events of one geodesic family that tie (the same pseudo-source
// reached through different windows) are thus fanned once.
constexpr float kTieSheet = 1e-3f;        // radians
constexpr double kTieDir = 1e-9;          // radians

__device__ __forceinline__ double2 cmul(double2 a, double2 b) {
    return make_double2(fma(a.x, b.x, -a.y * b.y), fma(a.x, b.y, a.y * b.x));
}
__device__ __forceinline__ double2 cmul_conj(double2 a, double2 b) {   // a * conj(b)
    return make_double2(fma(a.x, b.x, a.y * b.y), fma(a.y, b.x, -a.x * b.y));
}

// Where the ray from the apex v of o's face along z (relative to the direction
// v -> start(o), any length) meets o: distance from start(o), clamped to [0, L].
__device__ __forceinline__ double fan_hit(const HERec& Ro, double2 z) {
    const double ux = -Ro.u2x, uy = -Ro.u2y;                   // v -> start(o), unit
    const double dx = fma(ux, z.x, -uy * z.y), dy = fma(ux, z.y, uy * z.x);
    if (!(dy < 0.0)) return dx > 0.0 ? Ro.L : 0.0;             // parallel to o or turned away
    const double s = fma(-Ro.yc * dx, rcp_nr(dy), Ro.xc);
    return s < 0.0 ? 0.0 : (s > Ro.L ? Ro.L : s);
}

// kFanLanes lanes per fan candidate; lane j of the group handles corners j, j + 8, ...
// of the vertex's one-ring.  PROV: also record the distance events (geodesic paths).
template <bool PROV>
__global__ void __launch_bounds__(256) k_fan(Work w, int full_fan) {
    Counters* cnt = w.cnt;
    if (cnt->halt) return;
    const int lane = threadIdx.x & 31;
    const int sl = lane & (kFanLanes - 1);
    const int lead = lane & ~(kFanLanes - 1);
    const unsigned gmask = ((1u << kFanLanes) - 1u) << lead;
    const unsigned below = (1u << sl) - 1u;
    const int it = cnt->iter;
    const int nreq = min(cnt->n_req, w.req_cap);
    if (blockIdx.x == 0 && threadIdx.x == 0) atomicAdd(&cnt->fan_cand, (unsigned long long)nreq);
    const FanReq* req = w.req[it & 1];
    FanReq* req_nx = w.req[(it + 1) & 1];
    const unsigned stamp_fan = (unsigned)it + 1u;
    const int group0 = (blockIdx.x * blockDim.x + threadIdx.x) / kFanLanes;
    const int ngroups = (gridDim.x * blockDim.x) / kFanLanes;
    unsigned n_fans = 0, n_fwin = 0;
    for (int r = group0; r < nreq; r += ngroups) {     // uniform over the group
        const FanReq rq = req[r];
        const unsigned v = rq.v;
        const double D = rq.D;
        const Inst& I = w.inst[rq.inst];
        // 1: the iteration's fan of the vertex (a candidate from an event that lowered its
        // distance, carrying its final distance, the first this iteration); 2: a tie
        // deferred an iteration, fanned if its direction is new; 0: superseded, or
        // deferred now (a tie, or a candidate that did not make the fan but carries the
        // final distance within the margin)
        int kind = 0;
        if (sl == 0) {
            const unsigned long long gv = __ldcg(I.g + v), db = dbits(D);
            if (rq.tie == kReqLowered && db == gv && atomicExch(I.stamp + v, stamp_fan) != stamp_fan) {
                kind = 1;
            } else if (db <= gv + kDomUlps) {
                if (rq.tie == kReqDeferredTie) kind = 2;
                else push_fan(req_nx, &cnt->n_req_next, w.req_cap, &cnt->error, rq.inst, v, D, rq.href, rq.dx, rq.dy,
                              kReqDeferredTie);
            }
            n_fans += kind == 1 ? 1u : 0u;
        }
        kind = __shfl_sync(gmask, kind, lead);
        if (!kind) continue;
        const int s = I.vstart[v], e = I.vstart[v + 1];
        const bool boundary = (I.vflag[v] & 1) != 0;
        const bool all = full_fan != 0 || rq.href < 0;
        if (all && kind == 2) continue;            // a fan of every direction was made already
        // wedges in FP32 angular coordinates, unwrapped (interior ones are tested at
        // shifts of the total angle T): interior [phi + pi, phi + T - pi]; boundary
        // [-inf, phi - pi] and [phi + pi, +inf]
        const float T = I.vtheta[v];
        double2 za = make_double2(0.0, 0.0), zb = za, tr = make_double2(1.0, 0.0), zlo = za, zhi = za, tie_z = za;
        bool tie_lo = false, tie_hi = false;       // a tie's wedge cut to the part outside the last fan's
        float tie_w = 0.f;
        int nw = 0;
        float wlo[2] = {0.f, 0.f}, whi[2] = {0.f, 0.f};
        bool lo_open[2] = {false, false}, hi_open[2] = {false, false};
        if (!all) {
            float phi = I.vphi[rq.href] + atan2f((float)rq.dy, (float)rq.dx);
            // the incoming ray in the vertex's angular frame, turned by pi: the direction of
            // phi + pi (and of phi - pi); zb is that of phi + T - pi
            const double2 E = cmul(I.vrot[rq.href], make_double2(rq.dx, rq.dy));
            za = make_double2(-E.x, -E.y);
            tr = I.vtrot[v];
            zb = cmul(za, tr);
            if (boundary) phi = fminf(fmaxf(phi, 0.f), T);
            // the unit incoming direction and its angular position on the sheet [0, T) of an
            // interior vertex (positions phi and phi + T are one direction; their unit numbers
            // differ by the turn e^(i T), which is not 1 at a saddle)
            const double en_s = rsqrt(fma(E.x, E.x, E.y * E.y));
            double2 en = make_double2(E.x * en_s, E.y * en_s);
            float phic = phi;
            int kc = 0;
            if (!boundary) {
                kc = (int)floorf(phi / T);
                phic = phi - (float)kc * T;
                for (int q = 0; q < abs(kc) && q < 3; ++q) en = kc > 0 ? cmul_conj(en, tr) : cmul(en, tr);
            }
            if (kind == 2) {
                // a tie: fan only if its incoming direction differs from the last fan's
                const float fp = I.fan_phi[v];
                float dphi = fabsf(phic - fp);
                if (!boundary) {
                    dphi = fmodf(dphi, T);
                    dphi = fminf(dphi, T - dphi);
                }
                if (dphi < kTieSheet) {                // (a NaN, no fan recorded yet, fans)
                    // the same direction up to FP32: compare the FP64 directions on one
                    // sheet (the unit numbers of angular positions phi and phi + T differ
                    // by the turn e^(i T), which is not 1 at a saddle or boundary vertex)
                    const double2 fd = I.fan_dir[v];
                    const int sh = boundary ? 0 : (int)rintf((phic - fp) / T);
                    double2 ea = en;
                    for (int q = 0; q < abs(sh) && q < 3; ++q) ea = sh > 0 ? cmul_conj(ea, tr) : cmul(ea, tr);
                    if (fma(ea.x, fd.x, ea.y * fd.y) > 0.0 && fabs(fma(ea.x, fd.y, -ea.y * fd.x)) <= kTieDir) continue;
                }
                if (sl == 0) atomicAdd(&cnt->fan_ties, 1ull);
                // at an interior saddle whose two fanned areas overlap, only the part of this
                // candidate's area outside the last fan's is new: the wedge between the two
                // areas' upper (or lower) boundaries
                if (!boundary && fp == fp) {
                    const int sh = (int)rintf((phic - fp) / T);
                    const float delta = phic - (fp + (float)sh * T);
                    if (fabsf(delta) < T - 2.f * kPiF) {
                        const int s2 = sh + kc;                  // the last fan's direction in this frame
                        double2 fr = I.fan_dir[v];
                        for (int q = 0; q < abs(s2) && q < 3; ++q) fr = s2 > 0 ? cmul(fr, tr) : cmul_conj(fr, tr);
                        const float fraw = fp + (float)s2 * T;
                        if (delta > 0.f) {
                            tie_lo = true;
                            tie_w = fraw + T - kPiF;
                            const double2 t = cmul(fr, tr);
                            tie_z = make_double2(-t.x, -t.y);
                        } else {
                            tie_hi = true;
                            tie_w = fraw + kPiF;
                            tie_z = make_double2(-fr.x, -fr.y);
                        }
                    }
                }
            } else if (sl == 0) {
                I.fan_phi[v] = phic;
                I.fan_dir[v] = en;
            }
            if (boundary) {
                if (phi - kPiF > -kFanPickMargin) {
                    wlo[nw] = -1e30f; whi[nw] = phi - kPiF; lo_open[nw] = true; ++nw;
                }
                if (phi + kPiF < T + kFanPickMargin) {
                    wlo[nw] = phi + kPiF; whi[nw] = 1e30f; hi_open[nw] = true; ++nw;
                }
            } else if (T - 2.f * kPiF > -kFanPickMargin) {
                wlo[0] = phi + kPiF; whi[0] = phi + T - kPiF; nw = 1;
            }
            if (nw == 0) continue;
            zlo = za;
            zhi = boundary ? za : zb;
            if (tie_lo) { wlo[0] = tie_w; zlo = tie_z; }
            if (tie_hi) { whi[0] = tie_w; zhi = tie_z; }
        }
        bool deferred = false;
        for (int j0 = s; j0 < e && !deferred; j0 += kFanLanes) {
            const int j = j0 + sl;
            bool has = false;
            int o = 0;
            double s0 = 0.0, s1 = 0.0;
            HERec Ro;
            if (j < e) {
                const int hv = I.vlist[j];
                bool ex0 = false, ex1 = false;
                int shift = 0;
                if (all) {
                    has = true;
                } else {
                    const float c0 = I.vphi[hv], c1 = c0 + I.hang[hv];
                    for (int k = 0; k < nw && !has; ++k)
                        for (int sh = boundary ? 0 : -2; sh <= (boundary ? 0 : 1) && !has; ++sh) {
                            const float lo = wlo[k] + (float)sh * T, hi = whi[k] + (float)sh * T;
                            if (hi >= c0 - kFanPickMargin && lo <= c1 + kFanPickMargin) {
                                // a corner (under pi) meets at most one wedge at one shift
                                has = true;
                                shift = sh;
                                ex0 = !lo_open[k] && lo > c0 - kFanPickMargin;
                                ex1 = !hi_open[k] && hi < c1 + kFanPickMargin;
                            }
                        }
                }
                if (has) {
                    o = he_next(hv);                   // edge (a -> b) opposite v
                    Ro = I.rec[o];
                    s0 = 0.0;
                    s1 = Ro.L;
                    if (ex0 || ex1) {
                        // boundary directions in the corner's frame: z e^(i shift T) conj(rot(hv))
                        double2 t = make_double2(1.0, 0.0);
                        if (shift == 1) t = tr;
                        else if (shift == -1) t = make_double2(tr.x, -tr.y);
                        else if (shift == -2) t = cmul_conj(make_double2(tr.x, -tr.y), tr);
                        const double2 cr = I.vrot[hv];
                        if (ex0) s0 = fmax(fan_hit(Ro, cmul_conj(cmul(zlo, t), cr)) - kFanWiden * Ro.L, 0.0);
                        if (ex1) s1 = fmin(fan_hit(Ro, cmul_conj(cmul(zhi, t), cr)) + kFanWiden * Ro.L, Ro.L);
                    }
                }
            }
            const bool win = has && Ro.twin >= 0;
            const unsigned bal = (__ballot_sync(gmask, win) >> lead) & ((1u << kFanLanes) - 1u);
            const int cntw = __popc(bal);
            int base = 0;
            if (sl == 0 && cntw) base = atomicAdd(&cnt->n_child, cntw);
            base = __shfl_sync(gmask, base, lead);
            if (base + cntw > w.arena_cap) {
                // no room this iteration: mark the reserved slots empty, retry next iteration
                const int sl2 = base + __popc(bal & below);
                if (win && sl2 < w.arena_cap) w.arena.he[sl2] = -1;
                if (sl == 0) {
                    if (kind == 1) atomicExch(I.stamp + v, 0u);
                    push_fan(req_nx, &cnt->n_req_next, w.req_cap, &cnt->error, rq.inst, v, D, rq.href, rq.dx, rq.dy,
                             rq.tie);
                }
                deferred = true;
                continue;
            }
            if (!has) continue;
            const double Lo = Ro.L;
            if (!win) {
                // boundary edge: endpoint events for the covered endpoints
                const unsigned a = Ro.v0 & ~kPseudoBit, b = Ro.v1 & ~kPseudoBit;
                double ga = ldg_dist(I.g, a), gb = ldg_dist(I.g, b);
                const EvSrc es{rq.inst, o, (int)v, 1, 0.0, 0.0};   // along the edge from v (PROV only)
                // incoming directions: at a towards v, in o's frame; at b along next(o) = (b -> v)
                if (s0 <= 0.0)
                    if (const int ev = vertex_event<PROV>(I, Ro.v0, D + Ro.L2, ga, &w, &es))
                        push_fan(req_nx, &cnt->n_req_next, w.req_cap, &cnt->error, rq.inst, a, D + Ro.L2, o, Ro.xc, Ro.yc, ev);
                if (s1 >= Lo)
                    if (const int ev = vertex_event<PROV>(I, Ro.v1, D + Ro.L1, gb, &w, &es))
                        push_fan(req_nx, &cnt->n_req_next, w.req_cap, &cnt->error, rq.inst, b, D + Ro.L1, he_next(o), 1.0,
                                 0.0, ev);
                continue;
            }
            // window on twin(o) = (b -> a): I = v at (Lo - xc, -yc), interval [Lo - s1, Lo - s0]
            const int slot = base + __popc(bal & below);
            const double A = Lo - s1, B = Lo - s0;
            const double px = Lo - Ro.xc, py = -Ro.yc;
            const double IA = sqrt_nr(fma(A - px, A - px, py * py)), IB = sqrt_nr(fma(B - px, B - px, py * py));
            const double ga = ldg_dist(I.g, Ro.v0 & ~kPseudoBit), gb = ldg_dist(I.g, Ro.v1 & ~kPseudoBit);
            if (!(B - A > times_eps(Lo)) || dominated(D + IB, gb + B) || dominated(D + IA, ga + (Lo - A))) {
                w.arena.he[slot] = -1;
                continue;
            }
            const double key = D + (px < A ? IA : (px > B ? IB : -py));
            store_win(w.arena, slot, Ro.twin, rq.inst, D, A, B, px, py, key, (int)v, IA, IB);
            ++n_fwin;
        }
    }
    const unsigned f1 = __reduce_add_sync(0xffffffffu, n_fans), f2 = __reduce_add_sync(0xffffffffu, n_fwin);
    if (lane == 0 && f1) atomicAdd(&cnt->fans, (unsigned long long)f1);
    if (lane == 0 && f2) atomicAdd(&cnt->fan_windows, (unsigned long long)f2);
}

// ====================================================================== Step 3/4: append
__global__ void __launch_bounds__(256) k_append(Work w, const unsigned* __restrict__ keys, const int* __restrict__ vals,
                                                int trim) {
    __shared__ unsigned sh_hist[kShHistInst * kBins];
    Counters* cnt = w.cnt;
    if (cnt->halt) return;
    const int it = cnt->iter;
    const WinSoA nxt = w.pool[(it + 1) & 1];
    const int n = min(cnt->n_child, w.arena_cap);
    const int n_rest = cnt->n_rest;
    PoolStats ps{w.n_inst <= kShHistInst ? sh_hist : nullptr, w.hist[(it + 1) & 1], w.n_inst};
    if (ps.sh_hist) {
        for (int j = threadIdx.x; j < w.n_inst * kBins; j += blockDim.x) sh_hist[j] = 0u;
        __syncthreads();
    }
    constexpr int kTrimReach = 4;
    for (int base = blockIdx.x * blockDim.x; base < n; base += gridDim.x * blockDim.x) {
        const int i = base + threadIdx.x;
        // without a sort (keys == nullptr) the arena is appended in its own order
        unsigned k = i < n ? (keys ? keys[i] : (w.arena.he[i] < 0 ? ~0u : 0u)) : ~0u;
        bool keep = k != ~0u;
        int he = 0, inst = 0, src = -1;
        double d = 0, A = 0, B = 0, px = 0, py = 0, key = 0, IA = 0, IB = 0;
        int trimmed = 0;
        if (keep) {
            load_win(w.arena, keys ? vals[i] : i, he, inst, d, A, B, px, py, key, src, IA, IB);
            const Inst& I = w.inst[inst];
            const HERec R = I.rec[he];
            // re-filter against the distances after this iteration's events (the window
            // is nowhere closer than `key`)
            double g0 = ldg_dist(I.g, R.v0 & ~kPseudoBit), g1 = ldg_dist(I.g, R.v1 & ~kPseudoBit);
            if (dominated(key, g0 + B) || dominated(key, g1 + (R.L - A)) || stale_source(I, src, d)) keep = false;
            // per-edge trimming: a window on the same edge that covers [A, B] and is
            // everywhere shorter than this window's nearest point makes it useless
            if (keep && trim) {
                for (int dir = -1; dir <= 1 && keep; dir += 2) {
                    for (int s = 1; s <= kTrimReach && keep; ++s) {
                        int j = i + dir * s;
                        if (j < 0 || j >= n || keys[j] != k) break;
                        int jj = vals[j];
                        double A2 = w.arena.A[jj], B2 = w.arena.B[jj];
                        if (!(A2 <= A && B2 >= B)) continue;
                        double d2 = w.arena.d[jj], px2 = w.arena.px[jj], py2 = w.arena.py[jj];
                        double ea = A - px2, eb = B - px2;
                        double mx = d2 + sqrt(fmax(ea * ea, eb * eb) + py2 * py2);
                        if (dominated(key, mx)) { keep = false; trimmed = 1; }
                    }
                }
            }
        }
        int slot = warp_reserve(&cnt->n_app, keep ? 1 : 0);
        if (keep) {
            int pos = n_rest + slot;
            if (pos < w.pool_cap) store_win(nxt, pos, he, inst, d, A, B, px, py, key, src, IA, IB);
            else atomicOr(&cnt->error, kErrPoolFull);
        }
        pool_stat(w, ps, inst, key, keep);
        warp_add_ull(&cnt->trimmed, trimmed);
        warp_add_ull(&cnt->created, keep ? 1 : 0);
    }
    if (ps.sh_hist) {
        __syncthreads();
        for (int j = threadIdx.x; j < w.n_inst * kBins; j += blockDim.x)
            if (sh_hist[j]) atomicAdd(&ps.g_hist[j], sh_hist[j]);
    }
}

// ====================================================================== loop control
__global__ void k_finish(Work w, cudaGraphConditionalHandle handle, int use_cond, long long max_iters) {
    Counters* c = w.cnt;
    if (!c->halt) {
        c->scanned += (unsigned long long)min(c->n_pending, w.pool_cap);
        c->sorted += (unsigned long long)min(c->n_child, w.arena_cap);
        int np = c->n_rest + c->n_app;
        const float ratio = c->n_sel > 0 ? (float)c->n_app / (float)c->n_sel : 0.f;
        for (int i = 0; i < w.n_inst; ++i) w.ctl[i].last_ratio = ratio;
        c->n_pending = np;
        if ((unsigned long long)np > c->peak_pending) c->peak_pending = (unsigned long long)np;
        c->n_req = min(c->n_req_next, w.req_cap);
        c->n_req_next = 0;
        c->n_rest = 0;
        c->n_sel = 0;
        c->n_child = 0;
        c->n_app = 0;
        c->work_next = 0;
        c->iter += 1;
        c->done = (np == 0 && c->n_req == 0) ? 1 : 0;
        if (!c->done && c->iter >= max_iters) c->error |= kErrIter;
        // stop for the host: finished, an error, or the pool may not hold one more iteration
        c->halt = (c->done || c->error != 0 || np + w.arena_cap > w.pool_cap) ? 1 : 0;
    }
    if (use_cond) cudaGraphSetConditional(handle, c->halt ? 0u : 1u);
}

__global__ void k_copy_out(const unsigned long long* __restrict__ g, double* out, int n) {
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x) out[i] = bitsd(g[i]);
}

__global__ void k_min_into(const unsigned long long* __restrict__ g, unsigned long long* acc, int n) {
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x)
        if (g[i] < acc[i]) acc[i] = g[i];
}

// ====================================================================== host side
struct Alloc {
    std::vector<void*> ptrs;
    size_t bytes = 0;
    template <class T>
    cudaError_t get(T** p, size_t n) {
        if (n == 0) n = 1;
        cudaError_t e = cudaMalloc((void**)p, sizeof(T) * n);
        if (e == cudaSuccess) { ptrs.push_back(*p); bytes += sizeof(T) * n; }
        return e;
    }
    void release() {
        for (void* p : ptrs) cudaFree(p);
        ptrs.clear();
        bytes = 0;
    }
};

struct GraphKey {
    SolveCfg cfg;
    Work w;
};

struct Workspace {
    int device = 0;
    Alloc pools;            // pools, arena, sort buffers, requests (sized by caps)
    Alloc inst_mem;         // g / angle_split / stamps (sized by the instances)
    Alloc fixed;            // counters, tables
    Alloc sthr;             // strided-selection thresholds (PCH_CONTROL_STRIDED)
    int sthr_cap = 0;
    Alloc plog_mem;         // distance-event records (geodesic paths)
    int plog_cap = 0;
    ProvRec* plog = nullptr;
    Work w{};
    int pool_cap = 0, sel_cap = 0, arena_cap = 0, req_cap = 0;
    long long g_cap = 0, ang_cap = 0, st_cap = 0;
    int inst_cap = 0;
    unsigned long long* g_all = nullptr;
    unsigned long long* ang_all = nullptr;
    unsigned* stamp_all = nullptr;
    float* fanphi_all = nullptr;
    double2* fandir_all = nullptr;
    Counters* cnt_host = nullptr;
    cudaEvent_t ev[2] = {nullptr, nullptr};
    // graph cache: rebuilt when pointers or launch parameters change
    cudaGraph_t graph = nullptr;
    cudaGraphExec_t exec = nullptr;
    GraphKey gkey{};
    float* trace_buf = nullptr;
    int* trace_rows = nullptr;
    int trace_cap = 0;
    bool trace_on = false;
};

void destroy_workspace(Workspace* ws) {
    if (!ws) return;
    if (ws->exec) cudaGraphExecDestroy(ws->exec);
    if (ws->graph) cudaGraphDestroy(ws->graph);
    ws->pools.release();
    ws->inst_mem.release();
    ws->fixed.release();
    ws->sthr.release();
    ws->plog_mem.release();
    if (ws->cnt_host) cudaFreeHost(ws->cnt_host);
    for (auto& e : ws->ev) if (e) cudaEventDestroy(e);
    delete ws;
}

static void drop_graph(Workspace* ws) {
    if (ws->exec) cudaGraphExecDestroy(ws->exec);
    if (ws->graph) cudaGraphDestroy(ws->graph);
    ws->exec = nullptr;
    ws->graph = nullptr;
}

static cudaError_t alloc_soa(Alloc& a, WinSoA& s, int cap) {
    cudaError_t e;
    if ((e = a.get(&s.he, cap))) return e;
    if ((e = a.get(&s.inst, cap))) return e;
    if ((e = a.get(&s.d, cap))) return e;
    if ((e = a.get(&s.A, cap))) return e;
    if ((e = a.get(&s.B, cap))) return e;
    if ((e = a.get(&s.px, cap))) return e;
    if ((e = a.get(&s.py, cap))) return e;
    if ((e = a.get(&s.key, cap))) return e;
    if ((e = a.get(&s.IA, cap))) return e;
    if ((e = a.get(&s.IB, cap))) return e;
    return a.get(&s.src, cap);
}

// Capacities: the work list holds sel_cap windows (more selected windows simply stay
// pending), the child arena 6 * sel_cap (two children per selected window plus the half
// that chaining may fill, so it cannot overflow), the pending pools at least twice the
// arena (the loop halts for the host to grow them before they could overflow), and the
// fan requests req_cap (an overflow fails the attempt; the solve is then re-run with
// twice the room).
static pch_status ensure_pools(Workspace* ws, int sel_cap, int pool_cap, int req_min = 0) {
    int arena_cap = 6 * sel_cap;
    if (pool_cap < 2 * arena_cap) pool_cap = 2 * arena_cap;
    if (sel_cap <= ws->sel_cap && pool_cap <= ws->pool_cap && req_min <= ws->req_cap) return PCH_OK;
    sel_cap = std::max(sel_cap, ws->sel_cap);
    pool_cap = std::max(pool_cap, ws->pool_cap);
    arena_cap = 6 * sel_cap;
    const int req_cap = std::max({4 * sel_cap + (1 << 20), req_min, ws->req_cap});
    const int sort_blocks = 2 * sm_count();
    drop_graph(ws);
    Work& w = ws->w;
    Work nw = w;
    Alloc fresh;
    cudaError_t e = cudaSuccess;
    if (!e) e = alloc_soa(fresh, nw.pool[0], pool_cap);
    if (!e) e = alloc_soa(fresh, nw.pool[1], pool_cap);
    if (!e) e = alloc_soa(fresh, nw.sel, sel_cap);
    if (!e) e = alloc_soa(fresh, nw.arena, arena_cap);
    if (!e) e = fresh.get(&nw.req[0], req_cap);
    if (!e) e = fresh.get(&nw.req[1], req_cap);
    if (!e) e = fresh.get(&nw.sort_key[0], arena_cap);
    if (!e) e = fresh.get(&nw.sort_key[1], arena_cap);
    if (!e) e = fresh.get(&nw.sort_val[0], arena_cap);
    if (!e) e = fresh.get(&nw.sort_val[1], arena_cap);
    if (!e) e = fresh.get(&nw.sort_hist, (size_t)kRsDigits * sort_blocks);
    if (e) {
        fresh.release();
        return set_error(e == cudaErrorMemoryAllocation ? PCH_ERR_OOM : PCH_ERR_CUDA, "workspace allocation: %s",
                         cudaGetErrorString(e));
    }
    if (ws->pool_cap > 0) {
        // growth between iterations: keep the pending pools and the fan requests
        const size_t n = (size_t)ws->pool_cap;
        for (int p = 0; p < 2; ++p) {
            cudaMemcpy(nw.pool[p].he, w.pool[p].he, n * 4, cudaMemcpyDeviceToDevice);
            cudaMemcpy(nw.pool[p].inst, w.pool[p].inst, n * 4, cudaMemcpyDeviceToDevice);
            cudaMemcpy(nw.pool[p].d, w.pool[p].d, n * 8, cudaMemcpyDeviceToDevice);
            cudaMemcpy(nw.pool[p].A, w.pool[p].A, n * 8, cudaMemcpyDeviceToDevice);
            cudaMemcpy(nw.pool[p].B, w.pool[p].B, n * 8, cudaMemcpyDeviceToDevice);
            cudaMemcpy(nw.pool[p].px, w.pool[p].px, n * 8, cudaMemcpyDeviceToDevice);
            cudaMemcpy(nw.pool[p].py, w.pool[p].py, n * 8, cudaMemcpyDeviceToDevice);
            cudaMemcpy(nw.pool[p].key, w.pool[p].key, n * 8, cudaMemcpyDeviceToDevice);
            cudaMemcpy(nw.pool[p].src, w.pool[p].src, n * 4, cudaMemcpyDeviceToDevice);
            cudaMemcpy(nw.pool[p].IA, w.pool[p].IA, n * 8, cudaMemcpyDeviceToDevice);
            cudaMemcpy(nw.pool[p].IB, w.pool[p].IB, n * 8, cudaMemcpyDeviceToDevice);
            cudaMemcpy(nw.req[p], w.req[p], sizeof(FanReq) * (size_t)ws->req_cap, cudaMemcpyDeviceToDevice);
        }
        e = cudaDeviceSynchronize();
        if (e) { fresh.release(); return set_error(PCH_ERR_CUDA, "pool growth copy: %s", cudaGetErrorString(e)); }
    }
    ws->pools.release();
    ws->pools = fresh;
    w = nw;
    ws->pool_cap = w.pool_cap = pool_cap;
    ws->sel_cap = w.sel_cap = sel_cap;
    ws->arena_cap = w.arena_cap = arena_cap;
    ws->req_cap = w.req_cap = req_cap;
    w.sort_blocks = sort_blocks;
    return PCH_OK;
}

struct InstSpec {
    pch_mesh* m;
    long long goff, aoff;
    int k_src_begin, k_src_end;
};

static pch_status ensure_workspace(pch_mesh* owner, Workspace** out) {
    if (!owner->ws) {
        Workspace* ws = new Workspace();
        cudaGetDevice(&ws->device);
        if (cudaMallocHost(&ws->cnt_host, sizeof(Counters)) != cudaSuccess) {
            delete ws;
            return set_error(PCH_ERR_OOM, "pinned counter allocation failed");
        }
        cudaEventCreate(&ws->ev[0]);
        cudaEventCreate(&ws->ev[1]);
        if (ws->fixed.get(&ws->w.cnt, 1) != cudaSuccess) {
            destroy_workspace(ws);
            return set_error(PCH_ERR_OOM, "counter allocation failed");
        }
        owner->ws = ws;
    }
    *out = owner->ws;
    return PCH_OK;
}

static pch_status ensure_instances(Workspace* ws, int n_inst, long long g_total, long long a_total) {
    if (n_inst <= ws->inst_cap && g_total <= ws->g_cap && a_total <= ws->ang_cap) return PCH_OK;
    drop_graph(ws);
    ws->inst_mem.release();
    Work& w = ws->w;
    int ic = std::max(n_inst, ws->inst_cap);
    long long gc = std::max(g_total, ws->g_cap), ac = std::max(a_total, ws->ang_cap);
    cudaError_t e = cudaSuccess;
    if (!e) e = ws->inst_mem.get(&ws->g_all, gc);
    if (!e) e = ws->inst_mem.get(&ws->ang_all, ac);
    if (!e) e = ws->inst_mem.get(&ws->stamp_all, gc);
    if (!e) e = ws->inst_mem.get(&ws->fanphi_all, gc);
    if (!e) e = ws->inst_mem.get(&ws->fandir_all, gc);
    if (!e) e = ws->inst_mem.get(&w.inst, ic);
    if (!e) e = ws->inst_mem.get(&w.ctl, ic);
    if (!e) e = ws->inst_mem.get(&w.hist[0], (size_t)ic * kBins);
    if (!e) e = ws->inst_mem.get(&w.hist[1], (size_t)ic * kBins);
    if (e) {
        ws->inst_mem.release();
        ws->inst_cap = 0; ws->g_cap = ws->ang_cap = 0;
        return set_error(e == cudaErrorMemoryAllocation ? PCH_ERR_OOM : PCH_ERR_CUDA, "instance allocation: %s",
                         cudaGetErrorString(e));
    }
    ws->inst_cap = ic;
    ws->g_cap = gc;
    ws->ang_cap = ac;
    return PCH_OK;
}

static int grid_for(int blocks_per_sm) { return sm_count() * blocks_per_sm; }

// Kernels one iteration launches (for pch_stats.kernel_launches).
static int kernels_per_iteration(const SolveCfg& cfg) {
    int passes = (cfg.key_bits + kRsDigitBits - 1) / kRsDigitBits;
    return 6 + (cfg.stride_T > 0 ? 1 : 0) + sort_kernels_per_pass() * passes;
}

// Launch one iteration (all phases).  With `ev` (7 events) the phase boundaries are
// recorded for PCH_FLAG_PROFILE.  Returns a CUDA error if a launch failed.
static cudaError_t launch_iteration(Workspace* ws, cudaStream_t s, const SolveCfg& cfg, cudaGraphConditionalHandle h,
                                    int use_cond, cudaEvent_t* ev = nullptr) {
    Work& w = ws->w;
    const int tpb = 256;
    if (ev) cudaEventRecord(ev[0], s);
    k_tau<<<std::min(w.n_inst, 1024), 256, 0, s>>>(w, cfg.control, cfg.mlp);
    if (cfg.stride_T > 0) {
        const int g = std::min((cfg.stride_T + 255) / 256, grid_for(8));
        switch (cfg.stride_m) {
            case 1: k_strided<1><<<g, 256, 0, s>>>(w); break;
            case 2: k_strided<2><<<g, 256, 0, s>>>(w); break;
            case 4: k_strided<4><<<g, 256, 0, s>>>(w); break;
            case 8: k_strided<8><<<g, 256, 0, s>>>(w); break;
            default: k_strided<16><<<g, 256, 0, s>>>(w); break;
        }
    }
    k_compact<<<grid_for(4), tpb, 0, s>>>(w);
    if (ev) cudaEventRecord(ev[1], s);
    const dim3 pg(grid_for(cfg.prop_blocks_per_sm));
    const size_t psh = (size_t)cfg.prop_threads * kPropQueueBytesPerThread;
    if (cfg.prov) k_propagate<true><<<pg, cfg.prop_threads, psh, s>>>(w, cfg.hops, cfg.tail_cut, cfg.take_min);
    else k_propagate<false><<<pg, cfg.prop_threads, psh, s>>>(w, cfg.hops, cfg.tail_cut, cfg.take_min);
    if (ev) cudaEventRecord(ev[2], s);
    if (cfg.prov) k_fan<true><<<grid_for(2), 256, 0, s>>>(w, cfg.full_fan);
    else k_fan<false><<<grid_for(2), 256, 0, s>>>(w, cfg.full_fan);
    if (ev) cudaEventRecord(ev[3], s);
    unsigned* kb[2] = {w.sort_key[0], w.sort_key[1]};
    int* vb[2] = {w.sort_val[0], w.sort_val[1]};
    const int par = cfg.key_bits == 0 ? -1 :
        launch_sort_children(w.arena, w.inst, &w.cnt->n_child, w.arena_cap, cfg.key_bits, cfg.edge_sort, kb, vb, w.sort_hist,
                                   w.sort_blocks, s);
    if (ev) cudaEventRecord(ev[4], s);
    k_append<<<grid_for(4), tpb, 0, s>>>(w, par >= 0 ? kb[par] : nullptr, par >= 0 ? vb[par] : nullptr,
                                          cfg.trim && cfg.edge_sort);
    if (ev) cudaEventRecord(ev[5], s);
    k_finish<<<1, 1, 0, s>>>(w, h, use_cond, cfg.max_iters);
    if (ev) cudaEventRecord(ev[6], s);
    return cudaGetLastError();
}

static pch_status build_graph(Workspace* ws, cudaStream_t s, const SolveCfg& cfg) {
    drop_graph(ws);
    cudaGraph_t graph;
    PCH_CUDA(cudaGraphCreate(&graph, 0));
    cudaGraphConditionalHandle handle;
    cudaError_t e = cudaGraphConditionalHandleCreate(&handle, graph, 1, cudaGraphCondAssignDefault);
    if (e) { cudaGraphDestroy(graph); PCH_CUDA(e); }
    cudaGraphNodeParams cp{};
    cp.type = cudaGraphNodeTypeConditional;
    cp.conditional.handle = handle;
    cp.conditional.type = cudaGraphCondTypeWhile;
    cp.conditional.size = 1;
    cudaGraphNode_t node;
    e = cudaGraphAddNode(&node, graph, nullptr, nullptr, 0, &cp);
    if (e) { cudaGraphDestroy(graph); PCH_CUDA(e); }
    cudaGraph_t body = cp.conditional.phGraph_out[0];
    cudaStream_t cs;
    PCH_CUDA(cudaStreamCreateWithFlags(&cs, cudaStreamNonBlocking));
    e = cudaStreamBeginCaptureToGraph(cs, body, nullptr, nullptr, 0, cudaStreamCaptureModeRelaxed);
    if (!e) {
        for (int u = 0; u < cfg.unroll && !e; ++u) e = launch_iteration(ws, cs, cfg, handle, u == cfg.unroll - 1);
        cudaGraph_t outg = body;
        cudaError_t e2 = cudaStreamEndCapture(cs, &outg);
        if (!e) e = e2;
    }
    cudaStreamDestroy(cs);
    if (e) { cudaGraphDestroy(graph); PCH_CUDA(e); }
    cudaGraphExec_t exec;
    e = cudaGraphInstantiate(&exec, graph, 0);
    if (e) { cudaGraphDestroy(graph); PCH_CUDA(e); }
    ws->graph = graph;
    ws->exec = exec;
    (void)s;
    return PCH_OK;
}

static pch_status status_from_error(int err) {
    if (err & kErrIter) return set_error(PCH_ERR_TIMEOUT, "iteration cap reached before all windows were processed");
    if (err & (kErrPoolFull | kErrReqFull)) return set_error(PCH_ERR_CAPACITY, "window pool capacity exceeded (error %d)", err);
    if (err & kErrProvFull) return set_error(PCH_ERR_CAPACITY, "distance-event record capacity exceeded");
    return set_error(PCH_ERR_CUDA, "solver error flags %d", err);
}

// Common driver: runs the iterations of an initialised solve.
static pch_status run_solve(Workspace* ws, cudaStream_t s, const SolveCfg& cfg_in, pch_stats* stats) {
    SolveCfg cfg = cfg_in;
    Work& w = ws->w;
    long long launches = 0;
    double phase_ms[6] = {0, 0, 0, 0, 0, 0};
    PCH_CUDA(cudaEventRecord(ws->ev[0], s));
    if (cfg.loop == PCH_LOOP_HOST || cfg.profile) {
        cudaEvent_t pev[7];
        if (cfg.profile)
            for (auto& e : pev) PCH_CUDA(cudaEventCreate(&e));
        for (long long it = 0;; ++it) {
            cudaError_t le = launch_iteration(ws, s, cfg, 0, 0, cfg.profile ? pev : nullptr);
            if (le) {
                if (cfg.profile) for (auto& e : pev) cudaEventDestroy(e);
                PCH_CUDA(le);
            }
            launches += kernels_per_iteration(cfg);
            PCH_CUDA(cudaMemcpyAsync(ws->cnt_host, w.cnt, sizeof(Counters), cudaMemcpyDeviceToHost, s));
            PCH_CUDA(cudaStreamSynchronize(s));
            if (cfg.profile) {
                for (int p = 0; p < 6; ++p) {
                    float ms = 0.f;
                    cudaEventElapsedTime(&ms, pev[p], pev[p + 1]);
                    phase_ms[p] += ms;
                }
            }
            const Counters& c = *ws->cnt_host;
            if (c.error || c.done) break;
            if (c.n_pending + w.arena_cap > w.pool_cap) {
                pch_status st = ensure_pools(ws, ws->sel_cap, 2 * ws->pool_cap);
                if (st != PCH_OK) return st;
                PCH_CUDA(cudaMemsetAsync(&w.cnt->halt, 0, sizeof(int), s));
            }
        }
        if (cfg.profile) for (auto& e : pev) cudaEventDestroy(e);
    } else {
        while (true) {
            GraphKey key{};
            key.cfg = cfg;
            key.w = w;
            if (!(ws->exec && std::memcmp(&key, &ws->gkey, sizeof key) == 0)) {
                pch_status st = build_graph(ws, s, cfg);
                if (st != PCH_OK) return st;
                ws->gkey = key;
            }
            PCH_CUDA(cudaGraphLaunch(ws->exec, s));
            PCH_CUDA(cudaMemcpyAsync(ws->cnt_host, w.cnt, sizeof(Counters), cudaMemcpyDeviceToHost, s));
            PCH_CUDA(cudaStreamSynchronize(s));
            const Counters& c = *ws->cnt_host;
            // the WHILE body ran ceil(iterations / unroll) times
            if (c.error || c.done) break;
            if (c.n_pending + w.arena_cap > w.pool_cap) {
                pch_status st = ensure_pools(ws, ws->sel_cap, 2 * ws->pool_cap);
                if (st != PCH_OK) return st;
                PCH_CUDA(cudaMemsetAsync(&w.cnt->halt, 0, sizeof(int), s));
                continue;
            }
        }
        const long long it = ws->cnt_host->iter;
        launches += ((it + cfg.unroll - 1) / cfg.unroll) * cfg.unroll * kernels_per_iteration(cfg);
    }
    PCH_CUDA(cudaEventRecord(ws->ev[1], s));
    PCH_CUDA(cudaEventSynchronize(ws->ev[1]));
    const Counters& c = *ws->cnt_host;
    if (c.error) return status_from_error(c.error);
    if (stats) {
        float ms = 0.f;
        cudaEventElapsedTime(&ms, ws->ev[0], ws->ev[1]);
        stats->iterations = c.iter;
        stats->windows_created = (int64_t)c.created;
        stats->windows_propagated = (int64_t)c.propagated;
        stats->peak_pending = (int64_t)c.peak_pending;
        stats->ms_total = ms;
        stats->bytes_workspace = (int64_t)(ws->pools.bytes + ws->inst_mem.bytes + ws->fixed.bytes + ws->sthr.bytes);
        stats->kernel_launches += launches;
        stats->fans = (int64_t)c.fans;
        stats->fan_windows = (int64_t)c.fan_windows;
        stats->fan_candidates = (int64_t)c.fan_cand;
        stats->windows_chained = (int64_t)c.chained;
        stats->windows_scanned = (int64_t)c.scanned;
        stats->windows_sorted = (int64_t)c.sorted;
        stats->sort_passes = (cfg.key_bits + kRsDigitBits - 1) / kRsDigitBits;
        stats->windows_examined = (int64_t)c.examined;
        stats->windows_occupied = (int64_t)c.occupied;
        stats->children_computed = (int64_t)c.children;
        stats->fan_ties = (int64_t)c.fan_ties;
        // algorithmic FP64 operations of k_propagate (add, sub, mul, div, sqrt = 1; fma = 2),
        // counted per code path of propagate_window: a window taken from the work list 7
        // (2 offsets, 5 for the endpoint filter), a chained window 2 (its filter was its
        // parent's child filter), a window that passed +9 (occupancy test), an occupied
        // one +17 (crossing point and its angle_split position, |I v2|, event distance),
        // a child +25 (frame change 7: the child edge's unit axis comes with the half-edge
        // record; width 1, child filter 16, key 1) plus 8 per ray intersected (two per
        // child, one when the window occupies v2); the filter's test against the parent
        // edge's far vertex at the second end (+11) is not counted: it is evaluated only
        // where the first end's test holds (the warp runs it when any lane needs it)
        const unsigned long long fresh = c.examined > c.chained ? c.examined - c.chained : 0ull;
        stats->prop_fp64_ops = (int64_t)(7ull * fresh + 2ull * c.chained + 9ull * c.propagated +
                                         17ull * c.occupied + 25ull * c.children + 8ull * c.rays);
        for (int p = 0; p < 6; ++p) stats->ms_phase[p] = phase_ms[p];
    }
    return PCH_OK;
}

static SolveCfg make_cfg(const pch_options* opt, int n_inst, long long total_keys) {
    SolveCfg cfg{};
    cfg.control = opt ? opt->control : PCH_CONTROL_PLAIN;
    cfg.loop = opt ? opt->loop : PCH_LOOP_GRAPH;
    cfg.k = (opt && opt->k > 0) ? opt->k : default_k();
    cfg.max_iters = (opt && opt->max_iters > 0) ? opt->max_iters : (1LL << 31) - 1;
    cfg.prop_threads = (opt && opt->block > 0) ? opt->block : 64;
    cfg.prop_blocks_per_sm = default_prop_blocks_per_sm(cfg.prop_threads);
    cfg.trim = !(opt && (opt->flags & PCH_FLAG_NO_TRIM));
    cfg.full_fan = (opt && (opt->flags & PCH_FLAG_FULL_FAN)) ? 1 : 0;
    cfg.profile = (opt && (opt->flags & PCH_FLAG_PROFILE)) ? 1 : 0;
    cfg.hops = (opt && opt->hops > 0) ? opt->hops : default_hops();
    cfg.tail_cut = default_tail_cut();
    cfg.take_min = default_take_min();
    cfg.unroll = 2;
    // Step 3 organises the new windows into a gap-free pool; they are grouped by instance
    // (one 8-bit radix pass for up to 256 instances, none for one), or with
    // PCH_FLAG_EDGE_SORT ordered by (instance, half-edge) for the per-edge trimming
    cfg.edge_sort = (opt && (opt->flags & PCH_FLAG_EDGE_SORT)) ? 1 : 0;
    int bits = 0;
    if (cfg.edge_sort) {
        bits = 1;
        while ((1LL << bits) <= total_keys) ++bits;   // invalid key ~0u must exceed all valid keys
    } else {
        while ((1LL << bits) < n_inst) ++bits;
    }
    cfg.key_bits = bits;
    cfg.mlp = nullptr;
    cfg.stride_T = cfg.stride_m = 0;
    cfg.prov = 0;
    if (cfg.control == PCH_CONTROL_STRIDED) {
        // Section 5.1: T threads each select their ceil(k / T) nearest windows.  T is the
        // number of threads the GPU holds at once (2048 per SM); each selects M of them, M
        // rounded up to a power of two (at most 16, beyond which T grows instead), and
        // T = ceil(K / M) for K = k windows per instance.
        const long long K = std::max<long long>(1, cfg.k * (long long)n_inst);
        const long long Tmax = (long long)sm_count() * 2048;
        long long m = (K + Tmax - 1) / Tmax;
        int M = 1;
        while (M < m && M < 16) M <<= 1;
        long long T = (K + M - 1) / M;
        cfg.stride_m = M;
        cfg.stride_T = (int)std::min<long long>(T, 1LL << 30);
    }
    return cfg;
}

// Solve a set of instances.  srcs[i].inst says which instance a source seeds.
// Grow the distance-event records to hold `cap` (geodesic paths).
static pch_status ensure_plog(Workspace* ws, long long cap) {
    cap = std::min<long long>(cap, 1LL << 30);
    if (cap <= ws->plog_cap) return PCH_OK;
    drop_graph(ws);
    ws->plog_mem.release();
    ws->plog_cap = 0;
    ws->plog = nullptr;
    if (ws->plog_mem.get(&ws->plog, (size_t)cap) != cudaSuccess) {
        ws->plog_mem.release();
        ws->plog = nullptr;
        return set_error(PCH_ERR_OOM, "distance-event records: allocation of %lld failed", cap);
    }
    ws->plog_cap = (int)cap;
    return PCH_OK;
}

pch_status solve_instances(pch_mesh* const* meshes, int n_inst, const SrcDev* srcs, int n_src, const pch_options* opt,
                           double* const* outs, int out_mode, pch_stats* stats, int prov) {
    clear_error();
    if (!meshes || n_inst <= 0 || !srcs || n_src <= 0) return set_error(PCH_ERR_INVALID_ARG, "empty solve");
    for (int i = 0; i < n_inst; ++i)
        if (!meshes[i]) return set_error(PCH_ERR_INVALID_ARG, "null mesh for instance %d", i);
    for (int i = 0; i < n_src; ++i) {
        const SrcDev& sd = srcs[i];
        if (sd.inst < 0 || sd.inst >= n_inst) return set_error(PCH_ERR_INVALID_ARG, "bad source instance");
        const DevMesh& dm = meshes[sd.inst]->dm;
        if (sd.kind == 0) {
            if (sd.vertex < 0 || sd.vertex >= dm.nv) return set_error(PCH_ERR_INVALID_ARG, "source vertex %d out of range", sd.vertex);
        } else if (sd.kind == 1) {
            if (sd.face < 0 || sd.face >= dm.nf) return set_error(PCH_ERR_INVALID_ARG, "source face %d out of range", sd.face);
            double sb = sd.bary[0] + sd.bary[1] + sd.bary[2];
            for (int k = 0; k < 3; ++k)
                if (!(sd.bary[k] >= 0.0)) return set_error(PCH_ERR_INVALID_ARG, "negative barycentric weight");
            if (!(std::fabs(sb - 1.0) < 1e-9)) return set_error(PCH_ERR_INVALID_ARG, "barycentric weights must sum to 1");
        } else {
            return set_error(PCH_ERR_INVALID_ARG, "unknown source kind %d", sd.kind);
        }
    }
    if (opt && opt->block != 0 && (opt->block < 32 || opt->block > 256 || opt->block % 32 != 0))
        return set_error(PCH_ERR_INVALID_ARG, "block must be a multiple of 32 in [32, 256], got %d", opt->block);
    if (opt && opt->k < 0) return set_error(PCH_ERR_INVALID_ARG, "k must be >= 0");
    if (opt && (opt->control < PCH_CONTROL_PLAIN || opt->control > PCH_CONTROL_STRIDED))
        return set_error(PCH_ERR_INVALID_ARG, "unknown control %d", opt->control);
    cudaStream_t s = opt ? (cudaStream_t)opt->stream : (cudaStream_t)0;
    Workspace* ws;
    pch_status st = ensure_workspace(meshes[0], &ws);
    if (st != PCH_OK) return st;
    // instance layout
    std::vector<Inst> hinst(n_inst);
    std::vector<InstCtl> hctl(n_inst);
    long long goff = 0, aoff = 0, kbase = 0;
    std::vector<long long> gofs(n_inst), aofs(n_inst);
    for (int i = 0; i < n_inst; ++i) {
        gofs[i] = goff;
        aofs[i] = aoff;
        goff += meshes[i]->dm.nv;
        aoff += meshes[i]->dm.nh;
    }
    st = ensure_instances(ws, n_inst, goff, aoff);
    if (st != PCH_OK) return st;
    SolveCfg cfg = make_cfg(opt, n_inst, aoff);
    for (int i = 0; i < n_inst; ++i) {
        const DevMesh& dm = meshes[i]->dm;
        Inst& I = hinst[i];
        I.rec = dm.rec; I.vstart = dm.vstart; I.vlist = dm.vlist; I.vphi = dm.vphi; I.vtheta = dm.vtheta;
        I.hang = dm.hang; I.vflag = dm.vflag; I.vrot = dm.vrot; I.vtrot = dm.vtrot;
        I.g = ws->g_all + gofs[i];
        I.ang = ws->ang_all + aofs[i];
        I.stamp = ws->stamp_all + gofs[i];
        I.fan_phi = ws->fanphi_all + gofs[i];
        I.fan_dir = ws->fandir_all + gofs[i];
        I.nv = dm.nv; I.nh = dm.nh;
        I.keybase = kbase;
        kbase += dm.nh;
        I.lbar = dm.lbar; I.ilbar = 1.0 / dm.lbar;
        InstCtl& c = hctl[i];
        std::memset(&c, 0, sizeof c);
        c.kmin = ~0ull;
        c.ref = 0.0;
        c.k_target = cfg.k;
        c.active = 1;
    }
    // the work list never needs more than the pending windows, which rarely exceed the
    // half-edge count; a larger k only leaves the rest pending.  Under the learned control
    // the network may pick up to 2^26 windows an iteration: the list is sized for that
    // (within the same caps), not for the plain k it falls back to
    const long long k_size = cfg.control == PCH_CONTROL_LEARNED ? std::max<long long>(cfg.k, 1LL << 22) : cfg.k;
    long long sel_want = std::max<long long>(65536, 4LL * k_size * std::min(n_inst, 64));
    sel_want = std::min<long long>(sel_want, std::max<long long>(65536, aoff));
    sel_want = std::min<long long>(sel_want, 1 << 24);
    int pool_want = (int)std::min<long long>(std::max<long long>(2 * 6 * sel_want, 1 << 20), (1LL << 30));
    st = ensure_pools(ws, (int)sel_want, pool_want);
    if (st != PCH_OK) return st;
    Work& w = ws->w;
    w.n_inst = n_inst;
    if (cfg.stride_T > ws->sthr_cap) {
        drop_graph(ws);
        ws->sthr.release();
        ws->sthr_cap = 0;
        if (ws->sthr.get(&w.sthr_key, (size_t)cfg.stride_T) != cudaSuccess ||
            ws->sthr.get(&w.sthr_idx, (size_t)cfg.stride_T) != cudaSuccess) {
            ws->sthr.release();
            return set_error(PCH_ERR_OOM, "strided selection thresholds: allocation failed");
        }
        ws->sthr_cap = cfg.stride_T;
    }
    w.stride_T = cfg.stride_T;
    cfg.prov = prov ? 1 : 0;
    if (prov) {
        st = ensure_plog(ws, std::max<long long>(1 << 20, 4 * goff));
        if (st != PCH_OK) return st;
    }
    ws->trace_on = opt && (opt->flags & PCH_FLAG_TRACE);
    if (ws->trace_on && !ws->trace_buf) {
        ws->trace_cap = 1 << 18;
        if (ws->fixed.get(&ws->trace_buf, (size_t)ws->trace_cap * (kFeatures + 2)) != cudaSuccess ||
            ws->fixed.get(&ws->trace_rows, 1) != cudaSuccess)
            return set_error(PCH_ERR_OOM, "trace buffer allocation failed");
    }
    w.trace = ws->trace_on ? ws->trace_buf : nullptr;
    w.trace_cap = ws->trace_cap;
    w.trace_rows = ws->trace_rows;
    if (cfg.control == PCH_CONTROL_LEARNED) cfg.mlp = mlp_device_params();
    // a fan-request overflow fails the attempt (a lost request would lose a fan); the
    // solve is then run again from the start with twice the request room (the same for
    // the distance-event records of a geodesic-path solve)
    for (int attempt = 0;; ++attempt) {
        w.plog = prov ? ws->plog : nullptr;
        w.plog_cap = prov ? ws->plog_cap : 0;
        // upload tables, clear state
        PCH_CUDA(cudaMemcpyAsync(w.inst, hinst.data(), sizeof(Inst) * n_inst, cudaMemcpyHostToDevice, s));
        PCH_CUDA(cudaMemcpyAsync(w.ctl, hctl.data(), sizeof(InstCtl) * n_inst, cudaMemcpyHostToDevice, s));
        PCH_CUDA(cudaMemsetAsync(w.cnt, 0, sizeof(Counters), s));
        PCH_CUDA(cudaMemsetAsync(w.hist[0], 0, sizeof(unsigned) * kBins * n_inst, s));
        PCH_CUDA(cudaMemsetAsync(w.hist[1], 0, sizeof(unsigned) * kBins * n_inst, s));
        PCH_CUDA(cudaMemsetAsync(ws->ang_all, 0xff, sizeof(unsigned long long) * aoff, s));
        PCH_CUDA(cudaMemsetAsync(ws->stamp_all, 0, sizeof(unsigned) * goff, s));
        PCH_CUDA(cudaMemsetAsync(ws->fanphi_all, 0xff, sizeof(float) * goff, s));   // NaN: no fan yet
        if (w.trace_rows) PCH_CUDA(cudaMemsetAsync(w.trace_rows, 0, sizeof(int), s));
        if (stats) std::memset(stats, 0, sizeof(pch_stats));
        k_fill_inf<<<grid_for(4), 256, 0, s>>>(ws->g_all, goff);
        SrcDev* dsrc = nullptr;
        PCH_CUDA(cudaMallocAsync(&dsrc, sizeof(SrcDev) * n_src, s));
        PCH_CUDA(cudaMemcpyAsync(dsrc, srcs, sizeof(SrcDev) * n_src, cudaMemcpyHostToDevice, s));
        k_init_sources<<<(n_src + 127) / 128, 128, 0, s>>>(w, dsrc, n_src);
        k_init_face_sources<<<(n_src + 127) / 128, 128, 0, s>>>(w, dsrc, n_src);
        PCH_CUDA(cudaGetLastError());
        PCH_CUDA(cudaFreeAsync(dsrc, s));
        if (stats) stats->kernel_launches = 3;
        st = run_solve(ws, s, cfg, stats);
        if (st == PCH_ERR_CAPACITY && (ws->cnt_host->error & kErrReqFull) && attempt < 4) {
            st = ensure_pools(ws, ws->sel_cap, ws->pool_cap, 2 * ws->req_cap);
            if (st != PCH_OK) return st;
            clear_error();
            continue;
        }
        if (st == PCH_ERR_CAPACITY && (ws->cnt_host->error & kErrProvFull) && attempt < 4) {
            int most = 0;
            for (int r = 0; r < kPlogShards; ++r) most = std::max(most, ws->cnt_host->n_plog_shard[r]);
            st = ensure_plog(ws, std::max<long long>(2LL * ws->plog_cap, (long long)(most + 1) * kPlogShards * 5 / 4));
            if (st != PCH_OK) return st;
            clear_error();
            continue;
        }
        if (st != PCH_OK) return st;
        break;
    }
    // results
    for (int i = 0; i < n_inst; ++i) {
        const DevMesh& dm = meshes[i]->dm;
        if (out_mode == kOutNone) continue;
        if (out_mode == kOutDevice) {
            k_copy_out<<<grid_for(2), 256, 0, s>>>(ws->g_all + gofs[i], outs[i], dm.nv);
            if (stats) stats->kernel_launches += 1;
        } else if (out_mode == kOutHost) {
            PCH_CUDA(cudaMemcpyAsync(outs[i], ws->g_all + gofs[i], sizeof(double) * dm.nv, cudaMemcpyDeviceToHost, s));
        }
    }
    PCH_CUDA(cudaGetLastError());
    if (out_mode != kOutDevice) PCH_CUDA(cudaStreamSynchronize(s));
    return PCH_OK;
}

// ====================================================================== geodesic paths
// Section 4.4: the window that finally assigns a vertex its distance is the last of a
// window sequence carrying its shortest path; Section 3: that path is a straight segment
// in the unfolding of the faces the sequence crosses, from the window's pseudo-source,
// and from there the pseudo-source's own path.

constexpr int kNoPick = 0x7f7f7f7f;          // per-vertex pick before any record matched
constexpr long long kTraceMaxSteps = 1 << 22;

// Per vertex of instance 0: the first record (lowest index over the written part of every
// shard) whose distance is the vertex's final one.
__global__ void k_prov_pick(const ProvRec* __restrict__ log, int per, const Counters* __restrict__ cnt,
                            const unsigned long long* __restrict__ g, int nv, int* pick) {
    const long long n = (long long)per * kPlogShards;
    for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x) {
        const int shard = (int)(i / per);
        if (i - (long long)shard * per >= cnt->n_plog_shard[shard]) continue;
        const ProvRec r = log[i];
        if (r.inst == 0 && r.v >= 0 && r.v < nv && r.db == g[r.v]) atomicMin(pick + r.v, (int)i);
    }
}

// Barycentric weights over the stored corners of face(e) of the point (x, y) in e's frame.
__device__ __forceinline__ pch_path_point face_point(const HERec& E, int e, double x, double y) {
    const double b2 = y / E.yc, b1 = (x - b2 * E.xc) / E.L, b0 = 1.0 - b1 - b2;
    double b[3];
    const int i = e % 3;
    b[i] = b0;
    b[(i + 1) % 3] = b1;
    b[(i + 2) % 3] = b2;
    pch_path_point p;
    p.kind = PCH_POINT_FACE; p.id = e / 3; p.t0 = b[1]; p.t1 = b[2];
    return p;
}

// One thread per target.  A segment from vertex v back to its window's pseudo-source I
// (coordinates in the window's edge frame h) leaves v's position in that frame; it
// crosses h (unless v is an end of h) into twin(h)'s face.  In a face entered through
// half-edge e (the point P on e's axis, I beyond e's apex side, y > 0) the segment ends
// at the apex when that is the pseudo-source; else it leaves through edge v1 -> v2 or
// v2 -> v0, on the side of the line P -> apex where I lies, and P, I are carried into
// the frame of that edge's twin, the next face.  A crossing is reported on the edge of
// the face the path has just traversed (the side of the target), like a window's edge.
__global__ void k_trace(Inst In, const ProvRec* __restrict__ log, const int* __restrict__ pick,
                        const int* __restrict__ targets, int n_targets, int max_points, pch_path_point* out,
                        int* n_out) {
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n_targets; i += gridDim.x * blockDim.x) {
        pch_path_point* po = out + (size_t)i * max_points;
        int np = 0;
        auto emit = [&](const pch_path_point& p) {
            if (np < max_points) po[np] = p;
            ++np;
        };
        auto vertex_pt = [](int v) {
            pch_path_point p;
            p.kind = PCH_POINT_VERTEX; p.id = v; p.t0 = 0.0; p.t1 = 0.0;
            return p;
        };
        auto edge_pt = [](int h, double t) {
            pch_path_point p;
            p.kind = PCH_POINT_EDGE; p.id = h; p.t0 = t; p.t1 = 0.0;
            return p;
        };
        int v = targets[i];
        if (In.g[v] >= 0x7FF0000000000000ull) {   // +inf: unreachable, no path
            n_out[i] = 0;
            continue;
        }
        emit(vertex_pt(v));
        bool ok = false;
        long long steps = 0;
        while (steps++ < kTraceMaxSteps) {
            if (In.g[v] == 0ull) {              // a source
                ok = true;
                break;
            }
            const int pi = pick[v];
            if (pi == kNoPick) break;
            const ProvRec r = log[pi];
            if (r.kind == 1) {                   // along a boundary edge from the fan vertex
                if (r.src < 0 || r.src >= In.nv) break;
                v = r.src;
                emit(vertex_pt(v));
                continue;
            }
            if (r.h < 0 || r.h >= In.nh) break;
            const HERec R = In.rec[r.h];
            if (r.kind == 2) {                   // straight to the face-point source
                emit(face_point(R, r.h, r.px, r.py));
                ok = true;
                break;
            }
            // kind 0: v is an end or the apex of the window's edge h
            const double L = R.L;
            double x;
            if (v == (int)(R.v0 & ~kPseudoBit)) {
                x = 0.0;
            } else if (v == (int)(R.v1 & ~kPseudoBit)) {
                x = L;
            } else if (v == (int)(R.v2 & ~kPseudoBit)) {
                x = r.px + (R.xc - r.px) * (-r.py) / (R.yc - r.py);
                x = x < 0.0 ? 0.0 : (x > L ? L : x);
                emit(edge_pt(r.h, x / L));
            } else {
                break;
            }
            int e = R.twin;
            double Px = L - x, Ix = L - r.px, Iy = -r.py;
            const double seg = sqrt((Ix - Px) * (Ix - Px) + Iy * Iy);
            bool seg_done = false, path_done = false;
            while (e >= 0 && e < In.nh && steps++ < kTraceMaxSteps) {
                const HERec E = In.rec[e];
                const int a2 = (int)(E.v2 & ~kPseudoBit);
                const double tol = 1e-7 * (E.L + seg);
                if (r.src >= 0 && r.src == a2 && (Ix - E.xc) * (Ix - E.xc) + (Iy - E.yc) * (Iy - E.yc) <= tol * tol) {
                    v = a2;                      // reached the pseudo-source
                    emit(vertex_pt(v));
                    seg_done = true;
                    break;
                }
                if (r.src < 0) {                 // the face-point source inside this face?
                    const double b2 = Iy / E.yc, b1 = (Ix - b2 * E.xc) / E.L;
                    if (b2 >= -1e-9 && b1 >= -1e-9 && 1.0 - b1 - b2 >= -1e-9) {
                        emit(face_point(E, e, Ix, Iy));
                        path_done = true;
                        break;
                    }
                }
                // leave through v1 -> v2 (I right of P -> apex) or v2 -> v0; if the crossing
                // falls outside that edge (a near-vertex pass) take the other one
                const bool right0 = (E.xc - Px) * Iy - E.yc * (Ix - Px) < 0.0;
                bool crossed = false;
                for (int attempt = 0; attempt < 2 && !crossed; ++attempt) {
                    const bool right = attempt == 0 ? right0 : !right0;
                    const int f = right ? E.tw1 : E.tw2;
                    if (f < 0) continue;
                    const double Lf = right ? E.L1 : E.L2;
                    const double ox = right ? E.xc : 0.0, oy = right ? E.yc : 0.0;
                    const double ux = (right ? E.L - E.xc : E.xc) / Lf, uy = (right ? -E.yc : E.yc) / Lf;
                    const double prx = Px - ox, pry = -oy, irx = Ix - ox, iry = Iy - oy;
                    const double pfx = prx * ux + pry * uy, pfy = ux * pry - uy * prx;
                    const double ifx = irx * ux + iry * uy, ify = ux * iry - uy * irx;
                    const double den = ify - pfy;
                    if (!(den > 0.0)) continue;
                    double xf = pfx + (ifx - pfx) * (-pfy) / den;
                    const double slack = 1e-9 * Lf;
                    if (!(xf >= -slack && xf <= Lf + slack)) continue;
                    xf = xf < 0.0 ? 0.0 : (xf > Lf ? Lf : xf);
                    const int exit_he = right ? he_next(e) : 3 * (e / 3) + (e % 3 + 2) % 3;
                    emit(edge_pt(exit_he, 1.0 - xf / Lf));
                    e = f;
                    Px = xf;
                    Ix = ifx;
                    Iy = ify;
                    crossed = true;
                }
                if (!crossed) break;
            }
            if (path_done) {
                ok = true;
                break;
            }
            if (!seg_done) break;
        }
        n_out[i] = ok ? np : -1;
    }
}

// Solve with the distance events recorded, then trace every target's path.
static pch_status trace_paths(pch_mesh* m, const SrcDev* sd, int n_src, const pch_options* opt, const int* targets,
                              int n_targets, int max_points, pch_path_point* points, int* n_points, double* out_dist,
                              pch_stats* stats) {
    pch_options o = opt ? *opt : pch_options{};
    o.out_on_device = 0;
    double* outs[1] = {out_dist};
    pch_status st = solve_instances(&m, 1, sd, n_src, &o, outs, out_dist ? kOutHost : kOutNone, stats, 1);
    if (st != PCH_OK) return st;
    Workspace* ws = m->ws;
    cudaStream_t s = (cudaStream_t)o.stream;
    const int nv = m->dm.nv;
    const int per = ws->plog_cap / kPlogShards;
    Inst I{};
    PCH_CUDA(cudaMemcpyAsync(&I, ws->w.inst, sizeof(Inst), cudaMemcpyDeviceToHost, s));
    int *dpick = nullptr, *dtg = nullptr, *dn = nullptr;
    pch_path_point* dpts = nullptr;
    const size_t npts = (size_t)std::max(n_targets, 1) * (size_t)max_points;
    cudaError_t e = cudaMallocAsync(&dpick, sizeof(int) * (size_t)nv, s);
    if (!e) e = cudaMallocAsync(&dtg, sizeof(int) * (size_t)std::max(n_targets, 1), s);
    if (!e) e = cudaMallocAsync(&dn, sizeof(int) * (size_t)std::max(n_targets, 1), s);
    if (!e) e = cudaMallocAsync(&dpts, sizeof(pch_path_point) * npts, s);
    if (!e && n_targets > 0) e = cudaMemcpyAsync(dtg, targets, sizeof(int) * (size_t)n_targets, cudaMemcpyHostToDevice, s);
    if (!e) e = cudaMemsetAsync(dpick, 0x7f, sizeof(int) * (size_t)nv, s);
    if (!e) e = cudaStreamSynchronize(s);   // I (the instance table) is needed by value
    if (!e) {
        k_prov_pick<<<grid_for(4), 256, 0, s>>>(ws->plog, per, ws->w.cnt, I.g, nv, dpick);
        if (n_targets > 0)
            k_trace<<<(n_targets + 127) / 128, 128, 0, s>>>(I, ws->plog, dpick, dtg, n_targets, max_points, dpts, dn);
        e = cudaGetLastError();
    }
    if (!e && n_targets > 0) e = cudaMemcpyAsync(n_points, dn, sizeof(int) * (size_t)n_targets, cudaMemcpyDeviceToHost, s);
    if (!e && n_targets > 0)
        e = cudaMemcpyAsync(points, dpts, sizeof(pch_path_point) * (size_t)n_targets * max_points, cudaMemcpyDeviceToHost, s);
    cudaFreeAsync(dpick, s);
    cudaFreeAsync(dtg, s);
    cudaFreeAsync(dn, s);
    cudaFreeAsync(dpts, s);
    if (!e) e = cudaStreamSynchronize(s);
    if (e) return set_error(e == cudaErrorMemoryAllocation ? PCH_ERR_OOM : PCH_ERR_CUDA, "path trace: %s",
                            cudaGetErrorString(e));
    if (stats) stats->kernel_launches += n_targets > 0 ? 2 : 1;
    return PCH_OK;
}

// ====================================================================== Voronoi labels
// The geodesic Voronoi diagram of a source set (Section 7 names it as the use of the
// multiple-source field): every vertex is labelled with its nearest source.  After a
// recording solve, each vertex's final event names the pseudo-source vertex its shortest
// path bends at last (Section 3: a geodesic bends only at saddle or boundary vertices), or
// the face-point source itself; following those vertices back (their distances strictly
// fall along the chain) ends at a source, whose index is the label.
constexpr int kLabelNone = -1;        // unreachable vertex
constexpr int kLabelBroken = -2;      // no recorded event with the final distance (never expected)

__global__ void k_voronoi_prep(int* vsrc, int nv) {
    for (int v = blockIdx.x * blockDim.x + threadIdx.x; v < nv; v += gridDim.x * blockDim.x)
        if (vsrc[v] == 0x7f7f7f7f) vsrc[v] = -1;
}

// One thread per vertex: walk the chain of last pseudo-sources up to a source.
__global__ void k_voronoi(const unsigned long long* __restrict__ g, const ProvRec* __restrict__ log,
                          const int* __restrict__ pick, const int* __restrict__ vsrc, int nv, int* __restrict__ label) {
    for (int v0 = blockIdx.x * blockDim.x + threadIdx.x; v0 < nv; v0 += gridDim.x * blockDim.x) {
        int v = v0, lab = kLabelBroken;
        if (g[v0] >= 0x7FF0000000000000ull) {
            label[v0] = kLabelNone;
            continue;
        }
        for (int step = 0; step < nv; ++step) {
            if (vsrc[v] >= 0) {                 // a vertex source
                lab = vsrc[v];
                break;
            }
            const int pi = pick[v];
            if (pi == kNoPick) break;
            const int src = log[pi].src;
            if (src < 0) {                      // the face-point source -1 - src
                lab = -1 - src;
                break;
            }
            if (src >= nv || src == v) break;
            v = src;
        }
        label[v0] = lab;
    }
}

__global__ void k_vertex_sources(const SrcDev* __restrict__ srcs, int n, int* vsrc) {
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x)
        if (srcs[i].kind == 0) atomicMin(vsrc + srcs[i].vertex, srcs[i].label);
}

static pch_status voronoi(pch_mesh* m, const SrcDev* sd, int n_src, const pch_options* opt, int* labels,
                          double* out_dist, pch_stats* stats) {
    pch_options o = opt ? *opt : pch_options{};
    o.out_on_device = 0;
    double* outs[1] = {out_dist};
    pch_status st = solve_instances(&m, 1, sd, n_src, &o, outs, out_dist ? kOutHost : kOutNone, stats, 1);
    if (st != PCH_OK) return st;
    Workspace* ws = m->ws;
    cudaStream_t s = (cudaStream_t)o.stream;
    const int nv = m->dm.nv;
    const int per = ws->plog_cap / kPlogShards;
    Inst I{};
    PCH_CUDA(cudaMemcpyAsync(&I, ws->w.inst, sizeof(Inst), cudaMemcpyDeviceToHost, s));
    int *dpick = nullptr, *dvsrc = nullptr, *dlab = nullptr;
    SrcDev* dsd = nullptr;
    cudaError_t e = cudaMallocAsync(&dpick, sizeof(int) * (size_t)nv, s);
    if (!e) e = cudaMallocAsync(&dvsrc, sizeof(int) * (size_t)nv, s);
    if (!e) e = cudaMallocAsync(&dlab, sizeof(int) * (size_t)nv, s);
    if (!e) e = cudaMallocAsync(&dsd, sizeof(SrcDev) * (size_t)n_src, s);
    if (!e) e = cudaMemcpyAsync(dsd, sd, sizeof(SrcDev) * (size_t)n_src, cudaMemcpyHostToDevice, s);
    if (!e) e = cudaMemsetAsync(dpick, 0x7f, sizeof(int) * (size_t)nv, s);
    if (!e) e = cudaMemsetAsync(dvsrc, 0x7f, sizeof(int) * (size_t)nv, s);   // 0x7f7f7f7f: no source
    if (!e) e = cudaStreamSynchronize(s);   // I (the instance table) is needed by value
    if (!e) {
        k_vertex_sources<<<(n_src + 127) / 128, 128, 0, s>>>(dsd, n_src, dvsrc);
        k_prov_pick<<<grid_for(4), 256, 0, s>>>(ws->plog, per, ws->w.cnt, I.g, nv, dpick);
        // vsrc >= 0 marks a vertex source; the fill value 0x7f7f7f7f is turned into -1 here
        k_voronoi_prep<<<grid_for(4), 256, 0, s>>>(dvsrc, nv);
        k_voronoi<<<grid_for(4), 256, 0, s>>>(I.g, ws->plog, dpick, dvsrc, nv, dlab);
        e = cudaGetLastError();
    }
    if (!e) e = cudaMemcpyAsync(labels, dlab, sizeof(int) * (size_t)nv, cudaMemcpyDeviceToHost, s);
    cudaFreeAsync(dpick, s);
    cudaFreeAsync(dvsrc, s);
    cudaFreeAsync(dlab, s);
    cudaFreeAsync(dsd, s);
    if (!e) e = cudaStreamSynchronize(s);
    if (e) return set_error(e == cudaErrorMemoryAllocation ? PCH_ERR_OOM : PCH_ERR_CUDA, "voronoi: %s",
                            cudaGetErrorString(e));
    if (stats) stats->kernel_launches += 4;
    return PCH_OK;
}

}  // namespace pch

using namespace pch;

static SrcDev src_dev(const pch_source& s, int inst, int label) {
    SrcDev sd{};
    sd.inst = inst; sd.kind = s.kind; sd.vertex = s.vertex; sd.face = s.face; sd.label = label;
    for (int k = 0; k < 3; ++k) sd.bary[k] = s.bary[k];
    return sd;
}

extern "C" pch_status pch_solve(pch_mesh* m, const pch_source* src, const pch_options* opt, double* out_dist,
                                pch_stats* stats) {
    if (!m || !src || !out_dist) return set_error(PCH_ERR_INVALID_ARG, "null argument");
    SrcDev sd = src_dev(*src, 0, 0);
    double* outs[1] = {out_dist};
    return solve_instances(&m, 1, &sd, 1, opt, outs, (opt && opt->out_on_device) ? kOutDevice : kOutHost, stats);
}

extern "C" pch_status pch_solve_multi(pch_mesh* m, const pch_source* srcs, int32_t n_sources, const pch_options* opt,
                                      double* out_dist, pch_stats* stats) {
    if (!m || !srcs || !out_dist || n_sources <= 0) return set_error(PCH_ERR_INVALID_ARG, "null argument");
    std::vector<SrcDev> sd(n_sources);
    for (int i = 0; i < n_sources; ++i) sd[i] = src_dev(srcs[i], 0, i);
    double* outs[1] = {out_dist};
    return solve_instances(&m, 1, sd.data(), n_sources, opt, outs, (opt && opt->out_on_device) ? kOutDevice : kOutHost,
                           stats);
}

extern "C" pch_status pch_solve_batch(pch_mesh* const* meshes, const pch_source* srcs, int32_t n_instances,
                                      const pch_options* opt, double* const* out_dists, pch_stats* stats) {
    if (!meshes || !srcs || !out_dists || n_instances <= 0) return set_error(PCH_ERR_INVALID_ARG, "null argument");
    std::vector<SrcDev> sd(n_instances);
    for (int i = 0; i < n_instances; ++i) {
        if (!out_dists[i]) return set_error(PCH_ERR_INVALID_ARG, "null output for instance %d", i);
        sd[i] = src_dev(srcs[i], i, 0);
    }
    return solve_instances(meshes, n_instances, sd.data(), n_instances, opt, out_dists,
                           (opt && opt->out_on_device) ? kOutDevice : kOutHost, stats);
}

extern "C" pch_status pch_trace_paths(pch_mesh* m, const pch_source* srcs, int32_t n_sources, const pch_options* opt,
                                      const int32_t* targets, int32_t n_targets, int32_t max_points,
                                      pch_path_point* points, int32_t* n_points, double* out_dist, pch_stats* stats) {
    clear_error();
    if (!m || !srcs || n_sources <= 0 || n_targets < 0 || max_points < 1)
        return set_error(PCH_ERR_INVALID_ARG, "null argument, no source, n_targets < 0 or max_points < 1");
    if (n_targets > 0 && (!targets || !points || !n_points)) return set_error(PCH_ERR_INVALID_ARG, "null path buffers");
    if ((long long)n_targets * (long long)max_points > (1LL << 31))
        return set_error(PCH_ERR_CAPACITY, "n_targets * max_points exceeds 2^31 points");
    for (int i = 0; i < n_targets; ++i)
        if (targets[i] < 0 || targets[i] >= m->dm.nv) return set_error(PCH_ERR_INVALID_ARG, "target %d out of range", targets[i]);
    std::vector<SrcDev> sd(n_sources);
    for (int i = 0; i < n_sources; ++i) sd[i] = src_dev(srcs[i], 0, i);
    return trace_paths(m, sd.data(), n_sources, opt, targets, n_targets, max_points, points, n_points, out_dist, stats);
}

extern "C" pch_status pch_voronoi(pch_mesh* m, const pch_source* srcs, int32_t n_sources, const pch_options* opt,
                                  int32_t* labels, double* out_dist, pch_stats* stats) {
    clear_error();
    if (!m || !srcs || n_sources <= 0 || !labels) return set_error(PCH_ERR_INVALID_ARG, "null argument or no source");
    std::vector<SrcDev> sd(n_sources);
    for (int i = 0; i < n_sources; ++i) sd[i] = src_dev(srcs[i], 0, i);
    return voronoi(m, sd.data(), n_sources, opt, labels, out_dist, stats);
}

extern "C" pch_status pch_trace_fetch(pch_mesh* m, int32_t max_rows, float* features, float* chosen, int32_t* n_rows) {
    clear_error();
    if (!m || !n_rows) return set_error(PCH_ERR_INVALID_ARG, "null argument");
    Workspace* ws = m->ws;
    if (!ws || !ws->trace_buf) { *n_rows = 0; return PCH_OK; }
    int rows = 0;
    PCH_CUDA(cudaMemcpy(&rows, ws->trace_rows, sizeof(int), cudaMemcpyDeviceToHost));
    rows = std::min(rows, ws->trace_cap);
    if (max_rows < rows) rows = max_rows < 0 ? 0 : max_rows;
    std::vector<float> buf((size_t)rows * (kFeatures + 2));
    if (rows) PCH_CUDA(cudaMemcpy(buf.data(), ws->trace_buf, sizeof(float) * buf.size(), cudaMemcpyDeviceToHost));
    for (int r = 0; r < rows; ++r) {
        if (features) std::memcpy(features + (size_t)r * kFeatures, &buf[(size_t)r * (kFeatures + 2)], sizeof(float) * kFeatures);
        if (chosen) chosen[r] = buf[(size_t)r * (kFeatures + 2) + kFeatures];
    }
    *n_rows = rows;
    return PCH_OK;
}

// ---------------------------------------------------------------- autotuner
#include <fstream>
#include <sstream>
#include <string>

#ifndef PCH_BUILD_ID
#define PCH_BUILD_ID "unversioned"
#endif

extern "C" const char* pch_build_id(void) { return PCH_BUILD_ID; }

extern "C" pch_status pch_autotune(pch_mesh* m, const pch_source* src, pch_options* opt, const char* cache_path,
                                   double* best_ms) {
    clear_error();
    if (!m || !src || !opt) return set_error(PCH_ERR_INVALID_ARG, "null argument");
    cudaDeviceProp prop;
    int dev = 0;
    PCH_CUDA(cudaGetDevice(&dev));
    PCH_CUDA(cudaGetDeviceProperties(&prop, dev));
    std::string name(prop.name);
    for (auto& ch : name) if (ch == ' ' || ch == '|') ch = '_';
    std::ostringstream keyss;
    keyss << name << "|build=" << PCH_BUILD_ID << "|nv=" << m->dm.nv << "|nf=" << m->dm.nf
          << "|control=" << opt->control << "|flags=" << opt->flags;
    const std::string key = keyss.str();
    if (cache_path) {
        std::ifstream in(cache_path);
        std::string line;
        while (std::getline(in, line)) {
            std::istringstream ls(line);
            std::string k2;
            long long kk;
            int bb, hh;
            double ms;
            if (ls >> k2 >> kk >> bb >> hh >> ms && k2 == key) {
                opt->k = kk;
                opt->block = bb;
                opt->hops = hh;
                if (best_ms) *best_ms = ms;
                return PCH_OK;
            }
        }
    }
    SrcDev sd = src_dev(*src, 0, 0);
    pch_options trial = *opt;
    trial.out_on_device = 0;
    double best = 1e300;
    long long best_k = 0;
    int best_b = 0, best_h = 0;
    std::vector<long long> ks;
    for (long long k = 24576; k <= std::max<long long>(24576, 8LL * m->dm.nf); k *= 4) ks.push_back(k);
    const int blocks[3] = {64, 128, 256};
    const int hopss[5] = {4, 8, 16, 32, 64};
    auto time_cfg = [&](long long k, int b, int hp, double& ms) -> pch_status {
        trial.k = k;
        trial.block = b;
        trial.hops = hp;
        for (int rep = 0; rep < 2; ++rep) {   // the first run warms the graph cache
            pch_stats st{};
            pch_status rc = solve_instances(&m, 1, &sd, 1, &trial, nullptr, kOutNone, &st);
            if (rc != PCH_OK) return rc;
            ms = st.ms_total;
            if (rep == 0 && ms > 2.0 * best) break;   // far from the best: no second timing
        }
        return PCH_OK;
    };
    auto consider = [&](long long k, int b, int hp) -> pch_status {
        double ms = 0.0;
        pch_status rc = time_cfg(k, b, hp, ms);
        if (rc == PCH_OK && ms < best) { best = ms; best_k = k; best_b = b; best_h = hp; }
        return rc;
    };
    // the library's defaults first (so the result is never slower than them, up to the
    // noise of one timing), then a coordinate search: k at (128, 16) from the largest down
    // (stopping once a k is twice as slow as the best: smaller ones only add iterations),
    // then hops, then the block size
    // (under PCH_CONTROL_LEARNED the network picks k every iteration: only hops and the
    // block size are searched)
    const bool learned = opt->control == PCH_CONTROL_LEARNED;
    pch_status rc = consider(default_k(), 64, default_hops());
    if (rc != PCH_OK) return rc;
    if (learned) ks.clear();
    for (auto it = ks.rbegin(); it != ks.rend(); ++it) {
        double ms = 0.0;
        if ((rc = time_cfg(*it, 128, 16, ms)) != PCH_OK) return rc;
        if (ms < best) { best = ms; best_k = *it; best_b = 128; best_h = 16; }
        if (ms > 2.0 * best) break;
    }
    const long long k_sel = best_k;
    // hops from the most down, stopping once a setting is twice as slow as the best
    for (int q = 4; q >= 0; --q) {
        const int hp = hopss[q];
        if (!learned && hp == 16) continue;
        double ms = 0.0;
        if ((rc = time_cfg(k_sel, 128, hp, ms)) != PCH_OK) return rc;
        if (ms < best) { best = ms; best_k = k_sel; best_b = 128; best_h = hp; }
        if (ms > 2.0 * best) break;
    }
    const int h_sel = best_h;
    for (int b : blocks)
        if (b != 128 && (rc = consider(k_sel, b, h_sel)) != PCH_OK) return rc;
    opt->k = best_k;
    opt->block = best_b;
    opt->hops = best_h;
    if (best_ms) *best_ms = best;
    if (cache_path) {
        std::ofstream out(cache_path, std::ios::app);
        out.precision(17);
        out << key << " " << best_k << " " << best_b << " " << best_h << " " << best << "\n";
    }
    return PCH_OK;
}

// ---------------------------------------------------------------- math self-test
__global__ void k_selftest_math(const double* __restrict__ x, int n, unsigned long long* maxulp) {
    unsigned long long mr = 0, ms = 0;
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x) {
        const double v = x[i];
        const long long a = __double_as_longlong(rcp_nr(v)), b = __double_as_longlong(1.0 / v);

        const long long c = __double_as_longlong(sqrt_nr(fabs(v))), d = __double_as_longlong(sqrt(fabs(v)));
        unsigned long long ur = (unsigned long long)(a > b ? a - b : b - a);
        unsigned long long us = (unsigned long long)(c > d ? c - d : d - c);
        mr = ur > mr ? ur : mr;
        ms = us > ms ? us : ms;
    }
    atomicMax(maxulp, mr);
    atomicMax(maxulp + 1, ms);
}

extern "C" pch_status pch_selftest_math(const double* x_dev, int32_t n, unsigned long long* max_ulp_host) {
    clear_error();
    if (!x_dev || n <= 0 || !max_ulp_host) return set_error(PCH_ERR_INVALID_ARG, "bad arguments");
    unsigned long long* d = nullptr;
    PCH_CUDA(cudaMalloc(&d, 2 * sizeof(unsigned long long)));
    cudaMemset(d, 0, 2 * sizeof(unsigned long long));
    k_selftest_math<<<grid_for(2), 256>>>(x_dev, n, d);
    cudaError_t e = cudaMemcpy(max_ulp_host, d, 2 * sizeof(unsigned long long), cudaMemcpyDeviceToHost);
    cudaFree(d);
    PCH_CUDA(e);
    return PCH_OK;
}
