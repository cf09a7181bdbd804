// Internal device data layout of the PCH library (sm_103a).
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include "../../include/pch.h"

namespace pch {

// ---- tolerances (same values, independently written, as the CPU oracle) -------------
// "A = v0", "B = v1" and vertex occupancy are decided within kEpsSnap * |e| (2^-40,
// about 9.1e-13, a power of two so that the product is an exponent shift).
constexpr double kEpsSnap = 0x1p-40;
// Windows narrower than kEpsTiny * |e| are dropped (Section 5.3 drops tiny windows).
constexpr double kEpsTiny = 0x1p-40;
// kEpsSnap in units in the last place: B is at v1 when within 4096 ulp of |e| (between
// 2^-41 and 2^-40 of it, by where |e| falls in its binade).
constexpr long long kSnapUlps = 4096;
// A filter removes a window only when it is worse by more than this relative margin.
constexpr double kDomRel = 1e-12;

constexpr unsigned long long kEmptyAngle = ~0ull;
constexpr int kAngleXBits = 24;                       // low bits of a packed angle_split word
constexpr unsigned long long kAngleXMask = (1ull << kAngleXBits) - 1;
constexpr unsigned kPseudoBit = 0x80000000u;          // vertex id flag: saddle or boundary vertex

// Selection histogram: bin b covers (key - ref)/lbar in [(2^(b/16)-1)/4, (2^((b+1)/16)-1)/4).
constexpr int kBins = 256;
constexpr float kBinsPerOctave = 16.f;
constexpr float kBinScale = 4.f;

// Controller features (a8): see controller.cu.
constexpr int kFeatures = 24;
constexpr int kHidden = 64;

// ---- mesh (Section 4.1): one 96-byte record per half-edge --------------------------
// Frame of half-edge h = (v0 -> v1) in face f: v0 at the origin, v1 at (L, 0), the
// opposite vertex v2 at (xc, yc), yc > 0.  A window on h propagates into f.
struct __align__(16) HERec {
    double L, xc, yc;      // edge length and apex position
    double L1, L2;         // |v1 v2|, |v2 v0|
    double u1x, u1y;       // unit vector from v2 to v1: the right child's edge axis
    double u2x, u2y;       // unit vector from v0 to v2: the left child's edge axis
    int tw1;               // twin of next(h) = (v2 -> v1) in the neighbour: right child's edge
    int tw2;               // twin of prev(h) = (v0 -> v2) in the neighbour: left child's edge
    unsigned v0, v1, v2;   // vertex ids | kPseudoBit
    int twin;              // twin of h (-1 on the boundary)
};
static_assert(sizeof(HERec) == 96, "HERec layout");

struct DevMesh {
    int nv, nf, nh;
    double lbar;           // mean edge length
    HERec* rec;            // [nh]
    int* vstart;           // [nv + 1] CSR of outgoing half-edges, one-ring order
    int* vlist;            // [nh]
    // angles, kept in FP32: they only steer the pseudo-source fans, whose wedges are
    // widened far beyond FP32 rounding (the saddle test itself is made in FP64)
    float* hang;           // [nh] corner angle at the start vertex of each half-edge
    float* vtheta;         // [nv] total angle (Section 3)
    float* vphi;           // [nh] angular position of each outgoing half-edge around its start vertex
    double2* vrot;         // [nh] (cos, sin) of vphi, FP64: exact directions without trigonometry
    double2* vtrot;        // [nv] (cos, sin) of vtheta
    unsigned char* vflag;  // [nv] bit0 boundary, bit1 pseudo-source capable
};

// ---- windows: structure of arrays (Section 3's 6-tuple, with the pseudo-source kept
// as coordinates (px, py) in the edge frame instead of (d0, d1)) ------------------------
struct WinSoA {
    int* he;        // half-edge (local to the instance's mesh); -1 = empty slot
    int* inst;      // instance
    double* d;      // pseudo-source distance to the source
    double* A;      // interval [A, B] along the edge from its start vertex
    double* B;
    double* px;     // pseudo-source position in the edge frame (py < 0)
    double* py;
    double* key;    // d + dist(I, [A, B]): the window's distance back to the source
    int* src;       // mesh vertex at the pseudo-source (-1 for a point inside a face)
    double* IA;     // |I A|, |I B| (kept so that propagation never recomputes them)
    double* IB;
};

// ---- instances -------------------------------------------------------------------
struct Inst {
    const HERec* rec;
    const int* vstart;
    const int* vlist;
    const float* vphi;          // angular position of every half-edge around its start vertex
    const float* vtheta;        // total angle per vertex
    const float* hang;          // corner angle at the start vertex of every half-edge
    const double2* vrot;        // (cos, sin) of the angular position of every half-edge
    const double2* vtrot;       // (cos, sin) of the total angle of every vertex
    const unsigned char* vflag; // bit0: boundary vertex
    unsigned long long* g;      // geod_dist[] as ordered u64 images of nonnegative doubles
    unsigned long long* ang;    // angle_split[]: packed (rounded-up distance, crossing position)
    unsigned* stamp;            // per-vertex iteration stamp (one fan request per iteration)
    float* fan_phi;             // per-vertex angular position of the incoming ray of its last fan
    double2* fan_dir;           // per-vertex unit incoming direction of its last fan (angular frame)
    int nv, nh;
    long long keybase;          // sort key = keybase + half-edge
    double lbar;
    double ilbar;
};

struct InstCtl {
    double tau;                 // selection threshold of the current iteration
    double ref;                 // histogram reference (a lower bound of every pending key)
    unsigned long long kmin;    // running min of the keys written to the next pool (bits)
    int n_pending;              // pending windows of this instance in the current pool
    int n_next;                 // pending windows written to the next pool
    int n_sel;                  // selected this iteration
    int n_child;                // children written this iteration
    long long k_target;         // plain control: windows to select
    float last_ratio;           // children / selected of the previous iteration
    float ctl_out;              // last controller output
    int active;
    int pad;
};

// ---- global counters of one solve -------------------------------------------------
struct Counters {
    int n_pending;          // windows in the current pool
    int n_rest;             // not-selected windows copied to the next pool
    int n_sel;              // selected windows (work list)
    int n_child;            // slots used in the child arena
    int n_req;              // fan requests for this iteration
    int n_req_next;         // fan requests for the next iteration
    int n_app;              // windows appended to the next pool
    int iter;
    int error;              // bitmask of kErr*
    int done;
    int sort_bits;          // bits of the sort key
    int halt;               // set by k_finish when the loop must stop; every kernel no-ops
    unsigned long long created, propagated, filtered, trimmed, peak_pending;
    unsigned long long fans, fan_windows, fan_cand, chained;
    unsigned long long examined, occupied, children, rays;   // propagation path counts (FP64 op tally)
    unsigned long long scanned, sorted;               // windows read by compaction / sorted
    unsigned long long fan_ties;                      // deferred ties fanned (a new direction)
    int work_next;          // next work-list index handed to a propagation lane
    int n_plog;             // unused (kept for the layout); see n_plog_shard
    int n_plog_shard[32];   // provenance records reserved per shard (geodesic paths)
};
// Distance-event records are split into kPlogShards equal shards, one counter each, chosen
// by the SM a warp runs on: slot reservations then contend on 32 counters, not one.
constexpr int kPlogShards = 32;

enum : int {
    kErrPoolFull = 1,
    kErrReqFull = 2,
    kErrIter = 4,
    kErrNaN = 8,
    kErrProvFull = 16,
};

// Provenance of a distance event that lowered a vertex's distance (geodesic paths).  The
// record whose distance equals the vertex's final one comes from the last window of the
// window sequence that carries the vertex's shortest path (Section 4.4).
struct ProvRec {
    unsigned long long db;   // the event's distance (ordered bit image)
    int inst, v;             // instance, vertex
    int h;                   // kind 0: the window's half-edge; kind 2: a half-edge of the source's face
    int src;                 // pseudo-source vertex (-1: the face-point source)
    int kind;                // 0 window event, 1 along a boundary edge from src, 2 corner of the source's face
    int pad;
    double px, py;           // kind 0: pseudo-source, kind 2: the face point, in h's frame
};
static_assert(sizeof(ProvRec) == 48, "ProvRec layout");

// A pseudo-source fan candidate: a distance event at a saddle or boundary vertex, with
// the direction it arrived from.
struct FanReq {
    int inst;
    unsigned v;
    int href;       // half-edge leaving v whose frame holds (dx, dy); -1: every direction
    int tie;        // kind of candidate: from a lowering event, from a tying event, a deferred tie
    double D;       // the event's distance
    double dx, dy;  // from v towards the event's pseudo-source, in href's frame
};

// Capacities and buffers of the solve workspace.
struct Work {
    WinSoA pool[2];         // current / next pending pool
    WinSoA sel;             // selected windows
    WinSoA arena;           // children of this iteration (unsorted)
    int pool_cap, sel_cap, arena_cap, req_cap;
    FanReq* req[2];         // fan candidates of this and of the next iteration
    unsigned* sort_key[2];
    int* sort_val[2];
    int* sort_hist;         // radix histograms
    int sort_blocks;
    unsigned* hist[2];      // selection histograms [n_inst * kBins]
    Inst* inst;
    InstCtl* ctl;
    int n_inst;
    Counters* cnt;
    float* trace;           // controller trace rows
    int trace_cap;
    int* trace_rows;
    // strided approximate selection (Section 5.1): stride_T > 0 virtual threads, thread t
    // owns pool positions t, t + T, t + 2T, ... and selects its m nearest windows; the
    // m-th nearest (key bits, position) of each thread is its threshold
    int stride_T;
    unsigned long long* sthr_key;
    int* sthr_idx;
    // geodesic paths: distance events that lowered a vertex's distance (nullptr: off)
    ProvRec* plog;
    int plog_cap;
};

// Ordered u64 image of a nonnegative double (atomicMin-able, Section 4.2 Step 4).
__device__ __forceinline__ unsigned long long dbits(double x) { return (unsigned long long)__double_as_longlong(x); }
__device__ __forceinline__ double bitsd(unsigned long long b) { return __longlong_as_double((long long)b); }
// lhs > rhs (1 + kDomRel) for nonnegative lhs, rhs, decided on the ordered bit images so
// it costs no FP64 instruction: within a binade 9008 units in the last place are between
// 1e-12 and 2e-12 relative, so the test never removes a window the relative margin keeps.
constexpr unsigned long long kDomUlps = 9008;
__device__ __forceinline__ bool dominated(double lhs, double rhs) { return dbits(lhs) > dbits(rhs) + kDomUlps; }

// Order tests on the signed 64-bit images of doubles.  For non-NaN x, y of which at least
// one is >= +0 the images order exactly as the values (a negative operand has a negative
// image), except that -0 counts below +0.  They run on the integer pipe, which keeps the
// FP64 unit for arithmetic.
__device__ __forceinline__ long long sbits(double x) { return __double_as_longlong(x); }
__device__ __forceinline__ bool lt_s(double x, double y) { return sbits(x) < sbits(y); }
__device__ __forceinline__ bool le_s(double x, double y) { return sbits(x) <= sbits(y); }
__device__ __forceinline__ bool gt0_s(double x) { return sbits(x) > 0; }    // x > 0 (NaN: by sign)
__device__ __forceinline__ bool ge0_s(double x) { return sbits(x) >= 0; }   // x >= +0

// x * 2^-40 for a positive x by its exponent field (no FP64 instruction); x at or below
// 2^-900 takes the multiplication.
__device__ __forceinline__ double times_eps(double x) {
    const long long b = sbits(x);
    return b > 0x07B0000000000000ll ? __longlong_as_double(b - (40ll << 52)) : x * kEpsSnap;
}

}  // namespace pch
