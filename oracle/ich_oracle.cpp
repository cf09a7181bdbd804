// Sequential FP64 CPU oracle for exact polyhedral geodesic distance (Chen-Han with the
// Xin-Wang window filter, "ICH").  TEST INFRASTRUCTURE ONLY: the tests, the smoke check
// and the benchmark's CPU-baseline leg call it; the CUDA product path never does.
//
// It follows the paper's sequential reading (Section 3 and Section 4.2, Algorithm 2):
//  * a window is the 6-tuple (d, A, B, d0, d1, e) of Section 3 (Fig. `fig:window`):
//    interval [A,B] on oriented edge e, pseudo-source I at distance d from the source,
//    d0 = |I e.start|, d1 = |I e.end| in the unfolding (Fig. `fig:window`(b));
//  * windows are kept in a priority queue keyed by their distance back to the source,
//    as ICH does (Section 2, "Exact geodesic algorithms"; Section 6, ICH comparison);
//  * each popped window is propagated with Algorithm 2's steps in order: endpoint
//    events at v0 and v1 (with pseudo-source fans at saddle vertices, Fig.
//    `fig:propagation`(c)), occupancy of v2 and the "one angle one split" rule (Fig.
//    `fig:filter`(a)), the event at v2, then the ICH filter of Fig. `fig:filter`(b) on the
//    new windows.  Being sequential, events are applied at once (no event sort needed).
//  * initialisation per Algorithm 1: geod_dist = 0 at the source, +inf elsewhere; one
//    window on every edge opposite the source (Section 4.2, "Initialization").
//  * geodesic paths (TRACE): every window keeps its parent and its pseudo-source vertex,
//    every vertex the event that set its distance; a path is walked back along that
//    window sequence (Section 4.4) as straight unfolded segments (Section 3).
// Readings where the paper is silent (tolerances, which child a losing window keeps,
// boundary vertices, face-point sources) are stated next to the code that takes them.
#include <algorithm>
#include <cmath>
#include <cstdint>
#include <cstring>
#include <deque>
#include <limits>
#include <queue>
#include <unordered_map>
#include <vector>

namespace {

const double kInf = std::numeric_limits<double>::infinity();
const double kTwoPi = 6.283185307179586476925286766559;
// Relative snapping tolerance for "A = v0", "B = v1" and vertex occupancy (Algorithm 2
// tests endpoint equality exactly; rounding needs a band).
const double kEpsSnap = 1e-12;
// Windows narrower than kEpsTiny * |e| are dropped (Section 5.3 drops "tiny windows"
// with an absolute 1e-6; a relative 1e-12 keeps every window that can carry a distance).
const double kEpsTiny = 1e-12;
// A filter removes a window only when it is worse by more than this relative margin.
const double kDomRel = 1e-12;

enum {
    ORDER_PQ = 0, ORDER_FIFO = 1, ORDER_RANDOM = 2,
    ORDER_BATCH = 3,   // CPU PCH (Section 6): rounds of the k nearest windows, unordered
    ORDER_MASK = 3,
    NO_CH = 4,       // disable "one angle one split"
    NO_ICH = 8,      // disable the Xin-Wang filter
    TRACE = 16,      // keep every window and each vertex's final event (geodesic paths)
};

inline bool dominated(double lhs, double rhs) { return lhs > rhs * (1.0 + kDomRel); }

struct Mesh {
    int nv = 0, nf = 0;
    const double* xyz = nullptr;
    const int* tri = nullptr;
    std::vector<int> twin;          // 3F, -1 on the boundary
    std::vector<double> len;        // 3F, |start end|
    std::vector<char> pseudo;       // V: saddle (total angle >= 2 pi) or boundary vertex
    std::vector<std::vector<int>> out_he;   // V: outgoing half-edges
};

inline int nxt(int h) { return 3 * (h / 3) + (h % 3 + 1) % 3; }   // Section 4.1 formula
inline int prv(int h) { return 3 * (h / 3) + (h % 3 + 2) % 3; }
inline int hfrom(const Mesh& m, int h) { return m.tri[h]; }
inline int hto(const Mesh& m, int h) { return m.tri[nxt(h)]; }

double dist3(const Mesh& m, int a, int b) {
    double dx = m.xyz[3 * a] - m.xyz[3 * b], dy = m.xyz[3 * a + 1] - m.xyz[3 * b + 1],
           dz = m.xyz[3 * a + 2] - m.xyz[3 * b + 2];
    return std::sqrt(dx * dx + dy * dy + dz * dz);
}

// Half-edge structure of Section 4.1: he[3f+i] runs from tri[f][i] to tri[f][(i+1)%3].
int build_mesh(Mesh& m) {
    const int H = 3 * m.nf;
    m.twin.assign(H, -1);
    m.len.resize(H);
    std::unordered_map<uint64_t, int> dir;
    dir.reserve(2 * H);
    for (int h = 0; h < H; ++h) {
        int a = hfrom(m, h), b = hto(m, h);
        if (a < 0 || a >= m.nv || b < 0 || b >= m.nv || a == b) return -1;
        uint64_t k = (uint64_t)(uint32_t)a << 32 | (uint32_t)b;
        if (!dir.emplace(k, h).second) return -2;   // same directed edge twice: non-manifold
        m.len[h] = dist3(m, a, b);
    }
    for (int h = 0; h < H; ++h) {
        uint64_t k = (uint64_t)(uint32_t)hto(m, h) << 32 | (uint32_t)hfrom(m, h);
        auto it = dir.find(k);
        if (it != dir.end()) m.twin[h] = it->second;
    }
    // total angle per vertex (Section 3: spherical / Euclidean / saddle)
    std::vector<double> theta(m.nv, 0.0);
    std::vector<char> boundary(m.nv, 0);
    m.out_he.assign(m.nv, {});
    for (int h = 0; h < H; ++h) {
        int v = hfrom(m, h);
        m.out_he[v].push_back(h);
        double a = m.len[h], b = m.len[prv(h)], c = m.len[nxt(h)];
        if (a <= 0 || b <= 0) return -3;
        double cs = (a * a + b * b - c * c) / (2 * a * b);
        cs = std::max(-1.0, std::min(1.0, cs));
        theta[v] += std::acos(cs);
        if (m.twin[h] < 0) { boundary[hfrom(m, h)] = 1; boundary[hto(m, h)] = 1; }
    }
    m.pseudo.assign(m.nv, 0);
    for (int v = 0; v < m.nv; ++v)
        // A superset of the saddle vertices is sound (every fan window is a real path);
        // boundary vertices are included because geodesics may bend around them.
        m.pseudo[v] = boundary[v] || theta[v] > kTwoPi - 1e-9;
    return 0;
}

struct Window {
    double d, A, B, d0, d1;   // the paper's (d, A, B, d0, d1, e)
    int e;
    // path bookkeeping (TRACE only): the pseudo-source vertex (-1: the face-point source),
    // the window this one is a child of (-1: a fan or initial window) and its own index
    int src = -1, parent = -1, id = -1;
};

// A distance event with where it came from (TRACE only): a window event (kind 0, the
// window's index), a pseudo-source fan's event along a boundary edge (kind 1, from the
// vertex src), or the corner of a face-point source's face (kind 2).
struct Event {
    int v;
    double D;
    int kind = -1, wid = -1, src = -1;
};

struct Entry {
    double key;
    uint64_t seq;
    Window w;
};
struct EntryCmp {
    bool operator()(const Entry& a, const Entry& b) const {
        if (a.key != b.key) return a.key > b.key;
        return a.seq > b.seq;
    }
};

// Pseudo-source position in the frame of the window's edge (start at the origin, end at
// (L,0), propagation face on the +y side, I below): Fig. `fig:window`(b).
inline void pseudo_xy(const Window& w, double L, double& px, double& py) {
    px = ((w.d0 - w.d1) * (w.d0 + w.d1) + L * L) / (2 * L);
    double t = (w.d0 - px) * (w.d0 + px);
    py = -std::sqrt(t > 0 ? t : 0.0);
}

// Opposite vertex v2 of edge h, in h's frame (law of cosines on the three edge lengths:
// the method needs only the metric, Section 4.1).
inline void apex_xy(const Mesh& m, int h, double& xc, double& yc) {
    double L = m.len[h], a = m.len[prv(h)], b = m.len[nxt(h)];
    xc = ((a - b) * (a + b) + L * L) / (2 * L);
    double t = (a - xc) * (a + xc);
    yc = std::sqrt(t > 0 ? t : 0.0);
}

// Distance-to-source key of a window: d + distance from I to the segment [A,B]
// (the "shortest distance from the source to the interval" of Section 4.2, Step 4).
inline double window_key(const Window& w, double L) {
    double px, py;
    pseudo_xy(w, L, px, py);
    double x = px < w.A ? w.A : (px > w.B ? w.B : px);
    return w.d + std::hypot(x - px, py);
}

struct Solver {
    Mesh& m;
    int flags;
    std::vector<double> g;          // geod_dist[]
    std::vector<double> aD, aX;     // angle_split[]: best distance to v2 and where its ray crosses e
    std::priority_queue<Entry, std::vector<Entry>, EntryCmp> pq;
    std::deque<Entry> fifo;
    uint64_t seq = 0, rng = 0x9E3779B97F4A7C15ull;
    long long created = 0, propagated = 0, peak = 0, events = 0;
    long long max_windows;
    // ORDER_BATCH: the pending pool and the current round's selection
    long long batch_k = 1;
    std::vector<Entry> pool, batch;
    size_t bpos = 0;
    long long rounds = 0;
    // TRACE: every window pushed, and per vertex the event that set its distance
    std::vector<Window> hist;
    std::vector<Event> prov;

    Solver(Mesh& mm, int fl, long long cap) : m(mm), flags(fl), max_windows(cap) {
        g.assign(m.nv, kInf);
        aD.assign(3 * m.nf, kInf);
        aX.assign(3 * m.nf, 0.0);
        if (flags & TRACE) prov.assign(m.nv, Event{-1, kInf});
    }

    size_t qsize() const {
        const int order = flags & ORDER_MASK;
        if (order == ORDER_BATCH) return pool.size() + (batch.size() - bpos);
        return order == ORDER_PQ ? pq.size() : fifo.size();
    }

    double cap = kInf;   // NO_ICH only: drop windows beyond every vertex's edge-path distance

    void push(const Window& w) {
        double L = m.len[w.e];
        Entry en{window_key(w, L), seq++, w};
        if (en.key > cap) return;
        if (flags & TRACE) {
            en.w.id = (int)hist.size();
            hist.push_back(en.w);
        }
        int order = flags & ORDER_MASK;
        if (order == ORDER_PQ) {
            pq.push(en);
        } else if (order == ORDER_BATCH) {
            pool.push_back(en);
        } else if (order == ORDER_FIFO) {
            fifo.push_back(en);
        } else {   // seeded random order: insert at the front or the back
            rng ^= rng << 13; rng ^= rng >> 7; rng ^= rng << 17;
            if (rng & 1) fifo.push_front(en); else fifo.push_back(en);
        }
        ++created;
        peak = std::max<long long>(peak, (long long)qsize());
    }

    bool pop(Entry& out) {
        if ((flags & ORDER_MASK) == ORDER_PQ) {
            if (pq.empty()) return false;
            out = pq.top(); pq.pop(); return true;
        }
        if ((flags & ORDER_MASK) == ORDER_BATCH) {
            // Section 6, "The PCH algorithm on the CPU": each round takes the k windows
            // nearest the source by quickselect, without ordering them, and propagates
            // them one by one; windows created meanwhile wait for the next round.
            if (bpos == batch.size()) {
                batch.clear();
                bpos = 0;
                if (pool.empty()) return false;
                if ((long long)pool.size() > batch_k) {
                    std::nth_element(pool.begin(), pool.begin() + batch_k, pool.end(),
                                     [](const Entry& a, const Entry& b) {
                                         return a.key != b.key ? a.key < b.key : a.seq < b.seq;
                                     });
                    batch.assign(pool.begin(), pool.begin() + batch_k);
                    pool.erase(pool.begin(), pool.begin() + batch_k);
                } else {
                    batch.swap(pool);
                }
                ++rounds;
            }
            out = batch[bpos++];
            return true;
        }
        if (fifo.empty()) return false;
        out = fifo.front(); fifo.pop_front(); return true;
    }
    double min_key() const {
        return (flags & ORDER_MASK) == ORDER_PQ ? (pq.empty() ? kInf : pq.top().key) : -kInf;
    }

    // Xin-Wang filter (Fig. `fig:filter`(b)) on a new window lying on half-edge c
    // (start cs, end ce) inside face (v0,v1,v2), with |IX| at its endpoints given.
    // `third`, `dA_third`, `dB_third`: the vertex of the parent's edge that is not on the
    // new edge and its in-face distances to the window's ends A and B.  The paper tests
    // the third inequality at the end nearer the vertex that the new edge shares with the
    // parent edge, where d + |I x| - |third x| takes its smallest value over the interval;
    // here the window is dropped only when both ends are dominated: the same decision in
    // exact arithmetic, and the safe one when rounding puts one end's test on the wrong
    // side of the margin.
    bool ich_useless(double d, double a, double b, double Lc, double IA, double IB, int cs, int ce,
                     int third, double dA_third, double dB_third) const {
        if (flags & NO_ICH) return false;
        if (dominated(d + IB, g[cs] + b)) return true;            // vs the start vertex, at B
        if (dominated(d + IA, g[ce] + (Lc - a))) return true;     // vs the end vertex, at A
        if (third >= 0 && dominated(d + IA, g[third] + dA_third) && dominated(d + IB, g[third] + dB_third))
            return true;                                          // vs the parent edge's far vertex
        return false;
    }

    // Pseudo-source fan at vertex v with distance D (Fig. `fig:propagation`(c)).  The
    // oracle creates a window on every edge opposite v (the whole one-ring): a superset
    // of the fanned area, sound because each window is a real path from the source.
    void fan(int v, double D, std::vector<Event>& work) {
        for (int hv : m.out_he[v]) {
            int o = nxt(hv);          // edge (a -> b) opposite v in face(hv)
            int a = hfrom(m, o), b = hto(m, o);
            double va = m.len[hv], vb = m.len[nxt(o)];
            int t = m.twin[o];
            if (t < 0) {              // boundary: no face beyond, emit the endpoint events
                work.push_back(Event{a, D + va, 1, -1, v});
                work.push_back(Event{b, D + vb, 1, -1, v});
                continue;
            }
            Window w{D, 0.0, m.len[t], vb, va, t};   // on twin (b -> a): d0 = |vb|, d1 = |va|
            w.src = v;
            // ICH filter on the new window: vs b at B (the a end), vs a at A (the b end);
            // the third vertex is v itself, i.e. the test reads D > g[v].
            if (ich_useless(D, 0.0, m.len[t], m.len[t], vb, va, b, a, v, vb, va)) continue;
            push(w);
        }
    }

    void vertex_event(int v, double D, const Window& from, std::vector<Event>& work) {
        work.push_back(Event{v, D, 0, from.id, from.src});
    }

    // Apply queued distance events in order; saddle / boundary vertices spawn fans.
    void drain(std::vector<Event>& work) {
        while (!work.empty()) {
            const Event ev = work.back();
            work.pop_back();
            ++events;
            if (ev.D < g[ev.v]) {
                g[ev.v] = ev.D;
                if (flags & TRACE) prov[ev.v] = ev;
                if (m.pseudo[ev.v]) fan(ev.v, ev.D, work);
            }
        }
    }

    // A child window keeps its parent's pseudo-source and remembers its parent.
    static Window child(Window c, const Window& parent) {
        c.src = parent.src;
        c.parent = parent.id;
        return c;
    }

    // Ray from I through (x, 0) meets the line through Q0 with unit direction u at
    // Q0 + t u; returns t (NaN when parallel).
    static double hit(double px, double py, double x, double q0x, double q0y, double ux, double uy) {
        double rx = x - px, ry = -py;
        double den = ux * ry - uy * rx;
        if (std::fabs(den) < 1e-300) return std::nan("");
        double ix = px - q0x, iy = py - q0y;
        return (ix * ry - iy * rx) / den;
    }

    void propagate(const Window& w) {
        const int h = w.e;
        const int v0 = hfrom(m, h), v1 = hto(m, h), v2 = m.tri[prv(h)];
        const double L = m.len[h];
        double xc, yc, px, py;
        apex_xy(m, h, xc, yc);
        pseudo_xy(w, L, px, py);
        const double tol = kEpsSnap * L;
        std::vector<Event> work;

        // Algorithm 2: A = v0 -> distance event (v0, d0 + d) (+ fan, applied in drain)
        if (w.A <= tol) vertex_event(v0, w.d + w.d0, w, work);
        // B = v1 -> distance event (v1, d1 + d)
        if (w.B >= L - tol) vertex_event(v1, w.d + w.d1, w, work);

        // Does w occupy v2?  Where the ray I -> v2 crosses e.
        double xs = px + (xc - px) * (-py) / (yc - py);
        bool occ = (xs >= w.A - tol) && (xs <= w.B + tol);
        double Iv2 = std::hypot(xc - px, yc - py);
        bool left = false, right = false;
        if (occ) {
            double D2 = w.d + Iv2;
            if (flags & NO_CH) {
                left = right = true;
            } else if (D2 < aD[h]) {          // w gives v2 a shorter distance: two children
                aD[h] = D2;
                aX[h] = xs;
                left = right = true;
            } else {
                // "One angle one split": a window that loses at v2 keeps only the child
                // on its own side of the winner's ray to v2 (the rays on the other side
                // cross the winner's path to v2 and are longer than a path along it).
                // Reading: compare where the two rays to v2 cross e; keep both if equal.
                if (xs < aX[h] - tol) left = true;
                else if (xs > aX[h] + tol) right = true;
                else left = right = true;
            }
            vertex_event(v2, D2, w, work);
        } else if (xs < w.A) {
            right = true;                      // v2 lies left of the window: one child on (v2,v1)
        } else {
            left = true;                       // one child on (v0,v2)
        }
        drain(work);   // events (and fans) before the new windows are filtered

        const double xcl = std::min(std::max(xs, w.A), w.B);
        // |IA|, |IB| for the child endpoint distances
        if (left) {
            // child on edge v0 -> v2, living on twin(prev(h)) whose start is v0
            int hp = prv(h);
            int c = m.twin[hp];
            if (c >= 0) {
                double Lc = m.len[c];
                double ux = xc / Lc, uy = yc / Lc;
                double ta = hit(px, py, w.A, 0.0, 0.0, ux, uy);
                double tb = occ ? Lc : hit(px, py, w.B, 0.0, 0.0, ux, uy);
                if (occ && xcl - w.A <= kEpsTiny * L) ta = tb;   // empty left part
                if (std::isfinite(ta) && std::isfinite(tb)) {
                    ta = std::min(std::max(ta, 0.0), Lc);
                    tb = std::min(std::max(tb, 0.0), Lc);
                    if (tb - ta > kEpsTiny * Lc) {
                        double IA = std::hypot(ta * ux - px, ta * uy - py);
                        double IB = std::hypot(tb * ux - px, tb * uy - py);
                        // third vertex: v1 (parent edge {v0,v1})
                        double v1A = std::hypot(ta * ux - L, ta * uy), v1B = std::hypot(tb * ux - L, tb * uy);
                        if (!ich_useless(w.d, ta, tb, Lc, IA, IB, v0, v2, v1, v1A, v1B))
                            push(child(Window{w.d, ta, tb, w.d0, Iv2, c}, w));
                    }
                }
            }
        }
        if (right) {
            // child on edge v2 -> v1, living on twin(next(h)) whose start is v2
            int hn = nxt(h);
            int c = m.twin[hn];
            if (c >= 0) {
                double Lc = m.len[c];
                double ux = (L - xc) / Lc, uy = -yc / Lc;
                double ta = occ ? 0.0 : hit(px, py, w.A, xc, yc, ux, uy);
                double tb = hit(px, py, w.B, xc, yc, ux, uy);
                if (occ && w.B - xcl <= kEpsTiny * L) tb = ta;
                if (std::isfinite(ta) && std::isfinite(tb)) {
                    ta = std::min(std::max(ta, 0.0), Lc);
                    tb = std::min(std::max(tb, 0.0), Lc);
                    if (tb - ta > kEpsTiny * Lc) {
                        double ax = xc + ta * ux, ay = yc + ta * uy;
                        double bx = xc + tb * ux, by = yc + tb * uy;
                        double IA = std::hypot(ax - px, ay - py);
                        double IB = std::hypot(bx - px, by - py);
                        // third vertex: v0 (parent edge {v0,v1})
                        double v0A = std::hypot(ax, ay), v0B = std::hypot(bx, by);
                        if (!ich_useless(w.d, ta, tb, Lc, IA, IB, v2, v1, v0, v0A, v0B))
                            push(child(Window{w.d, ta, tb, Iv2, w.d1, c}, w));
                    }
                }
            }
        }
    }

    // Lazy check at pop time: the two endpoint tests of the filter against the current
    // distances (both are sound for any window: d + |IX| - |v0 X| falls and
    // d + |IX| - |v1 X| rises along the edge).
    bool stale(const Window& w) const {
        if (flags & NO_ICH) return false;
        double L = m.len[w.e], px, py;
        pseudo_xy(w, L, px, py);
        double IA = std::hypot(w.A - px, py), IB = std::hypot(w.B - px, py);
        int v0 = hfrom(m, w.e), v1 = hto(m, w.e);
        return dominated(w.d + IB, g[v0] + w.B) || dominated(w.d + IA, g[v1] + (L - w.A));
    }

    // ---- geodesic paths (TRACE) ---------------------------------------------------
    // A path point: a vertex (kind 0, id = vertex), a point on half-edge id at fraction t0
    // from its start (kind 1), or the face-point source in face id with barycentric
    // weights t0, t1 of the face's corners 1 and 2 (kind 2).
    struct Pt {
        int kind, id;
        double t0, t1;
    };
    int sface = -1;
    double sbary[3] = {0, 0, 0};

    Pt face_point() const { return Pt{2, sface, sbary[1], sbary[2]}; }

    // The geodesic path from vertex t back to a source, target first.  Section 4.4: the
    // window sequence w_1 ... w_l that gave t its distance, w_l the window of t's final
    // event; Section 3: the path is a straight segment through the unfolded faces that
    // sequence crosses, from the pseudo-source to t, then the path to the pseudo-source.
    // Each segment is walked back along the window chain: the point where it meets a
    // window's edge, expressed in the parent window's frame (the child edge is the
    // parent face's edge v0 -> v2 or v2 -> v1), is joined to the parent's pseudo-source
    // and the line's crossing with the parent's edge is the previous point.
    // Returns false if the chain is broken (no recorded event, a child not on its
    // parent's face); an unreachable t gives an empty path.
    bool trace(int t, std::vector<Pt>& out) const {
        out.clear();
        if (!(g[t] < kInf)) return true;
        int v = t;
        out.push_back(Pt{0, v, 0.0, 0.0});
        for (size_t guard = 0; guard <= hist.size() + (size_t)m.nv; ++guard) {
            const Event& ev = prov[v];
            if (ev.kind < 0) return g[v] == 0.0;                 // reached a source
            if (ev.kind == 1) {                                  // along an edge from the fan vertex
                v = ev.src;
                out.push_back(Pt{0, v, 0.0, 0.0});
                continue;
            }
            if (ev.kind == 2) {                                  // straight to the face-point source
                out.push_back(face_point());
                return true;
            }
            const Window* w = &hist[ev.wid];
            const int h = w->e;
            const double L = m.len[h];
            double px, py;
            pseudo_xy(*w, L, px, py);
            double x;                                            // where the segment meets w's edge
            if (v == hfrom(m, h)) {
                x = 0.0;
            } else if (v == hto(m, h)) {
                x = L;
            } else {                                             // v2: the ray I -> v2 crosses the edge
                double xc, yc;
                apex_xy(m, h, xc, yc);
                x = std::min(std::max(px + (xc - px) * (-py) / (yc - py), 0.0), L);
                out.push_back(Pt{1, h, x / L, 0.0});
            }
            while (w->parent >= 0) {
                const Window& p = hist[w->parent];
                const int hp = p.e;
                const double Lp = m.len[hp];
                double xc, yc;
                apex_xy(m, hp, xc, yc);
                const double f = x / m.len[w->e];
                double qx, qy;
                if (w->e == m.twin[prv(hp)]) {                   // left child: edge v0 -> v2
                    qx = f * xc;
                    qy = f * yc;
                } else if (w->e == m.twin[nxt(hp)]) {            // right child: edge v2 -> v1
                    qx = xc + f * (Lp - xc);
                    qy = yc - f * yc;
                } else {
                    return false;
                }
                double ppx, ppy;
                pseudo_xy(p, Lp, ppx, ppy);
                x = std::min(std::max(ppx + (qx - ppx) * (-ppy) / (qy - ppy), 0.0), Lp);
                out.push_back(Pt{1, hp, x / Lp, 0.0});
                w = &p;
            }
            if (w->src < 0) {                                    // an initial window of the face point
                out.push_back(face_point());
                return true;
            }
            v = w->src;
            out.push_back(Pt{0, v, 0.0, 0.0});
        }
        return false;
    }

    int run(const int* targets, int n_targets) {
        Entry en;
        for (long long pops = 0;; ++pops) {
            // every 1024 windows (the scan costs n_targets): stop once the targets are
            // final (keys never decrease); stopping later only propagates more windows
            if (n_targets > 0 && (pops & 1023) == 0) {
                double gmax = 0;
                for (int i = 0; i < n_targets; ++i) gmax = std::max(gmax, g[targets[i]]);
                if (min_key() >= gmax) break;
            }
            if (!pop(en)) break;
            if (stale(en.w)) continue;
            ++propagated;
            propagate(en.w);
            if (created > max_windows) return -5;
        }
        return 0;
    }
};

}  // namespace

// Output buffers of oracle_trace_paths.
struct PathOut {
    int n_targets;
    const int* targets;
    int max_points;
    int* kinds;
    int* ids;
    double* t0;
    double* t1;
    int* n_points;
};

static int solve_field(int nv, const double* xyz, int nf, const int* tri, int src_kind, int src_vertex,
                       int src_face, const double* src_bary, int n_src, const int* srcs, int flags,
                       long long max_windows, int n_targets, const int* targets, double* out,
                       long long* stats, long long batch_k, const PathOut* paths = nullptr) {
    Mesh m;
    m.nv = nv; m.nf = nf; m.xyz = xyz; m.tri = tri;
    int rc = build_mesh(m);
    if (rc != 0) return rc;
    Solver s(m, flags, max_windows > 0 ? max_windows : (1LL << 40));
    s.batch_k = batch_k > 0 ? batch_k : 1;
    std::vector<Event> work;
    if (src_kind == 0 || src_kind == 2) {
        // Algorithm 1: geod_dist = 0 at the sources; a window on every edge opposite them.
        int count = src_kind == 0 ? 1 : n_src;
        for (int i = 0; i < count; ++i) {
            int sv = src_kind == 0 ? src_vertex : srcs[i];
            if (sv < 0 || sv >= nv) return -1;
            s.g[sv] = 0.0;
        }
        for (int i = 0; i < count; ++i) {
            int sv = src_kind == 0 ? src_vertex : srcs[i];
            s.fan(sv, 0.0, work);
        }
        s.drain(work);
    } else if (src_kind == 1) {
        // Face-point source: windows on the three edges of its face (reading of the
        // source-point case; Algorithm 1 requires s in V).
        if (src_face < 0 || src_face >= nf) return -1;
        double p[3] = {0, 0, 0};
        for (int k = 0; k < 3; ++k)
            for (int c = 0; c < 3; ++c) p[c] += src_bary[k] * xyz[3 * tri[3 * src_face + k] + c];
        auto dp = [&](int v) {
            double dx = p[0] - xyz[3 * v], dy = p[1] - xyz[3 * v + 1], dz = p[2] - xyz[3 * v + 2];
            return std::sqrt(dx * dx + dy * dy + dz * dz);
        };
        s.sface = src_face;
        for (int k = 0; k < 3; ++k) s.sbary[k] = src_bary[k];
        for (int k = 0; k < 3; ++k) {
            int h = 3 * src_face + k;
            int a = hfrom(m, h), b = hto(m, h);
            work.push_back(Event{a, dp(a), 2, -1, -1});
            int t = m.twin[h];
            if (t >= 0) s.push(Window{0.0, 0.0, m.len[t], dp(b), dp(a), t});
        }
        s.drain(work);
    } else {
        return -1;
    }
    if (flags & NO_ICH) {
        // With the filter off nothing else retires circulating beams; a window whose key
        // exceeds the largest edge-path distance from the sources can improve no vertex.
        std::vector<double> dj(nv, kInf);
        std::priority_queue<std::pair<double, int>, std::vector<std::pair<double, int>>,
                            std::greater<std::pair<double, int>>> q;
        for (int v = 0; v < nv; ++v)
            if (s.g[v] < kInf) { dj[v] = s.g[v]; q.push({dj[v], v}); }
        while (!q.empty()) {
            auto [dd, u] = q.top(); q.pop();
            if (dd > dj[u]) continue;
            for (int h : m.out_he[u]) {
                int w2 = hto(m, h);
                if (dd + m.len[h] < dj[w2]) { dj[w2] = dd + m.len[h]; q.push({dj[w2], w2}); }
                int w3 = m.tri[prv(h)];
                if (dd + m.len[prv(h)] < dj[w3]) { dj[w3] = dd + m.len[prv(h)]; q.push({dj[w3], w3}); }
            }
        }
        double mx = 0;
        for (int v = 0; v < nv; ++v) if (dj[v] < kInf) mx = std::max(mx, dj[v]);
        s.cap = mx * (1 + 1e-9);
    }
    rc = s.run(targets, n_targets);
    for (int v = 0; v < nv; ++v) out[v] = s.g[v];
    if (rc == 0 && paths) {
        std::vector<Solver::Pt> pts;
        for (int i = 0; i < paths->n_targets; ++i) {
            const int t = paths->targets[i];
            if (t < 0 || t >= nv) return -1;
            if (!s.trace(t, pts)) {
                paths->n_points[i] = -1;
                continue;
            }
            paths->n_points[i] = (int)pts.size();
            const size_t base = (size_t)i * paths->max_points;
            for (size_t j = 0; j < pts.size() && (int)j < paths->max_points; ++j) {
                paths->kinds[base + j] = pts[j].kind;
                paths->ids[base + j] = pts[j].id;
                paths->t0[base + j] = pts[j].t0;
                paths->t1[base + j] = pts[j].t1;
            }
        }
    }
    if (stats) {
        stats[0] = s.created; stats[1] = s.propagated; stats[2] = s.peak; stats[3] = s.events;
        stats[4] = s.rounds;
    }
    return rc;
}

extern "C" {

// Exact geodesic distance from one source to every vertex.
//  src_kind 0: vertex source `src_vertex`; 1: point in face `src_face` with barycentric
//  `src_bary[3]`; 2: `n_src` vertex sources `srcs` (distance to the nearest one,
//  Section 4.2's source set S).
//  flags: ORDER_* | NO_CH | NO_ICH (ORDER_BATCH takes one window per round here; see
//  oracle_cpu_pch).  targets/n_targets: stop once those vertices are final (other
//  entries of out are then upper bounds; the priority-queue order only).
//  stats[0..4] = windows created, windows propagated, peak queue, distance events, rounds.
// Returns 0, or <0 on invalid / non-manifold / degenerate input or window cap exceeded.
int oracle_geodesic(int nv, const double* xyz, int nf, const int* tri, int src_kind, int src_vertex,
                    int src_face, const double* src_bary, int n_src, const int* srcs, int flags,
                    long long max_windows, int n_targets, const int* targets, double* out,
                    long long* stats) {
    return solve_field(nv, xyz, nf, tri, src_kind, src_vertex, src_face, src_bary, n_src, srcs, flags,
                       max_windows, n_targets, targets, out, stats, 1);
}

// The CPU PCH algorithm of Section 6: the same propagation with the selection of
// Algorithm 1 done sequentially, k windows a round (quickselect, not ordered), events
// applied as they arise (sequential code has no conflicting writers).  flags: NO_CH |
// NO_ICH; the order is ORDER_BATCH.  Same outputs and stats as oracle_geodesic.
int oracle_cpu_pch(int nv, const double* xyz, int nf, const int* tri, int src_vertex, long long k, int flags,
                   double* out, long long* stats) {
    if (k < 1) return -1;
    return solve_field(nv, xyz, nf, tri, 0, src_vertex, 0, nullptr, 0, nullptr,
                       (flags & ~ORDER_MASK) | ORDER_BATCH, 0, 0, nullptr, out, stats, k);
}

// Geodesic paths from the source(s) to `targets` (priority-queue order, TRACE on).
// Source arguments as oracle_geodesic.  For target i, n_points[i] points (target first,
// the source last; at most max_points stored from i * max_points on) of kinds[]: 0 vertex
// ids[], 1 point on half-edge ids[] at fraction t0[] from its start, 2 the face-point
// source in face ids[] with barycentric weights t0[], t1[] of corners 1 and 2;
// n_points[i] = 0 for an unreachable target, -1 if its window chain was broken.
// out receives the distance field.  Returns 0, or <0 as oracle_geodesic.
int oracle_trace_paths(int nv, const double* xyz, int nf, const int* tri, int src_kind, int src_vertex,
                       int src_face, const double* src_bary, int n_src, const int* srcs, int n_targets,
                       const int* targets, int max_points, int* kinds, int* ids, double* t0, double* t1,
                       int* n_points, double* out) {
    if (n_targets < 0 || max_points < 0) return -1;
    PathOut po{n_targets, targets, max_points, kinds, ids, t0, t1, n_points};
    return solve_field(nv, xyz, nf, tri, src_kind, src_vertex, src_face, src_bary, n_src, srcs, ORDER_PQ | TRACE,
                       0, 0, nullptr, out, nullptr, 1, &po);
}

// Total angle at every vertex and the pseudo-source flag the oracle uses (for tests).
int oracle_vertex_angles(int nv, const double* xyz, int nf, const int* tri, double* theta_out,
                         unsigned char* pseudo_out) {
    Mesh m;
    m.nv = nv; m.nf = nf; m.xyz = xyz; m.tri = tri;
    int rc = build_mesh(m);
    if (rc != 0) return rc;
    std::vector<double> th(nv, 0.0);
    for (int h = 0; h < 3 * nf; ++h) {
        double a = m.len[h], b = m.len[prv(h)], c = m.len[nxt(h)];
        double cs = std::max(-1.0, std::min(1.0, (a * a + b * b - c * c) / (2 * a * b)));
        th[hfrom(m, h)] += std::acos(cs);
    }
    for (int v = 0; v < nv; ++v) { theta_out[v] = th[v]; pseudo_out[v] = (unsigned char)m.pseudo[v]; }
    return 0;
}

}  // extern "C"
