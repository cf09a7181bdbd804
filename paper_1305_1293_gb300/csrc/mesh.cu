// Mesh preparation on the device (Section 4.1): half-edge table, edge lengths,
// per-half-edge unfolding frames, one-ring order, total angles and the saddle /
// boundary classification of Section 3.  Entry points pch_create_mesh, pch_mesh_info,
// pch_destroy, pch_last_error.
#include <cmath>
#include <cstring>
#include <mutex>
#include <string>
#include <vector>

#include "pch_host.h"

namespace pch {

static thread_local std::string g_err;

pch_status set_error(pch_status st, const char* fmt, ...) {
    char buf[512];
    va_list ap;
    va_start(ap, fmt);
    vsnprintf(buf, sizeof buf, fmt, ap);
    va_end(ap);
    g_err = buf;
    return st;
}
void clear_error() { g_err.clear(); }

int sm_count() {
    static int cached = -1;
    static int cached_dev = -1;
    int dev = 0;
    cudaGetDevice(&dev);
    if (cached < 0 || dev != cached_dev) {
        cudaDeviceGetAttribute(&cached, cudaDevAttrMultiProcessorCount, dev);
        cached_dev = dev;
    }
    return cached;
}

// The driver's cuCtxGetCurrent / cuCtxGetId, reached through the runtime so that the
// library does not link libcuda (it must load on a machine without a GPU driver).
typedef int (*CtxGetCurrentFn)(void**);
typedef int (*CtxGetIdFn)(void*, unsigned long long*);

unsigned long long current_context_id() {
    static CtxGetCurrentFn get_current = nullptr;
    static CtxGetIdFn get_id = nullptr;
    static std::once_flag once;
    std::call_once(once, [] {
        void* f = nullptr;
        cudaDriverEntryPointQueryResult q = cudaDriverEntryPointSymbolNotFound;
        if (cudaGetDriverEntryPointByVersion("cuCtxGetCurrent", &f, 12000, cudaEnableDefault, &q) == cudaSuccess &&
            q == cudaDriverEntryPointSuccess)
            get_current = reinterpret_cast<CtxGetCurrentFn>(f);
        f = nullptr;
        if (cudaGetDriverEntryPointByVersion("cuCtxGetId", &f, 12000, cudaEnableDefault, &q) == cudaSuccess &&
            q == cudaDriverEntryPointSuccess)
            get_id = reinterpret_cast<CtxGetIdFn>(f);
    });
    if (!get_current || !get_id) return 0;
    void* ctx = nullptr;
    if (get_current(&ctx) != 0 || !ctx) return 0;
    unsigned long long id = 0;
    return get_id(ctx, &id) == 0 ? id : 0;
}

// ---------------------------------------------------------------- exclusive scan
constexpr int kScanBlock = 1024;

__global__ void k_scan_block(const int* in, int* out, int n, int* block_sums) {
    __shared__ int sh[kScanBlock];
    int i = blockIdx.x * kScanBlock + threadIdx.x;
    int x = i < n ? in[i] : 0;
    sh[threadIdx.x] = x;
    __syncthreads();
    for (int off = 1; off < kScanBlock; off <<= 1) {
        int t = threadIdx.x >= off ? sh[threadIdx.x - off] : 0;
        __syncthreads();
        sh[threadIdx.x] += t;
        __syncthreads();
    }
    if (i < n) out[i] = sh[threadIdx.x] - x;
    if (threadIdx.x == kScanBlock - 1) block_sums[blockIdx.x] = sh[threadIdx.x];
}

__global__ void k_scan_sums(int* sums, int nb) {
    // single block: sequential chunks, deterministic
    __shared__ int carry;
    if (threadIdx.x == 0) carry = 0;
    __syncthreads();
    __shared__ int sh[kScanBlock];
    for (int base = 0; base < nb; base += kScanBlock) {
        int i = base + threadIdx.x;
        int x = i < nb ? sums[i] : 0;
        sh[threadIdx.x] = x;
        __syncthreads();
        for (int off = 1; off < kScanBlock; off <<= 1) {
            int t = threadIdx.x >= off ? sh[threadIdx.x - off] : 0;
            __syncthreads();
            sh[threadIdx.x] += t;
            __syncthreads();
        }
        if (i < nb) sums[i] = carry + sh[threadIdx.x] - x;
        __syncthreads();
        if (threadIdx.x == kScanBlock - 1) carry += sh[threadIdx.x];
        __syncthreads();
    }
}

__global__ void k_scan_add(int* out, int n, const int* sums) {
    int i = blockIdx.x * kScanBlock + threadIdx.x;
    if (i < n) out[i] += sums[blockIdx.x];
}

size_t scan_tmp_ints(int n) { return (size_t)(n + kScanBlock - 1) / kScanBlock + 1; }

cudaError_t exclusive_scan(const int* in, int* out, int n, int* tmp, cudaStream_t s) {
    if (n <= 0) return cudaSuccess;
    int nb = (n + kScanBlock - 1) / kScanBlock;
    k_scan_block<<<nb, kScanBlock, 0, s>>>(in, out, n, tmp);
    k_scan_sums<<<1, kScanBlock, 0, s>>>(tmp, nb);
    k_scan_add<<<nb, kScanBlock, 0, s>>>(out, n, tmp);
    return cudaGetLastError();
}

// ---------------------------------------------------------------- mesh kernels
enum : int { kMeshErrDegenerate = 1, kMeshErrDup = 2, kMeshErrFan = 4, kMeshErrProbe = 8 };

__device__ __forceinline__ int he_next(int h) { return 3 * (h / 3) + (h % 3 + 1) % 3; }
__device__ __forceinline__ int he_prev(int h) { return 3 * (h / 3) + (h % 3 + 2) % 3; }

__device__ __forceinline__ double dist3(const double* x, int a, int b) {
    double dx = x[3 * a] - x[3 * b], dy = x[3 * a + 1] - x[3 * b + 1], dz = x[3 * a + 2] - x[3 * b + 2];
    return sqrt(dx * dx + dy * dy + dz * dz);
}

// Edge lengths and the apex frame of every half-edge (the metric is all the method
// needs, Section 4.1).
__global__ void k_frames(int nh, const double* __restrict__ xyz, const int* __restrict__ tri, HERec* rec,
                         double* hang, int* err) {
    for (int h = blockIdx.x * blockDim.x + threadIdx.x; h < nh; h += gridDim.x * blockDim.x) {
        int a = tri[h], b = tri[he_next(h)], c = tri[he_prev(h)];
        double L = dist3(xyz, a, b), L1 = dist3(xyz, b, c), L2 = dist3(xyz, c, a);
        double xc = ((L2 - L1) * (L2 + L1) + L * L) / (2.0 * L);
        double t = (L2 - xc) * (L2 + xc);
        double yc = sqrt(t > 0.0 ? t : 0.0);
        HERec r;
        r.L = L; r.xc = xc; r.yc = yc; r.L1 = L1; r.L2 = L2;
        r.u1x = (L - xc) / L1; r.u1y = -yc / L1; r.u2x = xc / L2; r.u2y = yc / L2;
        r.tw1 = r.tw2 = r.twin = -1;
        r.v0 = a; r.v1 = b; r.v2 = c;
        rec[h] = r;
        hang[h] = atan2(yc, xc);
        if (a == b || b == c || c == a || !(yc > 1e-12 * L) || !(L > 1e-250)) atomicOr(err, kMeshErrDegenerate);
    }
}

__device__ __forceinline__ unsigned long long mix64(unsigned long long z) {
    z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
    z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
    return z ^ (z >> 31);
}

__global__ void k_hash_insert(int nh, const int* __restrict__ tri, unsigned long long* keys, int* vals,
                              unsigned long long mask, int* err) {
    for (int h = blockIdx.x * blockDim.x + threadIdx.x; h < nh; h += gridDim.x * blockDim.x) {
        unsigned long long k = (unsigned long long)(unsigned)tri[h] << 32 | (unsigned)tri[he_next(h)];
        unsigned long long s = mix64(k) & mask;
        for (unsigned long long probe = 0; probe <= mask; ++probe) {
            unsigned long long prev = atomicCAS(&keys[s], ~0ull, k);
            if (prev == ~0ull) { vals[s] = h; break; }
            if (prev == k) { atomicOr(err, kMeshErrDup); break; }
            s = (s + 1) & mask;
            if (probe == mask) atomicOr(err, kMeshErrProbe);
        }
    }
}

__global__ void k_twins(int nh, const int* __restrict__ tri, const unsigned long long* keys, const int* vals,
                        unsigned long long mask, int* twin, int* vcount, int* vout) {
    for (int h = blockIdx.x * blockDim.x + threadIdx.x; h < nh; h += gridDim.x * blockDim.x) {
        int a = tri[h], b = tri[he_next(h)];
        unsigned long long k = (unsigned long long)(unsigned)b << 32 | (unsigned)a;
        unsigned long long s = mix64(k) & mask;
        int t = -1;
        for (unsigned long long probe = 0; probe <= mask; ++probe) {
            unsigned long long kk = keys[s];
            if (kk == k) { t = vals[s]; break; }
            if (kk == ~0ull) break;
            s = (s + 1) & mask;
        }
        twin[h] = t;
        atomicAdd(&vcount[a], 1);
        atomicMin(&vout[a], h);
    }
}

// One thread per vertex: walk its one-ring (clockwise to a boundary, then
// counter-clockwise), record the ring order, angular positions and total angle.
__global__ void k_rings(int nv, const int* __restrict__ twin, const int* __restrict__ vout,
                        const int* __restrict__ vstart, const double* __restrict__ hang, int* vlist,
                        float* vphi, float* vtheta, float* hang_f, double2* vrot, double2* vtrot,
                        unsigned char* vflag, int* err) {
    const double kTwoPi = 6.283185307179586476925286766559;
    for (int v = blockIdx.x * blockDim.x + threadIdx.x; v < nv; v += gridDim.x * blockDim.x) {
        int cnt = vstart[v + 1] - vstart[v];
        if (cnt == 0) { vtheta[v] = 0; vtrot[v] = make_double2(1.0, 0.0); vflag[v] = 0; continue; }
        int h0 = vout[v];
        int start = h0;
        bool boundary = false;
        for (int s = 0; s <= cnt; ++s) {   // clockwise: h -> next(twin(h))
            int t = twin[start];
            if (t < 0) { boundary = true; break; }
            int hn = he_next(t);
            if (hn == h0) break;
            start = hn;
        }
        if (!boundary) start = h0;
        int h = start, k = 0;
        double phi = 0.0;
        while (k < cnt) {
            vlist[vstart[v] + k] = h;
            vphi[h] = (float)phi;
            hang_f[h] = (float)hang[h];
            double sp, cp;
            sincos(phi, &sp, &cp);
            vrot[h] = make_double2(cp, sp);
            phi += hang[h];
            ++k;
            int t = twin[he_prev(h)];           // counter-clockwise: h -> twin(prev(h))
            if (t < 0 || t == start) break;
            h = t;
        }
        if (k != cnt) atomicOr(err, kMeshErrFan);
        vtheta[v] = (float)phi;
        {
            double sp, cp;
            sincos(phi, &sp, &cp);
            vtrot[v] = make_double2(cp, sp);
        }
        unsigned char f = boundary ? 1 : 0;
        // Saddle (total angle above 2 pi, Section 3) or boundary vertex: a pseudo-source
        // candidate.  The 1e-9 band keeps flat vertices in the candidate set (superset).
        if (boundary || phi > kTwoPi - 1e-9) f |= 2;
        vflag[v] = f;
    }
}

__global__ void k_rec_ids(int nh, const int* __restrict__ twin, const unsigned char* __restrict__ vflag, HERec* rec) {
    for (int h = blockIdx.x * blockDim.x + threadIdx.x; h < nh; h += gridDim.x * blockDim.x) {
        HERec r = rec[h];
        r.twin = twin[h];
        r.tw1 = twin[he_next(h)];
        r.tw2 = twin[he_prev(h)];
        r.v0 |= (vflag[r.v0] & 2) ? kPseudoBit : 0u;
        r.v1 |= (vflag[r.v1] & 2) ? kPseudoBit : 0u;
        r.v2 |= (vflag[r.v2] & 2) ? kPseudoBit : 0u;
        rec[h] = r;
    }
}

// Deterministic mean edge length and counts: block b reduces a fixed contiguous range of
// half-edges and vertices in a fixed order, then k_stats_final adds the kStatBlocks
// partial results in a fixed tree, so the sum does not depend on scheduling.
constexpr int kStatBlocks = 256;

__device__ __forceinline__ void block_sum3(double& s, int& a, int& b) {
    __shared__ double sh[256];
    __shared__ int sa[256], sb[256];
    sh[threadIdx.x] = s; sa[threadIdx.x] = a; sb[threadIdx.x] = b;
    __syncthreads();
    for (int off = 128; off > 0; off >>= 1) {
        if (threadIdx.x < off) {
            sh[threadIdx.x] += sh[threadIdx.x + off];
            sa[threadIdx.x] += sa[threadIdx.x + off];
            sb[threadIdx.x] += sb[threadIdx.x + off];
        }
        __syncthreads();
    }
    s = sh[0]; a = sa[0]; b = sb[0];
}

__global__ void __launch_bounds__(256) k_stats(int nh, int nv, const HERec* rec, const int* twin,
                                               const unsigned char* vflag, double* part_l, int* part_c) {
    const long long h0 = (long long)nh * blockIdx.x / gridDim.x, h1 = (long long)nh * (blockIdx.x + 1) / gridDim.x;
    const long long v0 = (long long)nv * blockIdx.x / gridDim.x, v1 = (long long)nv * (blockIdx.x + 1) / gridDim.x;
    double s = 0.0;
    int nb = 0, np = 0;
    for (long long h = h0 + threadIdx.x; h < h1; h += blockDim.x) {
        s += rec[h].L;
        nb += twin[h] < 0;
    }
    for (long long v = v0 + threadIdx.x; v < v1; v += blockDim.x) np += (vflag[v] & 2) ? 1 : 0;
    block_sum3(s, nb, np);
    if (threadIdx.x == 0) { part_l[blockIdx.x] = s; part_c[2 * blockIdx.x] = nb; part_c[2 * blockIdx.x + 1] = np; }
}

__global__ void __launch_bounds__(256) k_stats_final(const double* part_l, const int* part_c, double* out_lsum,
                                                     int* out_counts) {
    double s = part_l[threadIdx.x];
    int nb = part_c[2 * threadIdx.x], np = part_c[2 * threadIdx.x + 1];
    block_sum3(s, nb, np);
    if (threadIdx.x == 0) { *out_lsum = s; out_counts[0] = nb; out_counts[1] = np; }
}

static void free_mesh(DevMesh& d) {
    cudaFree(d.rec); cudaFree(d.vstart); cudaFree(d.vlist); cudaFree(d.hang);
    cudaFree(d.vtheta); cudaFree(d.vphi); cudaFree(d.vflag); cudaFree(d.vrot); cudaFree(d.vtrot);
    d = DevMesh{};
}

void destroy_workspace(Workspace* w);   // solver.cu

}  // namespace pch

using namespace pch;

extern "C" const char* pch_last_error(void) { return pch::g_err.c_str(); }

extern "C" pch_status pch_create_mesh(const double* vertices, int32_t n_vertices, const int32_t* faces,
                                      int32_t n_faces, pch_mesh** out) {
    clear_error();
    if (!vertices || !faces || !out) return set_error(PCH_ERR_INVALID_ARG, "null pointer argument");
    if (n_vertices < 3 || n_faces < 1) return set_error(PCH_ERR_INVALID_ARG, "need >= 3 vertices and >= 1 face");
    if ((long long)n_faces * 3 >= (1LL << 31) - 1) return set_error(PCH_ERR_CAPACITY, "too many faces");
    for (long long i = 0; i < 3LL * n_vertices; ++i)
        if (!std::isfinite(vertices[i])) return set_error(PCH_ERR_INVALID_ARG, "non-finite coordinate at vertex %lld", i / 3);
    for (long long i = 0; i < 3LL * n_faces; ++i)
        if (faces[i] < 0 || faces[i] >= n_vertices)
            return set_error(PCH_ERR_INVALID_ARG, "face %lld references vertex %d out of range", i / 3, faces[i]);

    const int nv = n_vertices, nf = n_faces, nh = 3 * n_faces;
    DevMesh d{};
    d.nv = nv; d.nf = nf; d.nh = nh;
    double* xyz = nullptr;
    int *tri = nullptr, *twin = nullptr, *vcount = nullptr, *vout = nullptr, *err = nullptr, *scan_tmp = nullptr,
        *hvals = nullptr, *counts = nullptr;
    unsigned long long* hkeys = nullptr;
    double* lsum = nullptr;
    double* hang64 = nullptr;
    unsigned long long cap = 1;
    while (cap < 2ull * (unsigned long long)nh) cap <<= 1;
    pch_status st = PCH_OK;
    int herr = 0;
    double hl = 0.0;
    int hc[2] = {0, 0};
    auto fail = [&](pch_status s) { st = s; };
#define MCHK(call)                                                                              \
    do {                                                                                        \
        cudaError_t e_ = (call);                                                                \
        if (e_ != cudaSuccess) {                                                                \
            fail(set_error(e_ == cudaErrorMemoryAllocation ? PCH_ERR_OOM : PCH_ERR_CUDA, "%s: %s", #call, \
                           cudaGetErrorString(e_)));                                            \
            goto cleanup;                                                                       \
        }                                                                                       \
    } while (0)
    {
        MCHK(cudaMalloc(&xyz, sizeof(double) * 3 * nv));
        MCHK(cudaMalloc(&tri, sizeof(int) * nh));
        MCHK(cudaMalloc(&d.rec, sizeof(HERec) * nh));
        MCHK(cudaMalloc(&hang64, sizeof(double) * nh));
        MCHK(cudaMalloc(&d.hang, sizeof(float) * nh));
        MCHK(cudaMalloc(&d.vphi, sizeof(float) * nh));
        MCHK(cudaMalloc(&d.vlist, sizeof(int) * nh));
        MCHK(cudaMalloc(&d.vstart, sizeof(int) * (nv + 1)));
        MCHK(cudaMalloc(&d.vtheta, sizeof(float) * nv));
        MCHK(cudaMalloc(&d.vrot, sizeof(double2) * nh));
        MCHK(cudaMalloc(&d.vtrot, sizeof(double2) * nv));
        MCHK(cudaMalloc(&d.vflag, nv));
        MCHK(cudaMalloc(&twin, sizeof(int) * nh));
        MCHK(cudaMalloc(&vcount, sizeof(int) * (nv + 1)));
        MCHK(cudaMalloc(&vout, sizeof(int) * nv));
        MCHK(cudaMalloc(&err, sizeof(int)));
        MCHK(cudaMalloc(&counts, sizeof(int) * (2 + 2 * kStatBlocks)));
        MCHK(cudaMalloc(&lsum, sizeof(double) * (1 + kStatBlocks)));
        MCHK(cudaMalloc(&scan_tmp, sizeof(int) * scan_tmp_ints(nv + 1)));
        MCHK(cudaMalloc(&hkeys, sizeof(unsigned long long) * cap));
        MCHK(cudaMalloc(&hvals, sizeof(int) * cap));
        MCHK(cudaMemcpy(xyz, vertices, sizeof(double) * 3 * nv, cudaMemcpyHostToDevice));
        MCHK(cudaMemcpy(tri, faces, sizeof(int) * nh, cudaMemcpyHostToDevice));
        MCHK(cudaMemset(err, 0, sizeof(int)));
        MCHK(cudaMemset(vcount, 0, sizeof(int) * (nv + 1)));
        MCHK(cudaMemset(vout, 0x7f, sizeof(int) * nv));
        MCHK(cudaMemset(hkeys, 0xff, sizeof(unsigned long long) * cap));
        const int tb = 256;
        const int gb = std::max(1, std::min((nh + tb - 1) / tb, sm_count() * 8));
        const int gv = std::max(1, std::min((nv + tb - 1) / tb, sm_count() * 8));
        k_frames<<<gb, tb>>>(nh, xyz, tri, d.rec, hang64, err);
        k_hash_insert<<<gb, tb>>>(nh, tri, hkeys, hvals, cap - 1, err);
        k_twins<<<gb, tb>>>(nh, tri, hkeys, hvals, cap - 1, twin, vcount, vout);
        MCHK(cudaGetLastError());
        MCHK(exclusive_scan(vcount, d.vstart, nv + 1, scan_tmp, 0));
        k_rings<<<gv, tb>>>(nv, twin, vout, d.vstart, hang64, d.vlist, d.vphi, d.vtheta, d.hang, d.vrot, d.vtrot,
                            d.vflag, err);
        k_rec_ids<<<gb, tb>>>(nh, twin, d.vflag, d.rec);
        k_stats<<<kStatBlocks, 256>>>(nh, nv, d.rec, twin, d.vflag, lsum + 1, counts + 2);
        k_stats_final<<<1, kStatBlocks>>>(lsum + 1, counts + 2, lsum, counts);
        MCHK(cudaGetLastError());
        MCHK(cudaMemcpy(&herr, err, sizeof(int), cudaMemcpyDeviceToHost));
        MCHK(cudaMemcpy(&hl, lsum, sizeof(double), cudaMemcpyDeviceToHost));
        MCHK(cudaMemcpy(hc, counts, sizeof(int) * 2, cudaMemcpyDeviceToHost));
        if (herr & kMeshErrDup) { fail(set_error(PCH_ERR_NONMANIFOLD, "an oriented edge appears in two faces (non-manifold or inconsistent orientation)")); goto cleanup; }
        if (herr & kMeshErrDegenerate) { fail(set_error(PCH_ERR_DEGENERATE, "a face has a repeated vertex or (near) zero area")); goto cleanup; }
        if (herr & kMeshErrFan) { fail(set_error(PCH_ERR_NONMANIFOLD, "a vertex whose faces do not form a single fan")); goto cleanup; }
        if (herr & kMeshErrProbe) { fail(set_error(PCH_ERR_CUDA, "edge hash table overflow")); goto cleanup; }
        d.lbar = hl / nh;
        pch_mesh* m = new pch_mesh();
        m->dm = d;
        cudaGetDevice(&m->device);
        m->n_boundary_he = hc[0];
        m->n_pseudo = hc[1];
        m->ws = nullptr;
        *out = m;
    }
cleanup:
#undef MCHK
    cudaFree(xyz); cudaFree(tri); cudaFree(twin); cudaFree(vcount); cudaFree(vout); cudaFree(err);
    cudaFree(scan_tmp); cudaFree(hkeys); cudaFree(hvals); cudaFree(counts); cudaFree(lsum); cudaFree(hang64);
    if (st != PCH_OK) free_mesh(d);
    return st;
}

extern "C" pch_status pch_mesh_info(const pch_mesh* m, int32_t* n_vertices, int32_t* n_faces,
                                    int32_t* n_boundary_half_edges, int32_t* n_pseudo_vertices) {
    if (!m) return set_error(PCH_ERR_INVALID_ARG, "null mesh");
    if (n_vertices) *n_vertices = m->dm.nv;
    if (n_faces) *n_faces = m->dm.nf;
    if (n_boundary_half_edges) *n_boundary_half_edges = m->n_boundary_he;
    if (n_pseudo_vertices) *n_pseudo_vertices = m->n_pseudo;
    return PCH_OK;
}

extern "C" void pch_destroy(pch_mesh* m) {
    if (!m) return;
    int cur = 0;
    cudaGetDevice(&cur);
    cudaSetDevice(m->device);
    if (m->ws) destroy_workspace(m->ws);
    free_mesh(m->dm);
    cudaSetDevice(cur);
    delete m;
}
