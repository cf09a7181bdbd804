// Iso-contours of a distance field on the mesh (the iso-contours of the exact geodesic
// field that Section 2 cites as a use of exact distances, built from the field PCH
// computes).  On each face the field is taken as the linear interpolation of its three
// vertex distances; the contour at level L then crosses every edge whose ends lie on
// different sides of L (a vertex is inside when its distance is below L) at the
// interpolated point, and is one straight segment per crossed face and level.
// Entry point pch_iso_contours.
#include <algorithm>
#include <climits>
#include <cmath>
#include <vector>

#include "pch_host.h"

namespace pch {

__device__ __forceinline__ bool finite_d(double x) { return x <= 1.7976931348623157e308; }

// Crossing mask of face f at level L: bit i set when half-edge 3f+i (corner i -> corner
// i+1) has its ends on different sides.  A face with a non-finite distance has none.
__device__ __forceinline__ int face_mask(const double d[3], double L) {
    if (!(finite_d(d[0]) && finite_d(d[1]) && finite_d(d[2]))) return 0;
    int m = 0;
#pragma unroll
    for (int i = 0; i < 3; ++i)
        if ((d[i] < L) != (d[(i + 1) % 3] < L)) m |= 1 << i;
    return m;
}

__device__ __forceinline__ void face_dist(const HERec* __restrict__ rec, const double* __restrict__ dist, int f,
                                          double d[3]) {
#pragma unroll
    for (int i = 0; i < 3; ++i) d[i] = dist[rec[3 * f + i].v0 & ~kPseudoBit];
}

__global__ void k_contour_count(const HERec* __restrict__ rec, int nf, const double* __restrict__ dist,
                                const double* __restrict__ levels, int n_levels, int* count,
                                unsigned long long* total) {
    unsigned long long t = 0;
    for (int f = blockIdx.x * blockDim.x + threadIdx.x; f < nf; f += gridDim.x * blockDim.x) {
        double d[3];
        face_dist(rec, dist, f, d);
        int c = 0;
        for (int l = 0; l < n_levels; ++l) c += face_mask(d, levels[l]) != 0;
        count[f] = c;
        t += (unsigned long long)c;
    }
    if (t) atomicAdd(total, t);
}

// Segment endpoints: from the crossing on the edge whose start corner is inside to the
// crossing on the edge whose start corner is outside, so that the inside (distance
// below L) lies to the left of the segment seen from the face's front side (corners
// counter-clockwise).
__global__ void k_contour_write(const HERec* __restrict__ rec, int nf, const double* __restrict__ dist,
                                const double* __restrict__ levels, int n_levels, const int* __restrict__ offset,
                                long long capacity, pch_contour_segment* __restrict__ out) {
    for (int f = blockIdx.x * blockDim.x + threadIdx.x; f < nf; f += gridDim.x * blockDim.x) {
        double d[3];
        face_dist(rec, dist, f, d);
        long long o = offset[f];
        for (int l = 0; l < n_levels; ++l) {
            const double L = levels[l];
            const int m = face_mask(d, L);
            if (!m) continue;
            if (o < capacity) {
                pch_contour_segment sgm;
                sgm.level = l;
                sgm.face = f;
                int k = 0;
                // first the edge leaving the inside, then the edge entering it
                for (int pass = 0; pass < 2; ++pass)
                    for (int i = 0; i < 3; ++i) {
                        if (!(m >> i & 1)) continue;
                        const bool start_inside = d[i] < L;
                        if (start_inside != (pass == 0)) continue;
                        const double a = d[i], b = d[(i + 1) % 3];
                        sgm.half_edge[k] = 3 * f + i;
                        sgm.t[k] = (L - a) / (b - a);
                        ++k;
                    }
                out[o] = sgm;
            }
            ++o;
        }
    }
}

}  // namespace pch

using namespace pch;

extern "C" pch_status pch_iso_contours(const pch_mesh* m, const double* dist, int32_t dist_on_device,
                                       const double* levels, int32_t n_levels, pch_contour_segment* segments,
                                       int64_t capacity, int64_t* n_segments) {
    clear_error();
    if (!m || !dist || !levels || n_levels <= 0 || !n_segments || capacity < 0 || (capacity > 0 && !segments))
        return set_error(PCH_ERR_INVALID_ARG, "null argument, no level or negative capacity");
    for (int l = 0; l < n_levels; ++l)
        if (!std::isfinite(levels[l])) return set_error(PCH_ERR_INVALID_ARG, "level %d is not finite", l);
    const int nf = m->dm.nf, nv = m->dm.nv;
    double *ddist = nullptr, *dlev = nullptr;
    int *cnt = nullptr, *off = nullptr, *tmp = nullptr;
    unsigned long long* dtotal = nullptr;
    pch_contour_segment* dseg = nullptr;
    const size_t ntmp = scan_tmp_ints(nf);
    cudaStream_t s = 0;
    unsigned long long total = 0;
    pch_status st = PCH_OK;
    cudaError_t e = cudaSuccess;
    if (!dist_on_device) {
        e = cudaMalloc(&ddist, sizeof(double) * (size_t)nv);
        if (!e) e = cudaMemcpy(ddist, dist, sizeof(double) * (size_t)nv, cudaMemcpyHostToDevice);
    }
    if (!e) e = cudaMalloc(&dlev, sizeof(double) * (size_t)n_levels);
    if (!e) e = cudaMemcpy(dlev, levels, sizeof(double) * (size_t)n_levels, cudaMemcpyHostToDevice);
    if (!e) e = cudaMalloc(&cnt, sizeof(int) * (size_t)nf);
    if (!e) e = cudaMalloc(&off, sizeof(int) * (size_t)nf);
    if (!e) e = cudaMalloc(&tmp, sizeof(int) * std::max<size_t>(ntmp, 1));
    if (!e) e = cudaMalloc(&dtotal, sizeof(unsigned long long));
    if (!e) e = cudaMemset(dtotal, 0, sizeof(unsigned long long));
    const double* dd = dist_on_device ? dist : ddist;
    const int grid = sm_count() * 4;
    if (!e) {
        k_contour_count<<<grid, 256, 0, s>>>(m->dm.rec, nf, dd, dlev, n_levels, cnt, dtotal);
        e = cudaGetLastError();
    }
    if (!e) e = cudaMemcpy(&total, dtotal, sizeof(unsigned long long), cudaMemcpyDeviceToHost);
    if (!e && total > (unsigned long long)INT_MAX) {
        st = set_error(PCH_ERR_CAPACITY, "%llu contour segments exceed 2^31 - 1", total);
    } else if (!e) {
        const long long keep = std::min<long long>(capacity, (long long)total);
        e = exclusive_scan(cnt, off, nf, tmp, s);
        if (!e && keep > 0) e = cudaMalloc(&dseg, sizeof(pch_contour_segment) * (size_t)keep);
        if (!e && keep > 0) {
            k_contour_write<<<grid, 256, 0, s>>>(m->dm.rec, nf, dd, dlev, n_levels, off, keep, dseg);
            e = cudaGetLastError();
        }
        if (!e && keep > 0) e = cudaMemcpy(segments, dseg, sizeof(pch_contour_segment) * (size_t)keep, cudaMemcpyDeviceToHost);
    }
    cudaFree(ddist); cudaFree(dlev); cudaFree(cnt); cudaFree(off); cudaFree(tmp); cudaFree(dtotal); cudaFree(dseg);
    if (e) return set_error(e == cudaErrorMemoryAllocation ? PCH_ERR_OOM : PCH_ERR_CUDA, "iso-contours: %s",
                            cudaGetErrorString(e));
    if (st != PCH_OK) return st;
    *n_segments = (int64_t)total;
    return PCH_OK;
}
